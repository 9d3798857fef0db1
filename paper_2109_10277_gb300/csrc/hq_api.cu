// C ABI of libhq (declared in include/hq.h): grid lifecycle, the per-slice
// steps of the quasi-static loop (Sec. 2 enumerate; Sec. 3.1 per-slice beam
// work; Sec. 3.2 push, deposition, Poisson and predictor-corrector solvers)
// and the full sweep.  Host code only orders launches on the grid's stream.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hq_internal.cuh"

void graph_free(hq_grid_s* g);   // the captured sweep (defined before the C entry points)

using namespace hq;

namespace {

thread_local std::string g_global_err;

hq_status fail(hq_grid_s* g, hq_status st, const std::string& msg) {
  if (g) g->err = msg;
  else g_global_err = msg;
  return st;
}

#define HQ_CUDA(g, call)                                                                         \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail((g), e_ == cudaErrorMemoryAllocation ? HQ_ERR_OOM : HQ_ERR_CUDA, \
                                       std::string(#call) + ": " + cudaGetErrorString(e_));        \
  } while (0)

// FP32 value rounded to TF32 (11 significant bits, ties away from zero), as cvt.rna.tf32.f32
// rounds on the device.
float round_tf32_host(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  std::memcpy(&v, &u, 4);
  return v;
}

template <typename P>
cudaError_t dalloc(P** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

void adj_free(hq_grid_s* g);

void free_all(hq_grid_s* g) {
  auto F = [](void* p) { if (p) cudaFree(p); };
  for (hq::Plasma<double>* p : {&g->p64}) {
    F(p->x); F(p->y); F(p->psi); F(p->ux); F(p->uy); F(p->w); F(p->alive); F(p->hist);
  }
  {
    hq::Plasma<float>& p = g->p32;
    if (!g->fp64) {
      // x, y, psi, alive are shared with p64 storage (freed above); free the typed arrays
      F(p.ux); F(p.uy); F(p.w); F(p.hist); F(p.cell); F(p.fx); F(p.fy); F(p.opp); F(p.hsum); F(p.f4);
    }
  }
  if (g->det_arena) {
    // the deposit records are carved from the arena
    g->dep[0] = g->dep[1] = g->chi[0] = g->chi[1] = g->rho_ion = g->tj = g->bjn = nullptr;
    g->xs4 = g->xs1 = g->bjp = nullptr;
    F(g->det_arena);
    F(g->det_mirror);
  }
  for (int k = 0; k < kMaxSpecies; ++k) F(g->d_sp_prof[k]);
  F(g->c0);
  F(g->porigin); F(g->sort_key); F(g->sort_perm); F(g->sort_count); F(g->sort_offset); F(g->sort_tsum);
  F(g->sort_scratch);
  for (int i = 0; i < 2; ++i) { F(g->dep[i]); F(g->chi[i]); F(g->op_hi[i]); F(g->op_lo[i]); F(g->psrc[i]); }
  F(g->rho_ion); F(g->tj); F(g->bsrc0); F(g->bjn); F(g->bjp); F(g->xs4); F(g->xs1); F(g->pcg_r); F(g->pcg_p); F(g->pcg_s);
  F(g->pcg_part);
  F(g->d_pcres);
  F(g->scale_h); F(g->gf); F(g->bm); F(g->psi); F(g->bprev1); F(g->solved);
  F(g->f64_a); F(g->f64_b); F(g->f64_scale); F(g->tw_x); F(g->tw_y); F(g->sin_x); F(g->sin_y);
  F(g->sx_hi); F(g->sx_lo); F(g->sy_hi); F(g->sy_lo); F(g->f32_scale);
  for (int b = 0; b < kMaxBeams; ++b) {
    F(g->bins[b].bin); F(g->bins[b].count); F(g->bins[b].offset); F(g->bins[b].cursor); F(g->bins[b].perm);
  }
  adj_free(g);
  graph_free(g);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  g->cap_stream = nullptr;
  if (g->aux_stream) cudaStreamDestroy(g->aux_stream);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  g->aux_stream = nullptr;
  g->ev_fork = g->ev_join = nullptr;
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  g->ev_pool.clear();
  F(g->d_profile); F(g->d_status); F(g->d_removed); F(g->d_scratch_int); F(g->d_gbar);
  if (g->tmaps) dst_tc_free(g);
}

// (2/nx)(2/ny) / (lambda_kl - shift) for the 5-point Laplacian L (shift 0: Poisson; shift c > 0:
// the explicit solver's preconditioner (L - c)^{-1}); zero on mode 0 (wall).
std::vector<double> scale_table(const hq_grid_s* g, int rows, int cols, double shift = 0.0) {
  std::vector<double> t((size_t)rows * cols, 0.0);
  const double pi = M_PI;
  for (int l = 1; l < g->ny; ++l) {
    const double sy = std::sin(pi * l / (2.0 * g->ny));
    for (int k = 1; k < g->nx; ++k) {
      const double sx = std::sin(pi * k / (2.0 * g->nx));
      const double lam = -(4.0 / (g->geom.dx * g->geom.dx)) * sx * sx - (4.0 / (g->geom.dy * g->geom.dy)) * sy * sy;
      t[(size_t)l * cols + k] = (4.0 / ((double)g->nx * g->ny)) / (lam - shift);
    }
  }
  return t;
}

// sin(pi j k / n) with exact argument reduction.
double sin_jk(int64_t j, int64_t k, int n) {
  const int64_t m = (j * k) % (2 * (int64_t)n);
  return std::sin(M_PI * (double)m / (double)n);
}


// Fold matrix of the folded DST-I, [n][n/2]: row = output slot s (index k = fold_node(s)),
// column u = folded input column of pair (a, b) = fold_pair(u).  Odd k weigh the pair sum
// with sin(pi a k / n), even k the pair difference; the wall pair (0, n/2) stores x_{n/2}
// as its sum (weight sin(pi k / 2)) and nothing as its difference.
std::vector<double> fold_matrix(int n) {
  std::vector<double> c((size_t)n * (n / 2), 0.0);
  for (int s = 0; s < n; ++s) {
    const int k = fold_node(s, n);
    for (int u = 0; u < n / 2; ++u) {
      int pa, pb;
      fold_pair(u, n, pa, pb);
      const bool wall = pa == 0;
      double v;
      if (k & 1) v = wall ? sin_jk(pb, k, n) : sin_jk(pa, k, n);
      else v = wall ? 0.0 : sin_jk(pa, k, n);
      c[(size_t)s * (n / 2) + u] = v;
    }
  }
  return c;
}

// ---------------------------------------------------------------- checkpoints and tapes
// A stored plasma slice: the state a slice starts from (or is recomputed from).
struct Snap {
  double *x = nullptr, *y = nullptr, *psi = nullptr;
  void *ux = nullptr, *uy = nullptr, *hist = nullptr;
  uint8_t* alive = nullptr;
  int32_t* cell = nullptr;
  float *fx = nullptr, *fy = nullptr, *opp = nullptr, *hsum = nullptr;
};

// Checkpoints every k slices (plasma + the field records a slice starts from), the
// per-slice tapes of one segment (plasma, gather fields, B_perp of each predictor-
// corrector iterate), and the adjoint state.
struct AdjStore {
  int k = 0, nseg = 0;
  std::vector<Snap> ck;
  std::vector<void*> ck_dep0, ck_dep1, ck_chi0, ck_chi1, ck_b1, ck_b2, ck_ps0, ck_ps1;
  std::vector<Snap> tape;
  std::vector<void*> tape_gf, tape_b;
  int tape_slot = -1;       // tape slot of the slice being solved (-1: not taping)
  int fwd_done = 0;         // a checkpointed forward sweep is available
  int fwd_tape_base = -1;   // first slice held by the tape after the forward sweep
  std::vector<hq_beam_view> fwd_beams;
  int fwd_witness = -1;
  void *sx = nullptr, *sy = nullptr, *sux = nullptr, *suy = nullptr, *spsi = nullptr, *sh = nullptr, *sacc = nullptr;
  double* wbar_p = nullptr;
  void* dbar[3] = {nullptr, nullptr, nullptr};
  void* carry[3] = {nullptr, nullptr, nullptr};
  // adjoints of the gathered fields of one slice: ExmBy, EypBx, Ez, Bz (4 per node, from the
  // witness, final and trial adjoints) and Bx, By (2 per node, from the final adjoint)
  void *tbar = nullptr, *fbar_b = nullptr;
  void *bbar = nullptr, *jbar = nullptr, *jtot = nullptr, *rho_ion_bar = nullptr;
  std::vector<void*> allocs;
};

AdjStore* adj_of(const hq_grid_s* g) { return reinterpret_cast<AdjStore*>(g->adj); }

void snap_copy(hq_grid_s* g, Snap& d, bool save) {
  const size_t np = (size_t)g->np, ts = g->tsize;
  auto cp = [&](void* store, const void* live, size_t bytes) {
    if (save) cudaMemcpyAsync(store, live, bytes, cudaMemcpyDeviceToDevice, g->stream);
    else cudaMemcpyAsync(const_cast<void*>(live), store, bytes, cudaMemcpyDeviceToDevice, g->stream);
  };
  cp(d.x, g->p64.x, 8 * np);
  cp(d.y, g->p64.y, 8 * np);
  cp(d.psi, g->p64.psi, 8 * np);
  cp(d.alive, g->p64.alive, np);
  if (g->fp64) {
    cp(d.ux, g->p64.ux, ts * np);
    cp(d.uy, g->p64.uy, ts * np);
    cp(d.hist, g->p64.hist, ts * np * kRing * 5);
  } else {
    cp(d.ux, g->p32.ux, ts * np);
    cp(d.uy, g->p32.uy, ts * np);
    cp(d.hist, g->p32.hist, ts * np * kRing * 5);
    cp(d.cell, g->p32.cell, 4 * np);
    cp(d.fx, g->p32.fx, 4 * np);
    cp(d.fy, g->p32.fy, 4 * np);
    cp(d.opp, g->p32.opp, 4 * np);
    cp(d.hsum, g->p32.hsum, 4 * np * 5);
  }
}

// Tape hooks called by the forward solve of a slice.
void tape_slice_begin(hq_grid_s* g) {
  AdjStore* a = adj_of(g);
  if (a && a->tape_slot >= 0) snap_copy(g, a->tape[a->tape_slot], true);
}
void tape_b_iterate(hq_grid_s* g, int m) {
  AdjStore* a = adj_of(g);
  if (!a || a->tape_slot < 0) return;
  char* base = reinterpret_cast<char*>(a->tape_b[a->tape_slot]) + (size_t)m * 2 * g->tsize * g->nnode;
  cudaMemcpyAsync(base, g->bm, 2 * g->tsize * g->nnode, cudaMemcpyDeviceToDevice, g->stream);
}
// the slice's converged gather record followed by its converged B_perp record
void tape_slice_end(hq_grid_s* g) {
  AdjStore* a = adj_of(g);
  if (a && a->tape_slot >= 0) {
    const size_t gfb = kGF * g->tsize * g->nnode;
    char* t = reinterpret_cast<char*>(a->tape_gf[a->tape_slot]);
    cudaMemcpyAsync(t, g->gf, gfb, cudaMemcpyDeviceToDevice, g->stream);
    cudaMemcpyAsync(t + gfb, g->bm, 2 * g->tsize * g->nnode, cudaMemcpyDeviceToDevice, g->stream);
  }
}

void adj_free(hq_grid_s* g) {
  AdjStore* a = adj_of(g);
  if (!a) return;
  for (void* p : a->allocs) cudaFree(p);
  delete a;
  g->adj = nullptr;
}

// Counts the launches of one kernel group and, while profiling is on, brackets
// the group with a pair of CUDA events on the grid's stream.
struct Prof {
  hq_grid_s* g;
  bool on;
  Prof(hq_grid_s* g_, int cls, int nlaunch) : g(g_), on(g_->prof_on != 0) {
    g->launches[cls] += nlaunch;
    if (!on) return;
    if (g->ev_used + 2 > g->ev_pool.size()) {
      for (int k = 0; k < 256; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { on = false; return; }
        g->ev_pool.push_back(e);
      }
    }
    g->ev_class.push_back(cls);
    cudaEventRecord(g->ev_pool[g->ev_used], g->stream);
  }
  ~Prof() {
    if (!on) return;
    cudaEventRecord(g->ev_pool[g->ev_used + 1], g->stream);
    g->ev_used += 2;
  }
};

void dst_solve(hq_grid_s* g, int nrhs) {
  Prof p(g, HQ_K_DST, g->fp64 ? 4 : 1);   // FP64: four FFT passes; FP32: one fused cooperative launch
  if (g->fp64) dst_solve_f64(g, nrhs, g->stream);
  else dst_solve_tc(g, nrhs, g->stream);
}

template <typename T>
hq_status solve_fields_impl(hq_grid_s* g, int slice) {
  cudaStream_t s = g->stream;
  void* cur = g->dep[slice & 1];
  void* prev = g->dep[(slice + 1) & 1];
  void* chi_prev = g->chi[(slice + 1) & 1];
  tape_slice_begin(g);
  const bool fused_src = !g->fp64 && !g->sep_src;   // FP32: sources formed inside the solve launch
  if (fused_src) {
    Prof p(g, HQ_K_DST, 1);
    dst_solve_tc_main(g, cur, s);
  } else {
    { Prof p(g, HQ_K_FIELD, 1); launch_src_main<T>(g, cur, s); }
    dst_solve(g, 3);
  }
  { Prof p(g, HQ_K_FIELD, 1); launch_finish_main<T>(g, g->solved, slice == 0, s); }
  const int npc = g->d.n_pc_iter;
  if (g->explicit_b) {
    // explicit B_perp solver: source pass, then npc PCG iterations from the guess in bm
    const void* chi_cur = g->chi[slice & 1];
    { Prof p(g, HQ_K_TRIAL, 1); launch_explicit_src<T>(g, s); }
    if (g->det) {
      launch_fx_decode(g, g->xs4, 4 * g->nnode, nullptr, s);
      launch_fx_decode(g, g->xs1, g->nnode, nullptr, s);
    }
    { Prof p(g, HQ_K_FIELD, 1); launch_pcg_init<T>(g, slice, cur, chi_cur, prev, chi_prev, s); }
    for (int k = 0; k < npc; ++k) {
      {
        Prof p(g, HQ_K_DST, g->fp64 ? 4 : 1);
        if (g->fp64) dst_solve_f64(g, 2, s, reinterpret_cast<const double*>(g->scale_h));
        else dst_solve_tc_shifted(g, 2, s);
      }
      { Prof p(g, HQ_K_FIELD, 4); launch_pcg_iter<T>(g, slice, k, chi_cur, s); }
    }
    tape_slice_end(g);
    return HQ_OK;
  }
  for (int m = 0; m < npc; ++m) {
    const int last = m == npc - 1;
    // the last iteration's mixing adds its residual sums to this slice's pair
    g->pc_rsum = last && g->d_pcres ? g->d_pcres + 2 * kResLanes * (int64_t)slice : nullptr;   // (opt-in)
    tape_b_iterate(g, m);
    g->pc_iter = m;   // the B_perp sources of iteration 0 keep their invariant part for the others
    { Prof p(g, HQ_K_TRIAL, 1); launch_trial_pass<T>(g, slice, m, s); }
    if (m == 0) g->f4_slice = (g->fp64 || g->no_f4) ? -1 : slice;   // the final pass may reuse it
    if (g->det) launch_fx_decode(g, g->tj, 2 * g->nnode, nullptr, s);
    if (fused_src) {
      Prof p(g, HQ_K_DST, 1);   // sources, solve and the mixing in one launch
      dst_solve_tc_bmix_src(g, cur, prev, chi_prev, last, s);
      continue;
    }
    { Prof p(g, HQ_K_FIELD, 1); launch_src_bperp<T>(g, cur, prev, chi_prev, last, s); }
    if (g->fp64) {
      dst_solve(g, 2);
      Prof p(g, HQ_K_FIELD, 1);
      launch_finish_bperp<T>(g, g->solved, s);
    } else {
      Prof p(g, HQ_K_DST, 1);   // the mixing runs in the last product's epilogue
      dst_solve_tc_bmix(g, last, s);
    }
  }
  g->pc_rsum = nullptr;
  if (npc == 0) {
    // no predictor-corrector: B(i) is the guess; clear and reset without the source kernels
    Prof p(g, HQ_K_FIELD, 2);
    launch_zero<T>(g->bjn, 2 * g->nnode, s);
    launch_reset_dep<T>(g, prev, chi_prev, s);
  }
  tape_slice_end(g);
  return HQ_OK;
}

// Final AB5 pass of slice `slice_from` depositing into the record `parity`, which the
// last predictor-corrector source kernel of that slice reset to the ion background.
template <typename T>
void final_pass(hq_grid_s* g, int slice_from, int parity) {
  Prof p(g, HQ_K_FINAL, 1);
  launch_final_pass<T>(g, slice_from, g->dep[parity], g->chi[parity], g->f4_slice == slice_from, g->stream);
  if (g->det) {
    launch_fx_decode(g, g->dep[parity], 4 * g->nnode, nullptr, g->stream);
    launch_fx_decode(g, g->chi[parity], g->nnode, nullptr, g->stream);
  }
}

template <typename T>
void advance_impl(hq_grid_s* g, int slice) {
  cudaStream_t s = g->stream;
  if (slice == 0) {
    g->f4_slice = -1;
    Prof p(g, HQ_K_OTHER, g->bjp ? 9 : 8);
    launch_reset_dep<T>(g, g->dep[0], g->chi[0], s);
    launch_plasma_init<T>(g, s);
    launch_deposit_initial<T>(g, g->dep[0], g->chi[0], 0, s);
    if (g->det) {
      launch_fx_decode(g, g->dep[0], 4 * g->nnode, nullptr, s);
      launch_fx_decode(g, g->chi[0], g->nnode, nullptr, s);
    }
    launch_zero<T>(g->dep[1], 4 * g->nnode, s);   // J(-1) = 0 ahead of the box
    if (!g->fp64) launch_zero<float>(g->psrc[1], g->nnode, s);
    launch_zero<T>(g->bprev1, 2 * g->nnode, s);
    launch_zero<T>(g->bjn, 2 * g->nnode, s);
    launch_zero<T>(g->tj, 2 * g->nnode, s);
    if (g->bjp) launch_zero<T>(g->bjp, 4 * g->nnode, s);
    if (g->d_pcres) cudaMemsetAsync(g->d_pcres, 0, sizeof(double) * 2 * kResLanes * g->nz, s);
  } else {
    final_pass<T>(g, slice - 1, slice & 1);
    if (g->d.resort_every > 0 && slice % g->d.resort_every == 0) {
      Prof p(g, HQ_K_OTHER, 8);
      launch_resort(g, s);
    }
  }
}

bool same_view(const hq_beam_view& a, const hq_beam_view& b) {
  return a.n == b.n && a.x == b.x && a.y == b.y && a.zeta == b.zeta && a.ux == b.ux && a.uy == b.uy && a.uz == b.uz &&
         a.w == b.w && a.charge == b.charge && a.mass == b.mass;
}

hq_status check_views(hq_grid_s* g, const hq_beam_view* beams, int nb) {
  if (nb < 0 || nb > kMaxBeams) return fail(g, HQ_ERR_ARG, "nbeams must be 0..4");
  if (nb > 0 && !beams) return fail(g, HQ_ERR_ARG, "beams is NULL");
  for (int b = 0; b < nb; ++b) {
    const hq_beam_view& v = beams[b];
    if (v.n < 0 || v.n > 0x7fffffffLL) return fail(g, HQ_ERR_ARG, "beam size out of range");
    if (v.n > 0 && (!v.x || !v.y || !v.zeta || !v.ux || !v.uy || !v.uz || !v.w))
      return fail(g, HQ_ERR_ARG, "beam array is NULL");
    if (!(v.mass > 0.0) || !std::isfinite(v.charge)) return fail(g, HQ_ERR_ARG, "beam charge/mass invalid");
  }
  return HQ_OK;
}

int bound_index(const hq_grid_s* g, const hq_beam_view* v) {
  for (int b = 0; b < g->nbound; ++b)
    if (same_view(*v, g->bound[b])) return b;
  return -1;
}

hq_status check_launch(hq_grid_s* g) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(g, HQ_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return HQ_OK;
}


// ---------------------------------------------------------------- checkpointed forward and adjoint
hq_status adj_alloc(hq_grid_s* g, int k) {
  AdjStore* a = adj_of(g);
  if (a && a->k == k) return HQ_OK;
  adj_free(g);
  a = new (std::nothrow) AdjStore();
  if (!a) return fail(g, HQ_ERR_OOM, "host allocation failed");
  g->adj = a;
  a->k = k;
  a->nseg = (g->nz + k - 1) / k;
  const size_t np = (size_t)g->np, ts = g->tsize, nn = (size_t)g->nnode;
  const int npc = g->d.n_pc_iter;
  auto A = [&](void** p, size_t bytes) -> bool {
    *p = nullptr;
    if (bytes == 0) return true;
    if (cudaMalloc(p, bytes) != cudaSuccess) return false;
    a->allocs.push_back(*p);
    return true;
  };
  auto snap = [&](Snap& d) -> bool {
    bool ok = A((void**)&d.x, 8 * np) && A((void**)&d.y, 8 * np) && A((void**)&d.psi, 8 * np) &&
              A((void**)&d.alive, np) && A(&d.ux, ts * np) && A(&d.uy, ts * np) && A(&d.hist, ts * np * kRing * 5);
    if (ok && !g->fp64)
      ok = A((void**)&d.cell, 4 * np) && A((void**)&d.fx, 4 * np) && A((void**)&d.fy, 4 * np) &&
           A((void**)&d.opp, 4 * np) && A((void**)&d.hsum, 4 * np * 5);
    return ok;
  };
  bool ok = true;
  a->ck.resize(a->nseg);
  a->ck_dep0.resize(a->nseg); a->ck_dep1.resize(a->nseg); a->ck_chi0.resize(a->nseg); a->ck_chi1.resize(a->nseg);
  a->ck_b1.resize(a->nseg); a->ck_b2.resize(a->nseg);
  a->ck_ps0.assign(a->nseg, nullptr); a->ck_ps1.assign(a->nseg, nullptr);
  for (int i = 0; ok && i < a->nseg; ++i)
    ok = snap(a->ck[i]) && A(&a->ck_dep0[i], 4 * ts * nn) && A(&a->ck_dep1[i], 4 * ts * nn) &&
         A(&a->ck_chi0[i], ts * nn) && A(&a->ck_chi1[i], ts * nn) && A(&a->ck_b1[i], 2 * ts * nn) &&
         A(&a->ck_b2[i], 2 * ts * nn) && (g->fp64 || (A(&a->ck_ps0[i], 4 * nn) && A(&a->ck_ps1[i], 4 * nn)));
  a->tape.resize(k);
  a->tape_gf.resize(k);
  a->tape_b.resize(k);
  for (int i = 0; ok && i < k; ++i)
    ok = snap(a->tape[i]) && A(&a->tape_gf[i], (kGF + 2) * ts * nn) && A(&a->tape_b[i], (size_t)std::max(npc, 1) * 2 * ts * nn);
  ok = ok && A(&a->sx, ts * np) && A(&a->sy, ts * np) && A(&a->sux, ts * np) && A(&a->suy, ts * np) &&
       A(&a->spsi, ts * np) && A(&a->sh, ts * np * 20) && A(&a->sacc, ts * np * 5) && A((void**)&a->wbar_p, 8 * np) && A(&a->tbar, 4 * ts * nn) && A(&a->fbar_b, 2 * ts * nn) &&
       A(&a->bbar, (size_t)(npc + 1) * 2 * ts * nn) && A(&a->jbar, 2 * ts * nn) && A(&a->jtot, 2 * ts * nn) &&
       A(&a->rho_ion_bar, ts * nn);
  for (int i = 0; ok && i < 3; ++i) ok = A(&a->dbar[i], 4 * ts * nn) && A(&a->carry[i], 2 * ts * nn);
  if (!ok) {
    adj_free(g);
    return fail(g, HQ_ERR_OOM, "checkpoint/tape allocation failed (reduce ckpt_every)");
  }
  return HQ_OK;
}

void ckpt_copy(hq_grid_s* g, int seg, bool save) {
  AdjStore* a = adj_of(g);
  snap_copy(g, a->ck[seg], save);
  const size_t ts = g->tsize, nn = (size_t)g->nnode;
  auto cp = [&](void* store, void* live, size_t bytes) {
    if (save) cudaMemcpyAsync(store, live, bytes, cudaMemcpyDeviceToDevice, g->stream);
    else cudaMemcpyAsync(live, store, bytes, cudaMemcpyDeviceToDevice, g->stream);
  };
  cp(a->ck_dep0[seg], g->dep[0], 4 * ts * nn);
  cp(a->ck_dep1[seg], g->dep[1], 4 * ts * nn);
  cp(a->ck_chi0[seg], g->chi[0], ts * nn);
  cp(a->ck_chi1[seg], g->chi[1], ts * nn);
  // B_perp of the two previous slices: B(i-1) still in the B_perp record, B(i-2) in bprev1
  cp(a->ck_b1[seg], g->bm, 2 * ts * nn);
  cp(a->ck_b2[seg], g->bprev1, 2 * ts * nn);
  if (!g->fp64) {
    cp(a->ck_ps0[seg], g->psrc[0], 4 * nn);
    cp(a->ck_ps1[seg], g->psrc[1], 4 * nn);
  }
}

// Binds view `v` to bin slot k: counting sort of its particles by slice at their current zeta.
hq_status bind_view(hq_grid_s* g, int k, const hq_beam_view& v) {
  BeamBins& bb = g->bins[k];
  if (bb.cap < v.n) {
    if (bb.bin) cudaFree(bb.bin);
    if (bb.perm) cudaFree(bb.perm);
    bb.bin = bb.perm = nullptr;
    bb.cap = 0;
    HQ_CUDA(g, dalloc(&bb.bin, sizeof(int32_t) * v.n));
    HQ_CUDA(g, dalloc(&bb.perm, sizeof(int32_t) * v.n));
    bb.cap = v.n;
  }
  g->bound[k] = v;
  Prof p(g, HQ_K_BEAM, v.n > 0 ? 3 : 1);
  launch_beam_bin(g, k, v, g->stream);
  return HQ_OK;
}

template <typename T>
hq_status beam_deposit_impl(hq_grid_s* g, const hq_beam_view* beams, int nb, int slice) {
  cudaStream_t s = g->stream;
  // Slice 0 bins every view for the sweep.  A later slice keeps the bins of the views it was
  // already given (their particles of later slices have not been pushed) and bins a view it
  // has not seen before into a slot that no view of this call holds; views missing from the
  // call lose their slot.  This is how a beam arrives box by box (Sec. 5.2 temporal pipeline).
  int slot[kMaxBeams];
  hq_status st;
  if (slice == 0) {
    for (int b = 0; b < nb; ++b)
      if ((st = bind_view(g, slot[b] = b, beams[b])) != HQ_OK) return st;
    for (int k = nb; k < kMaxBeams; ++k) g->bound[k].n = -1;
  } else {
    bool held[kMaxBeams] = {};
    for (int b = 0; b < nb; ++b) {
      slot[b] = bound_index(g, &beams[b]);
      if (slot[b] >= 0) held[slot[b]] = true;
    }
    for (int b = 0; b < nb; ++b) {
      if (slot[b] >= 0) continue;
      int k = 0;
      while (held[k]) ++k;   // nb <= kMaxBeams views: a free slot exists
      held[k] = true;
      if ((st = bind_view(g, slot[b] = k, beams[b])) != HQ_OK) return st;
    }
    for (int k = 0; k < kMaxBeams; ++k)
      if (!held[k]) g->bound[k].n = -1;
  }
  g->nbound = kMaxBeams;
  // bjn (beam J_perp of slice i+1) was cleared at the end of the previous slice's solve
  for (int b = 0; b < nb; ++b) {
    if (beams[b].n == 0) continue;
    Prof p(g, HQ_K_BEAM, 1);
    launch_beam_deposit<T>(g, slot[b], beams[b], slice, g->dep[slice & 1], g->bjn, s);
  }
  if (g->det) {
    launch_fx_decode(g, g->dep[slice & 1], 4 * g->nnode, nullptr, s);
    launch_fx_decode(g, g->bjn, 2 * g->nnode, nullptr, s);
    if (g->bjp) launch_fx_decode(g, bjp_at(g, slice), 2 * g->nnode, nullptr, s);
  }
  return HQ_OK;
}

// Runs slices [a0, a1) from the state after hq_advance_slice(a0), taping slices >= tape_from.
template <typename T>
hq_status run_segment(hq_grid_s* g, const hq_beam_view* beams, int nb, int a0, int a1, int tape_from, int witness,
                      double* wsums) {
  AdjStore* a = adj_of(g);
  for (int i = a0; i < a1; ++i) {
    if (i > a0) advance_impl<T>(g, i);
    hq_status st = beam_deposit_impl<T>(g, beams, nb, i);
    if (st != HQ_OK) return st;
    a->tape_slot = i >= tape_from ? i - tape_from : -1;
    solve_fields_impl<T>(g, i);
    a->tape_slot = -1;
    if (witness >= 0 && wsums && beams[witness].n > 0) {
      Prof p(g, HQ_K_BEAM, 1);
      launch_witness<T>(g, witness, beams[witness], i, wsums, g->stream);
    }
  }
  return HQ_OK;
}

template <typename T>
hq_status forward_ckpt_impl(hq_grid_s* g, const hq_beam_view* beams, int nb, int witness, double* wsums) {
  AdjStore* a = adj_of(g);
  const int last_seg = a->nseg - 1;
  const int tape_from = last_seg * a->k;
  for (int seg = 0; seg < a->nseg; ++seg) {
    const int a0 = seg * a->k, a1 = std::min(g->nz, a0 + a->k);
    advance_impl<T>(g, a0);
    ckpt_copy(g, seg, true);
    hq_status st = run_segment<T>(g, beams, nb, a0, a1, seg == last_seg ? tape_from : g->nz, witness, wsums);
    if (st != HQ_OK) return st;
  }
  a->fwd_tape_base = tape_from;
  return HQ_OK;
}

template <typename T>
hq_status adjoint_impl(hq_grid_s* g, const hq_beam_view* beams, int nb, int witness, const double* sbar,
                       const hq_field_out* seeds, double* const* wbar_b, double* wbar_p_out, double* dn0,
                       double* dprof) {
  AdjStore* a = adj_of(g);
  cudaStream_t s = g->stream;
  const size_t np = (size_t)g->np, ts = g->tsize, nn = (size_t)g->nnode;
  const int npc = g->d.n_pc_iter;
  const size_t brec = 2 * ts * nn;
  for (void* p : {a->sx, a->sy, a->sux, a->suy, a->spsi}) cudaMemsetAsync(p, 0, ts * np, s);
  cudaMemsetAsync(a->sh, 0, ts * np * 20, s);
  cudaMemsetAsync(a->sacc, 0, ts * np * 5, s);
  cudaMemsetAsync(a->wbar_p, 0, 8 * np, s);
  for (int i = 0; i < 3; ++i) {
    cudaMemsetAsync(a->dbar[i], 0, 4 * ts * nn, s);
    cudaMemsetAsync(a->carry[i], 0, 2 * ts * nn, s);
  }
  cudaMemsetAsync(a->rho_ion_bar, 0, ts * nn, s);
  // cleared again by their consumers (main_post, bstart) for every next slice
  cudaMemsetAsync(a->tbar, 0, 4 * ts * nn, s);
  cudaMemsetAsync(a->fbar_b, 0, 2 * ts * nn, s);
  for (int b = 0; b < nb; ++b)
    if (wbar_b && wbar_b[b] && beams[b].n > 0) cudaMemsetAsync(wbar_b[b], 0, 8 * (size_t)beams[b].n, s);
  void* dnext = a->dbar[0];
  void* dcur = a->dbar[1];
  void* dprev = a->dbar[2];
  AdjView<T> av{reinterpret_cast<T*>(a->sx), reinterpret_cast<T*>(a->sy), reinterpret_cast<T*>(a->sux),
                reinterpret_cast<T*>(a->suy), reinterpret_cast<T*>(a->spsi), reinterpret_cast<T*>(a->sh),
                reinterpret_cast<T*>(a->sacc)};
  const T* w = g->fp64 ? reinterpret_cast<const T*>(g->p64.w) : reinterpret_cast<const T*>(g->p32.w);
  for (int seg = a->nseg - 1; seg >= 0; --seg) {
    const int a0 = seg * a->k, a1 = std::min(g->nz, a0 + a->k);
    if (!(seg == a->nseg - 1 && a->fwd_tape_base == a0)) {
      // recompute the segment from its checkpoint, taping every slice
      ckpt_copy(g, seg, false);
      cudaMemsetAsync(g->tj, 0, 2 * ts * nn, s);
      cudaMemsetAsync(g->bjn, 0, 2 * ts * nn, s);
      hq_status st = run_segment<T>(g, beams, nb, a0, a1, a0, -1, nullptr);
      if (st != HQ_OK) return st;
    }
    for (int i = a1 - 1; i >= a0; --i) {
      const int t = i - a0;
      const Snap& sn = a->tape[t];
      const bool f32 = !g->fp64;
      SnapView<T> sv{g->np, sn.x, sn.y, sn.psi, reinterpret_cast<const T*>(sn.ux), reinterpret_cast<const T*>(sn.uy), w,
                     sn.alive, reinterpret_cast<const T*>(sn.hist), f32 ? sn.hsum : nullptr, f32 ? sn.cell : nullptr,
                     f32 ? sn.fx : nullptr, f32 ? sn.fy : nullptr, f32 ? sn.opp : nullptr};
      const void* gf = a->tape_gf[t];
      cudaMemsetAsync(a->jtot, 0, 2 * ts * nn, s);
      if (seeds) {
        Prof p(g, HQ_K_FIELD, 1);
        launch_adj_seed<T>(g, *seeds, i, a->tbar, a->fbar_b, dcur, s);
      }
      if (witness >= 0 && beams[witness].n > 0) {
        Prof p(g, HQ_K_BEAM, 1);
        launch_adj_witness<T>(g, witness, beams[witness], i, gf, sbar, a->tbar,
                              wbar_b ? wbar_b[witness] : nullptr, s);
      }
      if (i < g->nz - 1) {
        Prof p(g, HQ_K_FINAL, 1);
        launch_adj_final<T>(g, sv, gf, i, dnext, av, a->tbar, a->fbar_b, a->wbar_p, s);
      }
      char* bb = reinterpret_cast<char*>(a->bbar);
      { Prof p(g, HQ_K_FIELD, 1); launch_adj_bstart<T>(g, a->fbar_b, a->carry[i % 3], bb + (size_t)npc * brec, s); }
      for (int m = npc; m >= 1; --m) {
        { Prof p(g, HQ_K_FIELD, 1); launch_adj_pc_pre<T>(g, bb + (size_t)m * brec, bb + (size_t)(m - 1) * brec, s); }
        dst_solve(g, 2);
        { Prof p(g, HQ_K_FIELD, 1); launch_adj_pc_post<T>(g, dcur, dprev, a->jbar, a->jtot, s); }
        {
          Prof p(g, HQ_K_TRIAL, 1);
          launch_adj_trial<T>(g, sv, gf, reinterpret_cast<char*>(a->tape_b[t]) + (size_t)(m - 1) * brec, i, a->jbar, av,
                              a->tbar, bb + (size_t)(m - 1) * brec, a->wbar_p, s);
        }
      }
      {
        Prof p(g, HQ_K_FIELD, 1);
        launch_adj_guess<T>(g, bb, i >= 1 ? a->carry[(i - 1) % 3] : nullptr, i >= 2 ? a->carry[(i - 2) % 3] : nullptr, s);
      }
      {
        Prof p(g, HQ_K_FIELD, 1);
        const void* sp = seeds && seeds->psi ? static_cast<const char*>(seeds->psi) + (size_t)i * nn * ts : nullptr;
        launch_adj_main_pre<T>(g, a->tbar, sp, s);
      }
      dst_solve(g, 3);
      { Prof p(g, HQ_K_FIELD, 1); launch_adj_main_post<T>(g, dcur, a->rho_ion_bar, a->tbar, s); }
      for (int b = 0; b < nb; ++b) {
        if (!wbar_b || !wbar_b[b] || beams[b].n == 0) continue;
        Prof p(g, HQ_K_BEAM, 1);
        launch_adj_beam<T>(g, b, beams[b], i, dcur, a->jtot, wbar_b[b], s);
      }
      // rotate: slice i's record becomes "next" for slice i-1; the old next is cleared for i-2
      void* old_next = dnext;
      dnext = dcur;
      dcur = dprev;
      dprev = old_next;
      cudaMemsetAsync(dprev, 0, 4 * ts * nn, s);
    }
  }
  { Prof p(g, HQ_K_OTHER, 1); launch_adj_init<T>(g, dnext, a->rho_ion_bar, a->wbar_p, s); }
  if (dn0) cudaMemsetAsync(dn0, 0, 8, s);
  if (dprof && !g->profile.empty()) cudaMemsetAsync(dprof, 0, 8 * g->profile.size(), s);
  if (dn0 || dprof) launch_adj_params(g, a->wbar_p, dn0, g->profile.empty() ? nullptr : dprof, s);
  if (wbar_p_out) cudaMemcpyAsync(wbar_p_out, a->wbar_p, 8 * np, cudaMemcpyDeviceToDevice, s);
  return HQ_OK;
}

}  // namespace

namespace hq {
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("HQ_NO_PDL");
    return !(e && e[0] == '1');
  }();
  return on;
}

// Error message for calls that have no grid (read back by hq_last_error(NULL)).
void set_global_error(const std::string& msg) { g_global_err = msg; }
hq_status static_sync();   // status of the allocation-free solves (k_dst_tc.cu)
}  // namespace hq

// The slice loop of one sweep (Sec. 2), issued on the grid's stream.
// The second stream of sweep_body's fork (false: the sweep runs on the grid's stream alone).
bool aux_ready(hq_grid_t g) {
  const char* nf = std::getenv("HQ_NO_FORK");
  if (nf && nf[0] == '1') return false;
  if (g->aux_stream) return true;
  if (cudaStreamCreateWithFlags(&g->aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (g->aux_stream) cudaStreamDestroy(g->aux_stream);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    g->aux_stream = nullptr;
    g->ev_fork = g->ev_join = nullptr;
    return false;
  }
  return true;
}

hq_status sweep_body(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, double dt, const hq_field_out* out,
                     int32_t witness_beam, double* witness_sums) {
  hq_status st;
  // Without a beam push, the witness sum of slice i-1 and the beam deposit of slice i do not
  // depend on slice i's final pass (disjoint buffers, or commutative atomics into the same
  // records), so from slice 1 on they run on a second stream beside it, forked and joined with
  // events (a graph capture records the fork as parallel branches).  Slice 0 stays in order
  // (the beams are binned and the records reset there).
  const bool fork = dt == 0.0 && !g->prof_on && !g->det && aux_ready(g);
  const bool wit = witness_beam >= 0;
  for (int i = 0; i < g->nz; ++i) {
    if (fork && i > 0) {
      cudaStream_t s = g->stream;
      cudaEventRecord(g->ev_fork, s);
      if ((st = hq_advance_slice(g, i)) != HQ_OK) return st;
      cudaStreamWaitEvent(g->aux_stream, g->ev_fork, 0);
      g->stream = g->aux_stream;
      st = wit ? hq_witness_accumulate(g, &beams[witness_beam], i - 1, witness_sums) : HQ_OK;
      if (st == HQ_OK) st = hq_beam_deposit(g, beams, nbeams, i);
      cudaEventRecord(g->ev_join, g->aux_stream);
      g->stream = s;
      cudaStreamWaitEvent(s, g->ev_join, 0);
      if (st != HQ_OK) return st;
    } else {
      if ((st = hq_advance_slice(g, i)) != HQ_OK) return st;
      if ((st = hq_beam_deposit(g, beams, nbeams, i)) != HQ_OK) return st;
    }
    if ((st = hq_solve_fields(g, i)) != HQ_OK) return st;
    if (out && (st = hq_store_fields(g, out, i)) != HQ_OK) return st;
    // forked sweeps sum slice i's witness beside the next slice's final pass
    if (wit && !(fork && i + 1 < g->nz) &&
        (st = hq_witness_accumulate(g, &beams[witness_beam], i, witness_sums)) != HQ_OK)
      return st;
    if (dt != 0.0 && (st = hq_push_beams(g, beams, nbeams, i, dt)) != HQ_OK) return st;
  }
  // advance once past the tail so the plasma state matches a completed sweep
  const int nz = g->nz;
  if (g->fp64) final_pass<double>(g, nz - 1, nz & 1);
  else final_pass<float>(g, nz - 1, nz & 1);
  g->last_adv = nz;
  return check_launch(g);
}

// A captured sweep and the arguments it was captured with (device pointers and values are
// baked into its kernel nodes).
struct SweepGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<hq_beam_view> beams;
  double dt = 0.0;
  bool has_out = false;
  hq_field_out out{};
  int witness = -1;
  double* sums = nullptr;
  bool matches(const hq_beam_view* b, int nb, double dt_, const hq_field_out* o, int w, double* s) const {
    if ((int)beams.size() != nb || dt != dt_ || has_out != (o != nullptr) || witness != w || sums != s) return false;
    for (int i = 0; i < nb; ++i)
      if (!same_view(beams[i], b[i])) return false;
    return !o || std::memcmp(&out, o, sizeof(hq_field_out)) == 0;
  }
};

void graph_free(hq_grid_s* g) {
  SweepGraph* sg = reinterpret_cast<SweepGraph*>(g->sweep_graph);
  if (!sg) return;
  if (sg->exec) cudaGraphExecDestroy(sg->exec);
  delete sg;
  g->sweep_graph = nullptr;
}

// Beam bin storage for the beams of a sweep, allocated ahead of a stream capture.
hq_status reserve_bins(hq_grid_s* g, const hq_beam_view* beams, int nb) {
  for (int b = 0; b < nb; ++b) {
    BeamBins& bb = g->bins[b];
    if (bb.cap >= beams[b].n) continue;
    if (bb.bin) cudaFree(bb.bin);
    if (bb.perm) cudaFree(bb.perm);
    bb.bin = bb.perm = nullptr;
    bb.cap = 0;
    HQ_CUDA(g, dalloc(&bb.bin, sizeof(int32_t) * beams[b].n));
    HQ_CUDA(g, dalloc(&bb.perm, sizeof(int32_t) * beams[b].n));
    bb.cap = beams[b].n;
  }
  return HQ_OK;
}

extern "C" {

hq_status hq_grid_create(const hq_grid_desc* desc, void* cuda_stream, hq_grid_t* out) {
  if (!desc || !out) return fail(nullptr, HQ_ERR_ARG, "desc and out must not be NULL");
  *out = nullptr;
  const hq_grid_desc& d = *desc;
  if (d.nx < 8 || d.ny < 8 || d.nx > 4096 || d.ny > 4096) return fail(nullptr, HQ_ERR_ARG, "nx, ny must be in 8..4096");
  if (d.nzeta < 1) return fail(nullptr, HQ_ERR_ARG, "nzeta must be >= 1");
  if (!(d.xmax > d.xmin) || !(d.ymax > d.ymin) || !(d.zeta_max > d.zeta_min) || !std::isfinite(d.xmin) ||
      !std::isfinite(d.xmax) || !std::isfinite(d.ymin) || !std::isfinite(d.ymax) || !std::isfinite(d.zeta_min) ||
      !std::isfinite(d.zeta_max))
    return fail(nullptr, HQ_ERR_ARG, "box bounds must be finite with max > min");
  if (d.shape_order < 0 || d.shape_order > 3) return fail(nullptr, HQ_ERR_ARG, "shape_order must be 0..3");
  if (d.ppc_x < 1 || d.ppc_y < 1 || d.ppc_x > 16 || d.ppc_y > 16) return fail(nullptr, HQ_ERR_ARG, "ppc must be 1..16");
  if (d.n_pc_iter < 0 || d.n_pc_iter > 1000) return fail(nullptr, HQ_ERR_ARG, "n_pc_iter must be 0..1000");
  if (!std::isfinite(d.pc_mix) || !std::isfinite(d.psi_guard) || !std::isfinite(d.n0_scale))
    return fail(nullptr, HQ_ERR_ARG, "pc_mix, psi_guard and n0_scale must be finite");
  if (d.precision != HQ_PREC_FP64 && d.precision != HQ_PREC_FP32_BF16X3 && d.precision != HQ_PREC_FP32_TF32X3)
    return fail(nullptr, HQ_ERR_ARG, "unknown precision");
  if (d.bperp_solver != HQ_BPERP_PC && d.bperp_solver != HQ_BPERP_EXPLICIT)
    return fail(nullptr, HQ_ERR_ARG, "unknown bperp_solver");
  if (d.bperp_solver == HQ_BPERP_EXPLICIT && (d.n_pc_iter < 1 || d.n_pc_iter > kMaxPcg))
    return fail(nullptr, HQ_ERR_ARG, "the explicit B_perp solver needs 1..64 iterations (n_pc_iter)");
  // the explicit solver's preconditioner shift: the unperturbed chi, n0_scale for the default
  // electrons, sum q^2 n0 / M over the species otherwise
  double xshift = d.n0_scale;
  if (d.n_species > 0 && d.species) {
    xshift = 0.0;
    for (int k = 0; k < d.n_species && k < kMaxSpecies; ++k)
      xshift += d.species[k].charge * d.species[k].charge * d.species[k].n0_scale / d.species[k].mass;
  }
  if (d.bperp_solver == HQ_BPERP_EXPLICIT && !(xshift > 0.0 && std::isfinite(xshift)))
    return fail(nullptr, HQ_ERR_ARG, "the explicit B_perp solver needs a positive preconditioner shift "
                                     "(n0_scale, or sum q^2 n0 / M over the species)");
  if (d.resort_every < 0) return fail(nullptr, HQ_ERR_ARG, "resort_every must be >= 0");
  if (d.pc_residuals != 0 && d.pc_residuals != 1) return fail(nullptr, HQ_ERR_ARG, "pc_residuals must be 0 or 1");
  if (d.deterministic != 0 && d.deterministic != 1) return fail(nullptr, HQ_ERR_ARG, "deterministic must be 0 or 1");
  if (d.deterministic && d.precision != HQ_PREC_FP64)
    return fail(nullptr, HQ_ERR_UNSUPPORTED, "deterministic accumulation is an FP64 mode");
  if (d.radial_profile && (d.n_profile < 2 || !(d.profile_rmax > 0.0)))
    return fail(nullptr, HQ_ERR_ARG, "radial profile needs n_profile >= 2 and profile_rmax > 0");
  if (d.n_species < 0 || d.n_species > kMaxSpecies || (d.n_species > 0 && !d.species))
    return fail(nullptr, HQ_ERR_ARG, "n_species must be 0..4 (with a species array)");
  for (int k = 0; k < d.n_species; ++k) {
    const hq_species_desc& sd = d.species[k];
    if (!std::isfinite(sd.charge) || sd.charge == 0.0 || !(sd.mass > 0.0) || !std::isfinite(sd.mass) ||
        !std::isfinite(sd.n0_scale))
      return fail(nullptr, HQ_ERR_ARG, "species charge must be finite and non-zero, mass positive and finite");
    if (sd.ppc_x < 1 || sd.ppc_y < 1 || sd.ppc_x > 16 || sd.ppc_y > 16)
      return fail(nullptr, HQ_ERR_ARG, "species ppc must be 1..16");
    if (sd.radial_profile && (sd.n_profile < 2 || !(sd.profile_rmax > 0.0)))
      return fail(nullptr, HQ_ERR_ARG, "species radial profile needs n_profile >= 2 and profile_rmax > 0");
    if (sd.neutralize != 0 && sd.neutralize != 1) return fail(nullptr, HQ_ERR_ARG, "species neutralize must be 0 or 1");
  }
  if (d.n_species > 0 && d.resort_every > 0)
    return fail(nullptr, HQ_ERR_UNSUPPORTED, "the plasma re-sort takes the default electron plasma only");
  int64_t np = 0;
  if (d.n_species == 0) np = (int64_t)d.nx * d.ny * d.ppc_x * d.ppc_y;
  for (int k = 0; k < d.n_species; ++k) np += (int64_t)d.nx * d.ny * d.species[k].ppc_x * d.species[k].ppc_y;
  if (np > (1LL << 31) - 1) return fail(nullptr, HQ_ERR_ARG, "too many plasma particles");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, HQ_ERR_CUDA, "no CUDA device");
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return fail(nullptr, HQ_ERR_CUDA, "cudaGetDeviceProperties failed");
  if (prop.major != 10 || prop.minor != 3)
    return fail(nullptr, HQ_ERR_UNSUPPORTED, "libhq is built for sm_103a (GB300) only; device is sm_" +
                                                 std::to_string(prop.major) + std::to_string(prop.minor));

  hq_grid_s* g = new (std::nothrow) hq_grid_s();
  if (!g) return fail(nullptr, HQ_ERR_OOM, "host allocation failed");
  g->d = d;
  if (d.radial_profile) g->profile.assign(d.radial_profile, d.radial_profile + d.n_profile);
  g->d.radial_profile = nullptr;
  // plasma species: the descriptors and their profiles are copied; the kernels' table gets the
  // device profiles below
  g->multi = d.n_species > 0;
  g->xshift = xshift;
  g->species.assign(d.species, d.species + d.n_species);
  g->sp_prof.resize(d.n_species);
  for (int k = 0; k < d.n_species; ++k) {
    if (d.species[k].radial_profile)
      g->sp_prof[k].assign(d.species[k].radial_profile, d.species[k].radial_profile + d.species[k].n_profile);
    g->species[k].radial_profile = nullptr;
  }
  g->d.species = nullptr;
  {
    SpeciesTab& t = g->sp;
    t = SpeciesTab{};
    const int ns = std::max(1, d.n_species);
    t.n = ns;
    int64_t off = 0;
    for (int k = 0; k < ns; ++k) {
      const bool def = d.n_species == 0;
      const double q = def ? -1.0 : d.species[k].charge, m = def ? 1.0 : d.species[k].mass;
      const int px = def ? d.ppc_x : d.species[k].ppc_x, py = def ? d.ppc_y : d.species[k].ppc_y;
      t.off[k] = off;
      off += (int64_t)d.nx * d.ny * px * py;
      t.q[k] = q;
      t.qm[k] = q / m;
      t.fq[k] = (float)q;
      t.fqm[k] = (float)(q / m);
      t.ppx[k] = px;
      t.ppy[k] = py;
      t.pow2[k] = (px & (px - 1)) == 0 && (py & (py - 1)) == 0;
      t.inv_px[k] = 1.0 / px;
      t.inv_py[k] = 1.0 / py;
      t.finv_px[k] = (float)t.inv_px[k];
      t.finv_py[k] = (float)t.inv_py[k];
      t.neutral[k] = def ? 1 : d.species[k].neutralize;
      t.n0[k] = def ? d.n0_scale : d.species[k].n0_scale;
      t.npf[k] = def ? 0 : (int)g->sp_prof[k].size();
      t.rmax[k] = def ? 0.0 : d.species[k].profile_rmax;
    }
    for (int k = ns; k <= kMaxSpecies; ++k) t.off[k] = off;
  }
  g->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  g->dev = dev;
  g->fp64 = d.precision == HQ_PREC_FP64;
  g->tf32 = d.precision == HQ_PREC_FP32_TF32X3;
  g->f4_slice = -1;
  g->explicit_b = d.bperp_solver == HQ_BPERP_EXPLICIT;
  g->nx = d.nx; g->ny = d.ny; g->nz = d.nzeta;
  g->nnode = (int64_t)d.nx * d.ny;
  g->np = np;
  g->tsize = g->fp64 ? sizeof(double) : sizeof(float);
  Geom& gm = g->geom;
  gm.nx = d.nx; gm.ny = d.ny;
  gm.xmin = d.xmin; gm.ymin = d.ymin; gm.xmax = d.xmax; gm.ymax = d.ymax;
  gm.dx = (d.xmax - d.xmin) / d.nx;
  gm.dy = (d.ymax - d.ymin) / d.ny;
  gm.inv_dx = 1.0 / gm.dx; gm.inv_dy = 1.0 / gm.dy;
  gm.dzeta = (d.zeta_max - d.zeta_min) / d.nzeta;
  gm.inv_area = 1.0 / (gm.dx * gm.dy);
  gm.inv2dx = 0.5 / gm.dx;
  gm.inv2dy = 0.5 / gm.dy;
  gm.inv2dz = 0.5 / gm.dzeta;
  gm.f_dz = (float)gm.dzeta;
  gm.f_dz_inv_dx = (float)(gm.dzeta * gm.inv_dx);
  gm.f_dz_inv_dy = (float)(gm.dzeta * gm.inv_dy);
  gm.f_inv_area = (float)gm.inv_area;
  gm.f_guard = (float)d.psi_guard;
  gm.f_inv_dx = (float)gm.inv_dx;
  gm.f_inv_dy = (float)gm.inv_dy;
  gm.f_inv2dx = (float)gm.inv2dx;
  gm.f_inv2dy = (float)gm.inv2dy;
  gm.f_inv2dz = (float)gm.inv2dz;
  g->last_adv = g->last_beam = g->last_solved = -1;

  auto bail = [&](hq_status st) {
    std::string msg = g->err;
    free_all(g);
    delete g;
    return fail(nullptr, st, msg);
  };
#define HQ_ALLOC(ptr, bytes)                                                                                   \
  do {                                                                                                         \
    cudaError_t e_ = dalloc(&(ptr), (bytes));                                                                  \
    if (e_ != cudaSuccess) {                                                                                   \
      g->err = std::string("cudaMalloc(" #ptr "): ") + cudaGetErrorString(e_);                                 \
      return bail(e_ == cudaErrorMemoryAllocation ? HQ_ERR_OOM : HQ_ERR_CUDA);                                 \
    }                                                                                                          \
  } while (0)

  const size_t ts = g->tsize, nn = (size_t)g->nnode;
  // plasma (x, y, psi and alive are shared between the two typed views)
  HQ_ALLOC(g->p64.x, 8 * np);
  HQ_ALLOC(g->p64.y, 8 * np);
  HQ_ALLOC(g->p64.psi, 8 * np);
  HQ_ALLOC(g->p64.alive, np);
  g->p64.n = g->p32.n = np;
  g->p32.x = g->p64.x; g->p32.y = g->p64.y; g->p32.psi = g->p64.psi; g->p32.alive = g->p64.alive;
  if (g->fp64) {
    HQ_ALLOC(g->p64.ux, 8 * np); HQ_ALLOC(g->p64.uy, 8 * np); HQ_ALLOC(g->p64.w, 8 * np);
    HQ_ALLOC(g->p64.hist, 8 * np * kRing * 5);
  } else {
    HQ_ALLOC(g->p32.ux, 4 * np); HQ_ALLOC(g->p32.uy, 4 * np); HQ_ALLOC(g->p32.w, 4 * np);
    HQ_ALLOC(g->p32.hist, 4 * np * kRing * 5);
    HQ_ALLOC(g->p32.cell, 4 * np); HQ_ALLOC(g->p32.fx, 4 * np); HQ_ALLOC(g->p32.fy, 4 * np); HQ_ALLOC(g->p32.opp, 4 * np);
    HQ_ALLOC(g->p32.hsum, 4 * np * 5);
    HQ_ALLOC(g->p32.f4, 16 * np);
  }
  if (d.resort_every > 0) {
    HQ_ALLOC(g->porigin, 4 * np);
    g->p64.origin = g->p32.origin = g->porigin;
    HQ_ALLOC(g->sort_key, 4 * np);
    HQ_ALLOC(g->sort_perm, 4 * np);
    HQ_ALLOC(g->sort_count, 4 * (nn + 1));
    HQ_ALLOC(g->sort_offset, 4 * (nn + 1));
    HQ_ALLOC(g->sort_tsum, 4 * (size_t)resort_tiles(g));
    HQ_ALLOC(g->sort_scratch, (size_t)resort_scratch_bytes(g));
  }
  // fields
  g->det = d.deterministic;
  if (g->det) {
    // one arena for the deposit records (and the witness accumulator), one for their
    // fixed-point mirrors at twice the stride: mirror(e) = 2 e + geom.det
    // (with the explicit solver also its source records xs4, xs1 and the beam J_perp pair bjp)
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const bool ex = g->explicit_b;
    const size_t sz[11] = {up(32 * nn), up(32 * nn), up(8 * nn), up(8 * nn), up(8 * nn), up(16 * nn), up(16 * nn), 256,
                           ex ? up(32 * nn) : 0, ex ? up(8 * nn) : 0, ex ? up(32 * nn) : 0};
    size_t tot = 0;
    for (size_t b : sz) tot += b;
    HQ_ALLOC(g->det_arena, tot);
    HQ_ALLOC(g->det_mirror, 2 * tot);
    cudaMemset(g->det_arena, 0, tot);
    cudaMemset(g->det_mirror, 0, 2 * tot);
    char* a = static_cast<char*>(g->det_arena);
    void* wsum = nullptr;
    void** dst[11] = {&g->dep[0], &g->dep[1], &g->chi[0], &g->chi[1], &g->rho_ion, &g->tj, &g->bjn, &wsum,
                      &g->xs4, &g->xs1, &g->bjp};
    for (int k = 0; k < 11; ++k) {
      if (sz[k]) *dst[k] = a;
      a += sz[k];
    }
    g->det_wsum = reinterpret_cast<double*>(wsum);
    g->geom.det = (int64_t)reinterpret_cast<uintptr_t>(g->det_mirror) - 2 * (int64_t)reinterpret_cast<uintptr_t>(g->det_arena);
  } else {
    for (int i = 0; i < 2; ++i) { HQ_ALLOC(g->dep[i], 4 * ts * nn); HQ_ALLOC(g->chi[i], ts * nn); }
    HQ_ALLOC(g->rho_ion, ts * nn);
    HQ_ALLOC(g->tj, 2 * ts * nn);
    if (!g->fp64) HQ_ALLOC(g->bsrc0, 8 * nn);
    HQ_ALLOC(g->bjn, 2 * ts * nn);
  }
  if (!g->fp64)
    for (int i = 0; i < 2; ++i) {
      HQ_ALLOC(g->psrc[i], 4 * nn);
      cudaMemset(g->psrc[i], 0, 4 * nn);
    }
  HQ_ALLOC(g->gf, kGF * ts * nn);
  HQ_ALLOC(g->bm, 2 * ts * nn);
  if (g->explicit_b) {
    if (!g->det) {
      HQ_ALLOC(g->bjp, 4 * ts * nn);
      HQ_ALLOC(g->xs4, 4 * ts * nn);
      HQ_ALLOC(g->xs1, ts * nn);
    } else {
      // deterministic mode: per-block partial dot products of the PCG
      const int64_t nb = std::max<int64_t>((nn + 255) / 256, (int64_t)((g->nx + 127) / 128) * g->ny);
      HQ_ALLOC(g->pcg_part, 16 * nb);
    }
    HQ_ALLOC(g->pcg_r, 2 * ts * nn);
    HQ_ALLOC(g->pcg_p, 2 * ts * nn);
    HQ_ALLOC(g->pcg_s, sizeof(double) * 4 * kMaxPcg * 2);
    for (void* p : {g->pcg_r, g->pcg_p}) cudaMemset(p, 0, 2 * ts * nn);
    cudaMemset(g->bjp, 0, 4 * ts * nn);
    cudaMemset(g->xs4, 0, 4 * ts * nn);
    cudaMemset(g->xs1, 0, ts * nn);
  }
  HQ_ALLOC(g->psi, ts * nn);
  HQ_ALLOC(g->bprev1, 2 * ts * nn);
  HQ_ALLOC(g->solved, kMaxRhs * ts * nn);
  HQ_ALLOC(g->d_status, sizeof(int));
  if (d.pc_residuals) {
    HQ_ALLOC(g->d_pcres, sizeof(double) * 2 * kResLanes * g->nz);
    cudaMemset(g->d_pcres, 0, sizeof(double) * 2 * kResLanes * g->nz);
  }
  if (g->det) g->geom.dstatus = g->d_status;   // fixed-point range overflows are reported here
  HQ_ALLOC(g->d_removed, sizeof(unsigned long long));
  for (int b = 0; b < kMaxBeams; ++b) {
    HQ_ALLOC(g->bins[b].count, sizeof(int32_t) * (g->nz + 1));
    HQ_ALLOC(g->bins[b].offset, sizeof(int32_t) * (g->nz + 1));
    HQ_ALLOC(g->bins[b].cursor, sizeof(int32_t) * (g->nz + 1));
  }
  for (int k = 0; k < d.n_species; ++k) {
    if (g->sp_prof[k].empty()) continue;
    HQ_ALLOC(g->d_sp_prof[k], 8 * g->sp_prof[k].size());
    if (cudaMemcpy(g->d_sp_prof[k], g->sp_prof[k].data(), 8 * g->sp_prof[k].size(), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      g->err = "species profile upload failed";
      return bail(HQ_ERR_CUDA);
    }
    g->sp.prof[k] = g->d_sp_prof[k];
  }
  if (!g->profile.empty()) {
    HQ_ALLOC(g->d_profile, 8 * g->profile.size());
    if (cudaMemcpy(g->d_profile, g->profile.data(), 8 * g->profile.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      g->err = "profile upload failed";
      return bail(HQ_ERR_CUDA);
    }
  }
  // zero everything the kernels accumulate into or read before writing
  for (void* p : {g->dep[0], g->dep[1]}) cudaMemset(p, 0, 4 * ts * nn);
  for (void* p : {g->chi[0], g->chi[1], g->rho_ion, g->psi}) cudaMemset(p, 0, ts * nn);
  for (void* p : {g->tj, g->bjn, g->bprev1, g->bm}) cudaMemset(p, 0, 2 * ts * nn);
  cudaMemset(g->gf, 0, kGF * ts * nn);
  cudaMemset(g->solved, 0, kMaxRhs * ts * nn);
  cudaMemset(g->d_status, 0, sizeof(int));
  cudaMemset(g->d_removed, 0, sizeof(unsigned long long));

  // DST tables
  if (g->fp64) {
    HQ_ALLOC(g->f64_a, 8 * kMaxRhs * nn);
    HQ_ALLOC(g->f64_b, 8 * kMaxRhs * nn);
    cudaMemset(g->f64_a, 0, 8 * kMaxRhs * nn);
    std::vector<double> sc = scale_table(g, g->ny, g->nx);
    HQ_ALLOC(g->f64_scale, 8 * nn);
    cudaMemcpy(g->f64_scale, sc.data(), 8 * nn, cudaMemcpyHostToDevice);
    if (g->explicit_b) {
      std::vector<double> sh = scale_table(g, g->ny, g->nx, g->xshift);
      HQ_ALLOC(g->scale_h, 8 * nn);
      cudaMemcpy(g->scale_h, sh.data(), 8 * nn, cudaMemcpyHostToDevice);
    }
    auto tables = [&](int n, double** tw, double** sn) -> hq_status {
      if (is_pow2(n)) {
        std::vector<double> t(2 * (size_t)n);
        for (int k = 0; k < n; ++k) {
          t[2 * k] = std::cos(M_PI * k / n);
          t[2 * k + 1] = -std::sin(M_PI * k / n);
        }
        if (dalloc(tw, 8 * t.size()) != cudaSuccess) return HQ_ERR_OOM;
        cudaMemcpy(*tw, t.data(), 8 * t.size(), cudaMemcpyHostToDevice);
      } else {
        std::vector<double> t((size_t)n * n);
        for (int j = 0; j < n; ++j)
          for (int k = 0; k < n; ++k) t[(size_t)j * n + k] = sin_jk(j, k, n);
        if (dalloc(sn, 8 * t.size()) != cudaSuccess) return HQ_ERR_OOM;
        cudaMemcpy(*sn, t.data(), 8 * t.size(), cudaMemcpyHostToDevice);
      }
      return HQ_OK;
    };
    if (tables(g->nx, &g->tw_x, &g->sin_x) != HQ_OK || tables(g->ny, &g->tw_y, &g->sin_y) != HQ_OK) {
      g->err = "DST table allocation failed";
      return bail(HQ_ERR_OOM);
    }
  } else {
    g->nxp = (int)round_up(g->nx, 128);
    g->nyp = (int)round_up(g->ny, 128);
    // folded DST-I (half the contraction) when both extents are multiples of 128
    const char* nf = std::getenv("HQ_NO_FOLD");
    g->fold = (g->nx % 128 == 0 && g->ny % 128 == 0 && !(nf && nf[0] == '1')) ? 1 : 0;
    const char* nsc = std::getenv("HQ_NO_SRCCACHE");
    g->no_srccache = nsc && nsc[0] == '1';
    const char* nf4 = std::getenv("HQ_NO_F4CACHE");
    g->no_f4 = nf4 && nf4[0] == '1';
    const char* ss = std::getenv("HQ_SEPARATE_SRC");
    g->sep_src = (ss && ss[0] == '1') ? 1 : 0;
    const char* fb = std::getenv("HQ_FAULT_BARRIER");
    g->fault_barrier = (fb && fb[0] == '1') ? 1 : 0;
    HQ_ALLOC(g->d_gbar, sizeof(unsigned long long));
    cudaMemset(g->d_gbar, 0, sizeof(unsigned long long));
    const size_t opn = (size_t)kMaxRhs * g->nxp * g->nyp;
    const size_t esz = g->tf32 ? 4 : 2;   // bytes per split operand element
    for (int i = 0; i < 2; ++i) {
      HQ_ALLOC(g->op_hi[i], esz * opn);
      HQ_ALLOC(g->op_lo[i], esz * opn);
      cudaMemset(g->op_hi[i], 0, esz * opn);
      cudaMemset(g->op_lo[i], 0, esz * opn);
    }
    // S (zero-padded [np][np]) or, folded, the fold matrix [n][n/2]; split into hi + lo (bf16,
    // or TF32 in FP32 words)
    auto smat = [&](int n, int np_, void** hi, void** lo) -> hq_status {
      const int cols = g->fold ? n / 2 : np_;
      const std::vector<double> fm = g->fold ? fold_matrix(n) : std::vector<double>();
      const size_t cnt = (size_t)np_ * cols;
      std::vector<__nv_bfloat16> h(g->tf32 ? 0 : cnt), l(g->tf32 ? 0 : cnt);
      std::vector<float> hf(g->tf32 ? cnt : 0), lf(g->tf32 ? cnt : 0);
      for (int k = 0; k < np_; ++k)
        for (int j = 0; j < cols; ++j) {
          const float v = g->fold ? (float)fm[(size_t)k * cols + j]
                                  : ((j < n && k < n) ? (float)sin_jk(j, k, n) : 0.0f);
          const size_t o = (size_t)k * cols + j;
          if (g->tf32) {
            hf[o] = round_tf32_host(v);
            lf[o] = v - hf[o];
          } else {
            const __nv_bfloat16 vh = __float2bfloat16_rn(v);
            h[o] = vh;
            l[o] = __float2bfloat16_rn(v - __bfloat162float(vh));
          }
        }
      if (dalloc(hi, esz * cnt) != cudaSuccess || dalloc(lo, esz * cnt) != cudaSuccess) return HQ_ERR_OOM;
      cudaMemcpy(*hi, g->tf32 ? (const void*)hf.data() : (const void*)h.data(), esz * cnt, cudaMemcpyHostToDevice);
      cudaMemcpy(*lo, g->tf32 ? (const void*)lf.data() : (const void*)l.data(), esz * cnt, cudaMemcpyHostToDevice);
      return HQ_OK;
    };
    if (smat(g->nx, g->nxp, &g->sx_hi, &g->sx_lo) != HQ_OK || smat(g->ny, g->nyp, &g->sy_hi, &g->sy_lo) != HQ_OK) {
      g->err = "DST matrix allocation failed";
      return bail(HQ_ERR_OOM);
    }
    std::vector<double> sc = scale_table(g, g->nyp, g->nxp);
    std::vector<float> scf(sc.size());
    for (int sy = 0; sy < g->nyp; ++sy)
      for (int sx = 0; sx < g->nxp; ++sx) {
        const int ky = g->fold ? fold_node(sy, g->ny) : sy, kx = g->fold ? fold_node(sx, g->nx) : sx;
        scf[(size_t)sy * g->nxp + sx] = (float)sc[(size_t)ky * g->nxp + kx];
      }
    HQ_ALLOC(g->f32_scale, 4 * scf.size());
    cudaMemcpy(g->f32_scale, scf.data(), 4 * scf.size(), cudaMemcpyHostToDevice);
    if (g->explicit_b) {
      std::vector<double> sh = scale_table(g, g->nyp, g->nxp, g->xshift);
      for (int sy = 0; sy < g->nyp; ++sy)
        for (int sx = 0; sx < g->nxp; ++sx) {
          const int ky = g->fold ? fold_node(sy, g->ny) : sy, kx = g->fold ? fold_node(sx, g->nx) : sx;
          scf[(size_t)sy * g->nxp + sx] = (float)sh[(size_t)ky * g->nxp + kx];
        }
      HQ_ALLOC(g->scale_h, 4 * scf.size());
      cudaMemcpy(g->scale_h, scf.data(), 4 * scf.size(), cudaMemcpyHostToDevice);
    }
    std::string err;
    if (dst_tc_init(g, err)) {
      g->err = err;
      return bail(HQ_ERR_CUDA);
    }
  }
  // ion background from the initial plasma
  if (g->fp64) {
    launch_plasma_init<double>(g, g->stream);
    launch_deposit_initial<double>(g, nullptr, nullptr, 1, g->stream);
    if (g->det) launch_fx_decode(g, g->rho_ion, nn, nullptr, g->stream);
  } else {
    launch_plasma_init<float>(g, g->stream);
    launch_deposit_initial<float>(g, nullptr, nullptr, 1, g->stream);
    bool bare = false;
    for (int k = 0; k < d.n_species; ++k) bare |= !d.species[k].neutralize;
    if (bare) {
      // the initial charge of the species without a background, for the ion-subtracted psi
      // source: summed in FP64 on the device, rounded once to FP32
      double* c0d = nullptr;
      HQ_ALLOC(c0d, 8 * nn);
      cudaMemsetAsync(c0d, 0, 8 * nn, g->stream);
      launch_species_c0(g, c0d, g->stream);
      std::vector<double> h(nn);
      std::vector<float> f(nn);
      const cudaError_t ec = cudaMemcpyAsync(h.data(), c0d, 8 * nn, cudaMemcpyDeviceToHost, g->stream);
      cudaStreamSynchronize(g->stream);
      cudaFree(c0d);
      if (ec != cudaSuccess) {
        g->err = "species charge download failed";
        return bail(HQ_ERR_CUDA);
      }
      for (size_t i = 0; i < nn; ++i) f[i] = (float)h[i];
      HQ_ALLOC(g->c0, 4 * nn);
      cudaMemcpy(g->c0, f.data(), 4 * nn, cudaMemcpyHostToDevice);
    }
  }
  cudaError_t e = cudaStreamSynchronize(g->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    g->err = std::string("grid initialization: ") + cudaGetErrorString(e);
    return bail(HQ_ERR_CUDA);
  }
#undef HQ_ALLOC
  *out = g;
  return HQ_OK;
}

hq_status hq_grid_destroy(hq_grid_t g) {
  if (!g) return HQ_OK;
  cudaStreamSynchronize(g->stream);
  free_all(g);
  delete g;
  return HQ_OK;
}

hq_status hq_advance_slice(hq_grid_t g, int32_t slice) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (slice < 0 || slice >= g->nz) return fail(g, HQ_ERR_ARG, "slice out of range");
  if (slice > 0 && !(g->last_solved == slice - 1 && g->last_adv == slice - 1))
    return fail(g, HQ_ERR_STATE, "hq_advance_slice(i) needs hq_solve_fields(i-1) first");
  if (g->fp64) advance_impl<double>(g, slice);
  else advance_impl<float>(g, slice);
  g->last_adv = slice;
  g->last_beam = -1;
  if (slice == 0) g->last_solved = -1;
  return check_launch(g);
}

hq_status hq_beam_deposit(hq_grid_t g, const hq_beam_view* beams, int32_t nbeams, int32_t slice) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (slice < 0 || slice >= g->nz) return fail(g, HQ_ERR_ARG, "slice out of range");
  if (g->last_adv != slice || g->last_beam == slice || g->last_solved == slice)
    return fail(g, HQ_ERR_STATE, "hq_beam_deposit(i) needs hq_advance_slice(i) first, once");
  hq_status st = check_views(g, beams, nbeams);
  if (st != HQ_OK) return st;
  st = g->fp64 ? beam_deposit_impl<double>(g, beams, nbeams, slice) : beam_deposit_impl<float>(g, beams, nbeams, slice);
  if (st != HQ_OK) return st;
  g->last_beam = slice;
  return check_launch(g);
}

hq_status hq_solve_fields(hq_grid_t g, int32_t slice) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (slice < 0 || slice >= g->nz) return fail(g, HQ_ERR_ARG, "slice out of range");
  if (g->last_beam != slice || g->last_solved == slice)
    return fail(g, HQ_ERR_STATE, "hq_solve_fields(i) needs hq_beam_deposit(i) first");
  if (g->fp64) solve_fields_impl<double>(g, slice);
  else solve_fields_impl<float>(g, slice);
  g->last_solved = slice;
  return check_launch(g);
}

hq_status hq_store_fields(hq_grid_t g, const hq_field_out* out, int64_t slot) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!out || slot < 0) return fail(g, HQ_ERR_ARG, "out is NULL or slot < 0");
  if (g->last_solved < 0) return fail(g, HQ_ERR_STATE, "no slice solved yet");
  const int i = g->last_solved;
  Prof p(g, HQ_K_FIELD, 1);
  if (g->fp64) launch_store<double>(g, out, slot, g->dep[i & 1], g->chi[i & 1], g->stream);
  else launch_store<float>(g, out, slot, g->dep[i & 1], g->chi[i & 1], g->stream);
  return check_launch(g);
}

hq_status hq_push_beams(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, int32_t slice, double dt) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (g->last_solved != slice) return fail(g, HQ_ERR_STATE, "hq_push_beams(i) needs hq_solve_fields(i)");
  hq_status st = check_views(g, beams, nbeams);
  if (st != HQ_OK) return st;
  if (!std::isfinite(dt)) return fail(g, HQ_ERR_ARG, "dt must be finite");
  for (int b = 0; b < nbeams; ++b) {
    const int k = bound_index(g, &beams[b]);
    if (k < 0) return fail(g, HQ_ERR_STATE, "beam was not given to hq_beam_deposit in this sweep");
    if (beams[b].n == 0) continue;
    Prof p(g, HQ_K_BEAM, 1);
    if (g->fp64) launch_beam_push<double>(g, k, beams[b], slice, dt, g->stream);
    else launch_beam_push<float>(g, k, beams[b], slice, dt, g->stream);
  }
  return check_launch(g);
}

hq_status hq_witness_accumulate(hq_grid_t g, const hq_beam_view* beam, int32_t slice, double* sums) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!beam || !sums) return fail(g, HQ_ERR_ARG, "beam and sums must not be NULL");
  if (g->last_solved != slice) return fail(g, HQ_ERR_STATE, "hq_witness_accumulate(i) needs hq_solve_fields(i)");
  const int k = bound_index(g, beam);
  if (k < 0) return fail(g, HQ_ERR_STATE, "beam was not given to hq_beam_deposit in this sweep");
  if (beam->n == 0) return HQ_OK;
  Prof p(g, HQ_K_BEAM, 1);
  if (g->fp64) {
    launch_witness<double>(g, k, *beam, slice, g->det ? g->det_wsum : sums, g->stream);
    if (g->det) launch_fx_decode(g, g->det_wsum, 3, sums, g->stream);
  }
  else launch_witness<float>(g, k, *beam, slice, sums, g->stream);
  return check_launch(g);
}

hq_status hq_beam_slices(hq_grid_t g, const hq_beam_view* beam, int32_t* slices) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!beam || (beam->n > 0 && !slices)) return fail(g, HQ_ERR_ARG, "beam and slices must not be NULL");
  hq_status st = check_views(g, beam, 1);
  if (st != HQ_OK) return st;
  if (beam->n == 0) return HQ_OK;
  Prof p(g, HQ_K_BEAM, 1);
  launch_beam_slices(g, *beam, slices, g->stream);
  return check_launch(g);
}

hq_status hq_pc_residuals(hq_grid_t g, double* out, int32_t n) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (n < 0 || (n > 0 && !out)) return fail(g, HQ_ERR_ARG, "out must hold n >= 0 doubles");
  if (!g->d_pcres) return fail(g, HQ_ERR_STATE, "the grid was created without pc_residuals = 1");
  HQ_CUDA(g, cudaStreamSynchronize(g->stream));
  std::vector<double> sums(2 * kResLanes * (size_t)g->nz);
  HQ_CUDA(g, cudaMemcpy(sums.data(), g->d_pcres, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    if (i >= g->nz) {
      out[i] = 0.0;
      continue;
    }
    double num = 0.0, den = 0.0;
    for (int l = 0; l < kResLanes; ++l) {
      num += sums[(2 * kResLanes * (size_t)i) + 2 * l];
      den += sums[(2 * kResLanes * (size_t)i) + 2 * l + 1];
    }
    out[i] = den > 0.0 ? std::sqrt(num / den) : 0.0;
  }
  return HQ_OK;
}

hq_status hq_beam_moments(hq_grid_t g, const hq_beam_view* beam, double* moments) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!beam || !moments) return fail(g, HQ_ERR_ARG, "beam and moments must not be NULL");
  hq_status st = check_views(g, beam, 1);
  if (st != HQ_OK) return st;
  if (beam->n == 0) return HQ_OK;
  Prof p(g, HQ_K_BEAM, 1);
  launch_beam_moments(*beam, moments, g->stream);
  return check_launch(g);
}

hq_status hq_sweep_step(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, double dt, const hq_field_out* out,
                        int32_t witness_beam, double* witness_sums) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  hq_status st = check_views(g, beams, nbeams);
  if (st != HQ_OK) return st;
  if (witness_beam >= nbeams || (witness_beam >= 0 && !witness_sums))
    return fail(g, HQ_ERR_ARG, "witness_beam must index a beam and witness_sums must be given");
  if (!std::isfinite(dt)) return fail(g, HQ_ERR_ARG, "dt must be finite");
  // The ~20 launches per slice are replayed from a CUDA graph when possible (off while
  // profiling, with HQ_NO_GRAPH=1, or after a capture was refused).
  const char* ng = std::getenv("HQ_NO_GRAPH");
  if (g->graph_off || g->prof_on || (ng && ng[0] == '1'))
    return sweep_body(g, beams, nbeams, dt, out, witness_beam, witness_sums);
  SweepGraph* sg = reinterpret_cast<SweepGraph*>(g->sweep_graph);
  if (!sg || !sg->exec || !sg->matches(beams, nbeams, dt, out, witness_beam, witness_sums)) {
    if ((st = reserve_bins(g, beams, nbeams)) != HQ_OK) return st;
    graph_free(g);
    if (!g->cap_stream && cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      g->cap_stream = nullptr;
      g->graph_off = 1;
      return sweep_body(g, beams, nbeams, dt, out, witness_beam, witness_sums);
    }
    // capture on the private stream (the caller's may be the legacy default stream, which
    // cannot be captured); nothing executes during the capture
    cudaStream_t user = g->stream;
    g->stream = g->cap_stream;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      g->stream = user;
      g->graph_off = 1;
      return sweep_body(g, beams, nbeams, dt, out, witness_beam, witness_sums);
    }
    st = sweep_body(g, beams, nbeams, dt, out, witness_beam, witness_sums);
    const cudaError_t ec = cudaStreamEndCapture(g->stream, &graph);
    g->stream = user;
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = (st == HQ_OK && ec == cudaSuccess && graph) ? cudaGraphInstantiate(&exec, graph, 0)
                                                                       : cudaErrorUnknown;
    if (graph) cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      // not capturable here: run the sweep on the stream (the capture executed nothing)
      cudaGetLastError();
      g->err.clear();
      g->graph_off = 1;
      return sweep_body(g, beams, nbeams, dt, out, witness_beam, witness_sums);
    }
    sg = new (std::nothrow) SweepGraph();
    if (!sg) {
      cudaGraphExecDestroy(exec);
      return fail(g, HQ_ERR_OOM, "host allocation failed");
    }
    sg->exec = exec;
    sg->beams.assign(beams, beams + nbeams);
    sg->dt = dt;
    sg->has_out = out != nullptr;
    if (out) sg->out = *out;
    sg->witness = witness_beam;
    sg->sums = witness_sums;
    g->sweep_graph = sg;
  }
  HQ_CUDA(g, cudaGraphLaunch(sg->exec, g->stream));
  // host bookkeeping of a completed sweep (the slice-order checks of the fine-grained calls)
  for (int b = 0; b < nbeams; ++b) g->bound[b] = beams[b];
  g->nbound = nbeams;
  g->last_adv = g->nz;
  g->last_beam = g->last_solved = g->nz - 1;
  return check_launch(g);
}


hq_status hq_sweep_slices(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, const hq_beam_view* next,
                          int32_t nnext, int32_t slice_begin, int32_t slice_end, double dt,
                          const hq_field_out* out, int32_t witness_beam, double* witness_sums) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (nbeams < 0 || nnext < 0 || nbeams + nnext > kMaxBeams || (nnext > 0 && !next))
    return fail(g, HQ_ERR_ARG, "nbeams + nnext must be 0..4 (next given when nnext > 0)");
  hq_status st = check_views(g, beams, nbeams);
  if (st != HQ_OK) return st;
  if ((st = check_views(g, next, nnext)) != HQ_OK) return st;
  if (slice_begin < 0 || slice_end > g->nz || slice_begin >= slice_end)
    return fail(g, HQ_ERR_ARG, "need 0 <= slice_begin < slice_end <= nzeta");
  if (slice_begin > 0 && g->last_solved != slice_begin - 1)
    return fail(g, HQ_ERR_STATE, "slice_begin must follow the previous call's slice_end");
  if (witness_beam >= nbeams || (witness_beam >= 0 && !witness_sums))
    return fail(g, HQ_ERR_ARG, "witness_beam must index a beam and witness_sums must be given");
  if (!std::isfinite(dt)) return fail(g, HQ_ERR_ARG, "dt must be finite");
  hq_beam_view views[kMaxBeams];
  for (int b = 0; b < nbeams; ++b) views[b] = beams[b];
  for (int b = 0; b < nnext; ++b) views[nbeams + b] = next[b];
  for (int i = slice_begin; i < slice_end; ++i) {
    if ((st = hq_advance_slice(g, i)) != HQ_OK) return st;
    const int nv = nbeams + (i == slice_end - 1 ? nnext : 0);
    if ((st = hq_beam_deposit(g, views, nv, i)) != HQ_OK) return st;
    if ((st = hq_solve_fields(g, i)) != HQ_OK) return st;
    if (out && (st = hq_store_fields(g, out, i)) != HQ_OK) return st;
    if (witness_beam >= 0 && (st = hq_witness_accumulate(g, &beams[witness_beam], i, witness_sums)) != HQ_OK)
      return st;
    if (dt != 0.0 && nbeams > 0 && (st = hq_push_beams(g, beams, nbeams, i, dt)) != HQ_OK) return st;
  }
  if (slice_end == g->nz) {
    // advance once past the tail so the plasma state matches a completed sweep
    if (g->fp64) final_pass<double>(g, g->nz - 1, g->nz & 1);
    else final_pass<float>(g, g->nz - 1, g->nz & 1);
    g->last_adv = g->nz;
  }
  return check_launch(g);
}

hq_status hq_sweep_forward_ckpt(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, int32_t witness_beam,
                                double* witness_sums, int32_t ckpt_every) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  hq_status st = check_views(g, beams, nbeams);
  if (st != HQ_OK) return st;
  if (witness_beam >= nbeams || (witness_beam >= 0 && !witness_sums))
    return fail(g, HQ_ERR_ARG, "witness_beam must index a beam and witness_sums must be given");
  if (ckpt_every < 1) return fail(g, HQ_ERR_ARG, "ckpt_every must be >= 1");
  if (g->explicit_b) return fail(g, HQ_ERR_UNSUPPORTED, "the adjoint supports the predictor-corrector B_perp solver only");
  if (g->d.resort_every > 0) return fail(g, HQ_ERR_UNSUPPORTED, "the adjoint needs the plasma in its initial order (resort_every = 0)");
  if (g->det) return fail(g, HQ_ERR_UNSUPPORTED, "deterministic accumulation is a forward-sweep mode");
  if (g->multi) return fail(g, HQ_ERR_UNSUPPORTED, "the adjoint takes the default electron plasma only");
  const int k = std::min<int>(ckpt_every, g->nz);
  if ((st = adj_alloc(g, k)) != HQ_OK) return st;
  AdjStore* a = adj_of(g);
  st = g->fp64 ? forward_ckpt_impl<double>(g, beams, nbeams, witness_beam, witness_sums)
               : forward_ckpt_impl<float>(g, beams, nbeams, witness_beam, witness_sums);
  if (st != HQ_OK) return st;
  a->fwd_done = 1;
  a->fwd_beams.assign(beams, beams + nbeams);
  a->fwd_witness = witness_beam;
  g->last_adv = g->nz - 1;
  g->last_beam = g->last_solved = g->nz - 1;
  return check_launch(g);
}

hq_status hq_sweep_adjoint(hq_grid_t g, hq_beam_view* beams, int32_t nbeams, int32_t witness_beam,
                           const double* dL_dsums, const hq_field_out* dL_dfields, double* const* dL_dbeam_w,
                           double* dL_dplasma_w, double* dL_dn0_scale, double* dL_dprofile) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  AdjStore* a = adj_of(g);
  if (!a || !a->fwd_done) return fail(g, HQ_ERR_STATE, "hq_sweep_adjoint needs hq_sweep_forward_ckpt first");
  if (nbeams != (int)a->fwd_beams.size() || witness_beam != a->fwd_witness)
    return fail(g, HQ_ERR_STATE, "beams/witness differ from the checkpointed forward sweep");
  for (int b = 0; b < nbeams; ++b)
    if (!same_view(beams[b], a->fwd_beams[b])) return fail(g, HQ_ERR_STATE, "beams differ from the forward sweep");
  if (witness_beam >= 0 && !dL_dsums) return fail(g, HQ_ERR_ARG, "dL_dsums (host double[3]) is needed");
  if (dL_dfields && dL_dfields->chi) return fail(g, HQ_ERR_ARG, "dL_dfields->chi is not supported (chi is output only)");
  const double zero[3] = {0.0, 0.0, 0.0};
  const double* sb = dL_dsums ? dL_dsums : zero;
  hq_status st = g->fp64 ? adjoint_impl<double>(g, beams, nbeams, witness_beam, sb, dL_dfields, dL_dbeam_w,
                                                dL_dplasma_w, dL_dn0_scale, dL_dprofile)
                         : adjoint_impl<float>(g, beams, nbeams, witness_beam, sb, dL_dfields, dL_dbeam_w,
                                               dL_dplasma_w, dL_dn0_scale, dL_dprofile);
  if (st != HQ_OK) return st;
  a->fwd_done = 0;
  g->last_adv = g->last_beam = g->last_solved = -1;
  return check_launch(g);
}

hq_status hq_poisson_solve(hq_grid_t g, const void* src, void* dst, int32_t nrhs) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!src || !dst || nrhs < 1 || nrhs > kMaxRhs) return fail(g, HQ_ERR_ARG, "src/dst NULL or nrhs not in 1..5");
  cudaStream_t s = g->stream;
  {
    Prof p(g, HQ_K_FIELD, 1);
    if (g->fp64) launch_src_copy<double>(g, src, nrhs, s);
    else launch_src_copy<float>(g, src, nrhs, s);
  }
  dst_solve(g, nrhs);
  HQ_CUDA(g, cudaMemcpyAsync(dst, g->solved, (size_t)nrhs * g->nnode * g->tsize, cudaMemcpyDeviceToDevice, s));
  return check_launch(g);
}

hq_status hq_plasma_state(hq_grid_t g, hq_plasma_view* out) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!out) return fail(g, HQ_ERR_ARG, "out is NULL");
  out->n = g->np;
  out->x = g->p64.x;
  out->y = g->p64.y;
  out->psi = g->p64.psi;
  out->alive = g->p64.alive;
  out->origin = g->porigin;
  if (g->fp64) { out->ux = g->p64.ux; out->uy = g->p64.uy; out->w = g->p64.w; }
  else { out->ux = g->p32.ux; out->uy = g->p32.uy; out->w = g->p32.w; }
  return HQ_OK;
}

hq_status hq_sync(hq_grid_t g, int64_t* removed) {
  if (!g) {
    if (removed) *removed = 0;
    return static_sync();
  }
  HQ_CUDA(g, cudaStreamSynchronize(g->stream));
  int status = 0;
  unsigned long long rm = 0;
  HQ_CUDA(g, cudaMemcpy(&status, g->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  HQ_CUDA(g, cudaMemcpy(&rm, g->d_removed, sizeof(rm), cudaMemcpyDeviceToHost));
  if (removed) *removed = (int64_t)rm;
  if (status) {
    HQ_CUDA(g, cudaMemset(g->d_status, 0, sizeof(int)));
    if (status & DEV_TIMEOUT) {
      if (g->d_gbar) HQ_CUDA(g, cudaMemset(g->d_gbar, 0, sizeof(unsigned long long)));  // an aborted solve left it
      return fail(g, HQ_ERR_TIMEOUT, "a bounded device wait ran out (tensor-core DST)");
    }
    if (status & DEV_NONFINITE)
      return fail(g, HQ_ERR_NUMERIC, "a non-finite value reached the field solve, or a deterministic-mode "
                                     "contribution left the fixed-point range");
  }
  return HQ_OK;
}

hq_status hq_profile_enable(hq_grid_t g, int32_t on) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  HQ_CUDA(g, cudaStreamSynchronize(g->stream));
  g->prof_on = on != 0;
  g->ev_used = 0;
  g->ev_class.clear();
  for (int k = 0; k < HQ_K_CLASSES; ++k) g->launches[k] = 0;
  return HQ_OK;
}

hq_status hq_profile_read(hq_grid_t g, hq_profile_t* out) {
  if (!g) return fail(nullptr, HQ_ERR_ARG, "grid is NULL");
  if (!out) return fail(g, HQ_ERR_ARG, "out is NULL");
  HQ_CUDA(g, cudaStreamSynchronize(g->stream));
  for (int k = 0; k < HQ_K_CLASSES; ++k) {
    out->ms[k] = 0.0;
    out->launches[k] = g->launches[k];
  }
  for (size_t i = 0; i < g->ev_class.size() && 2 * i + 1 < g->ev_used; ++i) {
    float ms = 0.0f;
    HQ_CUDA(g, cudaEventElapsedTime(&ms, g->ev_pool[2 * i], g->ev_pool[2 * i + 1]));
    out->ms[g->ev_class[i]] += ms;
  }
  return HQ_OK;
}

const char* hq_last_error(hq_grid_t g) { return g ? g->err.c_str() : g_global_err.c_str(); }

}  // extern "C"
