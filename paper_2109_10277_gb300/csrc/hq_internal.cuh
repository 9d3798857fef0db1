// Internal declarations shared by the CUDA translation units of libhq.
// Quasi-static PIC slice loop of arXiv:2109.10277 (Sec. 2, Sec. 3.2).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hq.h"

namespace hq {

// ---------------------------------------------------------------- device status bits
enum : int {
  DEV_TIMEOUT = 1,   // a bounded wait ran out
  DEV_NONFINITE = 2, // a non-finite value reached a field
};

constexpr int kMaxBeams = 4;
constexpr int kMaxRhs = 5;
constexpr int kRing = 4;  // AB5 history slots f_{i-1} .. f_{i-4}
constexpr int kMaxPcg = 64;   // explicit B_perp solver: at most this many PCG iterations

// Fifth-order Adams-Bashforth weights (Sec. 3.2 plasma push): beta_k for f_{i-k}.
__host__ __device__ constexpr double ab5(int k) {
  return k == 0 ? 1901.0 / 720.0 : k == 1 ? -2774.0 / 720.0 : k == 2 ? 2616.0 / 720.0
       : k == 3 ? -1274.0 / 720.0 : 251.0 / 720.0;
}

// Plain-value geometry passed to kernels.
struct Geom {
  int nx, ny;
  double xmin, ymin, dx, dy, inv_dx, inv_dy, dzeta;
  double xmax, ymax;
  double inv_area;  // 1 / (dx dy)
  double inv2dx, inv2dy, inv2dz;  // 1/(2 dx), 1/(2 dy), 1/(2 dzeta): central differences
  // FP32 copies for the FP32 kernels (no per-thread double-to-float conversion)
  float f_dz, f_dz_inv_dx, f_dz_inv_dy, f_inv_area, f_guard;
  float f_inv_dx, f_inv_dy, f_inv2dx, f_inv2dy, f_inv2dz;
  // deterministic FP64 accumulation (0: off): byte offset from twice a deposit record's
  // address to its fixed-point mirror (see fx_add), and the status word for overflows
  int64_t det;
  int* dstatus;
};

// A geometry constant in the kernel's arithmetic type: FP32 kernels take the host-rounded
// copy (on this GPU every FP64 conversion is an instruction of the slow FP64 pipe).
template <typename T> __device__ __forceinline__ T gsel(double d, float f) {
  if constexpr (sizeof(T) == 4) return f;
  else return d;
}

template <typename T> struct V4 { T a, b, c, d; };   // packed rho, jx, jy, jz

template <typename T> struct V2 { T a, b; };          // packed jx, jy or bx, by
// Gather fields packed per node: ExmBy, EypBx, Ez, Bz (one 16-byte record in FP32); the
// transverse magnetic field Bx, By of the predictor-corrector lives in a record of its own
// (V2 per node, hq_grid_s::bm), which the mixing updates in place.
constexpr int kGF = 4;

// Plasma slice, structure of arrays.  x, y, psi are FP64 accumulators in both
// modes; the rest is of the field type T.
template <typename T> struct Plasma {
  int64_t n;
  double *x, *y, *psi;
  T *ux, *uy, *w;
  uint8_t* alive;
  T* hist;           // [kRing][5][n]
  // FP32 mode: per-particle cell coordinates of the current slice, written by the
  // final pass so trial passes need no FP64 work (unused in FP64 mode).
  int32_t* cell;     // (iy << 16) | ix of floor(node coordinate)
  float* fx;         // fractional node coordinate in x, [0, 1)
  float* fy;
  float* opp;        // 1 + Psi, formed in FP64, rounded once
  // FP32 mode: the history part of the AB5 step of the current slice, sum_{k=1..4} beta_k
  // f_{i-k}, [5][n]: the same for all predictor-corrector trial passes of the slice, so they
  // read 5 values instead of the 20 of the ring (written by the final pass).
  float* hsum;
  // FP32 mode: ExmBy, EypBx, Ez, Bz gathered at the slice's first predictor-corrector iteration,
  // read by the later ones of the same slice (only Bx, By change between them)
  float4* f4;
  // With the re-sort (resort_every > 0): each particle's index in the initial placement (its
  // ion's position is recomputed from it); null otherwise (the array index is that index).
  int32_t* origin;
};

// Plasma species (hq_species_desc), as the particle kernels of a multi-species grid read them:
// species s holds particles [off[s], off[s + 1]) of the slice.
constexpr int kMaxSpecies = 4;
struct SpeciesTab {
  int n;
  int64_t off[kMaxSpecies + 1];
  double q[kMaxSpecies], qm[kMaxSpecies];     // charge (units of e), charge / mass (e / m_e)
  float fq[kMaxSpecies], fqm[kMaxSpecies];
  int ppx[kMaxSpecies], ppy[kMaxSpecies];
  int pow2[kMaxSpecies];                      // both particle counts per cell powers of two
  double inv_px[kMaxSpecies], inv_py[kMaxSpecies];
  float finv_px[kMaxSpecies], finv_py[kMaxSpecies];
  int neutral[kMaxSpecies];                   // immobile background of the opposite charge
  double n0[kMaxSpecies];
  const double* prof[kMaxSpecies];            // device radial profile or null
  int npf[kMaxSpecies];
  double rmax[kMaxSpecies];
};
__device__ __forceinline__ int species_of(const SpeciesTab& t, int64_t p) {
  int s = 0;
#pragma unroll
  for (int k = 1; k < kMaxSpecies; ++k) s += (k < t.n && p >= t.off[k]) ? 1 : 0;
  return s;
}

// Per-beam slice binning (counting sort by slice, Sec. 3.1).
struct BeamBins {
  int32_t* bin;      // per particle, -1 outside the box
  int32_t* count;    // nzeta + 1
  int32_t* offset;   // nzeta + 1 (exclusive scan)
  int32_t* cursor;   // nzeta
  int32_t* perm;     // particle indices grouped by slice
  int64_t cap;
};

struct TensorMaps;  // opaque, defined in the tensor-core DST unit

// Read-only view of a stored plasma slice (tape) for the adjoint kernels; w is the
// grid's (constant) weight array.
template <typename T> struct SnapView {
  int64_t n;
  const double *x, *y, *psi;
  const T *ux, *uy, *w;
  const uint8_t* alive;
  const T* hist;    // AB5 ring as stored: physical slot s holds f_k with k = s mod 4
  const float* hsum;   // FP32: the slice's AB5 history sum [5][n] (what the trial passes used); else null
  // FP32: the slice's cached cell index, fractional node coordinates and 1 + Psi (what the
  // trial passes and the final pass's gather used); else null
  const int32_t* cell;
  const float *fx, *fy, *opp;
};

// Per-particle adjoint state: x, y, ux, uy, Psi and the AB5 history in logical order
// (sh[j] is the adjoint of f_{i-1-j} at the current slice i), [4][5][n].
template <typename T> struct AdjView {
  T *sx, *sy, *sux, *suy, *spsi;
  T* sh;
  // [5][n]: sum of the predictor-corrector trial steps' AB5-combination adjoints of the slice
  // being reversed; their history adjoints (-dzeta beta_k times it) are folded into sh by the
  // next final-pass adjoint, so each trial adjoint updates 5 values instead of 20.
  T* sacc;
};

}  // namespace hq

// ---------------------------------------------------------------- grid object
struct hq_grid_s {
  hq_grid_desc d;
  std::vector<double> profile;
  cudaStream_t stream;
  int dev;
  int fp64;            // 1: FP64 everywhere; 0: FP32 + split tensor-core DST
  int tf32;            // FP32 mode: 1 TF32x3 operands, 0 bf16x3
  int nx, ny, nz;
  int64_t nnode, np;
  hq::Geom geom;
  size_t tsize;        // sizeof field type

  // plasma
  void* plasma;        // hq::Plasma<T>* host struct (typed by fp64)
  hq::Plasma<double> p64;
  hq::Plasma<float> p32;
  // plasma re-sort by cell every d.resort_every slices (null when off): initial index per
  // particle (shared by p64 and p32), sort keys, counts/cursor and offsets per cell (+1 for
  // non-finite positions), scan tile totals, the permutation, and the scratch copy
  int32_t* porigin;
  int32_t *sort_key, *sort_count, *sort_offset, *sort_tsum, *sort_perm;
  void* sort_scratch;
  // deterministic FP64 mode (d.deterministic): the deposit records dep[2], chi[2], tj, bjn,
  // rho_ion and the witness accumulator det_wsum live in one arena; the fixed-point mirrors
  // in a second one of twice its size (geom.det is their offset)
  int det;
  void *det_arena, *det_mirror;
  double* det_wsum;
  // plasma species (d.n_species > 0: multi = 1 and the particle kernels read sp); FP32: c0 is
  // the initial charge of the species without a neutralizing background, sum q w S(x0) / A,
  // added to the ion-subtracted psi source (null when every species is neutralized)
  // predictor-corrector residual of each slice of the last sweep (Sec. 3.2): sum (B_m - B_m-1)^2
  // and sum B_m^2 of the last iteration's mixing, [nzeta][kResLanes][2] (lanes spread the
  // atomics); pc_rsum points at the slice's lanes while its last iteration mixes (null otherwise)
  double* d_pcres;
  double* pc_rsum;
  int multi;
  double xshift;       // explicit B_perp solver: preconditioner shift c (the unperturbed chi)
  hq::SpeciesTab sp;
  std::vector<hq_species_desc> species;
  std::vector<std::vector<double>> sp_prof;
  double* d_sp_prof[hq::kMaxSpecies];
  float* c0;

  // fields (void* typed by fp64)
  void* dep[2];        // V4 per node: rho, jx, jy, jz   (ping-pong by slice parity)
  void* chi[2];
  void* rho_ion;
  void* tj;            // V2: trial plasma J_perp of slice i+1
  float* bsrc0;        // FP32: V2 per node, the predictor-corrector-invariant part of the B_perp sources
  int pc_iter;         // predictor-corrector iteration being issued (host side)
  int no_srccache;     // HQ_NO_SRCCACHE=1: every B_perp source phase reads all its records
  void* bjn;           // V2: beam J_perp of slice i+1
  void* bjp;           // 2 x V2: beam J_perp of slices i-1 and i by slice parity (explicit B_perp solver; null otherwise)
  // explicit B_perp solver (bperp_solver = 1): its source records, PCG vectors and scalars
  int explicit_b;
  void* xs4;           // V4: Fx, Fy, Jxx, Jyy (deposited by the explicit source pass)
  void* xs1;           // Jxy
  void* pcg_r;         // V2: residual r
  void* pcg_p;         // V2: search direction p
  double* pcg_s;       // [4][kMaxPcg][2]: r.z, p.Ap per iteration and right-hand side
  double* pcg_part;    // deterministic mode: per-block partial dot products (else null)
  void* scale_h;       // the preconditioner's spectral factors 1/(lambda - c), like f32_scale / f64_scale
  void* gf;            // kGF per node (gather fields ExmBy, EypBx, Ez, Bz of the current slice)
  void* bm;            // V2: Bx, By of the current slice (the predictor-corrector iterate, then converged);
                       // until finish_main of slice i it holds the converged B_perp of slice i-1
  void* psi;
  void* bprev1;        // V2: B_perp of slice i-2 until finish_main of slice i, then of slice i-1
                       // (B_perp of slice i-1 is gf[3..4] until then)
  void* solved;        // kMaxRhs x nnode: DST results

  // DST, FP64: [kMaxRhs][nnode] ping-pong buffers, per-mode scale, twiddles, sine tables
  double *f64_a, *f64_b, *f64_scale, *tw_x, *tw_y, *sin_x, *sin_y;
  // DST, FP32/bf16x3: padded operand buffers and sine matrices
  int nxp, nyp;
  // elements: bf16, or (tf32) FP32 words holding TF32 values
  void *op_hi[2], *op_lo[2];                // ping-pong [kMaxRhs * max(nxp,nyp)^2]
  void *sx_hi, *sx_lo, *sy_hi, *sy_lo;
  float* f32_scale;                          // [nyp][nxp] (1/lambda)(4/(nx ny)), slot order if folded
  hq::TensorMaps* tmaps;
  int fold;                                  // folded DST-I (nx, ny multiples of 128; FP32 mode)
  float* psrc[2];                            // FP32 mode: psi source rho - J_z of dep[0], dep[1]
  unsigned long long* d_gbar;                // grid-barrier counter of the fused solve kernel (zero between launches)
  int fault_barrier;                         // HQ_FAULT_BARRIER=1: the solve's first grid barrier never fills
  int no_f4;                                 // HQ_NO_F4CACHE=1: every trial pass gathers all six fields
  int f4_slice;                              // slice whose first trial pass filled p32.f4 (-1: none)
  int sep_src;                               // HQ_SEPARATE_SRC=1: source kernels ahead of the solve launches

  // beams
  hq::BeamBins bins[hq::kMaxBeams];
  hq_beam_view bound[hq::kMaxBeams];
  int nbound;

  double* d_profile;   // radial density profile (device copy)
  int* d_status;
  unsigned long long* d_removed;
  int* d_scratch_int;

  int last_adv, last_beam, last_solved;
  std::string err;

  // checkpoints, tapes and adjoint state (allocated by the first checkpointed sweep)
  void* adj;

  // hq_sweep_step replayed from a CUDA graph (captured once per argument set)
  void* sweep_graph;
  int graph_off;       // capture failed or was refused: plain stream launches from now on
  cudaStream_t cap_stream;   // private stream the sweep is captured on (the graph runs on `stream`)
  // second stream (and fork / join events) for the per-slice launches that can run beside the
  // final pass; created on first use
  cudaStream_t aux_stream;
  cudaEvent_t ev_fork, ev_join;

  // profiling: launch counters (always) and optional CUDA event pairs per launch group
  int64_t launches[HQ_K_CLASSES];
  int prof_on;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_class;   // class of each recorded pair (events 2k, 2k+1)
  size_t ev_used;
};

namespace hq {

// Programmatic dependent launch is on unless the environment sets HQ_NO_PDL=1.
bool pdl_enabled();

// Launch with programmatic stream serialization (see pdl_wait / pdl_trigger).
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------- launchers (kernels in *.cu)
// particles
template <typename T> void launch_plasma_init(const hq_grid_s* g, cudaStream_t s);
template <typename T> void launch_deposit_initial(const hq_grid_s* g, void* dep, void* chi, int ion_only, cudaStream_t s);
template <typename T> void launch_trial_pass(const hq_grid_s* g, int slice, int iter, cudaStream_t s);
template <typename T> void launch_final_pass(const hq_grid_s* g, int slice, void* dep, void* chi, bool f4,
                                             cudaStream_t s);
// fields
template <typename T> void launch_reset_dep(const hq_grid_s* g, void* dep, void* chi, cudaStream_t s);
template <typename T> void launch_src_main(const hq_grid_s* g, const void* dep, cudaStream_t s);
// reads and clears the trial J_perp; reset_prev != 0: after reading, resets dep_prev to the
// ion background (it receives the next slice's deposit)
template <typename T> void launch_src_bperp(const hq_grid_s* g, const void* dep_cur, void* dep_prev, void* chi_prev,
                                            int reset_prev, cudaStream_t s);
template <typename T> void launch_src_copy(const hq_grid_s* g, const void* src, int nrhs, cudaStream_t s);
// finish_main also sets the B_perp guess 2 B(i-1) - B(i-2) (first: slice 0, B(-1) = 0) and
// moves B(i-1) into bprev1
template <typename T> void launch_finish_main(const hq_grid_s* g, const void* res, int first, cudaStream_t s);
template <typename T> void launch_finish_bperp(const hq_grid_s* g, const void* res, cudaStream_t s);
template <typename T> void launch_store(const hq_grid_s* g, const hq_field_out* out, int64_t slot, const void* dep, const void* chi, cudaStream_t s);
template <typename T> void launch_zero(void* p, int64_t n, cudaStream_t s);
// DST backends: transform the nrhs sources prepared by the src kernels into g->solved
// scale: the spectral factors (null: the Poisson table f64_scale; scale_h: the shifted one)
void dst_solve_f64(hq_grid_s* g, int nrhs, cudaStream_t s, const double* scale = nullptr);
void dst_solve_tc(hq_grid_s* g, int nrhs, cudaStream_t s);
void dst_solve_tc_shifted(hq_grid_s* g, int nrhs, cudaStream_t s);   // (L - c)^{-1}: g->scale_h
void dst_solve_tc_bmix(hq_grid_s* g, int last, cudaStream_t s);   // B_perp solve + fused mixing (FP32)
// FP32 solves with the source assembly as their first phase (no separate source kernel)
void dst_solve_tc_main(hq_grid_s* g, const void* dep, cudaStream_t s);
void dst_solve_tc_bmix_src(hq_grid_s* g, const void* cur, void* prev, void* chi_prev, int last, cudaStream_t s);
int dst_tc_init(hq_grid_s* g, std::string& err);   // builds tensor maps; 0 on success
void dst_tc_free(hq_grid_s* g);
// beams
void launch_beam_bin(hq_grid_s* g, int b, const hq_beam_view& v, cudaStream_t s);
void launch_beam_slices(const hq_grid_s* g, const hq_beam_view& v, int32_t* out, cudaStream_t s);
// FP32 multi-species grids: sum q w S(x0) / A of the species without a neutralizing background,
// added in FP64 into out (nnode doubles, zeroed by the caller) (k_particles.cu)
void launch_species_c0(const hq_grid_s* g, double* out, cudaStream_t s);
// deterministic FP64 mode: adds the fixed-point mirrors of n elements of rec (a deposit record
// of the arena) to rec, or to dst when given, and clears the mirrors (k_fields.cu)
void launch_fx_decode(const hq_grid_s* g, void* rec, int64_t n, double* dst, cudaStream_t s);
// plasma re-sort by cell (k_sort.cu); the scratch size and scan tile count for allocation
void launch_resort(hq_grid_s* g, cudaStream_t s);
int64_t resort_scratch_bytes(const hq_grid_s* g);
int64_t resort_tiles(const hq_grid_s* g);
template <typename T> void launch_beam_deposit(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, void* dep, void* bjn, cudaStream_t s);
template <typename T> void launch_beam_push(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, double dt, cudaStream_t s);
template <typename T> void launch_witness(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, double* sums, cudaStream_t s);
void launch_beam_moments(const hq_beam_view& v, double* m, cudaStream_t s);   // m += 11 weighted moments
// explicit B_perp solver (k_explicit.cu): the particle source pass, the PCG start (right-hand
// side, initial residual into the solver's operand writer, reset of the slice i-1 record) and
// one PCG iteration after a shifted solve of the residual
template <typename T> void launch_explicit_src(const hq_grid_s* g, cudaStream_t s);
template <typename T> void launch_pcg_init(const hq_grid_s* g, int slice, const void* cur, const void* chi_cur, void* prev,
                                           void* chi_prev, cudaStream_t s);
template <typename T> void launch_pcg_iter(const hq_grid_s* g, int slice, int k, const void* chi_cur, cudaStream_t s);
// adjoint (k_adjoint.cu)
template <typename T> void launch_adj_final(const hq_grid_s* g, const SnapView<T>& s, const void* gf, int slice,
                                           const void* dbar_next, const AdjView<T>& a, void* tbar, void* fbar_b,
                                           double* wbar_p, cudaStream_t st);
template <typename T> void launch_adj_trial(const hq_grid_s* g, const SnapView<T>& s, const void* gf, const void* bm,
                                           int slice, const void* jbar, const AdjView<T>& a, void* tbar, void* bbar_m1,
                                           double* wbar_p, cudaStream_t st);
template <typename T> void launch_adj_bstart(const hq_grid_s* g, void* fbar_b, void* carry, void* bbar_n, cudaStream_t st);
template <typename T> void launch_adj_pc_pre(const hq_grid_s* g, const void* bbar_m, void* bbar_m1, cudaStream_t st);
template <typename T> void launch_adj_pc_post(const hq_grid_s* g, void* dcur, void* dprev, void* jbar, void* jtot, cudaStream_t st);
template <typename T> void launch_adj_guess(const hq_grid_s* g, const void* b0, void* c1, void* c2, cudaStream_t st);
template <typename T> void launch_adj_main_pre(const hq_grid_s* g, const void* tbar, const void* seed_psi, cudaStream_t st);
template <typename T> void launch_adj_seed(const hq_grid_s* g, const hq_field_out& seeds, int slice, void* tbar,
                                           void* fbar_b, void* dcur, cudaStream_t st);
template <typename T> void launch_adj_main_post(const hq_grid_s* g, void* dcur, void* rho_ion_bar, void* tbar,
                                               cudaStream_t st);
template <typename T> void launch_adj_beam(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, const void* dcur,
                                          const void* jtot, double* wbar, cudaStream_t st);
template <typename T> void launch_adj_witness(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, const void* gf,
                                             const double* sb, void* tbar, double* wbar, cudaStream_t st);
template <typename T> void launch_adj_init(const hq_grid_s* g, const void* d0, const void* rho_ion_bar, double* wbar_p,
                                          cudaStream_t st);
void launch_adj_params(const hq_grid_s* g, const double* wbar_p, double* dn0, double* dprof, cudaStream_t st);

}  // namespace hq

// ---------------------------------------------------------------- device helpers
namespace hq {

// Programmatic dependent launch: a kernel launched with launch_pdl may start while
// the previous kernel in the stream is still running; it must call pdl_wait()
// before touching memory that kernel reads or writes.  pdl_trigger() lets the next
// kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// B-spline weights of order P from the cell index jf = floor(u) and the fraction
// d = u - jf in [0, 1).  Node j0 + a carries weight w[a] (Sec. 3.2 deposition, orders 0-3).
template <int P, typename T>
__device__ __forceinline__ int shape_weights(int jf, T d, T* w) {
  if constexpr (P == 0) {
    w[0] = T(1);
    return jf + (d >= T(0.5) ? 1 : 0);
  } else if constexpr (P == 1) {
    w[0] = T(1) - d;
    w[1] = d;
    return jf;
  } else if constexpr (P == 2) {
    const bool up = d >= T(0.5);
    const T e = up ? d - T(1) : d;           // offset from the nearest node, [-0.5, 0.5)
    const T a = T(0.5) - e, b = T(0.5) + e;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - e * e;
    w[2] = T(0.5) * b * b;
    return jf + (up ? 1 : 0) - 1;
  } else {
    const T d2 = d * d, d3 = d2 * d, om = T(1) - d;
    w[0] = om * om * om * T(1.0 / 6.0);
    w[1] = (T(4) - T(6) * d2 + T(3) * d3) * T(1.0 / 6.0);
    w[2] = (T(1) + T(3) * d + T(3) * d2 - T(3) * d3) * T(1.0 / 6.0);
    w[3] = d3 * T(1.0 / 6.0);
    return jf - 1;
  }
}

// Node coordinate u = (x - x0) / dx split into floor and fraction, in FP64.
__device__ __forceinline__ void split_coord(double x, double x0, double dx, int& jf, double& d) {
  const double u = (x - x0) / dx;
  const double f = floor(u);
  jf = (int)f;
  d = u - f;
}

__device__ __forceinline__ bool in_interior(int j, int n) { return j >= 1 && j <= n - 1; }

// Deterministic FP64 accumulation (hq_grid_desc.deterministic).  A contribution v to an element
// of a deposit record is split into the fixed-point pair H = floor(v 2^32), L = round((v 2^32 - H)
// 2^40) and added with 64-bit integer atomics to the element's mirror, two words at byte address
// 2 * (element address) + det (the mirrors of all deposit records are laid out like the records,
// at twice the stride).  Integer sums do not depend on the order of the additions; k_fx_decode
// later adds H 2^-32 + L 2^-72 to the element and clears the mirror.  Resolution 2^-72; |v| and
// every partial sum must stay below 2^31 (else DEV_NONFINITE); up to 2^23 contributions per
// element between decodes.
__device__ __forceinline__ void fx_add(double* p, double v, int64_t det, int* status) {
  const double s = v * 4294967296.0;
  if (!(fabs(s) < 9.2e18)) {
    if (status) atomicOr(status, DEV_NONFINITE);
    return;
  }
  const double h = floor(s);
  const long long hi = (long long)h;
  const long long lo = llrint((s - h) * 1099511627776.0);
  unsigned long long* m = reinterpret_cast<unsigned long long*>(2ull * reinterpret_cast<uintptr_t>(p) + (uint64_t)det);
  atomicAdd(m, (unsigned long long)hi);
  if (lo) atomicAdd(m + 1, (unsigned long long)lo);
}
// Deposit add: fixed point in deterministic FP64 mode, a plain atomic otherwise.
__device__ __forceinline__ void dadd(double* p, double v, const Geom& gm) {
  if (gm.det) fx_add(p, v, gm.det, gm.dstatus);
  else atomicAdd(p, v);
}
__device__ __forceinline__ void dadd(float* p, float v, const Geom&) { atomicAdd(p, v); }

// Adds the block's (sum (B_m - B_m-1)^2, sum B_m^2) of the predictor-corrector mixing to the
// slice's residual sums rs: [kResLanes][2] pairs, the block's pair chosen by its index so that
// no address takes more than a few atomics (the host adds the lanes).  Warp shuffles, then a
// shared-memory sum over the warps; every thread of the block must call it (it synchronizes).
constexpr int kResLanes = 16;
__device__ __forceinline__ void pc_residual_add(double* rs, double d2, double b2) {
  __shared__ double part[2][32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    b2 += __shfl_down_sync(0xffffffffu, b2, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    part[0][w] = d2;
    part[1][w] = b2;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += part[threadIdx.x][k];
    const int lane = (int)((blockIdx.y * gridDim.x + blockIdx.x) % kResLanes);
    if (t != 0.0) atomicAdd(rs + 2 * lane + threadIdx.x, t);
  }
  __syncthreads();
}

// Folded DST-I order (Sec. 3.2 solver).  With S_jk = sin(pi j k / n),
// S_{n-j,k} = -(-1)^k S_jk: odd k see only x_j + x_{n-j}, even k only x_j - x_{n-j},
// so after folding the node pairs (j, n-j) every output needs n/2 terms.  The folded
// solver keeps each grid index in "slot order", pair u on slots 2u, 2u+1: pairs
// 0 .. n/4-1 are (1, n-1), (3, n-3), ...; pair n/4 is (0, n/2); the rest (2, n-2),
// (4, n-4), ...  Slots 0 .. n/2-1 thus hold the odd indices.  n must be a multiple of 4.
__host__ __device__ __forceinline__ void fold_pair(int u, int n, int& a, int& b) {
  if (u < n / 4) {
    a = 2 * u + 1;
    b = n - a;
  } else {
    a = 2 * (u - n / 4);
    b = a == 0 ? n / 2 : n - a;
  }
}
__host__ __device__ __forceinline__ int fold_node(int s, int n) {
  int a, b;
  fold_pair(s >> 1, n, a, b);
  return (s & 1) ? b : a;
}

}  // namespace hq

// ---------------------------------------------------------------- shared field helpers
namespace hq {

// DST operand writers: FP64 mode writes [rhs][ny][nx] doubles (g->f64_a); FP32 mode
// writes each value already split into hi + lo (bf16 or TF32), zero-padded [rhs][nyp][nxp]
// (g->op_hi[0], g->op_lo[0]), the tensor-core solver's input layout.
struct SinkF64 {
  static constexpr bool kFold = false;
  double* p;
  int nx, ny;
  __device__ void put(int r, int iy, int ix, double v) const { p[((int64_t)r * ny + iy) * nx + ix] = v; }
};

// The split of one FP32 value v into the tensor-core operand pair (hi, lo), v ~ hi + lo:
// bf16 (HQ_PREC_FP32_BF16X3: hi = bf16(v), lo = bf16(v - hi), 16 significant bits), or TF32 held
// in 32-bit words (HQ_PREC_FP32_TF32X3: hi = v rounded to 11 significant bits, lo = v - hi,
// which the tensor core reads truncated to TF32: 21 or more significant bits).
__device__ __forceinline__ float round_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return __uint_as_float(u);
}
__device__ __forceinline__ void put_split(__nv_bfloat16* hi, __nv_bfloat16* lo, int64_t o, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  hi[o] = h;
  lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
}
__device__ __forceinline__ void put_split(float* hi, float* lo, int64_t o, float v) {
  const float h = round_tf32(v);
  hi[o] = h;
  lo[o] = v - h;
}

// Plain operand layout [rhs][nyp][nxp] (E: __nv_bfloat16 or float for TF32).
template <typename E> struct SinkSplit {
  static constexpr bool kFold = false;
  E *hi, *lo;
  int nxp, nyp;
  __device__ void put(int r, int iy, int ix, float v) const { put_split(hi, lo, ((int64_t)r * nyp + iy) * nxp + ix, v); }
};

// FP32 mode with the folded solver (fold_pair): a thread owns the node pair (a, b) of
// folded column u in row slot sy and writes the sum x_a + x_b to column u and the
// difference x_a - x_b to column nx/2 + u (the pair (0, n/2) stores x_{n/2} and 0:
// node 0 is on the wall and never enters a DST-I).  Layout [rhs][ny slots][nx].
template <typename E> struct SinkFold {
  static constexpr bool kFold = true;
  E *hi, *lo;
  int nx, ny;
  __device__ void put_pair(int r, int sy, int u, float va, float vb) const {
    const bool wall = u == nx / 4;
    const int64_t row = ((int64_t)r * ny + sy) * nx;
    put_split(hi, lo, row + u, wall ? vb : va + vb);
    put_split(hi, lo, row + nx / 2 + u, wall ? 0.0f : va - vb);
  }
};

// Columns of one row of visit_one: nx/2 folded node pairs or nx nodes.
template <typename Sink> __host__ __device__ __forceinline__ int visit_width(const Geom& gm) {
  return Sink::kFold ? gm.nx / 2 : gm.nx;
}

// Runs f(iy, ix, v) for the node(s) of (row, tx) and hands the first nr values of v to the
// sink: one node for a plain sink (row = iy, tx = ix); for SinkFold the two nodes of folded
// column tx, the row taken in slot order.
template <int NR, typename T, typename Sink, typename F>
__device__ __forceinline__ void visit_one(const Geom& gm, const Sink& sink, int nr, F&& f, int row, int tx) {
  if constexpr (Sink::kFold) {
    const int iy = fold_node(row, gm.ny);
    int xa, xb;
    fold_pair(tx, gm.nx, xa, xb);
    T va[NR], vb[NR];
    f(iy, xa, va);
    f(iy, xb, vb);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) sink.put_pair(r, row, tx, va[r], vb[r]);
  } else {
    T v[NR];
    f(row, tx, v);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) sink.put(r, row, tx, v[r]);
  }
}

// One (row, column) of visit_one per thread: consecutive threads along the row, one row per
// block row.  Launch with src_grid().
template <int NR, typename T, typename Sink, typename F>
__device__ __forceinline__ void visit_nodes(const Geom& gm, const Sink& sink, int nr, F&& f) {
  const int tx = blockIdx.x * blockDim.x + threadIdx.x;
  if (tx >= visit_width<Sink>(gm)) return;
  visit_one<NR, T>(gm, sink, nr, f, (int)blockIdx.y, tx);
}

// Calls f(sink) with the DST operand writer of the grid's solver.
template <typename T, typename F>
inline void with_sink(const hq_grid_s* g, F&& f) {
  if constexpr (sizeof(T) == 8) {
    f(SinkF64{g->f64_a, g->nx, g->ny});
  } else {
    if (g->tf32) {
      float* hi = reinterpret_cast<float*>(g->op_hi[0]);
      float* lo = reinterpret_cast<float*>(g->op_lo[0]);
      if (g->fold) f(SinkFold<float>{hi, lo, g->nx, g->ny});
      else f(SinkSplit<float>{hi, lo, g->nxp, g->nyp});
    } else {
      __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(g->op_hi[0]);
      __nv_bfloat16* lo = reinterpret_cast<__nv_bfloat16*>(g->op_lo[0]);
      if (g->fold) f(SinkFold<__nv_bfloat16>{hi, lo, g->nx, g->ny});
      else f(SinkSplit<__nv_bfloat16>{hi, lo, g->nxp, g->nyp});
    }
  }
}

// Grid of the source kernels (visit_nodes): 128 threads per block along x, one row per block.
inline dim3 src_grid(const hq_grid_s* g) {
  const int w = g->fold ? g->nx / 2 : g->nx;
  return dim3((unsigned)((w + 127) / 128), (unsigned)g->ny);
}

// FP32 path: the psi source rho - J_z accumulated beside a deposit record (ion-subtracted per
// particle, see k_particles); null in FP64 mode, which forms rho - J_z from the record.
inline float* psrc_of(const hq_grid_s* g, const void* dep) {
  if (g->fp64) return nullptr;
  return dep == g->dep[0] ? g->psrc[0] : dep == g->dep[1] ? g->psrc[1] : nullptr;
}

// Explicit B_perp solver: the beam J_perp record of slice `slice` (parity-indexed pair; null
// without the explicit solver).  Slice i deposits into bjp_at(i) and reads bjp_at(i - 1).
inline void* bjp_at(const hq_grid_s* g, int slice) {
  if (!g->bjp) return nullptr;
  return static_cast<char*>(g->bjp) + (size_t)(slice & 1) * 2 * (g->fp64 ? 8 : 4) * (size_t)g->nnode;
}

template <typename T> struct SrcMain;
template <typename T> struct SrcBperp;
template <typename T> SrcMain<T> src_main_of(const hq_grid_s* g, const void* dep);
template <typename T> SrcBperp<T> src_bperp_of(const hq_grid_s* g, const void* cur, void* prev, void* chi_prev,
                                               int reset_prev);

// 1 - u_z / gamma without cancellation for u_z > 0: (1 + u_perp^2) / (gamma (gamma + u_z)).
__device__ __forceinline__ float one_minus_vz(float ux, float uy, float uz, float gamma) {
  return uz > 0.0f ? (1.0f + ux * ux + uy * uy) / (gamma * (gamma + uz)) : 1.0f - uz / gamma;
}

// Central difference helpers with wall nodes (index 0 and n) reading zero; the
// result on wall rows/columns is zero (matching the field layout convention).
template <typename A, typename C>
__device__ __forceinline__ auto dxc(const A& f, int iy, int ix, int nx, C inv2dx) -> decltype(f(0, 0)) {
  using T = decltype(f(0, 0));
  const T r = ix + 1 < nx ? f(iy, ix + 1) : T(0);
  const T l = f(iy, ix - 1);
  return (r - l) * T(inv2dx);
}
template <typename A, typename C>
__device__ __forceinline__ auto dyc(const A& f, int iy, int ix, int ny, C inv2dy) -> decltype(f(0, 0)) {
  using T = decltype(f(0, 0));
  const T u = iy + 1 < ny ? f(iy + 1, ix) : T(0);
  const T d = f(iy - 1, ix);
  return (u - d) * T(inv2dy);
}


// ---------------------------------------------------------------- per-node sources
// The field equations' sources (Sec. 2), one node at a time (visited by the source kernels
// of k_fields.cu through the grid's operand sink).

// psi: -(rho - Jz);  Ez: dx Jx + dy Jy;  Bz: dy Jx - dx Jy.  With ps (FP32 path) the psi
// source is the separately accumulated, ion-subtracted rho - Jz, plus c0 (multi-species grids:
// the initial charge of the species without a neutralizing background) when given.
template <typename T> struct SrcMain {
  static constexpr int NR = 3;
  static constexpr bool kEffects = false;
  const V4<T>* dep;
  const float* ps;
  Geom gm;
  const float* c0;
  // what one node's sources read: the psi source, and Jx, Jy at the four neighbours
  struct In {
    T p, jxr, jxl, jxu, jxd, jyr, jyl, jyu, jyd;
  };
  __device__ In load(int iy, int ix) const {
    In q{};
    if (ix > 0 && iy > 0) {
      const int nx = gm.nx;
      const int64_t o = (int64_t)iy * nx + ix;
      if (ps) {
        q.p = c0 ? T(-(ps[o] + c0[o])) : T(-ps[o]);
      } else {
        const V4<T> c = dep[o];
        q.p = -(c.a - c.d);
      }
      const bool r = ix + 1 < nx, u = iy + 1 < gm.ny;
      q.jxr = r ? dep[o + 1].b : T(0);
      q.jyr = r ? dep[o + 1].c : T(0);
      q.jxl = dep[o - 1].b;
      q.jyl = dep[o - 1].c;
      q.jxu = u ? dep[o + nx].b : T(0);
      q.jyu = u ? dep[o + nx].c : T(0);
      q.jxd = dep[o - nx].b;
      q.jyd = dep[o - nx].c;
    }
    return q;
  }
  __device__ void eval(int iy, int ix, const In& q, T* v) const {
    v[0] = v[1] = v[2] = T(0);
    if (ix > 0 && iy > 0) {
      const T i2x = gsel<T>(gm.inv2dx, gm.f_inv2dx), i2y = gsel<T>(gm.inv2dy, gm.f_inv2dy);
      v[0] = q.p;
      v[1] = (q.jxr - q.jxl) * i2x + (q.jyu - q.jyd) * i2y;
      v[2] = (q.jxu - q.jxd) * i2y - (q.jyr - q.jyl) * i2x;
    }
  }
  __device__ void effects(int, int) const {}
  __device__ void operator()(int iy, int ix, T* v) const { eval(iy, ix, load(iy, ix), v); }
};

// Bx: -dy Jz + dzeta Jy;  By: dx Jz - dzeta Jx, with dzeta J = (J(i-1) - J(i+1)) / (2 dzeta)
// and J(i+1) = trial plasma + beam of slice i+1 (Sec. 3.2 predictor-corrector).  The trial
// J_perp is cleared after reading (ready for the next trial pass); with reset_prev (the
// last iteration) the slice i-1 record is reset to the ion background, ready to receive
// the deposit of slice i+1, and the beam J_perp of slice i+1 is cleared for the next
// slice's beam deposit.
template <typename T> struct SrcBperp {
  static constexpr int NR = 2;
  static constexpr bool kEffects = true;
  const V4<T>* cur;
  V4<T>* prev;
  T* chi_prev;
  float* ps_prev;
  const T* rho_ion;
  V2<T>* tj;
  V2<T>* bjn;
  Geom gm;
  int reset_prev;
  // Only the trial J_perp changes between the predictor-corrector iterations of a slice: the
  // rest, a0 = -dy Jz + (Jy(i-1) - Jy_beam(i+1)) / 2dz and a1 = dx Jz - (Jx(i-1) - Jx_beam(i+1)) / 2dz,
  // is formed in the first iteration and kept per node in s0 (mode 1); the later ones read it
  // back with the trial J_perp alone (mode 2).  Mode 0 (FP64, or HQ_NO_SRCCACHE=1) forms
  // every term from the records.
  V2<T>* s0;
  int mode;
  // what one node's sources read: Jz at the four neighbours, J_perp of slices i-1 (record),
  // i+1 (trial plasma) and i+1 (beam); mode 2: a0, a1 (in pb, pc) and the trial J_perp
  struct In {
    T jzr, jzl, jzu, jzd, pb, pc, ta, tb, ba, bb;
  };
  __device__ In load(int iy, int ix) const {
    In q{};
    if (ix > 0 && iy > 0 && mode == 2) {
      const int64_t o = (int64_t)iy * gm.nx + ix;
      const V2<T> a = s0[o], t = tj[o];
      q.pb = a.a;
      q.pc = a.b;
      q.ta = t.a;
      q.tb = t.b;
    } else if (ix > 0 && iy > 0) {
      const int nx = gm.nx;
      const int64_t o = (int64_t)iy * nx + ix;
      q.jzr = ix + 1 < nx ? cur[o + 1].d : T(0);
      q.jzl = cur[o - 1].d;
      q.jzu = iy + 1 < gm.ny ? cur[o + nx].d : T(0);
      q.jzd = cur[o - nx].d;
      const V4<T> pv = prev[o];
      const V2<T> t = tj[o], b = bjn[o];
      q.pb = pv.b;
      q.pc = pv.c;
      q.ta = t.a;
      q.tb = t.b;
      q.ba = b.a;
      q.bb = b.b;
    }
    return q;
  }
  __device__ void eval(int iy, int ix, const In& q, T* v) const {
    v[0] = v[1] = T(0);
    if (ix > 0 && iy > 0) {
      const T i2z = gsel<T>(gm.inv2dz, gm.f_inv2dz);
      if (mode == 0) {
        const T dzjx = (q.pb - (q.ta + q.ba)) * i2z;
        const T dzjy = (q.pc - (q.tb + q.bb)) * i2z;
        v[0] = -((q.jzu - q.jzd) * gsel<T>(gm.inv2dy, gm.f_inv2dy)) + dzjy;
        v[1] = (q.jzr - q.jzl) * gsel<T>(gm.inv2dx, gm.f_inv2dx) - dzjx;
      } else {
        T a0 = q.pb, a1 = q.pc;
        if (mode == 1) {
          a0 = -((q.jzu - q.jzd) * gsel<T>(gm.inv2dy, gm.f_inv2dy)) + (q.pc - q.bb) * i2z;
          a1 = (q.jzr - q.jzl) * gsel<T>(gm.inv2dx, gm.f_inv2dx) - (q.pb - q.ba) * i2z;
          s0[(int64_t)iy * gm.nx + ix] = V2<T>{a0, a1};
        }
        v[0] = a0 - q.tb * i2z;
        v[1] = a1 + q.ta * i2z;
      }
    }
  }
  // after the node's reads: clear the trial J_perp, reset the slice i-1 record if asked
  __device__ void effects(int iy, int ix) const {
    const int64_t o = (int64_t)iy * gm.nx + ix;
    tj[o] = V2<T>{T(0), T(0)};
    if (reset_prev) {
      prev[o] = V4<T>{rho_ion[o], T(0), T(0), T(0)};
      chi_prev[o] = T(0);
      if (ps_prev) ps_prev[o] = 0.0f;
      bjn[o] = V2<T>{T(0), T(0)};
    }
  }
  __device__ void operator()(int iy, int ix, T* v) const {
    eval(iy, ix, load(iy, ix), v);
    effects(iy, ix);
  }
};

template <typename T> inline SrcMain<T> src_main_of(const hq_grid_s* g, const void* dep) {
  return SrcMain<T>{reinterpret_cast<const V4<T>*>(dep), psrc_of(g, dep), g->geom, g->c0};
}
template <typename T>
inline SrcBperp<T> src_bperp_of(const hq_grid_s* g, const void* cur, void* prev, void* chi_prev, int reset_prev) {
  const int mode = (sizeof(T) == 8 || !g->bsrc0 || g->no_srccache) ? 0 : (g->pc_iter == 0 ? 1 : 2);
  return SrcBperp<T>{reinterpret_cast<const V4<T>*>(cur), reinterpret_cast<V4<T>*>(prev), reinterpret_cast<T*>(chi_prev),
                     psrc_of(g, prev), reinterpret_cast<const T*>(g->rho_ion), reinterpret_cast<V2<T>*>(g->tj),
                     reinterpret_cast<V2<T>*>(g->bjn), g->geom, reset_prev,
                     reinterpret_cast<V2<T>*>(g->bsrc0), mode};
}

}  // namespace hq
