// Field-slice kernels around the Poisson solves (Sec. 2 steps 4-7, Eqs. psi,
// exmby, ez, bxby, bz): source assembly with second-order central differences,
// -grad(psi), the predictor-corrector mixing, the B_perp guess/shift and the
// per-slice output copy.  All are HBM/L2-streaming elementwise kernels over the
// ny x nx slice (one thread per node, consecutive threads along x).
//
// Sources are written through a "sink": FP64 mode writes doubles in the solver's
// [rhs][ny][nx] layout; FP32 mode writes each source already split into two bf16
// terms (hi + lo) in the operand layout of the tensor-core DST (zero-padded
// [rhs][nyp][nxp], or folded node pairs in slot order), so no separate conversion
// pass is needed.
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 256;

template <typename T>
__global__ void k_reset_dep(V4<T>* dep, T* chi, const T* rho_ion, float* ps, int64_t nn) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nn) return;
  dep[i] = V4<T>{rho_ion[i], T(0), T(0), T(0)};
  chi[i] = T(0);
  if (ps) ps[i] = 0.0f;   // ion-subtracted: the ion background enters per particle
}

// Source kernels: one node (or folded node pair) per thread; the arithmetic is in the
// per-node functors SrcMain and SrcBperp.
template <typename T, typename Sink>
__global__ void k_src_main(SrcMain<T> src, Sink sink) {
  pdl_trigger();
  pdl_wait();
  visit_nodes<3, T>(src.gm, sink, 3, src);
}

template <typename T, typename Sink>
__global__ void k_src_bperp(SrcBperp<T> src, Sink sink) {
  pdl_trigger();
  pdl_wait();
  visit_nodes<2, T>(src.gm, sink, 2, src);
}

template <typename T, typename Sink>
__global__ void k_src_copy(const T* __restrict__ src, int nrhs, Geom gm, Sink sink) {
  visit_nodes<kMaxRhs, T>(gm, sink, nrhs, [&](int iy, int ix, T* v) {
    for (int r = 0; r < kMaxRhs; ++r)
      v[r] = (r < nrhs && ix > 0 && iy > 0) ? src[((int64_t)r * gm.ny + iy) * gm.nx + ix] : T(0);
  });
}

// psi -> psi array; gf = (ExmBy, EypBx) = -grad psi, Ez, Bz; bm = the predictor-corrector
// guess B(i) = 2 B(i-1) - B(i-2).  On entry bm still holds the converged B(i-1) of the previous
// slice (taken as zero on the first slice) and b1 holds B(i-2); on exit b1 holds B(i-1).
template <typename T>
__global__ void k_finish_main(const T* __restrict__ res, T* psi, T* gf, V2<T>* bm, V2<T>* b1, int first, Geom gm,
                              int* status) {
  pdl_trigger();
  pdl_wait();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (ix >= gm.nx) return;
  const int nx = gm.nx;
  const int64_t nn = (int64_t)nx * gm.ny;
  const int64_t o = (int64_t)iy * nx + ix;
  auto ps = [&](int y, int x) { return res[(int64_t)y * nx + x]; };
  T ex = T(0), ey = T(0);
  if (ix > 0 && iy > 0) {
    ex = -dxc(ps, iy, ix, nx, gsel<T>(gm.inv2dx, gm.f_inv2dx));
    ey = -dyc(ps, iy, ix, gm.ny, gsel<T>(gm.inv2dy, gm.f_inv2dy));
  }
  const T p = res[o], ez = res[nn + o], bz = res[2 * nn + o];
  if (!(isfinite(p) && isfinite(ez) && isfinite(bz))) atomicOr(status, DEV_NONFINITE);
  psi[o] = p;
  T* q = gf + o * kGF;
  q[0] = ex;
  q[1] = ey;
  q[2] = ez;
  q[3] = bz;
  const V2<T> p1 = first ? V2<T>{T(0), T(0)} : bm[o];
  const V2<T> p2 = b1[o];
  bm[o] = V2<T>{T(2) * p1.a - p2.a, T(2) * p1.b - p2.b};
  b1[o] = p1;
}

// B <- w B_solved + (1 - w) B  (predictor-corrector mixing), into bm.
template <typename T>
__global__ void k_finish_bperp(const T* __restrict__ res, V2<T>* bm, int64_t nn, T w, int* status, double* rsum) {
  pdl_trigger();
  pdl_wait();
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double d2 = 0.0, b2 = 0.0;
  if (o < nn) {
    const T bx = res[o], by = res[nn + o];
    if (!(isfinite(bx) && isfinite(by))) atomicOr(status, DEV_NONFINITE);
    const V2<T> b = bm[o];
    const V2<T> nb{w * bx + (T(1) - w) * b.a, w * by + (T(1) - w) * b.b};
    bm[o] = nb;
    if (rsum) {
      const T dx = nb.a - b.a, dy = nb.b - b.b;
      d2 = (double)(dx * dx + dy * dy);
      b2 = (double)(nb.a * nb.a + nb.b * nb.b);
    }
  }
  if (rsum) pc_residual_add(rsum, d2, b2);
}

template <typename T>
__global__ void k_store(hq_field_out out, int64_t base, const V4<T>* dep, const float* ps, const T* chi,
                        const T* psi, const T* gf, const V2<T>* bm, int64_t nn) {
  pdl_trigger();
  pdl_wait();
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nn) return;
  const V4<T> d = dep[o];
  const T* q = gf + o * kGF;
  const int64_t t = base + o;
  // FP32 path: rho = (rho - J_z) + J_z from the ion-subtracted psi source (the rho record holds
  // the unit ion background, against which the plasma response is lost to rounding)
  if (out.rho) reinterpret_cast<T*>(out.rho)[t] = ps ? T(ps[o]) + d.d : d.a;
  if (out.jx) reinterpret_cast<T*>(out.jx)[t] = d.b;
  if (out.jy) reinterpret_cast<T*>(out.jy)[t] = d.c;
  if (out.jz) reinterpret_cast<T*>(out.jz)[t] = d.d;
  if (out.chi) reinterpret_cast<T*>(out.chi)[t] = chi[o];
  if (out.psi) reinterpret_cast<T*>(out.psi)[t] = psi[o];
  if (out.exmby) reinterpret_cast<T*>(out.exmby)[t] = q[0];
  if (out.eypbx) reinterpret_cast<T*>(out.eypbx)[t] = q[1];
  if (out.ez) reinterpret_cast<T*>(out.ez)[t] = q[2];
  if (out.bx) reinterpret_cast<T*>(out.bx)[t] = bm[o].a;
  if (out.by) reinterpret_cast<T*>(out.by)[t] = bm[o].b;
  if (out.bz) reinterpret_cast<T*>(out.bz)[t] = q[3];
}

template <typename T>
__global__ void k_zero(T* p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = T(0);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }
inline dim3 grid2d(const hq_grid_s* g) { return dim3((unsigned)((g->nx + 127) / 128), (unsigned)g->ny); }

}  // namespace

template <typename T>
void launch_reset_dep(const hq_grid_s* g, void* dep, void* chi, cudaStream_t s) {
  k_reset_dep<T><<<blocks_for(g->nnode), kThreads, 0, s>>>(reinterpret_cast<V4<T>*>(dep), reinterpret_cast<T*>(chi),
                                                         reinterpret_cast<const T*>(g->rho_ion), psrc_of(g, dep),
                                                         g->nnode);
}
template <typename T>
void launch_src_main(const hq_grid_s* g, const void* dep, cudaStream_t s) {
  with_sink<T>(g, [&](auto sink) {
    launch_pdl(k_src_main<T, decltype(sink)>, src_grid(g), 128, 0, s, src_main_of<T>(g, dep), sink);
  });
}
template <typename T>
void launch_src_bperp(const hq_grid_s* g, const void* cur, void* prev, void* chi_prev, int reset_prev, cudaStream_t s) {
  with_sink<T>(g, [&](auto sink) {
    launch_pdl(k_src_bperp<T, decltype(sink)>, src_grid(g), 128, 0, s,
               src_bperp_of<T>(g, cur, prev, chi_prev, reset_prev), sink);
  });
}
template <typename T>
void launch_src_copy(const hq_grid_s* g, const void* src, int nrhs, cudaStream_t s) {
  with_sink<T>(g, [&](auto sink) {
    k_src_copy<T, decltype(sink)><<<src_grid(g), 128, 0, s>>>(reinterpret_cast<const T*>(src), nrhs, g->geom, sink);
  });
}
template <typename T>
void launch_finish_main(const hq_grid_s* g, const void* res, int first, cudaStream_t s) {
  launch_pdl(k_finish_main<T>, grid2d(g), 128, 0, s, reinterpret_cast<const T*>(res), reinterpret_cast<T*>(g->psi),
             reinterpret_cast<T*>(g->gf), reinterpret_cast<V2<T>*>(g->bm), reinterpret_cast<V2<T>*>(g->bprev1), first,
             g->geom, g->d_status);
}
template <typename T>
void launch_finish_bperp(const hq_grid_s* g, const void* res, cudaStream_t s) {
  launch_pdl(k_finish_bperp<T>, blocks_for(g->nnode), kThreads, 0, s, reinterpret_cast<const T*>(res),
             reinterpret_cast<V2<T>*>(g->bm), g->nnode, T(g->d.pc_mix), g->d_status, g->pc_rsum);
}
template <typename T>
void launch_store(const hq_grid_s* g, const hq_field_out* out, int64_t slot, const void* dep, const void* chi, cudaStream_t s) {
  launch_pdl(k_store<T>, blocks_for(g->nnode), kThreads, 0, s, *out, slot * g->nnode,
             reinterpret_cast<const V4<T>*>(dep), static_cast<const float*>(psrc_of(g, dep)),
             reinterpret_cast<const T*>(chi), reinterpret_cast<const T*>(g->psi), reinterpret_cast<const T*>(g->gf),
             reinterpret_cast<const V2<T>*>(g->bm),
             g->nnode);
}
template <typename T>
void launch_zero(void* p, int64_t n, cudaStream_t s) {
  if (n > 0) k_zero<T><<<blocks_for(n), kThreads, 0, s>>>(reinterpret_cast<T*>(p), n);
}

// Deterministic FP64 mode: value of each element's fixed-point mirror (H 2^-32 + L 2^-72, see
// fx_add) added to the element (or to dst[i]); the mirror is cleared.  Elements whose mirror is
// zero are left untouched.
__global__ void k_fx_decode(double* rec, int64_t n, int64_t det, double* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long* m = reinterpret_cast<unsigned long long*>(2ull * reinterpret_cast<uintptr_t>(rec + i) + (uint64_t)det);
  const long long hi = (long long)m[0], lo = (long long)m[1];
  if ((hi | lo) == 0) return;
  const double v = (double)hi * 0x1p-32 + (double)lo * 0x1p-72;
  if (dst) dst[i] += v;
  else rec[i] += v;
  m[0] = 0ull;
  m[1] = 0ull;
}

void launch_fx_decode(const hq_grid_s* g, void* rec, int64_t n, double* dst, cudaStream_t s) {
  if (n > 0) k_fx_decode<<<blocks_for(n), kThreads, 0, s>>>(static_cast<double*>(rec), n, g->geom.det, dst);
}

#define HQ_INST(T)                                                                              \
  template void launch_reset_dep<T>(const hq_grid_s*, void*, void*, cudaStream_t);             \
  template void launch_src_main<T>(const hq_grid_s*, const void*, cudaStream_t);               \
  template void launch_src_bperp<T>(const hq_grid_s*, const void*, void*, void*, int, cudaStream_t); \
  template void launch_src_copy<T>(const hq_grid_s*, const void*, int, cudaStream_t);          \
  template void launch_finish_main<T>(const hq_grid_s*, const void*, int, cudaStream_t);       \
  template void launch_finish_bperp<T>(const hq_grid_s*, const void*, cudaStream_t);           \
  template void launch_store<T>(const hq_grid_s*, const hq_field_out*, int64_t, const void*, const void*, cudaStream_t); \
  template void launch_zero<T>(void*, int64_t, cudaStream_t);
HQ_INST(float)
HQ_INST(double)
#undef HQ_INST

}  // namespace hq
