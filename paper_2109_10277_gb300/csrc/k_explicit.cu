// Explicit B_perp field solver (Sec. 3.2, "explicit field solver": a Helmholtz-like equation
// instead of the predictor-corrector iterations).
//
// Reading (the paper cites the equation): differentiating the deposited plasma current
// J_perp = sum q w S u_perp / ((1 + Psi) A) along zeta with the particle equations of Sec. 3.2
// gives d(Jx)/d(zeta) = Tx - chi By and d(Jy)/d(zeta) = Ty + chi Bx, with chi the deposited
// susceptibility sum q^2 w S / (M (1 + Psi) A) (B taken at the node) and T the part without
// B_perp: force terms deposited from the gathered ExmBy, EypBx, Ez, Bz, convective terms as
// central differences of the deposited a g^2 u_a u_b, and the beams' central difference of
// their slice deposits.  Eq. bxby then reads
//   (L - chi) Bx = -dy Jz + Ty,   (L - chi) By = dx Jz - Tx,
// solved here by preconditioned conjugate gradients on (chi - L) B = -rhs, preconditioner
// (c - L)^{-1} with c = n0_scale (one shifted DST-I solve per iteration, on the tensor cores in
// FP32 mode), starting from the guess 2 B(i-1) - B(i-2), a fixed number of iterations.
//
// Kernels: the source pass over the plasma particles, and per-node PCG steps (the residual and
// direction vectors are V2 records (Bx, By); the scalars r.z and p.Ap are FP64 sums per
// iteration and right-hand side, accumulated with one atomic per block).
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 128;

// ---------------------------------------------------------------- source pass
// Per particle at its current (slice i) position: a = q w / A, g = 1 / (1 + Psi),
// Psi' = -(q/M)(g (ux ExmBy + uy EypBx) - Ez),
// Fx = a (g Gx - ux g^2 Psi'), Gx = -(q/M)(gamma g ExmBy + Bz g uy),
// Fy = a (g Gy - uy g^2 Psi'), Gy = -(q/M)(gamma g EypBx - Bz g ux),
// Jxx = a g^2 ux^2, Jxy = a g^2 ux uy, Jyy = a g^2 uy^2, deposited with the particle's shape.
// Written for electrons (q = -1, q/M = -1); a multi-species grid (MS) takes each particle's
// species constants.
template <int P, typename T, bool CACHE, bool MS>
__global__ void __launch_bounds__(kThreads) k_explicit_src(Plasma<T> pl, Geom gm, const T* __restrict__ gf,
                                                           V4<T>* xs4, T* xs1, SpeciesTab tab) {
  pdl_trigger();
  pdl_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n || !pl.alive[p]) return;
  int sp = 0;
  if constexpr (MS) sp = species_of(tab, p);
  T wx[P + 1], wy[P + 1];
  int ix0, iy0;
  T opp;
  if constexpr (CACHE) {
    const int cell = pl.cell[p];
    ix0 = shape_weights<P, T>(cell & 0xFFFF, T(pl.fx[p]), wx);
    iy0 = shape_weights<P, T>(cell >> 16, T(pl.fy[p]), wy);
    opp = T(pl.opp[p]);
  } else {
    int jx, jy;
    double fx, fy;
    split_coord(pl.x[p], gm.xmin, gm.dx, jx, fx);
    split_coord(pl.y[p], gm.ymin, gm.dy, jy, fy);
    ix0 = shape_weights<P, T>(jx, T(fx), wx);
    iy0 = shape_weights<P, T>(jy, T(fy), wy);
    opp = T(1.0 + pl.psi[p]);
  }
  T E[4] = {T(0), T(0), T(0), T(0)};   // ExmBy, EypBx, Ez, Bz
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, gm.nx)) continue;
      const T* q = gf + ((int64_t)iy * gm.nx + ix) * kGF;
      const T w = wx[a] * wy[b];
#pragma unroll
      for (int c = 0; c < 4; ++c) E[c] += w * q[c];
    }
  }
  const T ux = pl.ux[p], uy = pl.uy[p];
  const T g = T(1) / opp;
  const T gam = (T(1) + ux * ux + uy * uy + opp * opp) * T(0.5) * g;
  // electrons: q = -1, q/M = -1; other species: a = q w / A and the rates scaled by -q/M
  T a, dpsi, gx, gy;
  if constexpr (MS) {
    const T q = sizeof(T) == 8 ? T(tab.q[sp]) : T(tab.fq[sp]);
    const T mqm = sizeof(T) == 8 ? T(-tab.qm[sp]) : T(-tab.fqm[sp]);
    a = sizeof(T) == 8 ? T((tab.q[sp] * (double)pl.w[p]) / (gm.dx * gm.dy)) : q * pl.w[p] * gm.f_inv_area;
    dpsi = mqm * (g * (ux * E[0] + uy * E[1]) - E[2]);
    gx = mqm * (gam * g * E[0] + E[3] * g * uy);
    gy = mqm * (gam * g * E[1] - E[3] * g * ux);
  } else {
    a = sizeof(T) == 8 ? T((-1.0 * (double)pl.w[p]) / (gm.dx * gm.dy)) : -pl.w[p] * gm.f_inv_area;
    dpsi = g * (ux * E[0] + uy * E[1]) - E[2];
    gx = gam * g * E[0] + E[3] * g * uy;
    gy = gam * g * E[1] - E[3] * g * ux;
  }
  const T g2 = g * g;
  const T fx = a * (g * gx - ux * g2 * dpsi), fy = a * (g * gy - uy * g2 * dpsi);
  const T jxx = a * g2 * ux * ux, jxy = a * g2 * ux * uy, jyy = a * g2 * uy * uy;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a_ = 0; a_ <= P; ++a_) {
      const int ix = ix0 + a_;
      if (!in_interior(ix, gm.nx)) continue;
      const T w = wx[a_] * wy[b];
      const int64_t node = (int64_t)iy * gm.nx + ix;
      V4<T>* q = xs4 + node;
      if constexpr (sizeof(T) == 4) {
        atomicAdd(reinterpret_cast<float4*>(q), make_float4(w * fx, w * fy, w * jxx, w * jyy));
      } else {
        dadd(&q->a, w * fx, gm);
        dadd(&q->b, w * fy, gm);
        dadd(&q->c, w * jxx, gm);
        dadd(&q->d, w * jyy, gm);
      }
      dadd(xs1 + node, w * jxy, gm);
    }
  }
}

// ---------------------------------------------------------------- PCG on (chi - L) B = -rhs
// A v = chi v - L v at interior node (iy, ix) (wall nodes read 0; every PCG vector is 0 there).
template <typename T>
__device__ __forceinline__ V2<T> apply_A(const V2<T>* __restrict__ v, const T* __restrict__ chi, const Geom& gm, int iy,
                                         int ix) {
  const int nx = gm.nx;
  const int64_t o = (int64_t)iy * nx + ix;
  const V2<T> c = v[o], l = v[o - 1], d = v[o - nx];
  const V2<T> r = ix + 1 < nx ? v[o + 1] : V2<T>{T(0), T(0)};
  const V2<T> u = iy + 1 < gm.ny ? v[o + nx] : V2<T>{T(0), T(0)};
  const T k = chi[o];
  if constexpr (sizeof(T) == 8) {
    const double dx2 = gm.dx * gm.dx, dy2 = gm.dy * gm.dy;
    return V2<T>{k * c.a - ((r.a - 2.0 * c.a + l.a) / dx2 + (u.a - 2.0 * c.a + d.a) / dy2),
                 k * c.b - ((r.b - 2.0 * c.b + l.b) / dx2 + (u.b - 2.0 * c.b + d.b) / dy2)};
  } else {
    const float ix2 = gm.f_inv_dx * gm.f_inv_dx, iy2 = gm.f_inv_dy * gm.f_inv_dy;
    return V2<T>{k * c.a - ((r.a - 2.0f * c.a + l.a) * ix2 + (u.a - 2.0f * c.a + d.a) * iy2),
                 k * c.b - ((r.b - 2.0f * c.b + l.b) * ix2 + (u.b - 2.0f * c.b + d.b) * iy2)};
  }
}

// Block sum of two FP64 values, one atomic per block and value.
// Block sum of two FP64 values: one atomic per block and value into out, or (part non-null:
// deterministic FP64 mode) the block's pair stored at part[2 * block] for k_ordered_sum2.
__device__ __forceinline__ void block_sum2(double a, double b, double* out, double* part_out = nullptr) {
  __shared__ double part[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if ((threadIdx.x & 31) == 0) {
    part[0][w] = a;
    part[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += part[threadIdx.x][k];
    if (part_out) part_out[2 * (blockIdx.y * gridDim.x + blockIdx.x) + threadIdx.x] = t;
    else if (t != 0.0) atomicAdd(out + threadIdx.x, t);
  }
}

// out[c] = sum over the nb block pairs of part[2 b + c] in a fixed order (one block of 256
// threads: strided partial sums in increasing b, then a fixed tree): the deterministic mode's
// dot products.
__global__ void k_ordered_sum2(const double* __restrict__ part, int nb, double* out) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[0][threadIdx.x] += red[0][threadIdx.x + h];
      red[1][threadIdx.x] += red[1][threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x < 2) out[threadIdx.x] = red[threadIdx.x][0];
}

// Per-node right-hand side of the two Helmholtz-like equations and the initial residual
// r = -rhs - A x0 (x0 = the guess in bm), written to pcg_r and, through the grid's operand
// writer, as the preconditioner solve's sources.  Also resets the slice i-1 record (it receives
// the next slice's deposit), as the predictor-corrector's last source kernel does.
template <typename T> struct PcgInit {
  static constexpr int NR = 2;
  const V4<T>* cur;
  const T* chi;
  const V4<T>* xs4;
  const T* xs1;
  const V2<T>* bjp;
  const V2<T>* bjn;
  const V2<T>* x;
  V2<T>* r;
  V4<T>* prev;
  T* chi_prev;
  float* ps_prev;
  const T* rho_ion;
  Geom gm;
  __device__ void operator()(int iy, int ix, T* v) const {
    const int nx = gm.nx;
    const int64_t o = (int64_t)iy * nx + ix;
    v[0] = v[1] = T(0);
    if (ix > 0 && iy > 0) {
      auto jz = [&](int y, int x_) { return cur[(int64_t)y * nx + x_].d; };
      auto fxx = [&](int y, int x_) { return xs4[(int64_t)y * nx + x_].c; };
      auto fyy = [&](int y, int x_) { return xs4[(int64_t)y * nx + x_].d; };
      auto fxy = [&](int y, int x_) { return xs1[(int64_t)y * nx + x_]; };
      const T i2x = gsel<T>(gm.inv2dx, gm.f_inv2dx), i2y = gsel<T>(gm.inv2dy, gm.f_inv2dy);
      const T i2z = gsel<T>(gm.inv2dz, gm.f_inv2dz);
      const V4<T> s = xs4[o];
      const V2<T> bp = bjp[o], bn = bjn[o];
      const T tx = s.a + dxc(fxx, iy, ix, nx, i2x) + dyc(fxy, iy, ix, gm.ny, i2y) + (bp.a - bn.a) * i2z;
      const T ty = s.b + dxc(fxy, iy, ix, nx, i2x) + dyc(fyy, iy, ix, gm.ny, i2y) + (bp.b - bn.b) * i2z;
      const T rx = -dyc(jz, iy, ix, gm.ny, i2y) + ty;
      const T ry = dxc(jz, iy, ix, nx, i2x) - tx;
      const V2<T> ax = apply_A<T>(x, chi, gm, iy, ix);
      v[0] = -rx - ax.a;
      v[1] = -ry - ax.b;
    }
    r[o] = V2<T>{v[0], v[1]};
    prev[o] = V4<T>{rho_ion[o], T(0), T(0), T(0)};
    chi_prev[o] = T(0);
    if (ps_prev) ps_prev[o] = 0.0f;
  }
};

template <typename T, typename Sink>
__global__ void k_pcg_init(PcgInit<T> f, Sink sink) {
  pdl_trigger();
  pdl_wait();
  visit_nodes<2, T>(f.gm, sink, 2, f);
}

// z = P r = -(solved) (the shifted solve gives (L - c)^{-1} r); rz[k] += r . z.  Iteration 0 also
// clears the consumed source records.
template <typename T>
__global__ void k_pcg_z(const T* __restrict__ solved, const V2<T>* __restrict__ r, double* rz, int64_t nn, int first,
                        V4<T>* xs4, T* xs1, V2<T>* bjp, V2<T>* bjn, double* part) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0;
  if (o < nn) {
    const V2<T> q = r[o];
    a = -(double)q.a * (double)solved[o];
    b = -(double)q.b * (double)solved[nn + o];
    if (first) {
      xs4[o] = V4<T>{T(0), T(0), T(0), T(0)};
      xs1[o] = T(0);
      bjp[o] = V2<T>{T(0), T(0)};
      bjn[o] = V2<T>{T(0), T(0)};
    }
  }
  block_sum2(a, b, rz, part);
}

// p = z + beta p, beta = rz[k] / rz[k-1] (0 on the first iteration or a zero denominator).
template <typename T>
__global__ void k_pcg_p(const T* __restrict__ solved, V2<T>* p, const double* __restrict__ rz_k,
                        const double* __restrict__ rz_km1, int64_t nn) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nn) return;
  double be[2] = {0.0, 0.0};
  if (rz_km1)
    for (int c = 0; c < 2; ++c) be[c] = rz_km1[c] != 0.0 ? rz_k[c] / rz_km1[c] : 0.0;
  const V2<T> q = p[o];
  p[o] = V2<T>{T(-solved[o] + be[0] * q.a), T(-solved[nn + o] + be[1] * q.b)};
}

// pq[k] += p . (A p)
template <typename T>
__global__ void k_pcg_q(const V2<T>* __restrict__ p, const T* __restrict__ chi, Geom gm, double* pq, double* part) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  double a = 0.0, b = 0.0;
  if (ix < gm.nx && ix > 0 && iy > 0) {
    const V2<T> ap = apply_A<T>(p, chi, gm, iy, ix);
    const V2<T> q = p[(int64_t)iy * gm.nx + ix];
    a = (double)q.a * (double)ap.a;
    b = (double)q.b * (double)ap.b;
  }
  block_sum2(a, b, pq, part);
}

// x += alpha p, r -= alpha A p with alpha = rz[k] / pq[k] (0 for a zero denominator); the new r
// goes to the operand writer as the next preconditioner solve's sources.
template <typename T> struct PcgStep {
  static constexpr int NR = 2;
  const V2<T>* p;
  const T* chi;
  V2<T>* x;
  V2<T>* r;
  const double* rz;
  const double* pq;
  Geom gm;
  __device__ void operator()(int iy, int ix, T* v) const {
    const int64_t o = (int64_t)iy * gm.nx + ix;
    v[0] = v[1] = T(0);
    if (ix > 0 && iy > 0) {
      const V2<T> ap = apply_A<T>(p, chi, gm, iy, ix);
      const T al0 = T(pq[0] != 0.0 ? rz[0] / pq[0] : 0.0), al1 = T(pq[1] != 0.0 ? rz[1] / pq[1] : 0.0);
      const V2<T> pp = p[o], xx = x[o], rr = r[o];
      x[o] = V2<T>{xx.a + al0 * pp.a, xx.b + al1 * pp.b};
      v[0] = rr.a - al0 * ap.a;
      v[1] = rr.b - al1 * ap.b;
      r[o] = V2<T>{v[0], v[1]};
    }
  }
};

template <typename T, typename Sink>
__global__ void k_pcg_x(PcgStep<T> f, Sink sink) {
  visit_nodes<2, T>(f.gm, sink, 2, f);
}

template <typename T> Plasma<T> plasma_of(const hq_grid_s* g);
template <> Plasma<double> plasma_of<double>(const hq_grid_s* g) { return g->p64; }
template <> Plasma<float> plasma_of<float>(const hq_grid_s* g) { return g->p32; }

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// pcg_s layout: [which][k][rhs], which 0: r.z, 1: p.Ap
inline double* pcg_at(const hq_grid_s* g, int which, int k) { return g->pcg_s + ((size_t)which * kMaxPcg + k) * 2; }

template <typename T>
void launch_explicit_src(const hq_grid_s* g, cudaStream_t s) {
  const unsigned nb = blocks_for(g->np, kThreads);
  const T* gf = reinterpret_cast<const T*>(g->gf);
  V4<T>* xs4 = reinterpret_cast<V4<T>*>(g->xs4);
  T* xs1 = reinterpret_cast<T*>(g->xs1);
  constexpr bool C = sizeof(T) == 4;
  const SpeciesTab& t = g->sp;
#define HQ_XS(P)                                                                                          \
  (g->multi ? launch_pdl(k_explicit_src<P, T, C, true>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom, gf, xs4, xs1, t) \
            : launch_pdl(k_explicit_src<P, T, C, false>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom, gf, xs4, xs1, t))
  switch (g->d.shape_order) {
    case 0: HQ_XS(0); break;
    case 1: HQ_XS(1); break;
    case 2: HQ_XS(2); break;
    default: HQ_XS(3); break;
  }
#undef HQ_XS
}

template <typename T>
void launch_pcg_init(const hq_grid_s* g, int slice, const void* cur, const void* chi_cur, void* prev, void* chi_prev,
                     cudaStream_t s) {
  cudaMemsetAsync(g->pcg_s, 0, sizeof(double) * 4 * kMaxPcg * 2, s);
  PcgInit<T> f{reinterpret_cast<const V4<T>*>(cur), reinterpret_cast<const T*>(chi_cur),
               reinterpret_cast<const V4<T>*>(g->xs4), reinterpret_cast<const T*>(g->xs1),
               reinterpret_cast<const V2<T>*>(bjp_at(g, slice + 1)), reinterpret_cast<const V2<T>*>(g->bjn),
               reinterpret_cast<const V2<T>*>(g->bm), reinterpret_cast<V2<T>*>(g->pcg_r),
               reinterpret_cast<V4<T>*>(prev), reinterpret_cast<T*>(chi_prev), psrc_of(g, prev),
               reinterpret_cast<const T*>(g->rho_ion), g->geom};
  with_sink<T>(g, [&](auto sink) { launch_pdl(k_pcg_init<T, decltype(sink)>, src_grid(g), 128, 0, s, f, sink); });
}

template <typename T>
void launch_pcg_iter(const hq_grid_s* g, int slice, int k, const void* chi_cur, cudaStream_t s) {
  const int64_t nn = g->nnode;
  const T* solved = reinterpret_cast<const T*>(g->solved);
  const T* chi = reinterpret_cast<const T*>(chi_cur);
  V2<T>* r = reinterpret_cast<V2<T>*>(g->pcg_r);
  V2<T>* p = reinterpret_cast<V2<T>*>(g->pcg_p);
  double* part = g->pcg_part;   // deterministic mode: per-block partial dot products
  const unsigned nbz = blocks_for(nn, 256);
  k_pcg_z<T><<<nbz, 256, 0, s>>>(solved, r, pcg_at(g, 0, k), nn, k == 0, reinterpret_cast<V4<T>*>(g->xs4),
                                 reinterpret_cast<T*>(g->xs1), reinterpret_cast<V2<T>*>(bjp_at(g, slice + 1)),
                                 reinterpret_cast<V2<T>*>(g->bjn), part);
  if (part) k_ordered_sum2<<<1, 256, 0, s>>>(part, (int)nbz, pcg_at(g, 0, k));
  k_pcg_p<T><<<blocks_for(nn, 256), 256, 0, s>>>(solved, p, pcg_at(g, 0, k), k > 0 ? pcg_at(g, 0, k - 1) : nullptr, nn);
  const dim3 g2((unsigned)((g->nx + 127) / 128), (unsigned)g->ny);
  k_pcg_q<T><<<g2, 128, 0, s>>>(p, chi, g->geom, pcg_at(g, 1, k), part);
  if (part) k_ordered_sum2<<<1, 256, 0, s>>>(part, (int)(g2.x * g2.y), pcg_at(g, 1, k));
  PcgStep<T> f{p, chi, reinterpret_cast<V2<T>*>(g->bm), r, pcg_at(g, 0, k), pcg_at(g, 1, k), g->geom};
  with_sink<T>(g, [&](auto sink) { k_pcg_x<T, decltype(sink)><<<src_grid(g), 128, 0, s>>>(f, sink); });
}

template void launch_explicit_src<float>(const hq_grid_s*, cudaStream_t);
template void launch_explicit_src<double>(const hq_grid_s*, cudaStream_t);
template void launch_pcg_init<float>(const hq_grid_s*, int, const void*, const void*, void*, void*, cudaStream_t);
template void launch_pcg_init<double>(const hq_grid_s*, int, const void*, const void*, void*, void*, cudaStream_t);
template void launch_pcg_iter<float>(const hq_grid_s*, int, int, const void*, cudaStream_t);
template void launch_pcg_iter<double>(const hq_grid_s*, int, int, const void*, cudaStream_t);

}  // namespace hq
