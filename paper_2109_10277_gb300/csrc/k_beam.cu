// Beam kernels (Sec. 3.1: "beam particles are sorted per slice"; Sec. 3.2: beam
// deposition, order 0 longitudinally, and the second-order beam pusher).
//
// Binning is a counting sort on the device: slice index
// floor((zeta_max - zeta) / dzeta) per particle (FP64), a histogram with integer
// atomics, an exclusive scan and a scatter into a permutation, giving the CSR
// offsets of each slice.  The order of particles inside one slice is not fixed
// (atomic cursor); everything downstream is a sum over the slice.
#include <algorithm>

#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 256;

__global__ void k_bin_count(const double* __restrict__ zeta, int64_t n, double zmax, double dz, int nz,
                            int32_t* bin, int32_t* count) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double t = floor((zmax - zeta[p]) / dz);
  const bool ok = isfinite(t) && t >= 0.0 && t < (double)nz;
  const int b = ok ? (int)t : -1;
  bin[p] = b;
  if (ok) atomicAdd(count + b, 1);
}

// The slice of every particle with the binning's arithmetic: 0..nz-1 inside the box, -1 ahead
// of its head (zeta above zeta_max), nz behind its tail, -2 not finite.
__global__ void k_slice_of(const double* __restrict__ zeta, int64_t n, double zmax, double dz, int nz, int32_t* out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double t = floor((zmax - zeta[p]) / dz);
  out[p] = !isfinite(t) ? -2 : (t < 0.0 ? -1 : (t >= (double)nz ? nz : (int)t));
}

// Exclusive scan of count[0..nz) into offset[0..nz], cursor zeroed.  One block.
__global__ void k_scan(const int32_t* __restrict__ count, int32_t* offset, int32_t* cursor, int nz) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int chunk = (nz + nt - 1) / nt;
  const int lo = t * chunk, hi = min(nz, lo + chunk);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < nt; d <<= 1) {
    const int32_t v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;
  for (int i = lo; i < hi; ++i) {
    offset[i] = run;
    run += count[i];
    cursor[i] = 0;
  }
  if (t == nt - 1) offset[nz] = part[t];
}

__global__ void k_bin_scatter(const int32_t* __restrict__ bin, int64_t n, const int32_t* __restrict__ offset,
                              int32_t* cursor, int32_t* perm) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int b = bin[p];
  if (b < 0) return;
  const int pos = atomicAdd(cursor + b, 1);
  perm[offset[b] + pos] = (int32_t)p;
}

template <int P>
__device__ __forceinline__ int stencil1(double x, double x0, double dx, double* w) {
  int j;
  double d;
  split_coord(x, x0, dx, j, d);
  return shape_weights<P, double>(j, d, w);
}

// FP32 stencil of an FP64 position: node coordinate by multiplication (no FP64
// division), fraction rounded to FP32.
template <int P>
__device__ __forceinline__ int stencil1(double x, double x0, double inv_dx, float* w) {
  const double u = (x - x0) * inv_dx;
  const double f = floor(u);
  return shape_weights<P, float>((int)f, (float)(u - f), w);
}

template <int P, typename T>
__device__ __forceinline__ int stencil_t(double x, double x0, double dx, double inv_dx, T* w) {
  if constexpr (sizeof(T) == 8) return stencil1<P>(x, x0, dx, w);
  else return stencil1<P>(x, x0, inv_dx, w);
}

// Charge/current of the particles of slice i into dep (rho, Jx, Jy, Jz) and J_perp of
// slice i+1 into bjn: rho = q w S / (dx dy dzeta), J = rho u / gamma (in the field type).
// The explicit B_perp solver (bjc non-null) also keeps the beam's own J_perp of slice i in
// bjc, taken before the beam push moves these particles: slice i+1 reads it as J_perp(i-1).
template <int P, typename T>
__global__ void k_beam_deposit(hq_beam_view v, const int32_t* __restrict__ off, const int32_t* __restrict__ perm,
                               int slice, int nz, Geom gm, V4<T>* dep, V2<T>* bjn, V2<T>* bjc, float* ps) {
  pdl_trigger();
  pdl_wait();
  const int a0 = off[slice], a1 = off[slice + 1];
  const int b0 = slice + 1 < nz ? off[slice + 1] : 0, b1 = slice + 1 < nz ? off[slice + 2] : 0;
  const int na = a1 - a0, nb = b1 - b0;
  const double vol = gm.dx * gm.dy * gm.dzeta;
  const T rq = T(v.charge / vol);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < na + nb; t += gridDim.x * blockDim.x) {
    const bool cur = t < na;
    const int p = perm[cur ? a0 + t : b0 + (t - na)];
    const T ux = T(v.ux[p]), uy = T(v.uy[p]), uz = T(v.uz[p]);
    const T ig = T(1) / sqrt(T(1) + ux * ux + uy * uy + uz * uz);
    // FP64: (q w) / (dx dy dzeta) as in the oracle; FP32: precomputed q / volume
    const T r = sizeof(T) == 8 ? T((v.charge * v.w[p]) / vol) : rq * T(v.w[p]);
    T wx[P + 1], wy[P + 1];
    const int ix0 = stencil_t<P, T>(v.x[p], gm.xmin, gm.dx, gm.inv_dx, wx);
    const int iy0 = stencil_t<P, T>(v.y[p], gm.ymin, gm.dy, gm.inv_dy, wy);
    const T cx = ux * ig, cy = uy * ig, cz = uz * ig;
    // FP32 path: this particle's share of the psi source, rho (1 - v_z), without cancellation
    float omvz = 0.0f;
    if constexpr (sizeof(T) == 4) omvz = one_minus_vz(ux, uy, uz, 1.0f / ig);
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        const T s = wx[a] * wy[b] * r;
        const int64_t node = (int64_t)iy * gm.nx + ix;
        if (cur) {
          V4<T>* q = dep + node;
          dadd(&q->a, s, gm);
          dadd(&q->b, s * cx, gm);
          dadd(&q->c, s * cy, gm);
          dadd(&q->d, s * cz, gm);
          if (ps) atomicAdd(ps + node, float(s) * omvz);
          if (bjc) {
            dadd(&bjc[node].a, s * cx, gm);
            dadd(&bjc[node].b, s * cy, gm);
          }
        } else {
          V2<T>* q = bjn + node;
          dadd(&q->a, s * cx, gm);
          dadd(&q->b, s * cy, gm);
        }
      }
    }
  }
}

template <int P, typename T>
__device__ __forceinline__ void gather_all(const T* __restrict__ gf, const T* __restrict__ bm, const Geom& gm, double x,
                                           double y, double* F) {
  double wx[P + 1], wy[P + 1];
  const int ix0 = stencil1<P>(x, gm.xmin, gm.dx, wx);
  const int iy0 = stencil1<P>(y, gm.ymin, gm.dy, wy);
#pragma unroll
  for (int c = 0; c < 6; ++c) F[c] = 0.0;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, gm.nx)) continue;
      const int64_t node = (int64_t)iy * gm.nx + ix;
      const T* q = gf + node * kGF;   // ExmBy, EypBx, Ez, Bz
      const T* bq = bm + node * 2;    // Bx, By
      const double w = wx[a] * wy[b];
      F[0] += w * (double)q[0];
      F[1] += w * (double)q[1];
      F[2] += w * (double)q[2];
      F[3] += w * (double)bq[0];
      F[4] += w * (double)bq[1];
      F[5] += w * (double)q[3];
    }
  }
}

// Drift (dt/2) - Boris kick (dt) - drift (dt/2) in the fields of the particle's slice.
// E = (ExmBy + By, EypBx - Bx, Ez), B = (Bx, By, Bz); zeta advances with v_z - 1.
template <int P, typename T>
__global__ void k_beam_push(hq_beam_view v, const int32_t* __restrict__ off, const int32_t* __restrict__ perm,
                            int slice, Geom gm, const T* __restrict__ gf, const T* __restrict__ bm, double dt) {
  pdl_trigger();
  pdl_wait();
  const int a0 = off[slice], a1 = off[slice + 1];
  const double qm = v.charge / v.mass, h = 0.5 * dt;
  for (int t = a0 + blockIdx.x * blockDim.x + threadIdx.x; t < a1; t += gridDim.x * blockDim.x) {
    const int p = perm[t];
    double x = v.x[p], y = v.y[p], z = v.zeta[p], ux = v.ux[p], uy = v.uy[p], uz = v.uz[p];
    double ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    x += h * ux * ig;
    y += h * uy * ig;
    z += h * (uz * ig - 1.0);
    double F[6];
    gather_all<P, T>(gf, bm, gm, x, y, F);
    const double ex = F[0] + F[4], ey = F[1] - F[3], ez = F[2];
    ux += qm * h * ex;
    uy += qm * h * ey;
    uz += qm * h * ez;
    ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    const double tx = qm * h * F[3] * ig, ty = qm * h * F[4] * ig, tz = qm * h * F[5] * ig;
    const double s = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
    const double px = ux + (uy * tz - uz * ty);
    const double py = uy + (uz * tx - ux * tz);
    const double pz = uz + (ux * ty - uy * tx);
    ux += s * (py * tz - pz * ty);
    uy += s * (pz * tx - px * tz);
    uz += s * (px * ty - py * tx);
    ux += qm * h * ex;
    uy += qm * h * ey;
    uz += qm * h * ez;
    ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    x += h * ux * ig;
    y += h * uy * ig;
    z += h * (uz * ig - 1.0);
    v.x[p] = x;
    v.y[p] = y;
    v.zeta[p] = z;
    v.ux[p] = ux;
    v.uy[p] = uy;
    v.uz[p] = uz;
  }
}

// sums += (q w, q w Ez, q w Ez^2) over the particles of slice i (Ez gathered in the
// field type, sums in FP64).  Deterministic FP64 mode: every particle's terms go to the fixed-
// point mirror of sums (the grid's witness accumulator), independent of particle order.
template <int P, typename T>
__global__ void k_witness(hq_beam_view v, const int32_t* __restrict__ off, const int32_t* __restrict__ perm, int slice,
                          Geom gm, const T* __restrict__ gf, double* sums) {
  pdl_trigger();
  pdl_wait();
  const int a0 = off[slice], a1 = off[slice + 1];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (int t = a0 + blockIdx.x * blockDim.x + threadIdx.x; t < a1; t += gridDim.x * blockDim.x) {
    const int p = perm[t];
    T wx[P + 1], wy[P + 1];
    const int ix0 = stencil_t<P, T>(v.x[p], gm.xmin, gm.dx, gm.inv_dx, wx);
    const int iy0 = stencil_t<P, T>(v.y[p], gm.ymin, gm.dy, gm.inv_dy, wy);
    T ez = T(0);
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        ez += wx[a] * wy[b] * gf[((int64_t)iy * gm.nx + ix) * kGF + 2];
      }
    }
    const double qw = v.charge * v.w[p];
    const double e = (double)ez;
    if (gm.det) {
      fx_add(sums, qw, gm.det, gm.dstatus);
      fx_add(sums + 1, qw * e, gm.det, gm.dstatus);
      fx_add(sums + 2, qw * e * e, gm.det, gm.dstatus);
      continue;
    }
    s0 += qw;
    s1 += qw * e;
    s2 += qw * e * e;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0 && (s0 != 0.0 || s1 != 0.0 || s2 != 0.0)) {
    atomicAdd(sums, s0);
    atomicAdd(sums + 1, s1);
    atomicAdd(sums + 2, s2);
  }
}

// Weighted raw moments of a whole beam (Sec. 6 precision study: witness emittance), FP64:
// m += (w, w x, w y, w ux, w uy, w x^2, w y^2, w ux^2, w uy^2, w x ux, w y uy); a block sums
// its particles with warp shuffles and shared memory, then adds once per moment.
constexpr int kMoments = 11;
__global__ void k_beam_moments(hq_beam_view v, double* m) {
  __shared__ double part[kThreads / 32][kMoments];
  double a[kMoments];
#pragma unroll
  for (int k = 0; k < kMoments; ++k) a[k] = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < v.n; p += (int64_t)gridDim.x * blockDim.x) {
    const double w = v.w[p], x = v.x[p], y = v.y[p], ux = v.ux[p], uy = v.uy[p];
    a[0] += w;
    a[1] += w * x;
    a[2] += w * y;
    a[3] += w * ux;
    a[4] += w * uy;
    a[5] += w * x * x;
    a[6] += w * y * y;
    a[7] += w * ux * ux;
    a[8] += w * uy * uy;
    a[9] += w * x * ux;
    a[10] += w * y * uy;
  }
#pragma unroll
  for (int k = 0; k < kMoments; ++k)
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int k = 0; k < kMoments; ++k) part[warp][k] = a[k];
  __syncthreads();
  if (threadIdx.x < kMoments) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += part[w][threadIdx.x];
    atomicAdd(m + threadIdx.x, t);
  }
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }
constexpr unsigned kSliceBlocks = 152;  // grid-stride launches for per-slice beam work

}  // namespace

void launch_beam_slices(const hq_grid_s* g, const hq_beam_view& v, int32_t* out, cudaStream_t s) {
  if (v.n > 0) k_slice_of<<<blocks_for(v.n), kThreads, 0, s>>>(v.zeta, v.n, g->d.zeta_max, g->geom.dzeta, g->nz, out);
}

void launch_beam_bin(hq_grid_s* g, int b, const hq_beam_view& v, cudaStream_t s) {
  BeamBins& bb = g->bins[b];
  cudaMemsetAsync(bb.count, 0, sizeof(int32_t) * (g->nz + 1), s);
  if (v.n > 0) {
    k_bin_count<<<blocks_for(v.n), kThreads, 0, s>>>(v.zeta, v.n, g->d.zeta_max, g->geom.dzeta, g->nz, bb.bin, bb.count);
  }
  k_scan<<<1, 1024, 0, s>>>(bb.count, bb.offset, bb.cursor, g->nz);
  if (v.n > 0) k_bin_scatter<<<blocks_for(v.n), kThreads, 0, s>>>(bb.bin, v.n, bb.offset, bb.cursor, bb.perm);
}

#define HQ_SHAPE_SWITCH(ORDER, CALL) \
  switch (ORDER) {                   \
    case 0: { constexpr int P = 0; CALL; } break; \
    case 1: { constexpr int P = 1; CALL; } break; \
    case 2: { constexpr int P = 2; CALL; } break; \
    default: { constexpr int P = 3; CALL; } break; \
  }

template <typename T>
void launch_beam_deposit(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, void* dep, void* bjn, cudaStream_t s) {
  const BeamBins& bb = g->bins[b];
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (launch_pdl(k_beam_deposit<P, T>, dim3(kSliceBlocks), dim3(kThreads), (size_t)0, s, v, bb.offset, bb.perm,
                             slice, g->nz, g->geom, reinterpret_cast<V4<T>*>(dep), reinterpret_cast<V2<T>*>(bjn),
                             reinterpret_cast<V2<T>*>(bjp_at(g, slice)), psrc_of(g, dep))));
}
template <typename T>
void launch_beam_push(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, double dt, cudaStream_t s) {
  const BeamBins& bb = g->bins[b];
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (launch_pdl(k_beam_push<P, T>, dim3(kSliceBlocks), dim3(kThreads), (size_t)0, s, v, bb.offset, bb.perm,
                             slice, g->geom, reinterpret_cast<const T*>(g->gf), reinterpret_cast<const T*>(g->bm),
                             dt)));
}
template <typename T>
void launch_witness(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, double* sums, cudaStream_t s) {
  const BeamBins& bb = g->bins[b];
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (launch_pdl(k_witness<P, T>, dim3(kSliceBlocks), dim3(kThreads), (size_t)0, s, v, bb.offset, bb.perm,
                             slice, g->geom, reinterpret_cast<const T*>(g->gf), sums)));
}
#undef HQ_SHAPE_SWITCH

void launch_beam_moments(const hq_beam_view& v, double* m, cudaStream_t s) {
  const unsigned nb = (unsigned)std::min<int64_t>(4 * 152, std::max<int64_t>(1, (v.n + kThreads - 1) / kThreads));
  k_beam_moments<<<nb, kThreads, 0, s>>>(v, m);
}

template void launch_beam_deposit<float>(const hq_grid_s*, int, const hq_beam_view&, int, void*, void*, cudaStream_t);
template void launch_beam_deposit<double>(const hq_grid_s*, int, const hq_beam_view&, int, void*, void*, cudaStream_t);
template void launch_beam_push<float>(const hq_grid_s*, int, const hq_beam_view&, int, double, cudaStream_t);
template void launch_beam_push<double>(const hq_grid_s*, int, const hq_beam_view&, int, double, cudaStream_t);
template void launch_witness<float>(const hq_grid_s*, int, const hq_beam_view&, int, double*, cudaStream_t);
template void launch_witness<double>(const hq_grid_s*, int, const hq_beam_view&, int, double*, cudaStream_t);

}  // namespace hq
