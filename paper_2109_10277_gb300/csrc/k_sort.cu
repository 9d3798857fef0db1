// Plasma re-sort by cell (Sec. 3.1: the particle data is kept sorted; here a counting sort of
// the plasma slice by the cell each particle now lies in, every m slices), so that the
// particles one warp pushes stay neighbours on the grid as the wake displaces them, and their
// gathers and deposits touch few cache lines.
//
// Key: cell iy nx + ix of the particle's position (clamped to the grid), or nx ny for a
// non-finite position.  Histogram (integer atomics), a two-level exclusive scan, a scatter
// through an atomic cursor, then each cell's entries are put back in ascending previous
// index, so the sort is stable and the permutation depends on the positions alone.  Every
// per-particle array (the FP64 accumulators, momenta, weights, the AB5 ring, the FP32 caches
// and the particle's index in the initial placement) is gathered into a scratch copy in the
// new order and copied back, so the arrays keep their addresses (a captured sweep stays
// valid).
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 1024;   // scan tile: cells per block

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__global__ void k_sort_key(const double* __restrict__ x, const double* __restrict__ y, int64_t n, Geom gm,
                           int32_t* key, int32_t* count) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const double u = (x[p] - gm.xmin) * gm.inv_dx, v = (y[p] - gm.ymin) * gm.inv_dy;
  int k = gm.nx * gm.ny;
  if (isfinite(u) && isfinite(v)) {
    const int ix = (int)floor(fmin(fmax(u, 0.0), (double)(gm.nx - 1)));
    const int iy = (int)floor(fmin(fmax(v, 0.0), (double)(gm.ny - 1)));
    k = iy * gm.nx + ix;
  }
  key[p] = k;
  atomicAdd(count + k, 1);
}

// Exclusive scan of one tile of kTile counts (4 per thread) into offset; the tile's total
// into tsum[blockIdx.x].
__global__ void k_scan_tile(const int32_t* __restrict__ count, int64_t nb, int32_t* offset, int32_t* tsum) {
  __shared__ int32_t part[kThreads];
  const int64_t base = (int64_t)blockIdx.x * kTile + 4 * threadIdx.x;
  int32_t v[4], s = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    v[j] = base + j < nb ? count[base + j] : 0;
    s += v[j];
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int d = 1; d < kThreads; d <<= 1) {
    const int32_t t = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  int32_t run = part[threadIdx.x] - s;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (base + j < nb) offset[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == kThreads - 1) tsum[blockIdx.x] = part[kThreads - 1];
}

// Exclusive scan of the nt tile totals in place (one block, chunked).
__global__ void k_scan_totals(int32_t* tsum, int nt) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x, nth = blockDim.x;
  const int chunk = (nt + nth - 1) / nth;
  const int lo = t * chunk, hi = min(nt, lo + chunk);
  int32_t s = 0;
  for (int i = lo; i < hi; ++i) s += tsum[i];
  part[t] = s;
  __syncthreads();
  for (int d = 1; d < nth; d <<= 1) {
    const int32_t v = t >= d ? part[t - d] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;
  for (int i = lo; i < hi; ++i) {
    const int32_t c = tsum[i];
    tsum[i] = run;
    run += c;
  }
}

__global__ void k_scan_add(int32_t* offset, const int32_t* __restrict__ tsum, int32_t* cursor, int64_t nb) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  offset[i] += tsum[i / kTile];
  cursor[i] = 0;
}

__global__ void k_sort_scatter(const int32_t* __restrict__ key, int64_t n, const int32_t* __restrict__ offset,
                               int32_t* cursor, int32_t* perm) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int k = key[p];
  perm[offset[k] + atomicAdd(cursor + k, 1)] = (int32_t)p;
}

// Each cell's entries in ascending previous index (insertion sort: cells hold a few particles).
__global__ void k_sort_stable(const int32_t* __restrict__ offset, int64_t nb, int64_t n, int32_t* perm) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int32_t lo = offset[b], hi = b + 1 < nb ? offset[b + 1] : (int32_t)n;
  for (int32_t i = lo + 1; i < hi; ++i) {
    const int32_t v = perm[i];
    int32_t j = i - 1;
    while (j >= lo && perm[j] > v) {
      perm[j + 1] = perm[j];
      --j;
    }
    perm[j + 1] = v;
  }
}

// The per-particle arrays moved by the sort: column c is nsub[c] arrays of n elements of
// esize[c] bytes, the sub-arrays n elements apart.
constexpr int kMaxCols = 16;
struct SortCols {
  void* p[kMaxCols];
  int esize[kMaxCols];
  int nsub[kMaxCols];
  int64_t soff[kMaxCols];   // byte offset of the column in the scratch copy
  int ncols;
};

template <typename E>
__device__ __forceinline__ void move_elems(const void* src, void* dst, int64_t from, int64_t to, int nsub, int64_t n) {
  const E* s = static_cast<const E*>(src);
  E* d = static_cast<E*>(dst);
  for (int k = 0; k < nsub; ++k) d[(int64_t)k * n + to] = s[(int64_t)k * n + from];
}

// gather = 1: scratch[t] = array[perm[t]]; gather = 0: array[t] = scratch[t].
__global__ void k_sort_move(SortCols c, const int32_t* __restrict__ perm, int64_t n, uint8_t* scratch, int gather) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t from = gather ? (int64_t)perm[t] : t;
  for (int k = 0; k < c.ncols; ++k) {
    void* sc = scratch + c.soff[k];
    const void* src = gather ? c.p[k] : sc;
    void* dst = gather ? sc : c.p[k];
    switch (c.esize[k]) {
      case 8: move_elems<uint64_t>(src, dst, from, t, c.nsub[k], n); break;
      case 4: move_elems<uint32_t>(src, dst, from, t, c.nsub[k], n); break;
      default: move_elems<uint8_t>(src, dst, from, t, c.nsub[k], n); break;
    }
  }
}

SortCols sort_cols(const hq_grid_s* g) {
  SortCols c{};
  const int ts = g->fp64 ? 8 : 4;
  auto add = [&](void* p, int esize, int nsub) {
    if (!p) return;
    c.p[c.ncols] = p;
    c.esize[c.ncols] = esize;
    c.nsub[c.ncols] = nsub;
    ++c.ncols;
  };
  add(g->p64.x, 8, 1);
  add(g->p64.y, 8, 1);
  add(g->p64.psi, 8, 1);
  add(g->p64.alive, 1, 1);
  add(g->porigin, 4, 1);
  if (g->fp64) {
    add(g->p64.ux, 8, 1);
    add(g->p64.uy, 8, 1);
    add(g->p64.w, 8, 1);
    add(g->p64.hist, 8, kRing * 5);
  } else {
    add(g->p32.ux, ts, 1);
    add(g->p32.uy, ts, 1);
    add(g->p32.w, ts, 1);
    add(g->p32.hist, ts, kRing * 5);
    add(g->p32.cell, 4, 1);
    add(g->p32.fx, 4, 1);
    add(g->p32.fy, 4, 1);
    add(g->p32.opp, 4, 1);
    add(g->p32.hsum, 4, 5);
  }
  int64_t off = 0;
  for (int k = 0; k < c.ncols; ++k) {
    c.soff[k] = off;
    off += ((int64_t)c.esize[k] * c.nsub[k] * g->np + 255) / 256 * 256;
  }
  return c;
}

}  // namespace

int64_t resort_scratch_bytes(const hq_grid_s* g) {
  const SortCols c = sort_cols(g);
  const int k = c.ncols - 1;
  return c.soff[k] + ((int64_t)c.esize[k] * c.nsub[k] * g->np + 255) / 256 * 256;
}

int64_t resort_tiles(const hq_grid_s* g) { return ((int64_t)g->nnode + 1 + kTile - 1) / kTile; }

void launch_resort(hq_grid_s* g, cudaStream_t s) {
  const int64_t n = g->np, nb = (int64_t)g->nnode + 1;
  const int nt = (int)resort_tiles(g);
  cudaMemsetAsync(g->sort_count, 0, sizeof(int32_t) * nb, s);
  k_sort_key<<<blocks_for(n), kThreads, 0, s>>>(g->p64.x, g->p64.y, n, g->geom, g->sort_key, g->sort_count);
  k_scan_tile<<<nt, kThreads, 0, s>>>(g->sort_count, nb, g->sort_offset, g->sort_tsum);
  k_scan_totals<<<1, 1024, 0, s>>>(g->sort_tsum, nt);
  k_scan_add<<<blocks_for(nb), kThreads, 0, s>>>(g->sort_offset, g->sort_tsum, g->sort_count, nb);
  k_sort_scatter<<<blocks_for(n), kThreads, 0, s>>>(g->sort_key, n, g->sort_offset, g->sort_count, g->sort_perm);
  k_sort_stable<<<blocks_for(nb), kThreads, 0, s>>>(g->sort_offset, nb, n, g->sort_perm);
  const SortCols c = sort_cols(g);
  uint8_t* scratch = static_cast<uint8_t*>(g->sort_scratch);
  k_sort_move<<<blocks_for(n), kThreads, 0, s>>>(c, g->sort_perm, n, scratch, 1);
  k_sort_move<<<blocks_for(n), kThreads, 0, s>>>(c, g->sort_perm, n, scratch, 0);
}

}  // namespace hq
