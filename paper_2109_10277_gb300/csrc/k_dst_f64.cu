// FP64 DST-I for the plain-double path (Sec. 3.2, fast Poisson solver).
//
// One "pass" transforms every row of a [R][M][n] batch along its length n and
// writes the result transposed, out[r][k][m] = scale[k][m] * sum_j in[r][m][j]
// sin(pi j k / n).  Two passes give S_y s S_x, four a full solve.  With n a power
// of two each CTA packs two real rows into one complex sequence (odd extension of
// length 2n, Re = row a, Im = row b), runs an in-shared-memory radix-2 FFT in
// FP64 and reads both DST-I results back from the spectrum:
//   X_a[k] = -Im(Z_k)/2,  X_b[k] = Re(Z_k)/2.
// Other n use a direct O(n^2) sum against a precomputed sine table.  The FP64
// path is the double-precision baseline; the FP32 path uses tensor cores instead.
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// G rows per CTA (G/2 complex FFTs of length L = 2n); tw[t] = exp(-i pi t / n), t < n.
template <int G>
__global__ void __launch_bounds__(kThreads) k_dst_fft_pass(const double* __restrict__ in, double* __restrict__ out,
                                                           int n, int logL, int M, const double2* __restrict__ tw,
                                                           const double* __restrict__ scale) {
  extern __shared__ double2 sm[];
  pdl_trigger();
  pdl_wait();
  const int L = 2 * n;
  double2* twid = sm;
  double2* buf = sm + n;
  const int r = blockIdx.y;
  const int m0 = blockIdx.x * G;
  const double* src = in + (int64_t)r * M * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) twid[t] = tw[t];
  for (int t = threadIdx.x; t < (G / 2) * L; t += blockDim.x) {
    const int f = t / L, j = t - f * L;
    const int ma = m0 + 2 * f, mb = ma + 1;
    double ya = 0.0, yb = 0.0;
    int jj = 0;
    double sg = 0.0;
    if (j > 0 && j < n) { jj = j; sg = 1.0; }
    else if (j > n) { jj = L - j; sg = -1.0; }
    if (jj > 0) {
      if (ma < M) ya = sg * src[(int64_t)ma * n + jj];
      if (mb < M) yb = sg * src[(int64_t)mb * n + jj];
    }
    const int rev = (int)(__brev((unsigned)j) >> (32 - logL));
    buf[f * L + rev] = make_double2(ya, yb);
  }
  __syncthreads();
  const int half = L / 2;
  for (int s = 0; s < logL; ++s) {
    const int h = 1 << s;
    for (int t = threadIdx.x; t < (G / 2) * half; t += blockDim.x) {
      const int f = t / half, b = t - f * half;
      const int pos = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + pos, i1 = i0 + h;
      double2* x = buf + f * L;
      const double2 a = x[i0];
      const double2 wc = cmul(twid[pos << (logL - 1 - s)], x[i1]);
      x[i0] = make_double2(a.x + wc.x, a.y + wc.y);
      x[i1] = make_double2(a.x - wc.x, a.y - wc.y);
    }
    __syncthreads();
  }
  double* dst = out + (int64_t)r * n * M;
  for (int t = threadIdx.x; t < n * G; t += blockDim.x) {
    const int k = t / G, gi = t - k * G;
    const int m = m0 + gi;
    if (m >= M) continue;
    const double2 z = buf[(gi >> 1) * L + k];
    double v = (gi & 1) ? 0.5 * z.x : -0.5 * z.y;
    if (scale) v *= scale[(int64_t)k * M + m];
    dst[(int64_t)k * M + m] = v;
  }
}

// Direct sum for any n: sn[j*n + k] = sin(pi j k / n).
__global__ void k_dst_direct_pass(const double* __restrict__ in, double* __restrict__ out, int n, int M,
                                  const double* __restrict__ sn, const double* __restrict__ scale) {
  pdl_trigger();
  pdl_wait();
  const int r = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * M) return;
  const int k = (int)(t / M), m = (int)(t - (int64_t)k * M);
  const double* row = in + ((int64_t)r * M + m) * n;
  double acc = 0.0;
  for (int j = 1; j < n; ++j) acc += row[j] * sn[(int64_t)j * n + k];
  if (scale) acc *= scale[(int64_t)k * M + m];
  out[((int64_t)r * n + k) * M + m] = acc;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int n) { int l = 0; while ((1 << l) < n) ++l; return l; }

template <int G>
void fft_pass(const double* in, double* out, int n, int M, int R, const double* tw, const double* scale, cudaStream_t s) {
  const size_t smem = (size_t)(n + (G / 2) * 2 * n) * sizeof(double2);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_dst_fft_pass<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  dim3 grid((unsigned)((M + G - 1) / G), (unsigned)R);
  launch_pdl(k_dst_fft_pass<G>, grid, dim3(kThreads), smem, s, in, out, n, ilog2(2 * n), M,
             reinterpret_cast<const double2*>(tw), scale);
}

void pass(const double* in, double* out, int n, int M, int R, const double* tw, const double* sn, const double* scale,
          cudaStream_t s) {
  if (is_pow2(n) && n <= 4096) {
    if (n <= 512) fft_pass<16>(in, out, n, M, R, tw, scale, s);
    else if (n <= 1024) fft_pass<8>(in, out, n, M, R, tw, scale, s);
    else if (n <= 2048) fft_pass<4>(in, out, n, M, R, tw, scale, s);
    else fft_pass<2>(in, out, n, M, R, tw, scale, s);
  } else {
    dim3 grid((unsigned)(((int64_t)n * M + kThreads - 1) / kThreads), (unsigned)R);
    launch_pdl(k_dst_direct_pass, grid, dim3(kThreads), (size_t)0, s, in, out, n, M, sn, scale);
  }
}

}  // namespace

// sources in g->f64_a [R][ny][nx] -> solution in g->solved [R][ny][nx]
void dst_solve_f64(hq_grid_s* g, int R, cudaStream_t s, const double* scale) {
  if (!scale) scale = g->f64_scale;
  const int nx = g->nx, ny = g->ny;
  double* a = g->f64_a;
  double* b = g->f64_b;
  pass(a, b, nx, ny, R, g->tw_x, g->sin_x, nullptr, s);      // (s S_x)^T      [R][nx][ny]
  pass(b, a, ny, nx, R, g->tw_y, g->sin_y, scale, s); // S_y s S_x / lambda (normalized)
  pass(a, b, nx, ny, R, g->tw_x, g->sin_x, nullptr, s);
  pass(b, reinterpret_cast<double*>(g->solved), ny, nx, R, g->tw_y, g->sin_y, nullptr, s);
}

}  // namespace hq
