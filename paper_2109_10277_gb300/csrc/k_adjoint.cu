// Reverse-zeta adjoint of the quasi-static slice loop (hand-written discrete
// adjoint of the forward kernels; the paper has no adjoint, the structure
// follows its slice routine, Sec. 2, and predictor-corrector, Sec. 3.2).
//
// Transposes used:
//   gather  <-> deposit (same B-spline stencil), plus the stencil derivative for
//               the particle-position adjoints;
//   DST-I Dirichlet solve L^-1 is symmetric (self-adjoint);
//   masked central difference D (zero wall values/outputs): D^T = -D;
//   AB5 step y' = y - dzeta (b0 f + sum b_k H_k): ybar += y'bar, fbar = -dzeta b0 y'bar,
//               Hbar_k += -dzeta b_k y'bar;
//   push derivatives f(u, Psi, F): transposed Jacobian (derivs_adj).
// Per-particle adjoint state (x, y, ux, uy, Psi and the AB5 history, logical
// order f_{i-1}..f_{i-4}) is owned by one thread and updated in place from slice
// i+1 to slice i; field adjoints are accumulated with atomics.
#include "hq_internal.cuh"

namespace hq {

namespace {

constexpr int kThreads = 128;   // as the forward particle kernels: a shorter tail of partly filled waves

// B-spline weights and their derivatives d w / d u (u = node coordinate).
template <int P, typename T>
__device__ __forceinline__ int shape_wd(int jf, T d, T* w, T* dw) {
  if constexpr (P == 0) {
    w[0] = T(1);
    dw[0] = T(0);
    return jf + (d >= T(0.5) ? 1 : 0);
  } else if constexpr (P == 1) {
    w[0] = T(1) - d;
    w[1] = d;
    dw[0] = T(-1);
    dw[1] = T(1);
    return jf;
  } else if constexpr (P == 2) {
    const bool up = d >= T(0.5);
    const T e = up ? d - T(1) : d;
    const T a = T(0.5) - e, b = T(0.5) + e;
    w[0] = T(0.5) * a * a;
    w[1] = T(0.75) - e * e;
    w[2] = T(0.5) * b * b;
    dw[0] = -a;
    dw[1] = T(-2) * e;
    dw[2] = b;
    return jf + (up ? 1 : 0) - 1;
  } else {
    const T d2 = d * d, d3 = d2 * d, om = T(1) - d;
    w[0] = om * om * om * T(1.0 / 6.0);
    w[1] = (T(4) - T(6) * d2 + T(3) * d3) * T(1.0 / 6.0);
    w[2] = (T(1) + T(3) * d + T(3) * d2 - T(3) * d3) * T(1.0 / 6.0);
    w[3] = d3 * T(1.0 / 6.0);
    dw[0] = T(-0.5) * om * om;
    dw[1] = T(-2) * d + T(1.5) * d2;
    dw[2] = T(0.5) + d - T(1.5) * d2;
    dw[3] = T(0.5) * d2;
    return jf - 1;
  }
}

template <int P, typename T>
struct Stencil {
  int ix0, iy0;
  T wx[P + 1], wy[P + 1], dwx[P + 1], dwy[P + 1];  // dw*: derivative w.r.t. the physical coordinate
};

// FP64 forms the node coordinate by division (the oracle's arithmetic); FP32, like the FP32
// forward, by multiplication with the cell's inverse (no FP64 division per particle).
template <int P, typename T>
__device__ __forceinline__ void stencil_at(const Geom& gm, double x, double y, Stencil<P, T>& s) {
  int jx, jy;
  double fx, fy;
  if constexpr (sizeof(T) == 8) {
    split_coord(x, gm.xmin, gm.dx, jx, fx);
    split_coord(y, gm.ymin, gm.dy, jy, fy);
  } else {
    const double u = (x - gm.xmin) * gm.inv_dx, v = (y - gm.ymin) * gm.inv_dy;
    const double ufl = floor(u), vfl = floor(v);
    jx = (int)ufl;
    jy = (int)vfl;
    fx = u - ufl;
    fy = v - vfl;
  }
  s.ix0 = shape_wd<P, T>(jx, T(fx), s.wx, s.dwx);
  s.iy0 = shape_wd<P, T>(jy, T(fy), s.wy, s.dwy);
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    s.dwx[a] *= gsel<T>(gm.inv_dx, gm.f_inv_dx);
    s.dwy[a] *= gsel<T>(gm.inv_dy, gm.f_inv_dy);
  }
}

// NC components of a node record q: FP32 records whose components start on a 16-byte (4 of
// them) or 8-byte (2) boundary are read with one vector load.
template <int NC, typename T>
__device__ __forceinline__ void load_comp(const T* q, T* v) {
  if constexpr (sizeof(T) == 4 && NC == 4) {
    const float4 a = *reinterpret_cast<const float4*>(q);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (sizeof(T) == 4 && NC == 2) {
    const float2 a = *reinterpret_cast<const float2*>(q);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = q[c];
  }
}

// Interpolated values and x/y gradients of NC components at stride `st` (offset `off`);
// NC of 4 or 2 with st and off multiples of NC read one vector per node in FP32.
template <int P, typename T, int NC>
__device__ __forceinline__ void gather_g(const T* __restrict__ f, int st, int off, const Geom& gm, const Stencil<P, T>& s,
                                         T* val, T* gx, T* gy) {
#pragma unroll
  for (int c = 0; c < NC; ++c) val[c] = gx[c] = gy[c] = T(0);
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = s.iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = s.ix0 + a;
      if (!in_interior(ix, gm.nx)) continue;
      const T* q = f + ((int64_t)iy * gm.nx + ix) * st + off;
      const T w = s.wx[a] * s.wy[b], wxd = s.dwx[a] * s.wy[b], wyd = s.wx[a] * s.dwy[b];
      T v[NC];
      load_comp<NC, T>(q, v);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        val[c] += w * v[c];
        gx[c] += wxd * v[c];
        gy[c] += wyd * v[c];
      }
    }
  }
}

// f[node * st + off + c] += S * v[c] (atomics)
template <int P, typename T, int NC>
__device__ __forceinline__ void scatter(T* f, int st, int off, const Geom& gm, const Stencil<P, T>& s, const T* v) {
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = s.iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = s.ix0 + a;
      if (!in_interior(ix, gm.nx)) continue;
      T* q = f + ((int64_t)iy * gm.nx + ix) * st + off;
      const T w = s.wx[a] * s.wy[b];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (v[c] != T(0)) atomicAdd(q + c, w * v[c]);
    }
  }
}

// Adjoints of ExmBy, EypBx, Ez, Bz into a 4-per-node record: one float4 vector atomic per node
// in FP32 (a warp's 32 consecutive nodes span 512 contiguous bytes), one atomic per component
// in FP64.
template <int P, typename T>
__device__ __forceinline__ void scatter_v4(T* f, const Geom& gm, const Stencil<P, T>& s, const T* v) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = s.iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = s.ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        const float w = s.wx[a] * s.wy[b];
        atomicAdd(reinterpret_cast<float4*>(f) + ((int64_t)iy * gm.nx + ix),
                  make_float4(w * v[0], w * v[1], w * v[2], w * v[3]));
      }
    }
  } else {
    scatter<P, T, 4>(f, 4, 0, gm, s, v);
  }
}

// Adjoint pair (a, b) into a 2-per-node record: one float2 vector atomic per node in FP32.
template <int P, typename T>
__device__ __forceinline__ void scatter_v2(T* f, const Geom& gm, const Stencil<P, T>& s, const T* v) {
  if constexpr (sizeof(T) == 4) {
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = s.iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = s.ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        const float w = s.wx[a] * s.wy[b];
        atomicAdd(reinterpret_cast<float2*>(f) + ((int64_t)iy * gm.nx + ix), make_float2(w * v[0], w * v[1]));
      }
    }
  } else {
    scatter<P, T, 2>(f, 2, 0, gm, s, v);
  }
}

// Forward zeta-derivatives (identical to the forward kernels' formula).
template <typename T>
__device__ __forceinline__ void derivs_f(T ux, T uy, T opp, const T* F, T* f) {
  const T g = T(1) / opp;
  const T gam = (T(1) + ux * ux + uy * uy + opp * opp) * T(0.5) * g;
  f[0] = -ux * g;
  f[1] = -uy * g;
  f[2] = gam * g * F[0] + F[4] + F[5] * g * uy;
  f[3] = gam * g * F[1] - F[3] - F[5] * g * ux;
  f[4] = g * (ux * F[0] + uy * F[1]) - F[2];
}

// Transposed Jacobian of derivs: given fbar, accumulate (ux, uy, Psi) adjoints and the
// adjoints of the six gathered fields F = (ExmBy, EypBx, Ez, Bx, By, Bz).
template <typename T>
__device__ __forceinline__ void derivs_adj(T ux, T uy, T opp, const T* F, const T* fb, T& bux, T& buy, T& bpsi,
                                           T* bF) {
  const T g = T(1) / opp, g2 = g * g;
  const T q2 = T(1) + ux * ux + uy * uy;
  const T gam = q2 * T(0.5) * g + T(0.5) * opp;
  const T A = gam * g;
  const T dgam_dpsi = T(-0.5) * q2 * g2 + T(0.5);
  const T dA_dpsi = dgam_dpsi * g - gam * g2;
  const T E0 = F[0], E1 = F[1], Bz = F[5];
  bux = fb[0] * (-g) + fb[2] * (ux * g2 * E0) + fb[3] * (ux * g2 * E1 - Bz * g) + fb[4] * (g * E0);
  buy = fb[1] * (-g) + fb[2] * (uy * g2 * E0 + Bz * g) + fb[3] * (uy * g2 * E1) + fb[4] * (g * E1);
  bpsi = fb[0] * (ux * g2) + fb[1] * (uy * g2) + fb[2] * (dA_dpsi * E0 - Bz * g2 * uy) +
         fb[3] * (dA_dpsi * E1 + Bz * g2 * ux) - fb[4] * (g2 * (ux * E0 + uy * E1));
  bF[0] = fb[2] * A + fb[4] * g * ux;
  bF[1] = fb[3] * A + fb[4] * g * uy;
  bF[2] = -fb[4];
  bF[3] = -fb[3];
  bF[4] = fb[2];
  bF[5] = fb[2] * g * uy - fb[3] * g * ux;
}

template <typename T>
__device__ __forceinline__ T hist_at(const T* __restrict__ h, int64_t n, int64_t p, int slice, int k, int c) {
  const int slot = ((slice - k) % kRing + kRing) % kRing;  // physical slot of f_{slice-k}
  return h[((int64_t)slot * 5 + c) * n + p];
}

// Removal rule, identical to the forward passes.
__device__ __forceinline__ bool ok_state(const Geom& gm, double x, double y, double opp, double guard) {
  return isfinite(x) && isfinite(y) && isfinite(opp) && x > gm.xmin && x < gm.xmax && y > gm.ymin && y < gm.ymax &&
         opp >= guard;
}

template <typename T>
__device__ __forceinline__ T unit_charge_density(const Geom& gm) {  // q / A with q = -1
  if constexpr (sizeof(T) == 8) return T(-1.0) / (gm.dx * gm.dy);
  else return -gm.f_inv_area;
}

// Stencil (weights and derivatives w.r.t. the physical coordinate) at node coordinate
// (jx + fx, jy + fy), FP32: the cached split the forward kernels used.
template <int P>
__device__ __forceinline__ void stencil_split(const Geom& gm, int jx, float fx, int jy, float fy, Stencil<P, float>& s) {
  s.ix0 = shape_wd<P, float>(jx, fx, s.wx, s.dwx);
  s.iy0 = shape_wd<P, float>(jy, fy, s.wy, s.dwy);
#pragma unroll
  for (int a = 0; a <= P; ++a) {
    s.dwx[a] *= gm.f_inv_dx;
    s.dwy[a] *= gm.f_inv_dy;
  }
}

// ---------------------------------------------------------------- final pass adjoint
// Reverse of: gather at slice i, AB5 step to i+1, removal, deposit at i+1.
template <int P, typename T>
__global__ void __launch_bounds__(kThreads)
    k_adj_final(SnapView<T> s, const T* __restrict__ gf, Geom gm, int slice, double guard,
                const V4<T>* __restrict__ dbar_next, AdjView<T> a, T* tbar, V2<T>* fbar_b, double* wbar_p) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s.n || !s.alive[p]) return;
  const int64_t n = s.n;
  const double x = s.x[p], y = s.y[p], psi = s.psi[p];
  const T ux = s.ux[p], uy = s.uy[p], w = s.w[p];
  T opp;
  Stencil<P, T> st;
  if constexpr (sizeof(T) == 4) {
    // the forward final pass gathered at the cached cell coordinates, with the cached 1 + Psi
    const int cell = s.cell[p];
    stencil_split<P>(gm, cell & 0xFFFF, s.fx[p], cell >> 16, s.fy[p], st);
    opp = s.opp[p];
  } else {
    stencil_at<P, T>(gm, x, y, st);
    opp = T(1.0 + psi);
  }
  T F[6], Fx[6], Fy[6];
  {
    T v4[4], g4x[4], g4y[4];
    gather_g<P, T, 4>(gf, kGF, 0, gm, st, v4, g4x, g4y);   // ExmBy, EypBx, Ez, Bz
    T b[2], bx[2], by[2];
    gather_g<P, T, 2>(gf + kGF * (int64_t)gm.nx * gm.ny, 2, 0, gm, st, b, bx, by);   // Bx, By (converged)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      F[c] = v4[c];
      Fx[c] = g4x[c];
      Fy[c] = g4y[c];
    }
    F[3] = b[0]; F[4] = b[1]; F[5] = v4[3];
    Fx[3] = bx[0]; Fx[4] = bx[1]; Fx[5] = g4x[3];
    Fy[3] = by[0]; Fy[4] = by[1]; Fy[5] = g4y[3];
  }
  T f[5];
  derivs_f<T>(ux, uy, opp, F, f);
  T comb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    T acc = T(ab5(0)) * f[c];
#pragma unroll
    for (int k = 1; k <= 4; ++k) acc += T(ab5(k)) * hist_at<T>(s.hist, n, p, slice, k, c);
    comb[c] = acc;
  }
  const double dz = gm.dzeta;
  const T mdz = -gsel<T>(dz, gm.f_dz);   // -dzeta in the field type (no FP64 product per use)
  const double nxp = x - dz * (double)comb[0], nyp = y - dz * (double)comb[1];
  const double npsi = psi - dz * (double)comb[4];
  const T nux = ux + mdz * comb[2], nuy = uy + mdz * comb[3];
  if (!ok_state(gm, nxp, nyp, 1.0 + npsi, guard)) return;  // removed: nothing downstream depends on it
  // deposit at slice i+1: v = q w (gamma g, ux g, uy g, uz g) / A
  Stencil<P, T> sn;
  stencil_at<P, T>(gm, nxp, nyp, sn);
  T Dg[4], Dgx[4], Dgy[4];
  gather_g<P, T, 4>(reinterpret_cast<const T*>(dbar_next), 4, 0, gm, sn, Dg, Dgx, Dgy);
  const T nopp = T(1.0 + npsi), g = T(1) / nopp, g2 = g * g;
  const T q2 = T(1) + nux * nux + nuy * nuy;
  const T gg = q2 * T(0.5) * g2 + T(0.5);   // gamma g
  const T ug = q2 * T(0.5) * g2 - T(0.5);   // uz g
  const T qw1 = unit_charge_density<T>(gm), qw = qw1 * w;
  const T v[4] = {qw * gg, qw * nux * g, qw * nuy * g, qw * ug};
  T sb[5];
  sb[0] = a.sx[p] + v[0] * Dgx[0] + v[1] * Dgx[1] + v[2] * Dgx[2] + v[3] * Dgx[3];
  sb[1] = a.sy[p] + v[0] * Dgy[0] + v[1] * Dgy[1] + v[2] * Dgy[2] + v[3] * Dgy[3];
  sb[2] = a.sux[p] + qw * (Dg[0] * nux * g2 + Dg[1] * g + Dg[3] * nux * g2);
  sb[3] = a.suy[p] + qw * (Dg[0] * nuy * g2 + Dg[2] * g + Dg[3] * nuy * g2);
  sb[4] = a.spsi[p] + qw * (-(Dg[0] + Dg[3]) * q2 * g2 * g - Dg[1] * nux * g2 - Dg[2] * nuy * g2);
  wbar_p[p] += (double)(qw1 * (Dg[0] * gg + Dg[1] * nux * g + Dg[2] * nuy * g + Dg[3] * ug));
  // AB5 step and history shift
  T fb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    // history adjoints carried from slice i+1, with the trial steps' pending share folded in
    const T sacc = a.sacc[(int64_t)c * n + p];
    a.sacc[(int64_t)c * n + p] = T(0);
    T hn[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) hn[j] = a.sh[((int64_t)j * 5 + c) * n + p] + (mdz * T(ab5(j + 1))) * sacc;
    fb[c] = (mdz * T(ab5(0))) * sb[c] + hn[0];
#pragma unroll
    for (int j = 0; j < 4; ++j)
      a.sh[((int64_t)j * 5 + c) * n + p] = (mdz * T(ab5(j + 1))) * sb[c] + (j < 3 ? hn[j + 1] : T(0));
  }
  T bux, buy, bpsi, bF[6];
  derivs_adj<T>(ux, uy, opp, F, fb, bux, buy, bpsi, bF);
  {
    // ExmBy, EypBx, Ez, Bz into tbar; Bx, By into fbar_b
    const T v4[4] = {bF[0], bF[1], bF[2], bF[5]};
    scatter_v4<P, T>(tbar, gm, st, v4);
    const T v2b[2] = {bF[3], bF[4]};
    scatter_v2<P, T>(reinterpret_cast<T*>(fbar_b), gm, st, v2b);
  }
  T bx = sb[0], by = sb[1];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    bx += bF[c] * Fx[c];
    by += bF[c] * Fy[c];
  }
  a.sx[p] = bx;
  a.sy[p] = by;
  a.sux[p] = sb[2] + bux;
  a.suy[p] = sb[3] + buy;
  a.spsi[p] = sb[4] + bpsi;
}

// ---------------------------------------------------------------- trial pass adjoint
// Reverse of one predictor-corrector trial pass: gather with B^(m-1) at slice i,
// AB5 trial step to i+1, J_perp deposit of the trial particles.
template <int P, typename T>
__global__ void __launch_bounds__(kThreads)
    k_adj_trial(SnapView<T> s, const T* __restrict__ gf, const V2<T>* __restrict__ bm, Geom gm, int slice, double guard,
                const V2<T>* __restrict__ jbar, AdjView<T> a, T* tbar, V2<T>* bbar_m1, double* wbar_p) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s.n || !s.alive[p]) return;
  const int64_t n = s.n;
  const T ux = s.ux[p], uy = s.uy[p], w = s.w[p];
  // the forward trial pass's own arithmetic: FP32 from the cached cell coordinates and 1 + Psi
  // (FP32 mode), FP64 positions otherwise
  int jx = 0, jy = 0;
  T fxr = T(0), fyr = T(0);
  double x = 0.0, y = 0.0, psi = 0.0;
  T opp;
  Stencil<P, T> st;
  if constexpr (sizeof(T) == 4) {
    const int cell = s.cell[p];
    jx = cell & 0xFFFF;
    jy = cell >> 16;
    fxr = s.fx[p];
    fyr = s.fy[p];
    stencil_split<P>(gm, jx, fxr, jy, fyr, st);
    opp = s.opp[p];
  } else {
    x = s.x[p];
    y = s.y[p];
    psi = s.psi[p];
    stencil_at<P, T>(gm, x, y, st);
    opp = T(1.0 + psi);
  }
  T F[6], Fx[6], Fy[6];
  {
    T v4[4], g4x[4], g4y[4];
    gather_g<P, T, 4>(gf, kGF, 0, gm, st, v4, g4x, g4y);   // ExmBy, EypBx, Ez, Bz
    F[0] = v4[0]; F[1] = v4[1]; F[2] = v4[2];
    Fx[0] = g4x[0]; Fx[1] = g4x[1]; Fx[2] = g4x[2];
    Fy[0] = g4y[0]; Fy[1] = g4y[1]; Fy[2] = g4y[2];
    F[5] = v4[3]; Fx[5] = g4x[3]; Fy[5] = g4y[3];
    T b2[2], b2x[2], b2y[2];
    gather_g<P, T, 2>(reinterpret_cast<const T*>(bm), 2, 0, gm, st, b2, b2x, b2y);  // Bx, By of B^(m-1)
    F[3] = b2[0]; F[4] = b2[1];
    Fx[3] = b2x[0]; Fx[4] = b2x[1];
    Fy[3] = b2y[0]; Fy[4] = b2y[1];
  }
  T f[5];
  derivs_f<T>(ux, uy, opp, F, f);
  T comb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    if (s.hsum) {
      // FP32: the forward trial passes' own combination, beta_0 f_i + (stored history sum)
      comb[c] = T(ab5(0)) * f[c] + T(s.hsum[(int64_t)c * n + p]);
    } else {
      T acc = T(ab5(0)) * f[c];
#pragma unroll
      for (int k = 1; k <= 4; ++k) acc += T(ab5(k)) * hist_at<T>(s.hist, n, p, slice, k, c);
      comb[c] = acc;
    }
  }
  const T mdz = -gsel<T>(gm.dzeta, gm.f_dz);   // -dzeta in the field type
  const T tux = ux + mdz * comb[2], tuy = uy + mdz * comb[3];
  T topp;
  Stencil<P, T> sn;
  if constexpr (sizeof(T) == 4) {
    // trial step in cell-relative coordinates, as the forward FP32 trial pass takes it
    float ux_ = fxr - gm.f_dz_inv_dx * comb[0];
    float uy_ = fyr - gm.f_dz_inv_dy * comb[1];
    const float flx = floorf(ux_), fly = floorf(uy_);
    const int tjx = jx + (int)flx, tjy = jy + (int)fly;
    ux_ -= flx;
    uy_ -= fly;
    topp = opp + mdz * comb[4];
    const float ax = (float)tjx + ux_, ay = (float)tjy + uy_;
    const bool ok = isfinite(ax) && isfinite(ay) && isfinite(topp) && ax > 0.0f && ax < (float)gm.nx && ay > 0.0f &&
                    ay < (float)gm.ny && topp >= gm.f_guard;
    if (!ok) return;  // skipped by the trial deposit
    stencil_split<P>(gm, tjx, ux_, tjy, uy_, sn);
  } else {
    const double dz = gm.dzeta;
    const double tx = x - dz * (double)comb[0], ty = y - dz * (double)comb[1];
    const double tpsi = psi - dz * (double)comb[4];
    if (!ok_state(gm, tx, ty, 1.0 + tpsi, guard)) return;  // skipped by the trial deposit
    topp = T(1.0 + tpsi);
    stencil_at<P, T>(gm, tx, ty, sn);
  }
  T Jg[2], Jgx[2], Jgy[2];
  gather_g<P, T, 2>(reinterpret_cast<const T*>(jbar), 2, 0, gm, sn, Jg, Jgx, Jgy);
  const T tg = T(1) / topp;
  const T qw1 = unit_charge_density<T>(gm), qw = qw1 * w;
  const T v0 = qw * tux * tg, v1 = qw * tuy * tg;
  T stb[5];
  stb[0] = v0 * Jgx[0] + v1 * Jgx[1];
  stb[1] = v0 * Jgy[0] + v1 * Jgy[1];
  stb[2] = qw * Jg[0] * tg;
  stb[3] = qw * Jg[1] * tg;
  stb[4] = -qw * tg * tg * (Jg[0] * tux + Jg[1] * tuy);
  wbar_p[p] += (double)(qw1 * tg * (Jg[0] * tux + Jg[1] * tuy));
  T fb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    fb[c] = (mdz * T(ab5(0))) * stb[c];
    a.sacc[(int64_t)c * n + p] += stb[c];   // history share: folded into sh by the next final adjoint
  }
  T bux, buy, bpsi, bF[6];
  derivs_adj<T>(ux, uy, opp, F, fb, bux, buy, bpsi, bF);
  {
    // ExmBy, EypBx, Ez, Bz into tbar; Bx, By of B^(m-1) into bbar_m1
    const T v4[4] = {bF[0], bF[1], bF[2], bF[5]};
    scatter_v4<P, T>(tbar, gm, st, v4);
    const T v2b[2] = {bF[3], bF[4]};
    scatter_v2<P, T>(reinterpret_cast<T*>(bbar_m1), gm, st, v2b);
  }
  T bx = stb[0], by = stb[1];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    bx += bF[c] * Fx[c];
    by += bF[c] * Fy[c];
  }
  a.sx[p] += bx;
  a.sy[p] += by;
  a.sux[p] += stb[2] + bux;
  a.suy[p] += stb[3] + buy;
  a.spsi[p] += stb[4] + bpsi;
}

// ---------------------------------------------------------------- node-level adjoints
// Bbar^n = (Bx, By adjoints of the final pass's gather) + carry of B(i); both are consumed
// (cleared for the next slice).
template <typename T>
__global__ void k_adj_bstart(V2<T>* fbar_b, V2<T>* carry, V2<T>* bbar_n, int64_t nn) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nn) return;
  const V2<T> c = carry[o], f = fbar_b[o];
  bbar_n[o] = V2<T>{f.a + c.a, f.b + c.b};
  carry[o] = V2<T>{T(0), T(0)};
  fbar_b[o] = V2<T>{T(0), T(0)};
}

// Mixing B^m = w Bs + (1-w) B^(m-1): the solve gets w Bbar^m, Bbar^(m-1) starts at (1-w) Bbar^m.
template <typename T, typename Sink>
__global__ void k_adj_pc_pre(const V2<T>* __restrict__ bbar_m, V2<T>* bbar_m1, T w, Geom gm, Sink sink) {
  visit_nodes<2, T>(gm, sink, 2, [&](int iy, int ix, T* v) {
    const int64_t o = (int64_t)iy * gm.nx + ix;
    const V2<T> b = bbar_m[o];
    bbar_m1[o] = V2<T>{(T(1) - w) * b.a, (T(1) - w) * b.b};
    v[0] = w * b.a;
    v[1] = w * b.b;
  });
}

// Sources Bx = -dy Jz + (Jy(i-1) - Jy(i+1))/2dz, By = dx Jz - (Jx(i-1) - Jx(i+1))/2dz,
// transposed: res = L^-1 of the mixed B adjoints.
template <typename T>
__global__ void k_adj_pc_post(const T* __restrict__ res, V4<T>* dcur, V4<T>* dprev, V2<T>* jbar, V2<T>* jbar_tot,
                              Geom gm) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (ix >= gm.nx) return;
  const int nx = gm.nx;
  const int64_t nn = (int64_t)nx * gm.ny;
  const int64_t o = (int64_t)iy * nx + ix;
  T jz = T(0), jxp = T(0), jyp = T(0), jxn = T(0), jyn = T(0);
  if (ix > 0 && iy > 0) {
    auto r0 = [&](int y, int x) { return res[(int64_t)y * nx + x]; };
    auto r1 = [&](int y, int x) { return res[nn + (int64_t)y * nx + x]; };
    const T i2z = gsel<T>(gm.inv2dz, gm.f_inv2dz);
    jz = dyc(r0, iy, ix, gm.ny, gsel<T>(gm.inv2dy, gm.f_inv2dy)) - dxc(r1, iy, ix, nx, gsel<T>(gm.inv2dx, gm.f_inv2dx));
    const T a0 = res[o], a1 = res[nn + o];
    jxp = -a1 * i2z;
    jyp = a0 * i2z;
    jxn = a1 * i2z;
    jyn = -a0 * i2z;
  }
  dcur[o].d += jz;
  dprev[o].b += jxp;
  dprev[o].c += jyp;
  jbar[o] = V2<T>{jxn, jyn};
  const V2<T> t = jbar_tot[o];
  jbar_tot[o] = V2<T>{t.a + jxn, t.b + jyn};
}

// Guess B^0 = 2 B(i-1) - B(i-2): carries for the two previous slices.
template <typename T>
__global__ void k_adj_guess(const V2<T>* __restrict__ b0, V2<T>* c1, V2<T>* c2, int64_t nn) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nn) return;
  const V2<T> b = b0[o];
  if (c1) { c1[o].a += T(2) * b.a; c1[o].b += T(2) * b.b; }
  if (c2) { c2[o].a -= b.a; c2[o].b -= b.b; }
}

// psi_bar = Dx tbar0 + Dy tbar1 (ExmBy = -Dx psi, EypBx = -Dy psi), with Ez_bar, Bz_bar: tbar
// holds the adjoints of the gathered ExmBy, EypBx, Ez, Bz (witness, final and trial passes).
template <typename T, typename Sink>
__global__ void k_adj_main_pre(const T* __restrict__ tbar, const T* __restrict__ seed_psi, Geom gm, Sink sink) {
  const int nx = gm.nx;
  auto f0 = [&](int y, int x) { return tbar[((int64_t)y * nx + x) * 4 + 0]; };
  auto f1 = [&](int y, int x) { return tbar[((int64_t)y * nx + x) * 4 + 1]; };
  visit_nodes<3, T>(gm, sink, 3, [&](int iy, int ix, T* v) {
    const int64_t o = (int64_t)iy * nx + ix;
    v[0] = v[1] = v[2] = T(0);
    if (ix > 0 && iy > 0) {
      v[0] = dxc(f0, iy, ix, nx, gsel<T>(gm.inv2dx, gm.f_inv2dx)) + dyc(f1, iy, ix, gm.ny, gsel<T>(gm.inv2dy, gm.f_inv2dy));
      if (seed_psi) v[0] += seed_psi[o];   // the caller's dL/dpsi of this slice
      v[1] = tbar[o * 4 + 2];
      v[2] = tbar[o * 4 + 3];
    }
  });
}

// psi = L^-1(-(rho - Jz)), Ez = L^-1(dx Jx + dy Jy), Bz = L^-1(dy Jx - dx Jy), transposed.
// tbar of this slice is consumed: cleared for the next slice.
template <typename T>
__global__ void k_adj_main_post(const T* __restrict__ res, V4<T>* dcur, T* rho_ion_bar, V4<T>* tbar, Geom gm) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (ix >= gm.nx) return;
  const int nx = gm.nx;
  const int64_t nn = (int64_t)nx * gm.ny;
  const int64_t o = (int64_t)iy * nx + ix;
  tbar[o] = V4<T>{T(0), T(0), T(0), T(0)};
  V4<T> d = dcur[o];
  if (ix > 0 && iy > 0) {
    auto r1 = [&](int y, int x) { return res[nn + (int64_t)y * nx + x]; };
    auto r2 = [&](int y, int x) { return res[2 * nn + (int64_t)y * nx + x]; };
    const T i2x = gsel<T>(gm.inv2dx, gm.f_inv2dx), i2y = gsel<T>(gm.inv2dy, gm.f_inv2dy);
    const T sp = res[o];
    d.a += -sp;
    d.d += sp;
    d.b += -dxc(r1, iy, ix, nx, i2x) - dyc(r2, iy, ix, gm.ny, i2y);
    d.c += -dyc(r1, iy, ix, gm.ny, i2y) + dxc(r2, iy, ix, nx, i2x);
  }
  dcur[o] = d;
  rho_ion_bar[o] += d.a;
}


// ---------------------------------------------------------------- beams and parameters
template <int P>
__device__ __forceinline__ int stencil_b(double x, double x0, double dx, double* w) {
  int j;
  double d;
  split_coord(x, x0, dx, j, d);
  return shape_weights<P, double>(j, d, w);
}

template <int P, typename T, int NC>
__device__ __forceinline__ void gather_b(const T* __restrict__ f, int st, const Geom& gm, double x, double y, double* v) {
  double wx[P + 1], wy[P + 1];
  const int ix0 = stencil_b<P>(x, gm.xmin, gm.dx, wx), iy0 = stencil_b<P>(y, gm.ymin, gm.dy, wy);
#pragma unroll
  for (int c = 0; c < NC; ++c) v[c] = 0.0;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, gm.nx)) continue;
      const T* q = f + ((int64_t)iy * gm.nx + ix) * st;
#pragma unroll
      for (int c = 0; c < NC; ++c) v[c] += wx[a] * wy[b] * (double)q[c];
    }
  }
}

// Beam weights: deposit of slice i (rho, J) and the J_perp of slice i+1 used by the P-C.
template <int P, typename T>
__global__ void k_adj_beam(hq_beam_view v, const int32_t* __restrict__ off, const int32_t* __restrict__ perm, int slice,
                           int nz, Geom gm, const V4<T>* __restrict__ dcur, const V2<T>* __restrict__ jtot,
                           double* wbar) {
  const int a0 = off[slice], a1 = off[slice + 1];
  const int b0 = slice + 1 < nz ? off[slice + 1] : 0, b1 = slice + 1 < nz ? off[slice + 2] : 0;
  const int na = a1 - a0, nb = b1 - b0;
  const double rq = v.charge / (gm.dx * gm.dy * gm.dzeta);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < na + nb; t += gridDim.x * blockDim.x) {
    const bool cur = t < na;
    const int p = perm[cur ? a0 + t : b0 + (t - na)];
    const double ux = v.ux[p], uy = v.uy[p], uz = v.uz[p];
    const double ig = 1.0 / sqrt(1.0 + ux * ux + uy * uy + uz * uz);
    double g[4];
    double s;
    if (cur) {
      gather_b<P, T, 4>(reinterpret_cast<const T*>(dcur), 4, gm, v.x[p], v.y[p], g);
      s = g[0] + ux * ig * g[1] + uy * ig * g[2] + uz * ig * g[3];
    } else {
      gather_b<P, T, 2>(reinterpret_cast<const T*>(jtot), 2, gm, v.x[p], v.y[p], g);
      s = ux * ig * g[0] + uy * ig * g[1];
    }
    wbar[p] += rq * s;
  }
}

// Witness loss sums (S0, S1, S2) = sum q w (1, Ez, Ez^2) over slice i, with adjoints sb[0..2].
template <int P, typename T>
__global__ void k_adj_witness(hq_beam_view v, const int32_t* __restrict__ off, const int32_t* __restrict__ perm,
                              int slice, Geom gm, const T* __restrict__ gf, double sb0, double sb1, double sb2, T* tbar,
                              double* wbar) {
  const int a0 = off[slice], a1 = off[slice + 1];
  for (int t = a0 + blockIdx.x * blockDim.x + threadIdx.x; t < a1; t += gridDim.x * blockDim.x) {
    const int p = perm[t];
    double wx[P + 1], wy[P + 1];
    const int ix0 = stencil_b<P>(v.x[p], gm.xmin, gm.dx, wx), iy0 = stencil_b<P>(v.y[p], gm.ymin, gm.dy, wy);
    double ez = 0.0;
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        ez += wx[a] * wy[b] * (double)gf[((int64_t)iy * gm.nx + ix) * kGF + 2];
      }
    }
    const double qw = v.charge * v.w[p];
    if (wbar) wbar[p] += v.charge * (sb0 + ez * sb1 + ez * ez * sb2);
    const double e = qw * (sb1 + 2.0 * ez * sb2);
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        atomicAdd(tbar + ((int64_t)iy * gm.nx + ix) * 4 + 2, T(wx[a] * wy[b] * e));
      }
    }
  }
}

// Plasma weights at the initial slice: deposit of slice 0 (rho only: gamma g = 1) and
// the ion background rho_ion = -(q w / A) added to every slice.
template <int P, typename T>
__global__ void k_adj_init(int64_t np, Geom gm, int ppx, int ppy, const V4<T>* __restrict__ d0,
                           const T* __restrict__ rho_ion_bar, double* wbar_p) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int ppc = ppx * ppy;
  const int64_t c = p / ppc;
  const int sub = (int)(p - c * ppc);
  const int ix = (int)(c % gm.nx), iy = (int)(c / gm.nx);
  const int sx = sub % ppx, sy = sub / ppx;
  const double x = gm.xmin + ((double)ix + ((double)sx + 0.5) / ppx) * gm.dx;
  const double y = gm.ymin + ((double)iy + ((double)sy + 0.5) / ppy) * gm.dy;
  double g0[1], gi[1];
  gather_b<P, T, 1>(reinterpret_cast<const T*>(d0), 4, gm, x, y, g0);
  gather_b<P, T, 1>(rho_ion_bar, 1, gm, x, y, gi);
  wbar_p[p] += (-1.0 / (gm.dx * gm.dy)) * (g0[0] - gi[0]);
}

// dL/dn0_scale and dL/dprofile from the plasma weight adjoints (w = n0 dens(r) dx dy / ppc).
__global__ void k_adj_params(int64_t np, Geom gm, int ppx, int ppy, const double* __restrict__ prof, int npf,
                             double rmax, double n0s, const double* __restrict__ wbar_p, double* dn0, double* dprof) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double gn = 0.0;
  if (p < np) {
    const int ppc = ppx * ppy;
    const int64_t c = p / ppc;
    const int sub = (int)(p - c * ppc);
    const int ix = (int)(c % gm.nx), iy = (int)(c / gm.nx);
    const int sx = sub % ppx, sy = sub / ppx;
    const double x = gm.xmin + ((double)ix + ((double)sx + 0.5) / ppx) * gm.dx;
    const double y = gm.ymin + ((double)iy + ((double)sy + 0.5) / ppy) * gm.dy;
    const double cw = gm.dx * gm.dy / (double)ppc;
    double dens = 1.0;
    if (prof) {
      const double r = sqrt(x * x + y * y);
      double t = r / rmax * (npf - 1);
      t = fmin(fmax(t, 0.0), (double)(npf - 1));
      int k0 = (int)floor(t);
      k0 = k0 < 0 ? 0 : (k0 > npf - 2 ? npf - 2 : k0);
      const double fr = t - (double)k0;
      dens = prof[k0] * (1.0 - fr) + prof[k0 + 1] * fr;
      if (dprof) {
        atomicAdd(dprof + k0, wbar_p[p] * n0s * cw * (1.0 - fr));
        atomicAdd(dprof + k0 + 1, wbar_p[p] * n0s * cw * fr);
      }
    }
    gn = wbar_p[p] * dens * cw;
  }
  for (int o = 16; o > 0; o >>= 1) gn += __shfl_down_sync(0xffffffffu, gn, o);
  if (dn0 && (threadIdx.x & 31) == 0 && gn != 0.0) atomicAdd(dn0, gn);
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }
inline dim3 grid2d(const hq_grid_s* g) { return dim3((unsigned)((g->nx + 127) / 128), (unsigned)g->ny); }
constexpr unsigned kSliceBlocks = 152;

#define HQ_SHAPE_SWITCH(ORDER, CALL) \
  switch (ORDER) {                   \
    case 0: { constexpr int P = 0; CALL; } break; \
    case 1: { constexpr int P = 1; CALL; } break; \
    case 2: { constexpr int P = 2; CALL; } break; \
    default: { constexpr int P = 3; CALL; } break; \
  }

}  // namespace

template <typename T>
void launch_adj_final(const hq_grid_s* g, const SnapView<T>& s, const void* gf, int slice, const void* dbar_next,
                      const AdjView<T>& a, void* tbar, void* fbar_b, double* wbar_p, cudaStream_t st) {
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (k_adj_final<P, T><<<blocks_for(s.n), kThreads, 0, st>>>(
                      s, reinterpret_cast<const T*>(gf), g->geom, slice, g->d.psi_guard,
                      reinterpret_cast<const V4<T>*>(dbar_next), a, reinterpret_cast<T*>(tbar),
                      reinterpret_cast<V2<T>*>(fbar_b), wbar_p)));
}
template <typename T>
void launch_adj_trial(const hq_grid_s* g, const SnapView<T>& s, const void* gf, const void* bm, int slice,
                      const void* jbar, const AdjView<T>& a, void* tbar, void* bbar_m1, double* wbar_p,
                      cudaStream_t st) {
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (k_adj_trial<P, T><<<blocks_for(s.n), kThreads, 0, st>>>(
                      s, reinterpret_cast<const T*>(gf), reinterpret_cast<const V2<T>*>(bm), g->geom, slice,
                      g->d.psi_guard, reinterpret_cast<const V2<T>*>(jbar), a, reinterpret_cast<T*>(tbar),
                      reinterpret_cast<V2<T>*>(bbar_m1), wbar_p)));
}
template <typename T>
void launch_adj_bstart(const hq_grid_s* g, void* fbar_b, void* carry, void* bbar_n, cudaStream_t st) {
  k_adj_bstart<T><<<blocks_for(g->nnode), kThreads, 0, st>>>(reinterpret_cast<V2<T>*>(fbar_b),
                                                           reinterpret_cast<V2<T>*>(carry),
                                                           reinterpret_cast<V2<T>*>(bbar_n), g->nnode);
}
template <typename T>
void launch_adj_pc_pre(const hq_grid_s* g, const void* bbar_m, void* bbar_m1, cudaStream_t st) {
  with_sink<T>(g, [&](auto sink) {
    k_adj_pc_pre<T, decltype(sink)><<<src_grid(g), 128, 0, st>>>(
        reinterpret_cast<const V2<T>*>(bbar_m), reinterpret_cast<V2<T>*>(bbar_m1), T(g->d.pc_mix), g->geom, sink);
  });
}
template <typename T>
void launch_adj_pc_post(const hq_grid_s* g, void* dcur, void* dprev, void* jbar, void* jtot, cudaStream_t st) {
  k_adj_pc_post<T><<<grid2d(g), 128, 0, st>>>(reinterpret_cast<const T*>(g->solved), reinterpret_cast<V4<T>*>(dcur),
                                             reinterpret_cast<V4<T>*>(dprev), reinterpret_cast<V2<T>*>(jbar),
                                             reinterpret_cast<V2<T>*>(jtot), g->geom);
}
template <typename T>
void launch_adj_guess(const hq_grid_s* g, const void* b0, void* c1, void* c2, cudaStream_t st) {
  k_adj_guess<T><<<blocks_for(g->nnode), kThreads, 0, st>>>(reinterpret_cast<const V2<T>*>(b0),
                                                          reinterpret_cast<V2<T>*>(c1), reinterpret_cast<V2<T>*>(c2),
                                                          g->nnode);
}
template <typename T>
void launch_adj_main_pre(const hq_grid_s* g, const void* tbar, const void* seed_psi, cudaStream_t st) {
  with_sink<T>(g, [&](auto sink) {
    k_adj_main_pre<T, decltype(sink)><<<src_grid(g), 128, 0, st>>>(reinterpret_cast<const T*>(tbar),
                                                                   reinterpret_cast<const T*>(seed_psi), g->geom, sink);
  });
}

// Caller's adjoint seeds of slice i's output fields (hq_sweep_adjoint's dL_dfields, each a
// pointer to this slice's ny x nx values or null), added where the reverse sweep accumulates the
// adjoint of that field: ExmBy, EypBx, Ez, Bz into tbar, Bx, By into fbar_b, rho, Jx, Jy, Jz into
// the slice's deposit adjoint.  Wall nodes are fixed zeros in the forward: their seeds are ignored.
template <typename T>
__global__ void k_adj_seed(hq_field_out sd, int64_t off, V4<T>* tbar, V2<T>* fbar_b, V4<T>* dcur, Geom gm) {
  const int ix = blockIdx.x * blockDim.x + threadIdx.x, iy = blockIdx.y;
  if (ix >= gm.nx || ix == 0 || iy == 0) return;
  const int64_t o = (int64_t)iy * gm.nx + ix, t = off + o;
  auto at = [&](void* p) { return p ? reinterpret_cast<const T*>(p)[t] : T(0); };
  if (sd.exmby || sd.eypbx || sd.ez || sd.bz) {
    V4<T> q = tbar[o];
    q.a += at(sd.exmby);
    q.b += at(sd.eypbx);
    q.c += at(sd.ez);
    q.d += at(sd.bz);
    tbar[o] = q;
  }
  if (sd.bx || sd.by) {
    V2<T> q = fbar_b[o];
    q.a += at(sd.bx);
    q.b += at(sd.by);
    fbar_b[o] = q;
  }
  if (sd.rho || sd.jx || sd.jy || sd.jz) {
    V4<T> q = dcur[o];
    q.a += at(sd.rho);
    q.b += at(sd.jx);
    q.c += at(sd.jy);
    q.d += at(sd.jz);
    dcur[o] = q;
  }
}
template <typename T>
void launch_adj_seed(const hq_grid_s* g, const hq_field_out& sd, int slice, void* tbar, void* fbar_b, void* dcur,
                     cudaStream_t st) {
  k_adj_seed<T><<<grid2d(g), 128, 0, st>>>(sd, (int64_t)slice * g->nnode, reinterpret_cast<V4<T>*>(tbar),
                                          reinterpret_cast<V2<T>*>(fbar_b), reinterpret_cast<V4<T>*>(dcur), g->geom);
}
template <typename T>
void launch_adj_main_post(const hq_grid_s* g, void* dcur, void* rho_ion_bar, void* tbar, cudaStream_t st) {
  k_adj_main_post<T><<<grid2d(g), 128, 0, st>>>(reinterpret_cast<const T*>(g->solved), reinterpret_cast<V4<T>*>(dcur),
                                               reinterpret_cast<T*>(rho_ion_bar), reinterpret_cast<V4<T>*>(tbar),
                                               g->geom);
}
template <typename T>
void launch_adj_beam(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, const void* dcur, const void* jtot,
                     double* wbar, cudaStream_t st) {
  const BeamBins& bb = g->bins[b];
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (k_adj_beam<P, T><<<kSliceBlocks, kThreads, 0, st>>>(v, bb.offset, bb.perm, slice, g->nz, g->geom,
                                                                       reinterpret_cast<const V4<T>*>(dcur),
                                                                       reinterpret_cast<const V2<T>*>(jtot), wbar)));
}
template <typename T>
void launch_adj_witness(const hq_grid_s* g, int b, const hq_beam_view& v, int slice, const void* gf, const double* sb,
                        void* tbar, double* wbar, cudaStream_t st) {
  const BeamBins& bb = g->bins[b];
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (k_adj_witness<P, T><<<kSliceBlocks, kThreads, 0, st>>>(v, bb.offset, bb.perm, slice, g->geom,
                                                                          reinterpret_cast<const T*>(gf), sb[0], sb[1],
                                                                          sb[2], reinterpret_cast<T*>(tbar), wbar)));
}
template <typename T>
void launch_adj_init(const hq_grid_s* g, const void* d0, const void* rho_ion_bar, double* wbar_p, cudaStream_t st) {
  HQ_SHAPE_SWITCH(g->d.shape_order,
                  (k_adj_init<P, T><<<blocks_for(g->np), kThreads, 0, st>>>(
                      g->np, g->geom, g->d.ppc_x, g->d.ppc_y, reinterpret_cast<const V4<T>*>(d0),
                      reinterpret_cast<const T*>(rho_ion_bar), wbar_p)));
}
void launch_adj_params(const hq_grid_s* g, const double* wbar_p, double* dn0, double* dprof, cudaStream_t st) {
  k_adj_params<<<blocks_for(g->np), kThreads, 0, st>>>(g->np, g->geom, g->d.ppc_x, g->d.ppc_y,
                                                     g->profile.empty() ? nullptr : g->d_profile,
                                                     (int)g->profile.size(), g->d.profile_rmax, g->d.n0_scale, wbar_p,
                                                     dn0, dprof);
}

#define HQ_INST(T)                                                                                                   \
  template void launch_adj_final<T>(const hq_grid_s*, const SnapView<T>&, const void*, int, const void*,              \
                                    const AdjView<T>&, void*, void*, double*, cudaStream_t);                         \
  template void launch_adj_trial<T>(const hq_grid_s*, const SnapView<T>&, const void*, const void*, int, const void*, \
                                    const AdjView<T>&, void*, void*, double*, cudaStream_t);                         \
  template void launch_adj_bstart<T>(const hq_grid_s*, void*, void*, void*, cudaStream_t);                           \
  template void launch_adj_pc_pre<T>(const hq_grid_s*, const void*, void*, cudaStream_t);                            \
  template void launch_adj_pc_post<T>(const hq_grid_s*, void*, void*, void*, void*, cudaStream_t);                   \
  template void launch_adj_guess<T>(const hq_grid_s*, const void*, void*, void*, cudaStream_t);                      \
  template void launch_adj_main_pre<T>(const hq_grid_s*, const void*, const void*, cudaStream_t);                    \
  template void launch_adj_seed<T>(const hq_grid_s*, const hq_field_out&, int, void*, void*, void*, cudaStream_t);    \
  template void launch_adj_main_post<T>(const hq_grid_s*, void*, void*, void*, cudaStream_t);                        \
  template void launch_adj_beam<T>(const hq_grid_s*, int, const hq_beam_view&, int, const void*, const void*,        \
                                   double*, cudaStream_t);                                                           \
  template void launch_adj_witness<T>(const hq_grid_s*, int, const hq_beam_view&, int, const void*, const double*,   \
                                      void*, double*, cudaStream_t);                                                 \
  template void launch_adj_init<T>(const hq_grid_s*, const void*, const void*, double*, cudaStream_t);
HQ_INST(float)
HQ_INST(double)
#undef HQ_INST

}  // namespace hq
