// Plasma particle kernels: initialization, deposition (Sec. 3.2, "current
// deposition": order 0 longitudinally, orders 0-3 transversely, atomics to global
// memory), field gather and the fifth-order Adams-Bashforth push (Sec. 3.2,
// equations for d(x_perp)/d(zeta), d(u_perp)/d(zeta), d(Psi)/d(zeta)).
//
// Layout: structure of arrays, one thread per particle, consecutive threads take
// consecutive particles (coalesced streams).  Deposits go to a packed per-node
// (rho, Jx, Jy, Jz) record with one vector atomic per node in FP32 mode.
//
// FP32 mode keeps x, y and Psi as FP64 accumulators.  The final pass, which
// advances the state, derives each particle's cell index and fractional node
// coordinate (and 1 + Psi, formed in FP64 and rounded once) and caches them, so
// the n_pc trial passes of the predictor-corrector run without FP64 work.
#include "hq_internal.cuh"

namespace hq {

namespace {

// 128 threads per block: with one particle per thread, the finer blocks leave a shorter tail
// of partly filled waves (trial and final passes 2.4 % faster on the blowout512 sweep than 256)
constexpr int kThreads = 128;

__device__ __forceinline__ void atomic_add4(V4<float>* p, float a, float b, float c, float d, const Geom&) {
  atomicAdd(reinterpret_cast<float4*>(p), make_float4(a, b, c, d));
}
__device__ __forceinline__ void atomic_add4(V4<double>* p, double a, double b, double c, double d, const Geom& gm) {
  dadd(&p->a, a, gm);
  dadd(&p->b, b, gm);
  dadd(&p->c, c, gm);
  dadd(&p->d, d, gm);
}
__device__ __forceinline__ void atomic_add2(V2<float>* p, float a, float b, const Geom&) {
  atomicAdd(reinterpret_cast<float2*>(p), make_float2(a, b));
}
__device__ __forceinline__ void atomic_add2(V2<double>* p, double a, double b, const Geom& gm) {
  dadd(&p->a, a, gm);
  dadd(&p->b, b, gm);
}

// Six gathered fields: ExmBy, EypBx, Ez, Bx, By, Bz.
template <typename T> struct F6 { T v[6]; };

// The six fields of one node: ExmBy, EypBx, Ez, Bz from the gather record, Bx, By from the
// B_perp record; o = (ExmBy, EypBx, Ez, Bx, By, Bz).
__device__ __forceinline__ void load_node(const float* q, const float* b, float* o) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(q));
  const float2 c = __ldg(reinterpret_cast<const float2*>(b));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = c.x; o[4] = c.y; o[5] = a.w;
}
__device__ __forceinline__ void load_node(const double* q, const double* b, double* o) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(q));
  const double2 a2 = __ldg(reinterpret_cast<const double2*>(q + 2));
  const double2 c = __ldg(reinterpret_cast<const double2*>(b));
  o[0] = a.x; o[1] = a.y; o[2] = a2.x; o[3] = c.x; o[4] = c.y; o[5] = a2.y;
}

// Interpolate the packed fields at a particle whose x/y stencils start at ix0/iy0.
template <int P, typename T>
__device__ __forceinline__ F6<T> gather6(const T* __restrict__ gf, const T* __restrict__ bm, int nx, int ny, int ix0,
                                         int iy0, const T* wx, const T* wy) {
  F6<T> F;
#pragma unroll
  for (int c = 0; c < 6; ++c) F.v[c] = T(0);
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, nx)) continue;
      T q[6];
      const int64_t node = (int64_t)iy * nx + ix;
      load_node(gf + node * kGF, bm + node * 2, q);
      const T wgt = wx[a] * wy[b];
#pragma unroll
      for (int c = 0; c < 6; ++c) F.v[c] += wgt * q[c];
    }
  }
  return F;
}

// Bx, By alone at the same stencil, accumulated node by node exactly as gather6 does (the same
// products and sums in the same order, so the result is bit for bit gather6's v[3], v[4]).
template <int P>
__device__ __forceinline__ float2 gather_bperp(const float* __restrict__ bm, int nx, int ny, int ix0, int iy0,
                                               const float* wx, const float* wy) {
  float bx = 0.0f, by = 0.0f;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, nx)) continue;
      const float2 c = __ldg(reinterpret_cast<const float2*>(bm + ((int64_t)iy * nx + ix) * 2));
      const float wgt = wx[a] * wy[b];
      bx += wgt * c.x;
      by += wgt * c.y;
    }
  }
  return make_float2(bx, by);
}

// zeta-derivatives of a plasma particle, Sec. 3.2; opp = 1 + Psi.  Written for an electron
// (q/M = -1); a multi-species grid (MS) scales the momentum and Psi rates by mqm = -q/M.
template <typename T, bool MS = false>
__device__ __forceinline__ void derivs(T ux, T uy, T opp, const F6<T>& F, T* f, T mqm = T(1)) {
  const T g = T(1) / opp;
  const T gam = (T(1) + ux * ux + uy * uy + opp * opp) * T(0.5) * g;
  const T exmby = F.v[0], eypbx = F.v[1], ez = F.v[2], bx = F.v[3], by = F.v[4], bz = F.v[5];
  f[0] = -ux * g;
  f[1] = -uy * g;
  f[2] = gam * g * exmby + by + bz * g * uy;      // -(q/M)[...] with q/M = -1
  f[3] = gam * g * eypbx - bx - bz * g * ux;
  f[4] = g * (ux * exmby + uy * eypbx) - ez;
  if constexpr (MS) {
    f[2] = mqm * f[2];
    f[3] = mqm * f[3];
    f[4] = mqm * f[4];
  }
}

// A particle's species constants on a multi-species grid (MS), else the electron's: -q/M,
// q/M (the chi factor q^2/M over q) and q, in the kernel's type.
template <typename T> struct SpC {
  T mqm, qm, q;
};
template <typename T, bool MS>
__device__ __forceinline__ SpC<T> spc_of(const SpeciesTab& tab, int s) {
  if constexpr (MS) {
    if constexpr (sizeof(T) == 8) return SpC<T>{T(-tab.qm[s]), T(tab.qm[s]), T(tab.q[s])};
    else return SpC<T>{-tab.fqm[s], tab.fqm[s], tab.fq[s]};
  } else {
    return SpC<T>{T(1), T(-1), T(-1)};
  }
}

// AB5 combination sum_k beta_k f_{i-k} for component c; history slots hold f_{i-1..i-4}.
template <typename T>
__device__ __forceinline__ T ab5_comb(const T* __restrict__ hist, int64_t n, int64_t p, int slice,
                                      int c, T f0) {
  T acc = T(ab5(0)) * f0;
#pragma unroll
  for (int k = 1; k <= 4; ++k) {
    const int slot = ((slice - k) % kRing + kRing) % kRing;
    acc += T(ab5(k)) * hist[((int64_t)slot * 5 + c) * n + p];
  }
  return acc;
}

// u_z = (1 + u_perp^2 - (1 + psi)^2) / (2 (1 + psi)) (the quasi-static constant of motion
// gamma - u_z = 1 + psi).  FP64 evaluates it as written (the oracle's arithmetic); FP32 as
// (u_perp^2 - psi (2 + psi)) g / 2 with psi (2 + psi) from the FP64 psi, since in FP32 the
// written form subtracts numbers near 1 and loses the plasma's small u_z.
template <typename T>
__device__ __forceinline__ T uz_of(T ux, T uy, T opp, double psi, T g) {
  if constexpr (sizeof(T) == 8) return (T(1) + ux * ux + uy * uy - opp * opp) * T(0.5) * g;
  else return (ux * ux + uy * uy - T(psi * (2.0 + psi))) * T(0.5) * g;
}

template <int P, typename T>
__device__ __forceinline__ void deposit_full(V4<T>* dep, T* chi, const Geom& gm, int ix0, int iy0,
                                             const T* wx, const T* wy, T rho, T jx, T jy, T jz, T ch) {
  const int nx = gm.nx, ny = gm.ny;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, nx)) continue;
      const T wgt = wx[a] * wy[b];
      const int64_t node = (int64_t)iy * nx + ix;
      atomic_add4(dep + node, wgt * rho, wgt * jx, wgt * jy, wgt * jz, gm);
      if (chi) dadd(chi + node, wgt * ch, gm);
    }
  }
}

template <int P, typename T>
__device__ __forceinline__ void deposit_perp(V2<T>* tj, const Geom& gm, int ix0, int iy0,
                                             const T* wx, const T* wy, T jx, T jy) {
  const int nx = gm.nx, ny = gm.ny;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (!in_interior(ix, nx)) continue;
      const T wgt = wx[a] * wy[b];
      atomic_add2(tj + (int64_t)iy * nx + ix, wgt * jx, wgt * jy, gm);
    }
  }
}

// Stencil of a position given in FP64 (exact division, as in the oracle).
template <int P, typename T>
__device__ __forceinline__ void stencil_f64(const Geom& gm, double x, double y, int& ix0, int& iy0, T* wx, T* wy) {
  int jx, jy;
  double fx, fy;
  split_coord(x, gm.xmin, gm.dx, jx, fx);
  split_coord(y, gm.ymin, gm.dy, jy, fy);
  ix0 = shape_weights<P, T>(jx, T(fx), wx);
  iy0 = shape_weights<P, T>(jy, T(fy), wy);
}

// q w / A (an electron: q = -1).  FP64 mode divides by A = dx dy as the oracle does; FP32
// mode multiplies by the precomputed 1/A.
template <typename T>
__device__ __forceinline__ T charge_density(T w, const Geom& gm, T q = T(-1)) {
  if constexpr (sizeof(T) == 8) return (q * w) / (gm.dx * gm.dy);
  else return q * w * gm.f_inv_area;
}

// Removal rule (a reading; the paper is silent): finite, inside the open box,
// 1 + Psi >= psi_guard.
__device__ __forceinline__ bool state_ok(const Geom& gm, double x, double y, double opp, double guard) {
  return isfinite(x) && isfinite(y) && isfinite(opp) && x > gm.xmin && x < gm.xmax && y > gm.ymin &&
         y < gm.ymax && opp >= guard;
}

// ---------------------------------------------------------------- init
// Placement of plasma particle p (Sec. 2: unperturbed plasma ahead of the beams): cell-row-major,
// ppc_x x ppc_y at sub-cell centres, at rest.  A multi-species grid (MS) places each species'
// block [off[s], off[s + 1]) with that species' particles per cell, profile and density.
template <typename T, bool MS>
__global__ void k_plasma_init(Plasma<T> pl, Geom gm, int ppx, int ppy, const double* prof, int npf,
                              double rmax, double n0s, SpeciesTab tab) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n) return;
  int64_t lp = p;
  if constexpr (MS) {
    const int s = species_of(tab, p);
    lp = p - tab.off[s];
    ppx = tab.ppx[s];
    ppy = tab.ppy[s];
    prof = tab.prof[s];
    npf = tab.npf[s];
    rmax = tab.rmax[s];
    n0s = tab.n0[s];
  }
  const int ppc = ppx * ppy;
  const int64_t c = lp / ppc;
  const int sub = (int)(lp - c * ppc);
  const int ix = (int)(c % gm.nx), iy = (int)(c / gm.nx);
  const int sx = sub % ppx, sy = sub / ppx;
  const double x = gm.xmin + ((double)ix + ((double)sx + 0.5) / ppx) * gm.dx;
  const double y = gm.ymin + ((double)iy + ((double)sy + 0.5) / ppy) * gm.dy;
  double dens = 1.0;
  if (prof) {
    const double r = sqrt(x * x + y * y);
    double t = r / rmax * (npf - 1);
    t = fmin(fmax(t, 0.0), (double)(npf - 1));
    int k0 = (int)floor(t);
    k0 = k0 < 0 ? 0 : (k0 > npf - 2 ? npf - 2 : k0);
    const double fr = t - (double)k0;
    dens = prof[k0] * (1.0 - fr) + prof[k0 + 1] * fr;
  }
  pl.x[p] = x;
  pl.y[p] = y;
  pl.psi[p] = 0.0;
  pl.ux[p] = T(0);
  pl.uy[p] = T(0);
  pl.w[p] = T(n0s * dens * (gm.dx * gm.dy / (double)ppc));
  pl.alive[p] = 1;
  if (pl.origin) pl.origin[p] = (int32_t)p;
  for (int k = 0; k < kRing * 5; ++k) pl.hist[(int64_t)k * pl.n + p] = T(0);
  if (pl.hsum)
    for (int c = 0; c < 5; ++c) pl.hsum[(int64_t)c * pl.n + p] = 0.0f;
  if (pl.cell) {
    int jx, jy;
    double fx, fy;
    jx = (int)floor((x - gm.xmin) * gm.inv_dx);
    jy = (int)floor((y - gm.ymin) * gm.inv_dy);
    fx = (x - gm.xmin) * gm.inv_dx - jx;
    fy = (y - gm.ymin) * gm.inv_dy - jy;
    pl.cell[p] = (jy << 16) | jx;
    pl.fx[p] = (float)fx;
    pl.fy[p] = (float)fy;
    pl.opp[p] = 1.0f;
  }
}

// Deposit of the current plasma state (slice 0), or of the immobile background
// rho_ion = -(q w / A) deposited from the initial positions (ion_only; on a multi-species grid
// only the species with a neutralizing background).
template <int P, typename T, bool MS>
__global__ void k_deposit_initial(Plasma<T> pl, Geom gm, V4<T>* dep, T* chi, T* rho_ion, SpeciesTab tab) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n || !pl.alive[p]) return;
  int s = 0;
  if constexpr (MS) {
    s = species_of(tab, p);
    if (rho_ion && !tab.neutral[s]) return;
  }
  const SpC<T> sc = spc_of<T, MS>(tab, s);
  T wx[P + 1], wy[P + 1];
  int ix0, iy0;
  stencil_f64<P, T>(gm, pl.x[p], pl.y[p], ix0, iy0, wx, wy);
  const T qw = charge_density<T>(pl.w[p], gm, sc.q);
  if (rho_ion) {
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = iy0 + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = ix0 + a;
        if (!in_interior(ix, gm.nx)) continue;
        dadd(rho_ion + (int64_t)iy * gm.nx + ix, -(wx[a] * wy[b] * qw), gm);
      }
    }
    return;
  }
  const T ux = pl.ux[p], uy = pl.uy[p];
  const T opp = T(1.0 + pl.psi[p]);
  const T g = T(1) / opp;
  const T gam = (T(1) + ux * ux + uy * uy + opp * opp) * T(0.5) * g;
  const T uz = uz_of<T>(ux, uy, opp, pl.psi[p], g);
  deposit_full<P, T>(dep, chi, gm, ix0, iy0, wx, wy, qw * gam * g, qw * ux * g, qw * uy * g,
                     qw * uz * g, qw * sc.qm * g);
}

// FP32 multi-species grids: the initial charge of the species without a neutralizing
// background, sum q w S(x0) / A over their particles, accumulated in FP64 (c0 of the psi source).
template <int P>
__global__ void k_species_c0(Plasma<float> pl, Geom gm, double* out, SpeciesTab tab) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n) return;
  const int s = species_of(tab, p);
  if (tab.neutral[s]) return;
  double wx[P + 1], wy[P + 1];
  int ix0, iy0;
  stencil_f64<P, double>(gm, pl.x[p], pl.y[p], ix0, iy0, wx, wy);
  const double qw = tab.q[s] * (double)pl.w[p] * gm.inv_area;
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = iy0 + b;
    if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = ix0 + a;
      if (in_interior(ix, gm.nx)) atomicAdd(out + (int64_t)iy * gm.nx + ix, wx[a] * wy[b] * qw);
    }
  }
}

// ---------------------------------------------------------------- trial pass (predictor-corrector)
// Gather with B^(m-1), AB5 trial step to slice i+1, deposit J_perp of the trial
// particles into tj (Sec. 3.2, predictor-corrector field solver).  Within a slice only Bx, By
// change between the iterations: the FP32 path gathers the other four fields (ExmBy, EypBx,
// Ez, Bz) in the first iteration and keeps them per particle in pl.f4 (fmode 1), and the later
// iterations read them back and gather Bx, By alone (FM 2); FM 0 gathers all six.
template <int P, typename T, bool CACHE, bool MS, int FM>
__global__ void __launch_bounds__(kThreads) k_trial_pass(Plasma<T> pl, Geom gm, const T* __restrict__ gf, const T* __restrict__ bm,
                                                         V2<T>* tj, int slice, double guard, SpeciesTab tab) {
  pdl_trigger();
  pdl_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n || !pl.alive[p]) return;
  const SpC<T> sc = spc_of<T, MS>(tab, MS ? species_of(tab, p) : 0);
  const int64_t n = pl.n;
  T wx[P + 1], wy[P + 1];
  int ix0, iy0;
  T opp;
  int jx = 0, jy = 0;
  T fxr = T(0), fyr = T(0);
  if constexpr (CACHE) {
    const int cell = pl.cell[p];
    jx = cell & 0xFFFF;
    jy = cell >> 16;
    fxr = T(pl.fx[p]);
    fyr = T(pl.fy[p]);
    ix0 = shape_weights<P, T>(jx, fxr, wx);
    iy0 = shape_weights<P, T>(jy, fyr, wy);
    opp = T(pl.opp[p]);
  } else {
    stencil_f64<P, T>(gm, pl.x[p], pl.y[p], ix0, iy0, wx, wy);
    opp = T(1.0 + pl.psi[p]);
  }
  const T ux = pl.ux[p], uy = pl.uy[p];
  F6<T> F;
  if constexpr (CACHE && FM == 2) {
    const float4 c = pl.f4[p];
    const float2 b = gather_bperp<P>(bm, gm.nx, gm.ny, ix0, iy0, wx, wy);
    F.v[0] = c.x; F.v[1] = c.y; F.v[2] = c.z; F.v[3] = b.x; F.v[4] = b.y; F.v[5] = c.w;
  } else {
    F = gather6<P, T>(gf, bm, gm.nx, gm.ny, ix0, iy0, wx, wy);
    if constexpr (CACHE && FM == 1) pl.f4[p] = make_float4(F.v[0], F.v[1], F.v[2], F.v[5]);
  }
  T f[5];
  derivs<T, MS>(ux, uy, opp, F, f, sc.mqm);
  const T dz = CACHE ? T(gm.f_dz) : T(gm.dzeta);
  // AB5 combination beta_0 f_i + sum_{k>=1} beta_k f_{i-k}; FP32 reads the precomputed history part
  auto comb = [&](int c) -> T {
    if constexpr (CACHE) return T(ab5(0)) * f[c] + T(pl.hsum[(int64_t)c * n + p]);
    else return ab5_comb<T>(pl.hist, n, p, slice, c, f[c]);
  };
  const T cx = comb(0);
  const T cy = comb(1);
  const T tux = ux - dz * comb(2);
  const T tuy = uy - dz * comb(3);
  const T cpsi = comb(4);
  T twx[P + 1], twy[P + 1];
  int tix0, tiy0;
  T topp;
  if constexpr (CACHE) {
    // trial step in cell-relative coordinates (FP32 only)
    T ux_ = fxr - T(gm.f_dz_inv_dx) * cx;
    T uy_ = fyr - T(gm.f_dz_inv_dy) * cy;
    const T flx = floor(ux_), fly = floor(uy_);
    const int tjx = jx + (int)flx, tjy = jy + (int)fly;
    ux_ -= flx;
    uy_ -= fly;
    topp = opp - dz * cpsi;
    const T ax = T(tjx) + ux_, ay = T(tjy) + uy_;
    const bool ok = isfinite(ax) && isfinite(ay) && isfinite(topp) && ax > T(0) && ax < T(gm.nx) &&
                    ay > T(0) && ay < T(gm.ny) && topp >= T(gm.f_guard);
    if (!ok) return;
    tix0 = shape_weights<P, T>(tjx, ux_, twx);
    tiy0 = shape_weights<P, T>(tjy, uy_, twy);
  } else {
    const double tx = pl.x[p] - (double)dz * (double)cx;
    const double ty = pl.y[p] - (double)dz * (double)cy;
    const double tpsi = pl.psi[p] - (double)dz * (double)cpsi;
    if (!state_ok(gm, tx, ty, 1.0 + tpsi, guard)) return;
    topp = T(1.0 + tpsi);
    stencil_f64<P, T>(gm, tx, ty, tix0, tiy0, twx, twy);
  }
  const T qw = charge_density<T>(pl.w[p], gm, sc.q);
  const T tg = T(1) / topp;
  deposit_perp<P, T>(tj, gm, tix0, tiy0, twx, twy, qw * tux * tg, qw * tuy * tg);
}

// ---------------------------------------------------------------- FP32 psi source
// A plasma particle's share of the psi source rho - J_z (Eq. for psi) is q w S(x): rho_p - J_zp
// = q w (gamma - u_z) / (1 + psi) S with gamma - u_z = 1 + psi.  The FP32 path accumulates the
// source ion-subtracted, q w (S(x) - S(x0)) with x0 the particle's initial position (the ion
// it left behind), so the unit ion background never meets the small plasma response in an
// FP32 sum.  When both stencils share their base node the weight differences are formed as
// exact polynomial differences carrying the factor (x - x0); otherwise the two stencils are
// deposited with opposite signs.  Node coordinates u = (x - x_min) / dx enter split as cell +
// fraction; only the move u - u0 is formed from the FP64 fractions.

// Plasma particles per cell per axis, with the FP32 and FP64 reciprocals.
struct PpcInfo {
  int px, py;
  int pow2;   // both powers of two: the sub-cell offsets are exact in FP32
  float finv_x, finv_y;
  double inv_x, inv_y;
};

// Start (ion) node coordinate of plasma particle p, split as cell + fraction: u0 = cx + fx,
// v0 = cy + fy (the placement of k_plasma_init: 32-bit index arithmetic, the sub-cell offset
// (s + 1/2) / ppc).  With ppc a power of two the FP32 fraction is exact and the FP64 copy its
// widening (one conversion); otherwise the FP64 fraction is computed and rounded.  On this
// GPU every FP64 instruction issues on a slow pipe, so the split keeps them to a minimum.
struct Start {
  int cx, cy;
  float fx, fy;
  double dfx, dfy;
};
__device__ __forceinline__ Start start_coord(int64_t p, const Geom& gm, const PpcInfo& pc) {
  const int pi = (int)p;
  const int ppc = pc.px * pc.py;
  const int c = ppc == 1 ? pi : pi / ppc;
  const int sub = pi - c * ppc;
  Start s;
  s.cy = c / gm.nx;
  s.cx = c - s.cy * gm.nx;
  const int sy = pc.px == 1 ? sub : sub / pc.px, sx = sub - sy * pc.px;
  if (pc.pow2) {
    s.fx = ((float)sx + 0.5f) * pc.finv_x;
    s.fy = ((float)sy + 0.5f) * pc.finv_y;
    s.dfx = (double)s.fx;
    s.dfy = (double)s.fy;
  } else {
    s.dfx = ((double)sx + 0.5) * pc.inv_x;
    s.dfy = ((double)sy + 0.5) * pc.inv_y;
    s.fx = (float)s.dfx;
    s.fy = (float)s.dfy;
  }
  return s;
}

// u - u0 in FP32 for u = j + df (df the FP64 fraction) and the start j0 + df0: the FP64
// fraction difference is exact, so a small move keeps its full relative precision.
__device__ __forceinline__ float move_of(int j, double df, int j0, double df0) {
  return (float)(j - j0) + (float)(df - df0);
}

// Weights w at u = j + d, w0 at u0 = j0 + d0 (bases b, b0) and, when b == b0, dw = w - w0 from
// the polynomial differences (each proportional to dl = u - u0).
template <int P>
__device__ __forceinline__ void weight_diff(int j, float d, int j0, float d0, float dl, float* w, float* w0, float* dw,
                                            int& b, int& b0) {
  b = shape_weights<P, float>(j, d, w);
  b0 = shape_weights<P, float>(j0, d0, w0);
  if (b != b0) return;
  if constexpr (P == 0) {
    dw[0] = 0.0f;
  } else if constexpr (P == 1) {
    dw[0] = -dl;
    dw[1] = dl;
  } else if constexpr (P == 2) {
    // offsets from the shared nearest node: e - e0 = u - u0
    const float s = (d >= 0.5f ? d - 1.0f : d) + (d0 >= 0.5f ? d0 - 1.0f : d0);
    dw[0] = -0.5f * dl * (1.0f - s);
    dw[1] = -dl * s;
    dw[2] = 0.5f * dl * (1.0f + s);
  } else {
    const float s = d + d0, q = d * d + d * d0 + d0 * d0;
    const float a = (1.0f - d) * (1.0f - d) + (1.0f - d) * (1.0f - d0) + (1.0f - d0) * (1.0f - d0);
    const float k = dl * (1.0f / 6.0f);
    dw[0] = -k * a;
    dw[1] = k * (3.0f * q - 6.0f * s);
    dw[2] = k * (3.0f + 3.0f * s - 3.0f * q);
    dw[3] = k * q;
  }
}

template <int P>
__device__ __forceinline__ void add_stencil(float* ps, int nx, int ny, int bx, int by, const float* wx, const float* wy,
                                            float q) {
#pragma unroll
  for (int b = 0; b <= P; ++b) {
    const int iy = by + b;
    if (!in_interior(iy, ny)) continue;
#pragma unroll
    for (int a = 0; a <= P; ++a) {
      const int ix = bx + a;
      if (in_interior(ix, nx)) atomicAdd(ps + (int64_t)iy * nx + ix, q * wx[a] * wy[b]);
    }
  }
}

// Quadratic B-spline B2(t) (t = u - node) and B2(t0 + dl) - B2(t0) for an exact dl: within one
// polynomial piece the difference carries the factor dl; across a piece boundary tb it is split
// there, (B2(t) - B2(tb)) + (B2(tb) - B2(t0)), with t - tb = (t0 - tb) + dl.  t0 (a start offset
// on the half-cell lattice) and tb are exact in FP32, so every factor is formed without
// cancellation.
__device__ __forceinline__ int b2_piece(float t) {
  const float a = fabsf(t);
  return a < 0.5f ? 0 : (a < 1.5f ? (t > 0.0f ? 1 : -1) : (t > 0.0f ? 2 : -2));
}
__device__ __forceinline__ float b2_value(float t) {
  const float a = fabsf(t);
  return a < 0.5f ? 0.75f - t * t : (a < 1.5f ? 0.5f * (1.5f - a) * (1.5f - a) : 0.0f);
}
__device__ __forceinline__ float b2_within(float t, float t0, float dl, int pc) {
  if (pc == 0) return -dl * (t + t0);
  if (pc == 1 || pc == -1) return -0.5f * (pc > 0 ? dl : -dl) * (3.0f - fabsf(t) - fabsf(t0));
  return 0.0f;
}
__device__ __forceinline__ float b2_diff(float t0, float dl) {
  const float t = t0 + dl;
  const int p = b2_piece(t), p0 = b2_piece(t0);
  if (p == p0) return b2_within(t, t0, dl, p);
  const float tb = (float)(p < p0 ? p : p0) + 0.5f;   // adjacent pieces: boundary at lo + 1/2
  return b2_within(t, tb, (t0 - tb) + dl, p) + b2_within(tb, t0, tb - t0, p0);
}

// q w (S(u, v) - S(u0, v0)) into ps; the new position u = jx + fx (FP32 fraction fx, FP64 dfx),
// v = jy + fy, and the start s0.
template <int P>
__device__ __forceinline__ void deposit_psi_src(float* ps, const Geom& gm, int jx, float fx, double dfx, int jy, float fy,
                                                double dfy, const Start& s0, float qw) {
  const float dlx = move_of(jx, dfx, s0.cx, s0.dfx), dly = move_of(jy, dfy, s0.cy, s0.dfy);
  if constexpr (P == 2) {
    // quadratic: the cell-centred start sits on a piece boundary, so the two stencils' bases
    // differ by one for about half the particles; difference over the 4-node union support.
    // With |u - u0| < 1 each node's offset crosses at most one piece boundary (pieces are one
    // cell wide), which b2_diff handles; farther moves take the two-stencil path below.
    // Nearest-node bases: floor(u + 1/2) - 1 = j + [f >= 1/2] - 1.
    const int bx = jx + (fx >= 0.5f ? 1 : 0) - 1, bx0 = s0.cx + (s0.fx >= 0.5f ? 1 : 0) - 1;
    const int by = jy + (fy >= 0.5f ? 1 : 0) - 1, by0 = s0.cy + (s0.fy >= 0.5f ? 1 : 0) - 1;
    if (fabsf(dlx) < 1.0f && fabsf(dly) < 1.0f) {
      const int ux = bx < bx0 ? bx : bx0, uy = by < by0 ? by : by0;
      const float tx0 = (float)(s0.cx - ux) + s0.fx, ty0 = (float)(s0.cy - uy) + s0.fy;   // u0 - ux, v0 - uy
      float wy[4], w0x[4], dwx[4], dwy[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float sx0 = tx0 - (float)k, sy0 = ty0 - (float)k;
        w0x[k] = b2_value(sx0);
        wy[k] = b2_value(sy0 + dly);
        dwx[k] = b2_diff(sx0, dlx);
        dwy[k] = b2_diff(sy0, dly);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int iy = uy + b;
        if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const int ix = ux + a;
          const float val = dwx[a] * wy[b] + w0x[a] * dwy[b];
          if (val != 0.0f && in_interior(ix, gm.nx)) atomicAdd(ps + (int64_t)iy * gm.nx + ix, qw * val);
        }
      }
      return;
    }
  }
  float wx[P + 1], w0x[P + 1], dwx[P + 1], wy[P + 1], w0y[P + 1], dwy[P + 1];
  int bx, bx0, by, by0;
  weight_diff<P>(jx, fx, s0.cx, s0.fx, dlx, wx, w0x, dwx, bx, bx0);
  weight_diff<P>(jy, fy, s0.cy, s0.fy, dly, wy, w0y, dwy, by, by0);
  if (bx == bx0 && by == by0) {
    // S - S0 = (wx - w0x) wy + w0x (wy - w0y)
#pragma unroll
    for (int b = 0; b <= P; ++b) {
      const int iy = by + b;
      if (!in_interior(iy, gm.ny)) continue;
#pragma unroll
      for (int a = 0; a <= P; ++a) {
        const int ix = bx + a;
        if (in_interior(ix, gm.nx)) atomicAdd(ps + (int64_t)iy * gm.nx + ix, qw * (dwx[a] * wy[b] + w0x[a] * dwy[b]));
      }
    }
  } else {
    add_stencil<P>(ps, gm.nx, gm.ny, bx, by, wx, wy, qw);
    add_stencil<P>(ps, gm.nx, gm.ny, bx0, by0, w0x, w0y, -qw);
  }
}

// The ion left behind by a removed particle: -q w S(u0, v0).
template <int P>
__device__ __forceinline__ void deposit_ion_src(float* ps, const Geom& gm, const Start& s0, float qw) {
  float wx[P + 1], wy[P + 1];
  const int bx = shape_weights<P, float>(s0.cx, s0.fx, wx);
  const int by = shape_weights<P, float>(s0.cy, s0.fy, wy);
  add_stencil<P>(ps, gm.nx, gm.ny, bx, by, wx, wy, -qw);
}

// ---------------------------------------------------------------- final pass
// Gather with the converged fields of slice i, store f_i in the AB5 history,
// advance to slice i+1, apply the removal rule and deposit rho, J, chi there.
// Resident CTAs the FP32 final pass is compiled for: the pass is memory-latency bound, and a
// 48-register budget (64 for the cubic shape; neither spills) keeps 30 % more warps resident
// than its unconstrained 62 (70) registers allow: 3 % of the blowout512 sweep.
template <int P, typename T> constexpr int final_min_blocks() {
  return sizeof(T) == 4 ? 65536 / ((P == 3 ? 64 : 48) * kThreads) : 1;
}

// FM 2 (FP32, after a predictor-corrector whose first iteration kept the slice's ExmBy, EypBx,
// Ez, Bz per particle in pl.f4): read those back and gather the converged Bx, By alone.
template <int P, typename T, bool CACHE, bool MS, int FM>
__global__ void __launch_bounds__(kThreads, final_min_blocks<P, T>()) k_final_pass(Plasma<T> pl, Geom gm, const T* __restrict__ gf, const T* __restrict__ bm,
                                                         V4<T>* dep, T* chi, float* ps, PpcInfo pc, int slice,
                                                         double guard, unsigned long long* removed, SpeciesTab tab) {
  pdl_trigger();
  pdl_wait();
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= pl.n) return;
  int sp = 0;
  int64_t lp = pl.origin ? (int64_t)pl.origin[p] : p;   // index in the initial placement (of its species)
  if constexpr (MS) {
    sp = species_of(tab, p);
    lp = p - tab.off[sp];
    pc.px = tab.ppx[sp];
    pc.py = tab.ppy[sp];
    pc.pow2 = tab.pow2[sp];
    pc.inv_x = tab.inv_px[sp];
    pc.inv_y = tab.inv_py[sp];
    pc.finv_x = tab.finv_px[sp];
    pc.finv_y = tab.finv_py[sp];
  }
  const SpC<T> sc = spc_of<T, MS>(tab, sp);
  Start s0{};
  if (ps) s0 = start_coord(lp, gm, pc);
  if (!pl.alive[p]) {
    if constexpr (sizeof(T) == 4)
      if (ps) deposit_ion_src<P>(ps, gm, s0, charge_density<T>(pl.w[p], gm, sc.q));
    return;
  }
  const int64_t n = pl.n;
  T wx[P + 1], wy[P + 1];
  int ix0, iy0;
  T opp;
  if constexpr (CACHE) {
    const int cell = pl.cell[p];
    ix0 = shape_weights<P, T>(cell & 0xFFFF, T(pl.fx[p]), wx);
    iy0 = shape_weights<P, T>(cell >> 16, T(pl.fy[p]), wy);
    opp = T(pl.opp[p]);
  } else {
    stencil_f64<P, T>(gm, pl.x[p], pl.y[p], ix0, iy0, wx, wy);
    opp = T(1.0 + pl.psi[p]);
  }
  const T ux = pl.ux[p], uy = pl.uy[p];
  F6<T> F;
  if constexpr (CACHE && FM == 2) {
    const float4 c = pl.f4[p];
    const float2 b = gather_bperp<P>(bm, gm.nx, gm.ny, ix0, iy0, wx, wy);
    F.v[0] = c.x; F.v[1] = c.y; F.v[2] = c.z; F.v[3] = b.x; F.v[4] = b.y; F.v[5] = c.w;
  } else {
    F = gather6<P, T>(gf, bm, gm.nx, gm.ny, ix0, iy0, wx, wy);
  }
  T f[5];
  derivs<T, MS>(ux, uy, opp, F, f, sc.mqm);
  T comb[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    T h[kRing + 1];   // h[k] = f_{i-k}
#pragma unroll
    for (int k = 1; k <= kRing; ++k) h[k] = pl.hist[((int64_t)(((slice - k) % kRing + kRing) % kRing) * 5 + c) * n + p];
    T acc = T(ab5(0)) * f[c];
#pragma unroll
    for (int k = 1; k <= kRing; ++k) acc += T(ab5(k)) * h[k];
    comb[c] = acc;
    if constexpr (CACHE) {
      // history part of the next slice's step: beta_1 f_i + beta_2 f_{i-1} + ... + beta_4 f_{i-3}
      T hn = T(ab5(1)) * f[c];
#pragma unroll
      for (int k = 2; k <= kRing; ++k) hn += T(ab5(k)) * h[k - 1];
      pl.hsum[(int64_t)c * n + p] = float(hn);
    }
  }
  const int slot = slice % kRing;
#pragma unroll
  for (int c = 0; c < 5; ++c) pl.hist[((int64_t)slot * 5 + c) * n + p] = f[c];
  const double dz = gm.dzeta;
  const double nxp = pl.x[p] - dz * (double)comb[0];
  const double nyp = pl.y[p] - dz * (double)comb[1];
  const double npsi = pl.psi[p] - dz * (double)comb[4];
  const T nux = ux - gsel<T>(dz, gm.f_dz) * comb[2];
  const T nuy = uy - gsel<T>(dz, gm.f_dz) * comb[3];
  const double nopp = 1.0 + npsi;
  if (!state_ok(gm, nxp, nyp, nopp, guard)) {
    pl.alive[p] = 0;
    atomicAdd(removed, 1ull);
    if constexpr (sizeof(T) == 4)
      if (ps) deposit_ion_src<P>(ps, gm, s0, charge_density<T>(pl.w[p], gm, sc.q));
    return;
  }
  pl.x[p] = nxp;
  pl.y[p] = nyp;
  pl.psi[p] = npsi;
  pl.ux[p] = nux;
  pl.uy[p] = nuy;
  T topp;
  int jx = 0, jy = 0;           // FP32 path: cell, FP64 and FP32 fraction of the new position
  double dfx = 0.0, dfy = 0.0;
  float frx = 0.0f, fry = 0.0f;
  if constexpr (CACHE) {
    const double ux_ = (nxp - gm.xmin) * gm.inv_dx, uy_ = (nyp - gm.ymin) * gm.inv_dy;
    const double flx = floor(ux_), fly = floor(uy_);
    jx = (int)flx;
    jy = (int)fly;
    dfx = ux_ - flx;
    dfy = uy_ - fly;
    frx = (float)dfx;
    fry = (float)dfy;
    pl.cell[p] = (jy << 16) | jx;
    pl.fx[p] = frx;
    pl.fy[p] = fry;
    topp = (float)nopp;
    pl.opp[p] = topp;
    ix0 = shape_weights<P, T>(jx, T(frx), wx);
    iy0 = shape_weights<P, T>(jy, T(fry), wy);
  } else {
    topp = T(nopp);
    stencil_f64<P, T>(gm, nxp, nyp, ix0, iy0, wx, wy);
  }
  const T qw = charge_density<T>(pl.w[p], gm, sc.q);
  const T g = T(1) / topp;
  const T gam = (T(1) + nux * nux + nuy * nuy + topp * topp) * T(0.5) * g;
  const T uz = uz_of<T>(nux, nuy, topp, npsi, g);
  deposit_full<P, T>(dep, chi, gm, ix0, iy0, wx, wy, qw * gam * g, qw * nux * g, qw * nuy * g,
                     qw * uz * g, qw * sc.qm * g);
  if constexpr (CACHE)
    if (ps) deposit_psi_src<P>(ps, gm, jx, frx, dfx, jy, fry, dfy, s0, qw);
}

template <typename T> Plasma<T> plasma_of(const hq_grid_s* g);
template <> Plasma<double> plasma_of<double>(const hq_grid_s* g) { return g->p64; }
template <> Plasma<float> plasma_of<float>(const hq_grid_s* g) { return g->p32; }

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

// Shape-order and species dispatch of the particle kernels: the default electron plasma runs
// the MS = false instances (electron constants folded in), multi-species grids MS = true.
#define HQ_PDISPATCH(ORDER, MULTI, CALL)                                                  \
  switch ((ORDER) * 2 + ((MULTI) ? 1 : 0)) {                                                \
    case 0: { constexpr int P = 0; constexpr bool M = false; CALL; } break;                 \
    case 1: { constexpr int P = 0; constexpr bool M = true; CALL; } break;                  \
    case 2: { constexpr int P = 1; constexpr bool M = false; CALL; } break;                 \
    case 3: { constexpr int P = 1; constexpr bool M = true; CALL; } break;                  \
    case 4: { constexpr int P = 2; constexpr bool M = false; CALL; } break;                 \
    case 5: { constexpr int P = 2; constexpr bool M = true; CALL; } break;                  \
    case 6: { constexpr int P = 3; constexpr bool M = false; CALL; } break;                 \
    default: { constexpr int P = 3; constexpr bool M = true; CALL; } break;                 \
  }

template <typename T>
void launch_plasma_init(const hq_grid_s* g, cudaStream_t s) {
  const double* prof = g->profile.empty() ? nullptr : g->d_profile;
  if (g->multi)
    k_plasma_init<T, true><<<blocks_for(g->np), kThreads, 0, s>>>(plasma_of<T>(g), g->geom, 1, 1, nullptr, 0, 0.0,
                                                                   0.0, g->sp);
  else
    k_plasma_init<T, false><<<blocks_for(g->np), kThreads, 0, s>>>(
        plasma_of<T>(g), g->geom, g->d.ppc_x, g->d.ppc_y, prof, (int)g->profile.size(), g->d.profile_rmax,
        g->d.n0_scale, g->sp);
}

template <typename T>
void launch_deposit_initial(const hq_grid_s* g, void* dep, void* chi, int ion_only, cudaStream_t s) {
  const unsigned nb = blocks_for(g->np);
  V4<T>* d = reinterpret_cast<V4<T>*>(dep);
  T* c = reinterpret_cast<T*>(chi);
  T* ion = ion_only ? reinterpret_cast<T*>(g->rho_ion) : nullptr;
  HQ_PDISPATCH(g->d.shape_order, g->multi,
               (k_deposit_initial<P, T, M><<<nb, kThreads, 0, s>>>(plasma_of<T>(g), g->geom, d, c, ion, g->sp)));
}

void launch_species_c0(const hq_grid_s* g, double* out, cudaStream_t s) {
  const unsigned nb = blocks_for(g->np);
  switch (g->d.shape_order) {
    case 0: k_species_c0<0><<<nb, kThreads, 0, s>>>(g->p32, g->geom, out, g->sp); break;
    case 1: k_species_c0<1><<<nb, kThreads, 0, s>>>(g->p32, g->geom, out, g->sp); break;
    case 2: k_species_c0<2><<<nb, kThreads, 0, s>>>(g->p32, g->geom, out, g->sp); break;
    default: k_species_c0<3><<<nb, kThreads, 0, s>>>(g->p32, g->geom, out, g->sp); break;
  }
}

template <typename T>
void launch_trial_pass(const hq_grid_s* g, int slice, int iter, cudaStream_t s) {
  const unsigned nb = blocks_for(g->np);
  // FP32: the first predictor-corrector iteration of a slice keeps the four static gathered
  // fields per particle, the others read them (HQ_NO_F4CACHE=1: every pass gathers all six)
  const int fmode = (sizeof(T) == 8 || g->no_f4) ? 0 : (iter == 0 ? 1 : 2);
  const T* gf = reinterpret_cast<const T*>(g->gf);
  const T* bm = reinterpret_cast<const T*>(g->bm);
  V2<T>* tj = reinterpret_cast<V2<T>*>(g->tj);
  constexpr bool C = sizeof(T) == 4;
  const double gd = g->d.psi_guard;
  HQ_PDISPATCH(g->d.shape_order, g->multi,
               (fmode == 2 ? launch_pdl(k_trial_pass<P, T, C, M, C ? 2 : 0>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom,
                                        gf, bm, tj, slice, gd, g->sp)
                : fmode == 1 ? launch_pdl(k_trial_pass<P, T, C, M, C ? 1 : 0>, nb, kThreads, 0, s, plasma_of<T>(g),
                                          g->geom, gf, bm, tj, slice, gd, g->sp)
                             : launch_pdl(k_trial_pass<P, T, C, M, 0>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom, gf,
                                          bm, tj, slice, gd, g->sp)));
}

template <typename T>
void launch_final_pass(const hq_grid_s* g, int slice, void* dep, void* chi, bool f4, cudaStream_t s) {
  const unsigned nb = blocks_for(g->np);
  const T* gf = reinterpret_cast<const T*>(g->gf);
  const T* bm = reinterpret_cast<const T*>(g->bm);
  V4<T>* d = reinterpret_cast<V4<T>*>(dep);
  T* c = reinterpret_cast<T*>(chi);
  constexpr bool C = sizeof(T) == 4;
  const double gd = g->d.psi_guard;
  unsigned long long* rm = g->d_removed;
  float* ps = psrc_of(g, dep);
  PpcInfo pc;
  pc.px = g->d.ppc_x;
  pc.py = g->d.ppc_y;
  pc.pow2 = (pc.px & (pc.px - 1)) == 0 && (pc.py & (pc.py - 1)) == 0;
  pc.inv_x = 1.0 / pc.px;
  pc.inv_y = 1.0 / pc.py;
  pc.finv_x = (float)pc.inv_x;
  pc.finv_y = (float)pc.inv_y;
  HQ_PDISPATCH(g->d.shape_order, g->multi,
               (f4 && C ? launch_pdl(k_final_pass<P, T, C, M, C ? 2 : 0>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom,
                                     gf, bm, d, c, ps, pc, slice, gd, rm, g->sp)
                        : launch_pdl(k_final_pass<P, T, C, M, 0>, nb, kThreads, 0, s, plasma_of<T>(g), g->geom, gf, bm,
                                     d, c, ps, pc, slice, gd, rm, g->sp)));
}
#undef HQ_PDISPATCH

template void launch_plasma_init<float>(const hq_grid_s*, cudaStream_t);
template void launch_plasma_init<double>(const hq_grid_s*, cudaStream_t);
template void launch_deposit_initial<float>(const hq_grid_s*, void*, void*, int, cudaStream_t);
template void launch_deposit_initial<double>(const hq_grid_s*, void*, void*, int, cudaStream_t);
template void launch_trial_pass<float>(const hq_grid_s*, int, int, cudaStream_t);
template void launch_trial_pass<double>(const hq_grid_s*, int, int, cudaStream_t);
template void launch_final_pass<float>(const hq_grid_s*, int, void*, void*, bool, cudaStream_t);
template void launch_final_pass<double>(const hq_grid_s*, int, void*, void*, bool, cudaStream_t);

}  // namespace hq
