// DST-I as dense matrix products on the 5th-generation tensor cores (tcgen05),
// for the FP32 path of the fast Poisson solver (Sec. 3.2: "fast Poisson solvers
// based on a Discrete Sine Transform of the first type").
//
// A Dirichlet solve is f = (2/nx)(2/ny) S_y [ (S_y s S_x) / lambda ] S_x.  With
// every operand kept K-major, each of the four products is a "TN" GEMM
//   D[m][n] = sum_k A[m][k] S[n][k]          (S symmetric)
// whose epilogue stores D transposed, so that the next product again reads its
// operand K-major: two such products give S_y s S_x.  R right-hand sides are
// stacked along m (R * 128-padded rows), so one launch transforms them all.
//
// Precision ("bf16x3"): every FP32 operand a is carried as a_hi + a_lo with
// a_hi = bf16(a), a_lo = bf16(a - a_hi) (16 significant bits); a product uses
// a_hi b_hi + a_hi b_lo + a_lo b_hi, accumulated in FP32 in tensor memory.
// The epilogue of each product re-splits its FP32 result for the next one and
// fuses the 1/lambda scaling (second product) or the final FP32 store (fourth).
// Precision "TF32x3" (the fused streamed solve below, instantiated on FP32 words): a_hi =
// a rounded to TF32 (cvt.rna), a_lo = a - a_hi, tcgen05.mma kind::tf32 (K = 8 per
// instruction); the byte layout of every stage, box and swizzle is the bf16 one, a 128-byte
// K block holding 32 elements instead of 64.
//
// Per-product kernel (k_dst_gemm, one product per launch; the allocation-free entry point
// at the end of this file runs it), one 128 x 128 output tile per CTA, 4 warps:
//   warp 0 lane 0  TMA producer: 128B-swizzled 128x64 bf16 boxes of A_hi, A_lo,
//                  S_hi, S_lo per stage (64 KB), 3-stage mbarrier ring;
//   warp 1 lane 0  MMA issuer: 12 tcgen05.mma (M=128, N=128, K=16) per stage,
//                  tcgen05.commit releases the stage, a final commit signals
//                  the epilogue;
//   warps 0-3      epilogue: tcgen05.ld 32x32b (lane = row), transposed store.
// Every wait on an mbarrier is bounded; on expiry the kernel sets a status bit,
// still drains its MMAs, frees its tensor memory and returns.
#include "hq_internal.cuh"

#include <algorithm>
#include <cstdlib>

namespace hq {

struct TensorMaps {
  CUtensorMap a0_hi, a0_lo;   // op[0] as [kMaxRhs * nyp][nxp]
  CUtensorMap a1_hi, a1_lo;   // op[1] as [kMaxRhs * nxp][nyp]
  CUtensorMap sx_hi[2], sx_lo[2];   // [nxp][nxp], boxes of 128 ([0]) or 64 ([1]) rows (per-product path)
  CUtensorMap sy_hi[2], sy_lo[2];   // [nyp][nyp]
  // fused solve, per N-tile width ([0]: 64, [1]: 32): S_x [nxp][nxp], or the fold matrix
  // [nxp][nxp/2], in boxes of BN rows; the FP32 scale [nyp][nxp] in 128 (x) by BN (y) boxes
  CUtensorMap bx_hi[2], bx_lo[2];
  CUtensorMap by_hi[2], by_lo[2];
  CUtensorMap scale[2];
  CUtensorMap scale_h[2];     // the shifted (Helmholtz) spectral factors, same boxes (explicit solver)
  int ctas[2];                // co-resident CTAs of each width
  bool wide_only;             // HQ_SOLVE_BN=64: never use the 32-wide tiles
  // resident fold-matrix solve (square folded grids, n = 256 or 512): the fold matrix in
  // 128-row boxes, op[0] and op[1] in BN-row boxes ([0]: 64, [1]: 32)
  bool rs;
  CUtensorMap rf_hi, rf_lo;
  CUtensorMap rx_hi[2][2], rx_lo[2][2];   // [operand][width]
  int rs_ctas[2];
};

namespace {

// A K block is 128 bytes of every operand row (one 128B-swizzle atom row): BK = 64 bf16
// elements, or 32 TF32 elements held in FP32 words (the TF32x3 split); byte sizes below are
// the same for both.
constexpr int BM = 128, BK = 64;
constexpr int A_BYTES = BM * 128;                  // 16 KB per A box
template <typename E> constexpr int kb_elems() { return 128 / (int)sizeof(E); }
// Tile shape per N-tile width: 128 (3 stages of 64 KB) or 64 (4 stages of 48 KB).
template <int BN, typename E = __nv_bfloat16> struct Cfg {
  static constexpr int B_BYTES = BN * 128;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // A_hi, A_lo, B_hi, B_lo
  static constexpr int STAGES = BN == 128 ? 3 : 4;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr uint32_t TMEM_COLS = BN;
  // instruction descriptor (kind::f16 with A = B = BF16 (1), or kind::tf32 with A = B = TF32
  // (2)): D = F32, both K-major, M = BM, N = BN
  static constexpr uint32_t FMT = sizeof(E) == 4 ? 2u : 1u;
  static constexpr uint32_t IDESC =
      (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  // the same with N = 2 BN: B_hi and B_lo, adjacent in a stage, read as one operand
  static constexpr uint32_t IDESC2 =
      (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(BN >> 2) << 17) | ((uint32_t)(BM >> 4) << 24);
};

struct Epi {
  int mode;          // 0: split + transposed bf16 store; 1: scale, split, store; 2: FP32 transposed store
  int P1;            // rows per right-hand side (padded), i.e. m extent per rhs
  int P2;            // padded n extent
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  const float* scale;   // [P2][P1]
  float* out_f32;       // [R][n_real][m_real]
  int m_real, n_real;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (about two seconds of SM clock); false and a status bit on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* status) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (4ll << 30)) {
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile, 128B swizzle: rows of 64 bf16 (128 B), 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t desc_k_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address, 16 B units
  d |= (uint64_t)1 << 16;                      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;            // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                      // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                      // layout: SWIZZLE_128B
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
// TF32 operands (kind::tf32, K = 8 per instruction: 32 bytes of each row, as for bf16)
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}
template <typename E>
__device__ __forceinline__ void mma_op(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  if constexpr (sizeof(E) == 4) mma_tf32(tmem_d, a, b, idesc, accum);
  else mma_bf16(tmem_d, a, b, idesc, accum);
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  tmem_ld32_issue(taddr, v);
  tmem_ld_wait();
}
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
// W (16 or 32) columns of a stacked accumulator: x[j] = D[c0 + j] + D[BN + c0 + j] of this
// thread's lane
template <int BN, int W>
__device__ __forceinline__ void tmem_ld_pair(uint32_t taddr, float* x) {
  uint32_t v[W], u[W];
  if constexpr (W == 32) {
    tmem_ld32_issue(taddr, v);
    tmem_ld32_issue(taddr + (uint32_t)BN, u);
  } else {
    static_assert(W == 16, "16 or 32 columns");
    tmem_ld16_issue(taddr, v);
    tmem_ld16_issue(taddr + (uint32_t)BN, u);
  }
  tmem_ld_wait();
#pragma unroll
  for (int j = 0; j < W; ++j) x[j] = __uint_as_float(v[j]) + __uint_as_float(u[j]);
}

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_dst_gemm(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
               const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo, int K, Epi ep,
               int* status) {
  using C = Cfg<BN>;
  constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES;
  constexpr uint32_t TMEM_COLS = C::TMEM_COLS;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* basep = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(basep + STAGES * STAGE_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // everything above overlaps the previous kernel (programmatic dependent launch)
  pdl_trigger();
  pdl_wait();

  if (warp == 0 && lane == 0) {
    // TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES && !mbar_wait(empty0 + 8 * s, ((kb / STAGES) - 1) & 1, status)) break;
      const uint32_t st = base + s * STAGE_BYTES;
      const uint32_t fb = full0 + 8 * s;
      mbar_expect_tx(fb, STAGE_BYTES);
      tma_load_2d(st, &ta_hi, kb * BK, m0, fb);
      tma_load_2d(st + A_BYTES, &ta_lo, kb * BK, m0, fb);
      tma_load_2d(st + 2 * A_BYTES, &tb_hi, kb * BK, n0, fb);
      tma_load_2d(st + 2 * A_BYTES + C::B_BYTES, &tb_lo, kb * BK, n0, fb);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(full0 + 8 * s, (kb / STAGES) & 1, status)) break;
      tc_fence_after();
      const uint32_t st = base + s * STAGE_BYTES;
      const uint64_t ah = desc_k_sw128(st), al = desc_k_sw128(st + A_BYTES);
      const uint64_t bh = desc_k_sw128(st + 2 * A_BYTES), bl = desc_k_sw128(st + 2 * A_BYTES + C::B_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        const uint64_t off = (uint64_t)((k * 32) >> 4);  // 16 bf16 = 32 B along K inside the swizzle row
        mma_bf16(tmem, ah + off, bh + off, C::IDESC, (kb | k) != 0 ? 1u : 0u);
        mma_bf16(tmem, ah + off, bl + off, C::IDESC, 1u);
        mma_bf16(tmem, al + off, bh + off, C::IDESC, 1u);
      }
      mma_commit(empty0 + 8 * s);
    }
    mma_commit(done);
  }
  __syncwarp();
  mbar_wait(done, 0, status);
  tc_fence_after();

  // ---------------------------------------------------------------- epilogue
  const int row = warp * 32 + lane;
  const int m = m0 + row;
  const int r = m / ep.P1, ml = m - r * ep.P1;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (ep.mode == 2) {
      if (ml < ep.m_real) {
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c0 + j;
          const float x = __uint_as_float(v[j]);
          bad |= !isfinite(x);
          if (n < ep.n_real) ep.out_f32[((int64_t)r * ep.n_real + n) * ep.m_real + ml] = x;
        }
        if (bad) atomicOr(status, DEV_NONFINITE);
      }
    } else {
      float sc[32];
      if (ep.mode == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j) sc[j] = __ldg(ep.scale + (int64_t)(n0 + c0 + j) * ep.P1 + ml);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = n0 + c0 + j;
        float x = __uint_as_float(v[j]);
        if (ep.mode == 1) x *= sc[j];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        const int64_t o = ((int64_t)r * ep.P2 + n) * ep.P1 + ml;
        ep.out_hi[o] = h;
        ep.out_lo[o] = l;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------- fused persistent solve
// A whole Dirichlet solve in one cooperative launch: the four products run as
// phases separated by grid-wide barriers, with tensor memory, mbarriers and the
// shared-memory ring set up once and the intermediates kept in L2.  Phase p
// contracts along x (p = 0, 2: operand op[0], matrix S_x) or along y (p = 1, 3:
// op[1], S_y); its epilogue writes the next phase's operand transposed.
//
// Folded order (fold_pair; n a multiple of 128): every operand row holds its n/2
// pair sums followed by its n/2 pair differences, the output columns are slots, and
// an N-tile of odd (even) slots contracts over the sums (differences) only, K = n/2,
// against the fold matrix.  Rows 2u, 2u+1 of a tile are a pair, i.e. adjacent TMEM
// lanes, so the epilogue folds the next operand with one warp shuffle.
//
// Tiles are 128 x BN (BN = 32 when every tile still gets its own CTA, else 64), one CTA
// of 256 threads per SM: warp 0 lane 0 issues the TMA loads (A_hi, A_lo, B_hi, B_lo of a
// 128-byte K block per stage, 4-stage ring), warp 1 lane 0 the MMAs (two per K step:
// A_hi x [B_hi; B_lo] with N = 2 BN, A_lo x B_hi with N = BN, into a 2 BN-column TMEM
// accumulator), and all 8 warps the epilogue, each warpgroup half of the columns.
struct SolveArgs {
  int R;                               // right-hand sides
  int nxp, nyp;                        // operand extents (= nx, ny when folded)
  int fold;
  void *op_hi[2], *op_lo[2];           // op[0]: [R][nyp][nxp], op[1]: [R][nxp][nyp] (bf16 or TF32 words)
  const float* scale;                  // [nyp][nxp]: (4/(nx ny)) / lambda, slot order when folded
  int final_mode;                      // 2: FP32 store into out [R][ny][nx]; 3: predictor-corrector mixing
  float* out;
  int nx, ny;
  float* bm;                           // mode 3: B <- w B_solved + (1 - w) B in bm[node * 2 + r]
  float w;
  double* rsum;                        // mode 3: sum (B_new - B_old)^2, sum B_new^2 added here (or null)
  unsigned long long* gbar;            // grid-barrier counter (zero at launch, reset by the last CTA)
  int* status;
  int barrier_skew;                    // added to the first barrier's target (fault injection; 0)
  // source phase ahead of the four products: 0 none (sources already in op[0]); 1 the psi,
  // Ez, Bz sources of a deposit record (sm); 2 the B_perp sources of the predictor-corrector (sb)
  int pre;
  SrcMain<float> sm;
  SrcBperp<float> sb;
};

// Source phase: every thread of the launch takes (row, column) items of the operand writer
// in turn (consecutive threads along a row), KB items at a time: all their reads are issued
// before any write, then the sources are evaluated, split into op[0] and the functor's own
// writes (clearing the trial J_perp) follow.
template <typename Sink, typename F, int NR>
__device__ __forceinline__ void solve_sources(const Geom& gm, const Sink& sink, const F& f) {
  constexpr int KB = 4;
  constexpr int NN = Sink::kFold ? 2 : 1;   // nodes per item
  const int w = visit_width<Sink>(gm);
  const int total = w * gm.ny;
  const int stride = gridDim.x * blockDim.x;
  for (int t0 = blockIdx.x * blockDim.x + threadIdx.x; t0 < total; t0 += KB * stride) {
    int iy[KB][NN], ix[KB][NN];
    typename F::In in[KB][NN];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int t = t0 + k * stride;
      const int row = t < total ? t / w : 0, tx = t < total ? t % w : 0;
      if constexpr (Sink::kFold) {
        iy[k][0] = iy[k][NN - 1] = fold_node(row, gm.ny);
        fold_pair(tx, gm.nx, ix[k][0], ix[k][NN - 1]);
      } else {
        iy[k][0] = row;
        ix[k][0] = tx;
      }
#pragma unroll
      for (int j = 0; j < NN; ++j) in[k][j] = t < total ? f.load(iy[k][j], ix[k][j]) : typename F::In{};
    }
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int t = t0 + k * stride;
      if (t >= total) break;
      float v[NN][NR];
#pragma unroll
      for (int j = 0; j < NN; ++j) f.eval(iy[k][j], ix[k][j], in[k][j], v[j]);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if constexpr (Sink::kFold) sink.put_pair(r, t / w, t % w, v[0][r], v[NN - 1][r]);
        else sink.put(r, t / w, t % w, v[0][r]);
      }
      if constexpr (F::kEffects) {
#pragma unroll
        for (int j = 0; j < NN; ++j) f.effects(iy[k][j], ix[k][j]);
      }
    }
  }
}
// Bounded mbarrier wait that also gives up once another thread of the CTA has.
__device__ __forceinline__ bool mbar_wait_a(uint32_t bar, uint32_t parity, int* status, volatile int* abort_f) {
  const long long t0 = clock64();
  uint32_t it = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 63u) == 0 && (*abort_f || clock64() - t0 > (4ll << 30))) {
      atomicOr(status, DEV_TIMEOUT);
      *abort_f = 1;
      return false;
    }
  }
  return true;
}

// Grid-wide barrier (all CTAs co-resident: cooperative launch).  The counter is zero at
// launch and only grows within it: barrier b completes at (b + 1) * gridDim.x arrivals; after
// the last barrier every CTA arrives once more and the last one resets the counter to zero,
// so a launch needs no host-side state (and can be replayed from a CUDA graph).  The proxy
// fences order the epilogue's generic stores before the other CTAs' TMA (async-proxy)
// loads of the next phase.  Bounded: on expiry, or once another CTA has reported a
// timeout, the CTA sets DEV_TIMEOUT and leaves.
__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned long long target, int* status,
                                             volatile int* abort_f) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!*abort_f) {
      asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
      const long long t0 = clock64();
      uint32_t it = 0;
      while (true) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) break;
        if ((++it & 15u) == 0 &&
            ((*reinterpret_cast<volatile int*>(status) & DEV_TIMEOUT) || clock64() - t0 > (4ll << 30))) {
          atomicOr(status, DEV_TIMEOUT);
          *abort_f = 1;
          break;
        }
      }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  return !*abort_f;
}

// The fused solve runs 256 threads per CTA (warps 0, 1: TMA producer, MMA issuer; all 8
// warps: epilogue) on N tiles 64 wide, or 32 wide when that still gives every tile its own
// CTA (twice the tiles, so more of the SMs take part in each product).
constexpr int kSolveThreads = 256;

// Shared memory of the solve: the stage ring, the FP32 scale tile of phase 1
// ([BN n][128 rows]), then the barriers (full, empty, done, scale) and the TMEM slot.
template <int BN> struct SolveSmem {
  static constexpr int STAGES = Cfg<BN>::STAGES;
  static constexpr int RING = STAGES * Cfg<BN>::STAGE_BYTES;
  static constexpr int SCALE = RING;
  static constexpr int BARS = SCALE + BN * BM * 4;
  static constexpr int BYTES = BARS + 256 + 1024 /*alignment*/;
};

template <int BN, bool RES, typename E>
__global__ void __launch_bounds__(kSolveThreads, 1)
    k_dst_solve(const __grid_constant__ CUtensorMap a0h, const __grid_constant__ CUtensorMap a0l,
                const __grid_constant__ CUtensorMap a1h, const __grid_constant__ CUtensorMap a1l,
                const __grid_constant__ CUtensorMap bxh, const __grid_constant__ CUtensorMap bxl,
                const __grid_constant__ CUtensorMap byh, const __grid_constant__ CUtensorMap byl,
                const __grid_constant__ CUtensorMap scm, const SolveArgs a) {
  using C = Cfg<BN, E>;
  using L = SolveSmem<BN>;
  constexpr int STAGES = C::STAGES, STAGE_BYTES = C::STAGE_BYTES;
  constexpr int KE = kb_elems<E>();   // elements per K block
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* basep = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(basep + L::BARS);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  const uint32_t sbar = smem_u32(bars + 2 * STAGES + 1);
  const float* scale_s = reinterpret_cast<const float*>(basep + L::SCALE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_f = &s_abort;

  if (threadIdx.x == 0) {
    for (const CUtensorMap* m : {&a0h, &a0l, &a1h, &a1l, &bxh, &bxl, &byh, &byl, &scm})
      prefetch_map(m);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    mbar_init(sbar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // stage-ring, accumulator and scale-tile counters across tiles
  uint32_t kb_run = 0, tiles_run = 0, scales_run = 0;
  auto phase_geom = [&](int q, int& P1, int& P2, int& mt, int& tiles, int& nk) {
    const bool ax = (q & 1) == 0;
    P1 = ax ? a.nyp : a.nxp;
    P2 = ax ? a.nxp : a.nyp;
    mt = a.R * P1 / BM;
    tiles = mt * (P2 / BN);
    nk = (a.fold ? P2 / 2 : P2) / KE;
  };
  // both axes' geometry and this CTA's first tile, computed before the first phase (after a
  // grid barrier they would sit on the path to the phase's first TMA issue)
  int P1x, P2x, mtx, tilesx, nkx, P1y, P2y, mty, tilesy, nky;
  phase_geom(0, P1x, P2x, mtx, tilesx, nkx);
  phase_geom(1, P1y, P2y, mty, tilesy, nky);
  const int final_mode = a.final_mode;
  const int t0 = (int)blockIdx.x;
  const int m0x = (t0 % mtx) * BM, n0x = (t0 / mtx) * BN, rx = m0x / P1x;
  const int m0y = (t0 % mty) * BM, n0y = (t0 / mty) * BN, ry = m0y / P1y;
  // source phase (its writes reach the other CTAs' TMA loads through the barrier's proxy fences)
  const unsigned nb0 = a.pre ? 1u : 0u;   // barriers before phase 0
  bool go = true;
  if (a.pre) {
    const Geom& gm = a.pre == 1 ? a.sm.gm : a.sb.gm;
    E* hi0 = reinterpret_cast<E*>(a.op_hi[0]);
    E* lo0 = reinterpret_cast<E*>(a.op_lo[0]);
    if (a.fold) {
      const SinkFold<E> sink{hi0, lo0, a.nx, a.ny};
      if (a.pre == 1) solve_sources<SinkFold<E>, SrcMain<float>, 3>(gm, sink, a.sm);
      else solve_sources<SinkFold<E>, SrcBperp<float>, 2>(gm, sink, a.sb);
    } else {
      const SinkSplit<E> sink{hi0, lo0, a.nxp, a.nyp};
      if (a.pre == 1) solve_sources<SinkSplit<E>, SrcMain<float>, 3>(gm, sink, a.sm);
      else solve_sources<SinkSplit<E>, SrcBperp<float>, 2>(gm, sink, a.sb);
    }
    go = grid_barrier(a.gbar, (unsigned long long)gridDim.x + (unsigned)a.barrier_skew, a.status, abort_f);
  }
  for (int p = 0; p < 4 && go; ++p) {
    const bool along_x = (p & 1) == 0;
    // rows per rhs, output columns (= contraction extent), tiles, K blocks
    const int P1 = along_x ? P1x : P1y, P2 = along_x ? P2x : P2y, mt = along_x ? mtx : mty;
    const int tiles = along_x ? tilesx : tilesy, nk = along_x ? nkx : nky;
    const CUtensorMap* tah = along_x ? &a0h : &a1h;
    const CUtensorMap* tal = along_x ? &a0l : &a1l;
    const CUtensorMap* tbh = along_x ? &bxh : &byh;
    const CUtensorMap* tbl = along_x ? &bxl : &byl;
    const int mode = p == 3 ? final_mode : (p == 1 ? 1 : 0);
    if (p == 3) pdl_trigger();
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const bool first = tile == t0;
      const int m0 = first ? (along_x ? m0x : m0y) : (tile % mt) * BM;
      const int n0 = first ? (along_x ? n0x : n0y) : (tile / mt) * BN;
      const int r = first ? (along_x ? rx : ry) : m0 / P1, ml0 = m0 - r * P1;   // a tile lies within one rhs
      const int koff = (a.fold && n0 >= P2 / 2) ? P2 / 2 : 0;
      if (warp == 0 && lane == 0) {
        // TMA producer (and the scale tile of the spectral division)
        if (mode == 1) {
          mbar_expect_tx(sbar, BN * BM * 4);
          tma_load_2d(base + L::SCALE, &scm, ml0, n0, sbar);
        }
        for (int kb = 0; kb < nk; ++kb) {
          const uint32_t g = kb_run + kb;
          const int s = g % STAGES;
          const uint32_t st = base + s * STAGE_BYTES;
          const uint32_t fb = full0 + 8 * s;
          // a tile starts on a drained ring (every thread waited for the previous tile's last
          // MMA), so only a stage reused within the tile needs its release
          if (kb >= STAGES && !mbar_wait_a(empty0 + 8 * s, ((g / STAGES) - 1) & 1, a.status, abort_f)) break;
          mbar_expect_tx(fb, STAGE_BYTES);
          tma_load_2d(st, tah, koff + kb * KE, m0, fb);
          tma_load_2d(st + A_BYTES, tal, koff + kb * KE, m0, fb);
          tma_load_2d(st + 2 * A_BYTES, tbh, kb * KE, n0, fb);
          tma_load_2d(st + 2 * A_BYTES + C::B_BYTES, tbl, kb * KE, n0, fb);
        }
      } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (int kb = 0; kb < nk; ++kb) {
          const uint32_t g = kb_run + kb;
          const int s = g % STAGES;
          if (!mbar_wait_a(full0 + 8 * s, (g / STAGES) & 1, a.status, abort_f)) break;
          tc_fence_after();
          const uint32_t st = base + s * STAGE_BYTES;
          const uint64_t ah = desc_k_sw128(st), al = desc_k_sw128(st + A_BYTES);
          const uint64_t bh = desc_k_sw128(st + 2 * A_BYTES);
          // columns [0, BN): A_hi B_hi + A_lo B_hi; columns [BN, 2 BN): A_hi B_lo (one MMA
          // with N = 2 BN covers both A_hi products: the tensor core's cost here is per instruction);
          // four 32-byte K steps per block (K = 16 bf16 or 8 TF32 each)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint64_t off = (uint64_t)((k * 32) >> 4);
            mma_op<E>(tmem, ah + off, bh + off, C::IDESC2, (kb | k) != 0 ? 1u : 0u);
            mma_op<E>(tmem, al + off, bh + off, C::IDESC, 1u);
          }
          mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);
      }
      __syncwarp();
      mbar_wait_a(done, tiles_run & 1, a.status, abort_f);
      if (mode == 1) mbar_wait_a(sbar, scales_run & 1, a.status, abort_f);
      tc_fence_after();

      // ------------------------------------------------ epilogue: TMEM lane = tile row; the
      // two warpgroups take one half of the columns each (a warp reads the lanes of its
      // quarter of the tile, warp % 4)
      constexpr int CH = BN / 2;
      const int row = (warp & 3) * 32 + lane;
      const int ml = ml0 + row;
      const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
      const int c0 = (warp >> 2) * CH;
      if (mode <= 1) {
        // scale (phase 1), fold with the pair partner (one shuffle), split and store the next
        // operand transposed: folded, even rows hold pair sums (column u), odd rows pair
        // differences (column P1/2 + u)
        const bool odd = (ml & 1) != 0, wall = a.fold && (ml >> 1) == P1 / 4;
        const int fcol = a.fold ? (odd ? P1 / 2 + (ml >> 1) : (ml >> 1)) : ml;
        E* oh = reinterpret_cast<E*>(a.op_hi[along_x ? 1 : 0]);
        E* ol = reinterpret_cast<E*>(a.op_lo[along_x ? 1 : 0]);
        {
          float x[CH];
          tmem_ld_pair<BN, CH>(tl + (uint32_t)c0, x);
          if (mode == 1) {
#pragma unroll
            for (int j = 0; j < CH; ++j) x[j] *= scale_s[(c0 + j) * BM + row];
          }
          if (a.fold) {
            // all exchanges first, so that the warp's shuffles overlap
            float y[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) y[j] = __shfl_xor_sync(0xffffffffu, x[j], 1);
#pragma unroll
            for (int j = 0; j < CH; ++j) x[j] = odd ? (wall ? 0.0f : y[j] - x[j]) : (wall ? y[j] : x[j] + y[j]);
          }
#pragma unroll
          for (int j = 0; j < CH; ++j) put_split(oh, ol, ((int64_t)r * P2 + n0 + c0 + j) * P1 + fcol, x[j]);
        }
      } else {
        // node of this row (rows run along x in the last phase)
        const int xn = a.fold ? fold_node(ml, a.nx) : ml;
        float x[CH];
        tmem_ld_pair<BN, CH>(tl + (uint32_t)c0, x);
        float d2 = 0.0f, b2 = 0.0f;   // mode 3 with RES: this thread's share of the residual (FP32)
        if (xn < a.nx) {
          auto ynode = [&](int j) { return a.fold ? fold_node(n0 + c0 + j, a.ny) : n0 + c0 + j; };
          if (mode == 2) {
#pragma unroll
            for (int j = 0; j < CH; ++j) {
              const int yn = ynode(j);
              if (yn < a.ny) a.out[((int64_t)r * a.ny + yn) * a.nx + xn] = x[j];
            }
          } else {
            // predictor-corrector mixing into bm[r] (all loads first, then mix and store)
            float old[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
              const int yn = ynode(j);
              const int64_t node = (int64_t)yn * a.nx + xn;
              old[j] = yn < a.ny ? a.bm[node * 2 + r] : 0.0f;
            }
            bool bad = false;
#pragma unroll
            for (int j = 0; j < CH; ++j) {
              const int yn = ynode(j);
              if (yn >= a.ny) continue;
              bad |= !isfinite(x[j]);
              const int64_t node = (int64_t)yn * a.nx + xn;
              const float nb = a.w * x[j] + (1.0f - a.w) * old[j];
              a.bm[node * 2 + r] = nb;
              if constexpr (RES) {
                const float d = nb - old[j];
                d2 += d * d;
                b2 += nb * nb;
              }
            }
            if (bad) atomicOr(a.status, DEV_NONFINITE);
          }
        }
        if constexpr (RES)
          if (mode == 3) pc_residual_add(a.rsum, (double)d2, (double)b2);   // every lane (mode is uniform)
      }
      kb_run += nk;
      ++tiles_run;
      if (mode == 1) ++scales_run;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (*abort_f) break;
    }
    if (p < 3 && !grid_barrier(a.gbar,
                               (unsigned long long)(nb0 + p + 1) * gridDim.x +
                                   (nb0 == 0 && p == 0 ? (unsigned)a.barrier_skew : 0u),
                               a.status, abort_f))
      break;
  }
  // exit arrival: the last CTA through resets the counter for the next launch
  if (threadIdx.x == 0 && !*abort_f) {
    const unsigned long long seen = atomicAdd(a.gbar, 1ull);
    if (seen == (nb0 + 4ull) * gridDim.x - 1ull) atomicExch(a.gbar, 0ull);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)) : "memory");
  }
}

// ---------------------------------------------------------------- resident fold-matrix solve
// The same four products for a square folded grid (nx = ny = n, n = 256 or 512) with the
// operand roles swapped: each CTA owns one block of 128 output slots for the whole launch,
// so its 128 x n/2 slice of the fold matrix (bf16 hi + lo, 64 or 128 KB) is loaded into
// shared memory once, while the source phase runs, and only the data operand (BN rows of
// the previous phase's output) is streamed per tile:
//   D[s][c] = sum_u F[s][u] X[c][koff + u]   (A = F in shared memory, B = X streamed),
// with koff = 0 for the odd-index slots (pair sums) and n/2 for the even ones (differences).
// TMEM lane = output slot s, column = data row c.  The fold of the next operand pairs
// adjacent columns of one thread (no shuffle), and each thread stores its row of the next
// operand as contiguous 16-byte runs.  The third product writes its rows in node order, so
// the last one's output columns are consecutive x nodes.
template <int BN> struct RsSmem {
  static constexpr int KB_MAX = 4;                          // folded K = n/2 <= 256
  static constexpr int F = 0;                               // F_hi blocks 0..3, F_lo blocks 4..7
  static constexpr int STAGE = 2 * BN * BK * 2;             // X_hi + X_lo rows of one K block
  static constexpr int RING = 2 * KB_MAX * A_BYTES;
  static constexpr int BARS = RING + KB_MAX * STAGE;
  static constexpr int BYTES = BARS + 256 + 1024 /*alignment*/;
};

// bf16 hi/lo split of 8 values packed for two 16-byte stores.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * k]), h1 = __float2bfloat16_rn(v[2 * k + 1]);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * k] - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * k + 1] - __bfloat162float(h1));
    h[k] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
    l[k] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Epilogue of one thread's CH consecutive columns (data rows i0 .. i0 + CH - 1 of rhs r) of
// output slot s.  Modes 0/1 (1: times the 1/lambda factors sc) fold adjacent column pairs into
// the next operand's row (r, orow) (orow = s, or its node for the third product): pair sums at column v, differences at n/2 + v (the wall
// pair (0, n/2) keeps x_{n/2} as its sum and 0 as its difference).  Mode 2 stores the
// solution (rows in node order: columns are consecutive x nodes); mode 3 is rs_mix.
template <int CH>
__device__ __forceinline__ void rs_epilogue(const SolveArgs& a, int mode, int s, int orow, int r, int i0, float* x,
                                            const float* sc, __nv_bfloat16* oh, __nv_bfloat16* ol) {
  const int n = a.nx, H = n / 2;
  if (mode <= 1) {
    if (mode == 1) {
#pragma unroll
      for (int j = 0; j < CH; ++j) x[j] *= sc[j];
    }
    float sum[CH / 2], dif[CH / 2];
    const int v0 = i0 >> 1;
#pragma unroll
    for (int k = 0; k < CH / 2; ++k) {
      const bool wall = v0 + k == n / 4;
      sum[k] = wall ? x[2 * k + 1] : x[2 * k] + x[2 * k + 1];
      dif[k] = wall ? 0.0f : x[2 * k] - x[2 * k + 1];
    }
    const int64_t base = ((int64_t)r * n + orow) * n;
#pragma unroll
    for (int k = 0; k < CH / 2; k += 8) {
      uint4 h, l;
      split8(sum + k, h, l);
      *reinterpret_cast<uint4*>(oh + base + v0 + k) = h;
      *reinterpret_cast<uint4*>(ol + base + v0 + k) = l;
      split8(dif + k, h, l);
      *reinterpret_cast<uint4*>(oh + base + H + v0 + k) = h;
      *reinterpret_cast<uint4*>(ol + base + H + v0 + k) = l;
    }
  } else if (mode == 2) {
    const int yn = fold_node(s, n);
    float4* o = reinterpret_cast<float4*>(a.out + ((int64_t)r * a.ny + yn) * a.nx + i0);
#pragma unroll
    for (int q = 0; q < CH / 4; ++q) o[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  }
}

// Source phase of the resident fold-matrix solve (square folded grid, n <= 512): a CTA takes
// whole rows (RPP per pass, all their reads issued first), its threads read and evaluate the
// sources at consecutive nodes of a row (coalesced), stage them in shared memory S
// ([RPP rows][NR][n] floats), and then write the folded pairs (x_a + x_b, x_a - x_b) of
// consecutive folded columns.
template <typename F, int NR>
__device__ __forceinline__ void solve_sources_rows(const Geom& gm, const F& f, const SinkFold<__nv_bfloat16>& sink,
                                                   float* S) {
  constexpr int NPT = 2;   // nodes per thread per row (n <= 2 x 256)
  constexpr int RPP = 4;   // rows per pass
  const int n = gm.nx, w = n / 2;
  for (int sy0 = blockIdx.x; sy0 < gm.ny; sy0 += RPP * gridDim.x) {
    typename F::In in[RPP][NPT];
    int iy[RPP];
#pragma unroll
    for (int q = 0; q < RPP; ++q) {
      const int sy = sy0 + q * gridDim.x;
      iy[q] = sy < gm.ny ? fold_node(sy, gm.ny) : -1;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int x = threadIdx.x + k * kSolveThreads;
        in[q][k] = (iy[q] >= 0 && x < n) ? f.load(iy[q], x) : typename F::In{};
      }
    }
#pragma unroll
    for (int q = 0; q < RPP; ++q) {
      if (iy[q] < 0) continue;
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int x = threadIdx.x + k * kSolveThreads;
        if (x >= n) continue;
        float v[NR];
        f.eval(iy[q], x, in[q][k], v);
#pragma unroll
        for (int r = 0; r < NR; ++r) S[(q * NR + r) * n + x] = v[r];
        if constexpr (F::kEffects) f.effects(iy[q], x);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RPP; ++q) {
      if (iy[q] < 0) continue;
      const int sy = sy0 + q * gridDim.x;
      for (int u = threadIdx.x; u < w; u += kSolveThreads) {
        int xa, xb;
        fold_pair(u, n, xa, xb);
#pragma unroll
        for (int r = 0; r < NR; ++r) sink.put_pair(r, sy, u, S[(q * NR + r) * n + xa], S[(q * NR + r) * n + xb]);
      }
    }
    __syncthreads();
  }
}

// Predictor-corrector mixing B <- w B_solved + (1 - w) B of one tile (128 slots of y x BN
// consecutive x nodes from xb, component r) staged in shared memory ([128][BN + 1]): element
// e = (row, j) is taken by thread e mod 256, so a warp covers consecutive x nodes of one row;
// up to sixteen elements' loads are issued before their stores.
template <int BN, bool RES>
__device__ __forceinline__ void rs_mix(const SolveArgs& a, const float* tile, int s0, int r, int xb) {
  constexpr int LD = BN + 1, NE = BM * BN, UN = NE / kSolveThreads < 16 ? NE / kSolveThreads : 16;
  const int n = a.nx;
  bool bad = false;
  float d2 = 0.0f, b2 = 0.0f;   // RES (the slice's last iteration): residual sums in FP32
  for (int e0 = threadIdx.x; e0 < NE; e0 += UN * kSolveThreads) {
    float v[UN], old[UN];
    int64_t at[UN];
#pragma unroll
    for (int k = 0; k < UN; ++k) {
      const int e = e0 + k * kSolveThreads;
      const int row = e / BN, j = e - row * BN;
      v[k] = e < NE ? tile[row * LD + j] : 0.0f;
      at[k] = e < NE ? ((int64_t)fold_node(s0 + row, n) * a.nx + xb + j) * 2 + r : -1;
      old[k] = e < NE ? a.bm[at[k]] : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < UN; ++k) {
      if (at[k] < 0) continue;
      bad |= !isfinite(v[k]);
      const float nb = a.w * v[k] + (1.0f - a.w) * old[k];
      a.bm[at[k]] = nb;
      if constexpr (RES) {
        const float d = nb - old[k];
        d2 += d * d;
        b2 += nb * nb;
      }
    }
  }
  if (bad) atomicOr(a.status, DEV_NONFINITE);
  if constexpr (RES) pc_residual_add(a.rsum, (double)d2, (double)b2);
}

template <int BN, bool RES>
__global__ void __launch_bounds__(kSolveThreads, 1)
    k_dst_solve_rs(const __grid_constant__ CUtensorMap fh, const __grid_constant__ CUtensorMap fl,
                   const __grid_constant__ CUtensorMap x0h, const __grid_constant__ CUtensorMap x0l,
                   const __grid_constant__ CUtensorMap x1h, const __grid_constant__ CUtensorMap x1l, const SolveArgs a) {
  using L = RsSmem<BN>;
  constexpr int STAGES = L::KB_MAX;
  constexpr int CH = BN / 2;
  extern __shared__ uint8_t smem_raw[];
  __shared__ int s_abort;
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* basep = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(basep + L::BARS);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 2);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done = smem_u32(bars + 2 * STAGES);
  const uint32_t fbar = smem_u32(bars + 2 * STAGES + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_f = &s_abort;
  const int n = a.nx, H = n / 2, nk = H / BK, MB = n / BM;
  const int mb = (int)blockIdx.x % MB, s0 = mb * BM;
  const int koff = s0 < H ? 0 : H;          // odd slots (first half) contract over the pair sums
  const int NT = a.R * n / BN;               // data-row tiles per product
  const int nt0 = (int)blockIdx.x / MB, ntstep = (int)gridDim.x / MB;

  if (threadIdx.x == 0) {
    for (const CUtensorMap* m : {&fh, &fl, &x0h, &x0l, &x1h, &x1l}) prefetch_map(m);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    mbar_init(done, 1);
    mbar_init(fbar, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // this CTA's fold-matrix slice (rows s0 .. s0 + 127, all n/2 columns), resident for the launch
  if (threadIdx.x == 0) {
    mbar_expect_tx(fbar, (uint32_t)(2 * nk * A_BYTES));
    for (int kb = 0; kb < nk; ++kb) {
      tma_load_2d(base + L::F + kb * A_BYTES, &fh, kb * BK, s0, fbar);
      tma_load_2d(base + L::F + (STAGES + kb) * A_BYTES, &fl, kb * BK, s0, fbar);
    }
  }
  const unsigned nb0 = a.pre ? 1u : 0u;
  bool go = true;
  if (a.pre) {
    // (the stage ring is idle until the first product: it holds the staged sources)
    const SinkFold<__nv_bfloat16> sink{reinterpret_cast<__nv_bfloat16*>(a.op_hi[0]),
                                       reinterpret_cast<__nv_bfloat16*>(a.op_lo[0]), a.nx, a.ny};
    float* S = reinterpret_cast<float*>(basep + L::RING);   // 4 rows x 3 x 512 floats = 24 KB
    if (a.pre == 1) solve_sources_rows<SrcMain<float>, 3>(a.sm.gm, a.sm, sink, S);
    else solve_sources_rows<SrcBperp<float>, 2>(a.sb.gm, a.sb, sink, S);
    go = grid_barrier(a.gbar, (unsigned long long)gridDim.x + (unsigned)a.barrier_skew, a.status, abort_f);
  }
  uint32_t kb_run = 0, tiles_run = 0;
  bool f_ready = false;
  for (int p = 0; p < 4 && go; ++p) {
    const CUtensorMap* xh = (p & 1) ? &x1h : &x0h;
    const CUtensorMap* xl = (p & 1) ? &x1l : &x0l;
    const int mode = p == 3 ? a.final_mode : (p == 1 ? 1 : 0);
    if (p == 3) pdl_trigger();   // the next kernel may be scheduled (it waits for this grid's end)
    for (int nt = nt0; nt < NT; nt += ntstep) {
      const int c0 = nt * BN;
      if (warp == 0 && lane == 0) {
        // data-tile producer: the whole folded K of BN rows, one stage per 64-wide K block
        for (int kb = 0; kb < nk; ++kb) {
          const uint32_t g = kb_run + kb;
          const int s = g % STAGES;
          const uint32_t st = base + L::RING + s * L::STAGE;
          const uint32_t fb = full0 + 8 * s;
          if (g >= (uint32_t)STAGES && !mbar_wait_a(empty0 + 8 * s, ((g / STAGES) - 1) & 1, a.status, abort_f)) break;
          mbar_expect_tx(fb, L::STAGE);
          tma_load_2d(st, xh, koff + kb * BK, c0, fb);
          tma_load_2d(st + BN * BK * 2, xl, koff + kb * BK, c0, fb);
        }
      } else if (warp == 1 && lane == 0) {
        // MMA issuer: A = fold-matrix slice (resident), B = [X_hi; X_lo] (N = 2 BN) and X_hi
        bool ok = f_ready || mbar_wait_a(fbar, 0, a.status, abort_f);
        f_ready = ok;
        for (int kb = 0; ok && kb < nk; ++kb) {
          const uint32_t g = kb_run + kb;
          const int s = g % STAGES;
          if (!mbar_wait_a(full0 + 8 * s, (g / STAGES) & 1, a.status, abort_f)) break;
          tc_fence_after();
          const uint32_t st = base + L::RING + s * L::STAGE;
          const uint64_t ah = desc_k_sw128(base + L::F + kb * A_BYTES);
          const uint64_t al = desc_k_sw128(base + L::F + (STAGES + kb) * A_BYTES);
          const uint64_t bh = desc_k_sw128(st);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t off = (uint64_t)((k * 32) >> 4);
            mma_bf16(tmem, ah + off, bh + off, Cfg<BN>::IDESC2, (kb | k) != 0 ? 1u : 0u);
            mma_bf16(tmem, al + off, bh + off, Cfg<BN>::IDESC, 1u);
          }
          mma_commit(empty0 + 8 * s);
        }
        mma_commit(done);
      }
      __syncwarp();
      // epilogue: TMEM lane = slot s0 + row, the two warpgroups take one half of the columns each
      const int row = (warp & 3) * 32 + lane;
      const int s = s0 + row;
      const int half = warp >> 2;
      const int r = c0 / n;
      const int i0 = c0 - r * n + half * CH;
      float sc[CH];   // the 1/lambda factors of this thread's elements, read while the MMAs run
      if (mode == 1) {
        const float4* q = reinterpret_cast<const float4*>(a.scale + (int64_t)s * n + i0);
#pragma unroll
        for (int k = 0; k < CH / 4; ++k) {
          const float4 f = __ldg(q + k);
          sc[4 * k] = f.x;
          sc[4 * k + 1] = f.y;
          sc[4 * k + 2] = f.z;
          sc[4 * k + 3] = f.w;
        }
      }
      mbar_wait_a(done, tiles_run & 1, a.status, abort_f);
      tc_fence_after();
      {
        float x[CH];
        tmem_ld_pair<BN, CH>(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * CH), x);
        const int orow = p == 2 ? fold_node(s, n) : s;
        if (mode == 3) {
          // predictor-corrector mixing into bm[node][r]: the tile goes through shared memory (the
          // drained stage ring) so that a warp updates consecutive nodes of one row
          constexpr int LD = BN + 1;
          float* tile = reinterpret_cast<float*>(basep + L::RING);
#pragma unroll
          for (int j = 0; j < CH; ++j) tile[row * LD + half * CH + j] = x[j];
          __syncthreads();
          if (!*abort_f) rs_mix<BN, RES>(a, tile, s0, r, c0 - r * n);
        } else if (!*abort_f) {
          rs_epilogue<CH>(a, mode, s, orow, r, i0, x, sc, reinterpret_cast<__nv_bfloat16*>(a.op_hi[(p + 1) & 1]),
                          reinterpret_cast<__nv_bfloat16*>(a.op_lo[(p + 1) & 1]));
        }
      }
      kb_run += nk;
      ++tiles_run;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      if (*abort_f) break;
    }
    if (*abort_f) break;
    if (p < 3 && !grid_barrier(a.gbar,
                               (unsigned long long)(nb0 + p + 1) * gridDim.x +
                                   (nb0 == 0 && p == 0 ? (unsigned)a.barrier_skew : 0u),
                               a.status, abort_f))
      break;
  }
  // the fold-matrix load must have landed before the CTA leaves (a CTA without tiles, or one
  // that gave up, may not have waited for it): a bounded wait that ignores the abort flag
  if (threadIdx.x == 0) mbar_wait(fbar, 0, a.status);
  // exit arrival: the last CTA through resets the counter for the next launch
  if (threadIdx.x == 0 && !*abort_f) {
    const unsigned long long seen = atomicAdd(a.gbar, 1ull);
    if (seen == (nb0 + 4ull) * gridDim.x - 1ull) atomicExch(a.gbar, 0ull);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)) : "memory");
  }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                              const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// A split operand [rows][cols] in 128B-swizzled boxes of one K block (128 bytes) by box_rows:
// bf16 elements, or (tf32) FP32 words.
int make_map(EncodeFn enc, CUtensorMap* map, void* ptr, uint64_t rows, uint64_t cols, std::string& err,
             uint32_t box_rows = 128, bool tf32 = false) {
  const uint32_t es = tf32 ? 4 : 2;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * es};
  cuuint32_t box[2] = {128 / es, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult rc = enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)rc) + ")";
    return 1;
  }
  return 0;
}

// Unswizzled map with an arbitrary box (the FP32 scale tile).
int make_map_plain(EncodeFn enc, CUtensorMap* map, CUtensorMapDataType dt, uint32_t esize, void* ptr, uint64_t rows,
                   uint64_t cols, uint32_t box_x, uint32_t box_y, std::string& err) {
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * esize};
  cuuint32_t box[2] = {box_x, box_y};
  cuuint32_t estr[2] = {1, 1};
  CUresult rc = enc(map, dt, 2, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (rc != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)rc) + ")";
    return 1;
  }
  return 0;
}

// N-tile width: 64 when 128-wide tiles would leave most of the 152 SMs idle.
inline int pick_bn(int M, int N) { return (M / BM) * (N / 128) < 152 ? 64 : 128; }

void gemm(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap* bh, const CUtensorMap* bl, int M, int N,
          int K, const Epi& ep, int* status, cudaStream_t s) {
  if (pick_bn(M, N) == 128) {
    dim3 grid((unsigned)(M / BM), (unsigned)(N / 128));
    launch_pdl(k_dst_gemm<128>, grid, dim3(128), (size_t)Cfg<128>::SMEM_BYTES, s, ah, al, bh[0], bl[0], K, ep, status);
  } else {
    dim3 grid((unsigned)(M / BM), (unsigned)(N / 64));
    launch_pdl(k_dst_gemm<64>, grid, dim3(128), (size_t)Cfg<64>::SMEM_BYTES, s, ah, al, bh[1], bl[1], K, ep, status);
  }
}

}  // namespace

int dst_tc_init(hq_grid_s* g, std::string& err) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      fn == nullptr || q != cudaDriverEntryPointSuccess) {
    err = "cuTensorMapEncodeTiled not available from the driver";
    return 1;
  }
  EncodeFn enc = reinterpret_cast<EncodeFn>(fn);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->dev) != cudaSuccess) {
    err = "cannot read the SM count";
    return 1;
  }
  auto size_solve = [&](auto kern, int smem, int& ctas) {
    int per_sm = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSolveThreads, smem) != cudaSuccess || per_sm < 1) {
      err = "cannot size the cooperative DST solve";
      return false;
    }
    ctas = per_sm * sms;
    return true;
  };
  g->tmaps = new TensorMaps();
  TensorMaps& t = *g->tmaps;
  int spare = 0;   // the residual-accumulating instances (the last P-C iteration): same resources
  const bool tf = g->tf32 != 0;
  if (tf ? (!size_solve(k_dst_solve<64, false, float>, SolveSmem<64>::BYTES, t.ctas[0]) ||
            !size_solve(k_dst_solve<32, false, float>, SolveSmem<32>::BYTES, t.ctas[1]) ||
            !size_solve(k_dst_solve<64, true, float>, SolveSmem<64>::BYTES, spare) ||
            !size_solve(k_dst_solve<32, true, float>, SolveSmem<32>::BYTES, spare))
         : (!size_solve(k_dst_solve<64, false, __nv_bfloat16>, SolveSmem<64>::BYTES, t.ctas[0]) ||
            !size_solve(k_dst_solve<32, false, __nv_bfloat16>, SolveSmem<32>::BYTES, t.ctas[1]) ||
            !size_solve(k_dst_solve<64, true, __nv_bfloat16>, SolveSmem<64>::BYTES, spare) ||
            !size_solve(k_dst_solve<32, true, __nv_bfloat16>, SolveSmem<32>::BYTES, spare)))
    return 1;
  const char* bn = std::getenv("HQ_SOLVE_BN");
  t.wide_only = bn != nullptr && std::atoi(bn) == 64;
  const char* nors = std::getenv("HQ_NO_RS");
  // (the resident fold matrix is bf16: as TF32 words it would need 256 KB of shared memory at 512^2)
  t.rs = !tf && g->fold && g->nx == g->ny && (g->nx == 256 || g->nx == 512) && !(nors && nors[0] == '1');
  if (t.rs && (!size_solve(k_dst_solve_rs<64, false>, RsSmem<64>::BYTES, t.rs_ctas[0]) ||
               !size_solve(k_dst_solve_rs<32, false>, RsSmem<32>::BYTES, t.rs_ctas[1]) ||
               !size_solve(k_dst_solve_rs<64, true>, RsSmem<64>::BYTES, spare) ||
               !size_solve(k_dst_solve_rs<32, true>, RsSmem<32>::BYTES, spare)))
    return 1;
  const uint64_t nxp = g->nxp, nyp = g->nyp;
  int bad = 0;
  bad |= make_map(enc, &t.a0_hi, g->op_hi[0], kMaxRhs * nyp, nxp, err, 128, tf);
  bad |= make_map(enc, &t.a0_lo, g->op_lo[0], kMaxRhs * nyp, nxp, err, 128, tf);
  bad |= make_map(enc, &t.a1_hi, g->op_hi[1], kMaxRhs * nxp, nyp, err, 128, tf);
  bad |= make_map(enc, &t.a1_lo, g->op_lo[1], kMaxRhs * nxp, nyp, err, 128, tf);
  // S_x, S_y (or the fold matrices, half as wide) as [rows][K]
  const uint64_t kx = g->fold ? nxp / 2 : nxp, ky = g->fold ? nyp / 2 : nyp;
  for (int i = 0; i < 2; ++i) {
    const uint32_t bn = i == 0 ? 64 : 32;
    bad |= make_map(enc, &t.bx_hi[i], g->sx_hi, nxp, kx, err, bn, tf);
    bad |= make_map(enc, &t.bx_lo[i], g->sx_lo, nxp, kx, err, bn, tf);
    bad |= make_map(enc, &t.by_hi[i], g->sy_hi, nyp, ky, err, bn, tf);
    bad |= make_map(enc, &t.by_lo[i], g->sy_lo, nyp, ky, err, bn, tf);
    bad |= make_map_plain(enc, &t.scale[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->f32_scale, nyp, nxp, BM, bn, err);
    if (g->scale_h)
      bad |= make_map_plain(enc, &t.scale_h[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g->scale_h, nyp, nxp, BM, bn, err);
  }
  if (t.rs) {
    bad |= make_map(enc, &t.rf_hi, g->sx_hi, nxp, kx, err, 128);
    bad |= make_map(enc, &t.rf_lo, g->sx_lo, nxp, kx, err, 128);
    for (int o = 0; o < 2; ++o)
      for (int i = 0; i < 2; ++i) {
        const uint32_t bn = i == 0 ? 64 : 32;
        bad |= make_map(enc, &t.rx_hi[o][i], g->op_hi[o], kMaxRhs * nyp, nxp, err, bn);
        bad |= make_map(enc, &t.rx_lo[o][i], g->op_lo[o], kMaxRhs * nyp, nxp, err, bn);
      }
  }
  return bad;
}

void dst_tc_free(hq_grid_s* g) {
  delete g->tmaps;
  g->tmaps = nullptr;
}

namespace {

// One cooperative launch of k_dst_solve: on the sources in op[0] (pre = 0), or forming them
// first from the deposit records (pre = 1: psi, Ez, Bz of dep_cur; pre = 2: B_perp).
void solve_fused(hq_grid_s* g, int R, int final_mode, int last, cudaStream_t s, int pre = 0,
                 const void* dep_cur = nullptr, void* dep_prev = nullptr, void* chi_prev = nullptr,
                 bool shifted = false) {
  const TensorMaps& t = *g->tmaps;
  SolveArgs a{};
  a.R = R;
  a.nxp = g->nxp;
  a.nyp = g->nyp;
  a.fold = g->fold;
  a.op_hi[0] = g->op_hi[0];
  a.op_lo[0] = g->op_lo[0];
  a.op_hi[1] = g->op_hi[1];
  a.op_lo[1] = g->op_lo[1];
  a.scale = reinterpret_cast<const float*>(shifted ? g->scale_h : g->f32_scale);
  a.final_mode = final_mode;
  a.out = reinterpret_cast<float*>(g->solved);
  a.nx = g->nx;
  a.ny = g->ny;
  a.bm = reinterpret_cast<float*>(g->bm);
  a.w = (float)g->d.pc_mix;
  a.rsum = g->pc_rsum;
  a.gbar = g->d_gbar;
  a.status = g->d_status;
  a.barrier_skew = g->fault_barrier;
  a.pre = pre;
  if (pre == 1) a.sm = src_main_of<float>(g, dep_cur);
  if (pre == 2) a.sb = src_bperp_of<float>(g, dep_cur, dep_prev, chi_prev, last);
  if (t.rs) {
    // resident fold-matrix solve: MB slot blocks x (R n / BN) data-row tiles per product; the
    // grid is a multiple of MB (a CTA keeps its slot block)
    const int n = g->nx, MB = n / BM;
    const int tiles32 = MB * (R * n / 32);
    const bool narrow = !t.wide_only && tiles32 <= t.rs_ctas[1];
    const int v = narrow ? 1 : 0;
    const int tiles_v = MB * (R * n / (narrow ? 32 : 64));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min(tiles_v, t.rs_ctas[v] / MB * MB));
    cfg.blockDim = dim3(kSolveThreads);
    cfg.dynamicSmemBytes = narrow ? RsSmem<32>::BYTES : RsSmem<64>::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto kern = a.rsum ? (narrow ? k_dst_solve_rs<32, true> : k_dst_solve_rs<64, true>)
                       : (narrow ? k_dst_solve_rs<32, false> : k_dst_solve_rs<64, false>);
    cudaLaunchKernelEx(&cfg, kern, t.rf_hi, t.rf_lo, t.rx_hi[0][v], t.rx_lo[0][v], t.rx_hi[1][v], t.rx_lo[1][v], a);
    return;
  }
  // tiles of one product (the larger of the x and y products) at N-tile width bn
  auto tiles = [&](int bn) {
    return std::max(R * (g->nyp / BM) * (g->nxp / bn), R * (g->nxp / BM) * (g->nyp / bn));
  };
  const bool narrow = !t.wide_only && tiles(32) <= t.ctas[1];
  const int v = narrow ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)std::min(t.ctas[v], tiles(narrow ? 32 : 64)));
  cfg.blockDim = dim3(kSolveThreads);
  cfg.dynamicSmemBytes = narrow ? SolveSmem<32>::BYTES : SolveSmem<64>::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // a launch error is reported by the caller's launch check
  auto kern = g->tf32 ? (a.rsum ? (narrow ? k_dst_solve<32, true, float> : k_dst_solve<64, true, float>)
                                : (narrow ? k_dst_solve<32, false, float> : k_dst_solve<64, false, float>))
                      : (a.rsum ? (narrow ? k_dst_solve<32, true, __nv_bfloat16> : k_dst_solve<64, true, __nv_bfloat16>)
                                : (narrow ? k_dst_solve<32, false, __nv_bfloat16>
                                          : k_dst_solve<64, false, __nv_bfloat16>));
  cudaLaunchKernelEx(&cfg, kern, t.a0_hi, t.a0_lo, t.a1_hi, t.a1_lo, t.bx_hi[v], t.bx_lo[v], t.by_hi[v], t.by_lo[v],
                     shifted ? t.scale_h[v] : t.scale[v], a);
}

}  // namespace

// B_perp solve with the predictor-corrector mixing fused into the last product's epilogue:
// sources (split, 2 rhs) in op[0] -> bm <- w B + (1 - w) bm.
void dst_solve_tc_bmix(hq_grid_s* g, int last, cudaStream_t s) { solve_fused(g, 2, 3, last, s); }

// sources (split) in op[0] -> FP32 solution in g->solved [R][ny][nx]
void dst_solve_tc(hq_grid_s* g, int R, cudaStream_t s) { solve_fused(g, R, 2, 0, s); }
void dst_solve_tc_shifted(hq_grid_s* g, int R, cudaStream_t s) {
  solve_fused(g, R, 2, 0, s, 0, nullptr, nullptr, nullptr, true);
}

// The same with the source kernels folded into the launch as its first phase: psi, Ez, Bz of
// the deposit record dep -> g->solved; the B_perp sources of the predictor-corrector (which
// clear the trial J_perp and, on the last iteration, reset dep_prev) -> mixing into bm.
void dst_solve_tc_main(hq_grid_s* g, const void* dep, cudaStream_t s) { solve_fused(g, 3, 2, 0, s, 1, dep); }
void dst_solve_tc_bmix_src(hq_grid_s* g, const void* cur, void* prev, void* chi_prev, int last, cudaStream_t s) {
  solve_fused(g, 2, 3, last, s, 2, cur, prev, chi_prev);
}

}  // namespace hq

// ---------------------------------------------------------------- allocation-free variant
// hq_poisson_solve_static: the same tensor-core Dirichlet solve for callers that
// cannot allocate device memory (all scratch in one file-scope static array).
#include <map>
#include <mutex>

namespace hq {
void set_global_error(const std::string& msg);  // defined in hq_api.cu

namespace {

constexpr int kStaticMaxN = 512;   // nx, ny <= 512 (so the padded extents are <= 512)
constexpr int kStaticMaxRhs = 3;
constexpr size_t kStaticOpBytes = (size_t)kStaticMaxRhs * kStaticMaxN * kStaticMaxN * 2;  // one bf16 operand buffer
constexpr size_t kStaticSBytes = (size_t)kStaticMaxN * kStaticMaxN * 2;                    // one bf16 sine matrix
constexpr size_t kStaticScaleBytes = (size_t)kStaticMaxN * kStaticMaxN * 4;                // FP32 1/lambda table
// layout: status word (256 B) | op_hi0 op_lo0 op_hi1 op_lo1 | sx_hi sx_lo sy_hi sy_lo | scale  (9 MiB + 256 B)
constexpr size_t kStaticBytes = 256 + 4 * kStaticOpBytes + 4 * kStaticSBytes + kStaticScaleBytes;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticDev {
  uint8_t* base = nullptr;   // device address of g_static_scratch on this device
  int nx = 0, ny = 0;        // geometry the tables in the array hold (nx = 0: unknown, rebuild)
  double dx = 0.0, dy = 0.0;
  TensorMaps maps;           // encoded for (map_nx, map_ny)
  int map_nx = 0, map_ny = 0;
};
std::mutex g_static_mu;
std::map<int, StaticDev> g_static_dev;

// S_x, S_y (bf16 hi/lo, zero-padded) and the scale (4/(nx ny))/lambda for one grid.
__global__ void k_static_tables(__nv_bfloat16* sxh, __nv_bfloat16* sxl, __nv_bfloat16* syh, __nv_bfloat16* syl,
                                float* scale, int nx, int ny, int nxp, int nyp, double dx, double dy) {
  const int64_t tot = (int64_t)kStaticMaxN * kStaticMaxN;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / kStaticMaxN), c = (int)(t % kStaticMaxN);
    if (r < nxp && c < nxp) {
      const float v = (r < nx && c < nx) ? (float)sinpi((double)(((int64_t)r * c) % (2 * nx)) / nx) : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      sxh[(int64_t)r * nxp + c] = h;
      sxl[(int64_t)r * nxp + c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    if (r < nyp && c < nyp) {
      const float v = (r < ny && c < ny) ? (float)sinpi((double)(((int64_t)r * c) % (2 * ny)) / ny) : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      syh[(int64_t)r * nyp + c] = h;
      syl[(int64_t)r * nyp + c] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
    if (r < nyp && c < nxp) {
      float s = 0.0f;
      if (r >= 1 && r < ny && c >= 1 && c < nx) {
        const double sx = sinpi(c / (2.0 * nx)), sy = sinpi(r / (2.0 * ny));
        const double lam = -(4.0 / (dx * dx)) * sx * sx - (4.0 / (dy * dy)) * sy * sy;
        s = (float)((4.0 / ((double)nx * ny)) / lam);
      }
      scale[(int64_t)r * nxp + c] = s;
    }
  }
}

// Sources into the zero-padded split operand layout [R][nyp][nxp]; every padded entry
// is written, so nothing left over from an earlier call of another size survives.
__global__ void k_static_src(const float* __restrict__ src, __nv_bfloat16* hi, __nv_bfloat16* lo, int R, int nx, int ny,
                             int nxp, int nyp) {
  const int64_t tot = (int64_t)R * nyp * nxp;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(t % nxp);
    const int64_t ry = t / nxp;
    const int iy = (int)(ry % nyp), r = (int)(ry / nyp);
    const float v = (ix >= 1 && ix < nx && iy >= 1 && iy < ny) ? src[((int64_t)r * ny + iy) * nx + ix] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[t] = h;
    lo[t] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

EncodeFn static_encoder(std::string& err) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      fn == nullptr || q != cudaDriverEntryPointSuccess) {
    err = "cuTensorMapEncodeTiled not available from the driver";
    return nullptr;
  }
  return reinterpret_cast<EncodeFn>(fn);
}

hq_status static_fail(hq_status st, const std::string& msg) {
  set_global_error(msg);
  return st;
}

}  // namespace
}  // namespace hq

using namespace hq;

extern "C" hq_status hq_poisson_solve_static(const float* src, float* dst, int32_t nx, int32_t ny, double dx, double dy,
                                             int32_t nrhs, void* cuda_stream) {
  if (!src || !dst) return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: src and dst must not be NULL");
  if (nx < 8 || ny < 8 || nx > kStaticMaxN || ny > kStaticMaxN)
    return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: nx and ny must be in 8..512 (static scratch limit)");
  if (nrhs < 1 || nrhs > kStaticMaxRhs)
    return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: nrhs must be in 1..3 (static scratch limit)");
  if (!(dx > 0.0) || !(dy > 0.0) || !std::isfinite(dx) || !std::isfinite(dy))
    return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: dx and dy must be finite and positive");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sdev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(HQ_ERR_CUDA, "hq_poisson_solve_static: no CUDA device");
  if (cudaStreamGetDevice(s, &sdev) != cudaSuccess)
    return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: cuda_stream is not a valid stream");
  if (sdev != dev)
    return static_fail(HQ_ERR_ARG, "hq_poisson_solve_static: cuda_stream belongs to device " + std::to_string(sdev) +
                                        ", not the current device " + std::to_string(dev));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
    return static_fail(HQ_ERR_CUDA, "hq_poisson_solve_static: cannot query the stream's capture state");
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lock(g_static_mu);
  StaticDev& sd = g_static_dev[dev];
  std::string err;
  if (!sd.base) {
    // once per device: resolve the static array's device address (the host-side symbol is
    // only a stand-in) and allow the GEMM's shared-memory footprint
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess || prop.major != 10 || prop.minor != 3)
      return static_fail(HQ_ERR_UNSUPPORTED, "hq_poisson_solve_static: needs an sm_103a (GB300) device");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return static_fail(HQ_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    if (cudaFuncSetAttribute(k_dst_gemm<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<128>::SMEM_BYTES) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_dst_gemm<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<64>::SMEM_BYTES) !=
            cudaSuccess)
      return static_fail(HQ_ERR_CUDA, "hq_poisson_solve_static: cannot raise the GEMM shared-memory limit");
    sd.base = static_cast<uint8_t*>(p);
  }
  uint8_t* b = sd.base;
  int* status = reinterpret_cast<int*>(b);
  __nv_bfloat16* op_hi0 = reinterpret_cast<__nv_bfloat16*>(b + 256);
  __nv_bfloat16* op_lo0 = reinterpret_cast<__nv_bfloat16*>(b + 256 + kStaticOpBytes);
  __nv_bfloat16* op_hi1 = reinterpret_cast<__nv_bfloat16*>(b + 256 + 2 * kStaticOpBytes);
  __nv_bfloat16* op_lo1 = reinterpret_cast<__nv_bfloat16*>(b + 256 + 3 * kStaticOpBytes);
  uint8_t* sb = b + 256 + 4 * kStaticOpBytes;
  __nv_bfloat16* sxh = reinterpret_cast<__nv_bfloat16*>(sb);
  __nv_bfloat16* sxl = reinterpret_cast<__nv_bfloat16*>(sb + kStaticSBytes);
  __nv_bfloat16* syh = reinterpret_cast<__nv_bfloat16*>(sb + 2 * kStaticSBytes);
  __nv_bfloat16* syl = reinterpret_cast<__nv_bfloat16*>(sb + 3 * kStaticSBytes);
  float* scale = reinterpret_cast<float*>(sb + 4 * kStaticSBytes);
  const int nxp = (nx + 127) / 128 * 128, nyp = (ny + 127) / 128 * 128;
  if (sd.map_nx != nx || sd.map_ny != ny) {
    // new extents: re-encode the tensor maps over the new padded extents (host-side, no
    // allocation)
    EncodeFn enc = static_encoder(err);
    if (!enc) return static_fail(HQ_ERR_CUDA, err);
    TensorMaps& t = sd.maps;
    int bad = 0;
    bad |= make_map(enc, &t.a0_hi, op_hi0, (uint64_t)kStaticMaxRhs * nyp, nxp, err);
    bad |= make_map(enc, &t.a0_lo, op_lo0, (uint64_t)kStaticMaxRhs * nyp, nxp, err);
    bad |= make_map(enc, &t.a1_hi, op_hi1, (uint64_t)kStaticMaxRhs * nxp, nyp, err);
    bad |= make_map(enc, &t.a1_lo, op_lo1, (uint64_t)kStaticMaxRhs * nxp, nyp, err);
    for (int i = 0; i < 2; ++i) {
      const uint32_t rows = i == 0 ? 128 : 64;
      bad |= make_map(enc, &t.sx_hi[i], sxh, nxp, nxp, err, rows);
      bad |= make_map(enc, &t.sx_lo[i], sxl, nxp, nxp, err, rows);
      bad |= make_map(enc, &t.sy_hi[i], syh, nyp, nyp, err, rows);
      bad |= make_map(enc, &t.sy_lo[i], syl, nyp, nyp, err, rows);
    }
    if (bad) {
      sd.map_nx = sd.map_ny = 0;
      sd.nx = sd.ny = 0;
      return static_fail(HQ_ERR_CUDA, err);
    }
    sd.map_nx = nx;
    sd.map_ny = ny;
  }
  // The sine matrices and the 1/lambda table in the array are rebuilt for a new (nx, ny, dx,
  // dy), and by every call made while the stream is being captured: what such a call enqueues
  // runs later, so the array's contents can no longer be tracked here and the next call
  // rebuilds them too.
  if (capturing || sd.nx != nx || sd.ny != ny || sd.dx != dx || sd.dy != dy) {
    sd.nx = sd.ny = 0;
    k_static_tables<<<256, 256, 0, s>>>(sxh, sxl, syh, syl, scale, nx, ny, nxp, nyp, dx, dy);
    const cudaError_t te = cudaGetLastError();
    if (te != cudaSuccess)
      return static_fail(HQ_ERR_CUDA, std::string("hq_poisson_solve_static: table build: ") + cudaGetErrorString(te));
    if (!capturing) {
      sd.nx = nx;
      sd.ny = ny;
      sd.dx = dx;
      sd.dy = dy;
    }
  }
  const TensorMaps& t = sd.maps;
  // the status word at the start of the array is not cleared here: a timeout or a non-finite
  // result stays flagged until hq_sync(NULL, ...) reads and clears it
  k_static_src<<<256, 256, 0, s>>>(src, op_hi0, op_lo0, nrhs, nx, ny, nxp, nyp);
  Epi e{};
  e = Epi{0, nyp, nxp, op_hi1, op_lo1, nullptr, nullptr, 0, 0};
  gemm(t.a0_hi, t.a0_lo, t.sx_hi, t.sx_lo, nrhs * nyp, nxp, nxp, e, status, s);
  e = Epi{1, nxp, nyp, op_hi0, op_lo0, scale, nullptr, 0, 0};
  gemm(t.a1_hi, t.a1_lo, t.sy_hi, t.sy_lo, nrhs * nxp, nyp, nyp, e, status, s);
  e = Epi{0, nyp, nxp, op_hi1, op_lo1, nullptr, nullptr, 0, 0};
  gemm(t.a0_hi, t.a0_lo, t.sx_hi, t.sx_lo, nrhs * nyp, nxp, nxp, e, status, s);
  e = Epi{2, nxp, nyp, nullptr, nullptr, nullptr, dst, nx, ny};
  gemm(t.a1_hi, t.a1_lo, t.sy_hi, t.sy_lo, nrhs * nxp, nyp, nyp, e, status, s);
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) return static_fail(HQ_ERR_CUDA, std::string("hq_poisson_solve_static: ") + cudaGetErrorString(le));
  return HQ_OK;
}

namespace hq {
// Status of the allocation-free solves on the current device (hq_sync(NULL, ...)): waits for
// the device, reads the status word at the start of the static array and clears it.  A device
// on which no such solve was set up reports HQ_OK.
hq_status static_sync() {
  if (cudaDeviceSynchronize() != cudaSuccess) {
    const cudaError_t e = cudaGetLastError();
    return static_fail(HQ_ERR_CUDA, std::string("hq_sync(NULL): ") + cudaGetErrorString(e));
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(HQ_ERR_CUDA, "hq_sync(NULL): no CUDA device");
  uint8_t* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    auto it = g_static_dev.find(dev);
    if (it != g_static_dev.end()) base = it->second.base;
  }
  if (!base) return HQ_OK;
  int status = 0;
  if (cudaMemcpy(&status, base, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return static_fail(HQ_ERR_CUDA, "hq_sync(NULL): status read failed");
  if (!status) return HQ_OK;
  if (cudaMemset(base, 0, sizeof(int)) != cudaSuccess) return static_fail(HQ_ERR_CUDA, "hq_sync(NULL): status reset failed");
  if (status & DEV_TIMEOUT)
    return static_fail(HQ_ERR_TIMEOUT, "hq_poisson_solve_static: a bounded device wait ran out");
  return static_fail(HQ_ERR_NUMERIC, "hq_poisson_solve_static: a non-finite value reached the solution");
}
}  // namespace hq
