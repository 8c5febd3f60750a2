// Trailing Schur-complement update of the mixed-precision sampler on the
// fifth-generation tensor cores (tcgen05, sm_103a):
//
//     C[i, c] -= sum_t W[i, t] L[c, t]      (lower triangle, i >= c)
//
// which is the rank-NB update A22 -= W L21^T = L21 D1 L21^T of the blocked
// LDL^T sampler (Algorithm 3's Schur complement, Hermitian form), i.e. the
// contraction that carries asymptotically all of the work (Section 4). In
// full mode every tile of the square trailing block is updated: the LU form
// A22 -= L21 U12 = (L21 D1) (D1^{-1} U12), with L the rows of D1^{-1} U12
// transposed.
//
// Precision (chosen per call):
//   3xTF32 : W = Wh + Wl, L = Lh + Ll (TF32 pairs); per 8-deep k-step
//            Wl Lh^T + Wh Ll^T + Wh Lh^T (kind::tf32).
//   BF16x6 : W = W0 + W1 + W2, L = L0 + L1 + L2 (three BF16 pieces, which
//            represent an FP32 value exactly); per 16-deep k-step the six
//            products with combined order <= 2 (kind::f16, BF16 runs at twice
//            the TF32 rate, so this costs the same as 3xTF32 and reaches FP32
//            accuracy). Small products are issued first.
// Both splits are produced by the panel kernel; FP32 accumulation.
//
// Accuracy: the tensor core's in-instruction FP32 accumulation is not
// round-to-nearest, so a long chain of MMAs into one accumulator drifts. Each
// group of MMAs (one 32-deep k-block for 3xTF32, one 16-deep k-step for
// BF16x6) therefore goes into a fresh TMEM accumulator that the epilogue drains
// into FP32 registers with ordinary round-to-nearest adds.
//
// Structure (persistent, one CTA per SM, 320 threads, 128 x 128 tiles of the
// lower triangle assigned round-robin):
//   warp 0 / lane 0 : TMA producer, ring of operand stages (128 rows per split;
//                     3xTF32: 128-byte rows, SWIZZLE_128B, 3 stages; BF16x6:
//                     64-byte rows, SWIZZLE_64B, 4 stages)
//   warp 1          : allocates 4 x 128 TMEM columns (a ring of accumulators,
//                     so the MMAs run ahead of the epilogue); lane 0 issues
//                     tcgen05.mma (M = N = 128) and tcgen05.commit
//   warps 2-9       : epilogue; each thread owns half a row of the tile (64
//                     columns): it accumulates minus every drained partial
//                     (tcgen05.ld 32x32b) in registers, fetches its C values
//                     at the start of the tile and stores C + sum at its end.
// Every mbarrier wait is bounded; on expiry the kernel records an error,
// drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"

namespace dpp {
namespace {

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kThreads = 320;          // producer, MMA, 8 epilogue warps
constexpr int kEpiThreads = 256;
constexpr int kEpiCols = kBN / 2;
constexpr int kAccBufs = 4;
constexpr int kTmemCols = kAccBufs * kBN;  // all 512 columns

template <int MODE>
struct TcBase;

// 3xTF32: 2 splits (TF32 hi, lo in FP32 containers), three products per
// 8-deep k-step.
template <>
struct TcBase<kSplit3xTf32> {
  static constexpr int kOps = 2;
  static constexpr int kEsz = 4;
  static constexpr int kProducts = 3;
  // D = F32 (bits 4-5 = 1), A = B = TF32 (2), K-major, N >> 3, M >> 4
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                     ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  __device__ static void product(int p, int* ia, int* ib) {
    const int A[3] = {1, 0, 0}, B[3] = {0, 1, 0};
    *ia = A[p];
    *ib = B[p];
  }
};

// BF16x6: 3 splits, the six products of combined order <= 2 per 16-deep step.
template <>
struct TcBase<kSplitBf16x6> {
  static constexpr int kOps = 3;
  static constexpr int kEsz = 2;
  static constexpr int kProducts = 6;
  // D = F32, A = B = BF16 (1), K-major, N >> 3, M >> 4
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                                     ((uint32_t)(kBN >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
  __device__ static void product(int p, int* ia, int* ib) {
    const int A[6] = {1, 0, 2, 0, 1, 0}, B[6] = {1, 2, 0, 1, 0, 0};
    *ia = A[p];
    *ib = B[p];
  }
};

// Operand ring and drain interval of a variant (DPP_TUNE_UPDATE_VARIANT).
// Every MMA k-step consumes 32 bytes of each operand row (8 TF32 or 16 BF16).
//   3xTF32 V0: 32-deep stages of 128-byte rows (SWIZZLE_128B), 3 stages,
//              a fresh accumulator every 32 deep (12 MMAs);
//   3xTF32 V1: the same ring, a fresh accumulator every 64 deep;
//   3xTF32 V2: 16-deep stages of 64-byte rows (SWIZZLE_64B), 6 stages (more
//              bytes in flight per SM), a fresh accumulator every 32 deep;
//   3xTF32 V3: the V2 ring, every 64 deep.
//   BF16x6 V0/V2: 32-deep stages of 64-byte rows, 4 stages, every 16 deep;
//   BF16x6 V1/V3: the same ring, every 32 deep.
// A drain may span stages; the last one of a tile may be shorter.
template <int MODE, int V>
struct TcCfg : TcBase<MODE> {
  static constexpr bool kDeep = MODE == kSplit3xTf32 && V >= 2;
  static constexpr int kBK = kDeep ? 16 : 32;
  static constexpr int kRowBytes = kBK * TcBase<MODE>::kEsz;  // 128 or 64
  static constexpr int kStages = MODE == kSplit3xTf32 ? (kDeep ? 6 : 3) : 4;
  static constexpr int kSteps = kRowBytes / 32;  // MMA k-steps per stage
  static constexpr int kStepsPerDrain =
      MODE == kSplit3xTf32 ? ((V & 1) ? 8 : 4) : ((V & 1) ? 2 : 1);
};

template <class Cfg>
__host__ __device__ constexpr int tile_bytes() {
  return kBM * Cfg::kRowBytes;  // 128 rows of one split
}
template <class Cfg>
__host__ __device__ constexpr int stage_bytes() {
  return 2 * Cfg::kOps * tile_bytes<Cfg>();
}
template <class Cfg>
__host__ __device__ constexpr int smem_bytes() {
  return Cfg::kStages * stage_bytes<Cfg>() + 1024 + 256;
}

__device__ inline uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ inline bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on phase `parity` of an mbarrier.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ inline void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                   uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand with rows of ROW bytes
// swizzled over ROW bytes (128 or 64), 8-row swizzle atoms 8 ROW bytes apart.
template <int ROW>
__device__ inline uint64_t sw_desc(uint32_t saddr) {
  static_assert(ROW == 128 || ROW == 64, "row width");
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(16u >> 4) << 16;             // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)((8u * ROW) >> 4) << 32;      // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                      // descriptor version
  d |= (uint64_t)(ROW == 128 ? 2 : 4) << 61;   // 128-byte or 64-byte swizzle
  return d;
}

__device__ inline void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int MODE>
__device__ inline void mma_issue(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (MODE == kSplit3xTf32) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(TcBase<MODE>::kIdesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(TcBase<MODE>::kIdesc), "r"(accumulate)
        : "memory");
  }
}

struct TcMaps {
  CUtensorMap W[3];
  CUtensorMap L[3];
};

struct TcArgs {
  float* C;
  int64_t ldc, n, r0;
  int kblocks;
  int64_t tiles;   // tiles along one side of the trailing block
  int64_t ntiles;  // tiles updated: the lower triangle's, or tiles^2 if full
  int full;        // 1: every tile of the square block (LU), 0: lower triangle
  int* err;
};

// Row and column of lower-triangle tile x (row-major order). The estimate is
// FP32 (the FP64 pipe is the GPU's slowest and every epilogue thread calls
// this per tile) and the integer loops make it exact.
__device__ inline void tile_coords(int64_t x, int64_t* tr, int64_t* tc) {
  int64_t r = (int64_t)((sqrtf(8.f * (float)x + 1.f) - 1.f) * 0.5f);
  while (r > 0 && r * (r + 1) / 2 > x) --r;
  while ((r + 1) * (r + 2) / 2 <= x) ++r;
  *tr = r;
  *tc = x - r * (r + 1) / 2;
}

// Row and column of tile x of this launch (row-major order in either mode).
__device__ inline void tile_of(const TcArgs& a, int64_t x, int64_t* tr, int64_t* tc) {
  if (a.full) {
    *tr = x / a.tiles;
    *tc = x - *tr * a.tiles;
  } else {
    tile_coords(x, tr, tc);
  }
}

__device__ inline void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Ten warps are allocated registers as twelve, so a thread may hold 168; the
// epilogue's two 64-value arrays and a 16-column TMEM slice fit in that.
template <int MODE, int V>
__global__ void __launch_bounds__(kThreads, 1)
    k_update_tc(const __grid_constant__ TcMaps maps, TcArgs a) {
  using Cfg = TcCfg<MODE, V>;
  constexpr int kStages = Cfg::kStages;
  constexpr int kStageBytes = stage_bytes<Cfg>();
  constexpr int kTileBytes = tile_bytes<Cfg>();
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + kStages * kStageBytes);
  uint64_t* full = bars;                      // [kStages]
  uint64_t* empty = bars + kStages;           // [kStages]
  uint64_t* acc_full = bars + 2 * kStages;    // [kAccBufs]
  uint64_t* acc_empty = acc_full + kAccBufs;  // [kAccBufs]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + kAccBufs);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < kAccBufs; ++b) {
      mbar_init(smem_u32(&acc_full[b]), 1);
      mbar_init(smem_u32(&acc_empty[b]), kEpiThreads);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int KB = a.kblocks;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer ----
      int64_t g = 0;  // k-blocks issued so far
      bool ok = true;
      for (int64_t x = blockIdx.x; x < a.ntiles && ok; x += gridDim.x) {
        int64_t tr, tc;
        tile_of(a, x, &tr, &tc);
        const int i0 = (int)(a.r0 + tr * kBM), c0 = (int)(a.r0 + tc * kBN);
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t ph = (uint32_t)((g / kStages) & 1);
          if (!mbar_wait(smem_u32(&empty[s]), ph ^ 1u) || *(volatile int*)&s_fail) {
            atomicExch(&s_fail, 1);
            ok = false;
            break;
          }
          unsigned char* st = base + s * kStageBytes;
          const uint32_t fb = smem_u32(&full[s]);
          mbar_expect_tx(fb, kStageBytes);
          const int kx = kb * Cfg::kBK;
#pragma unroll
          for (int o = 0; o < Cfg::kOps; ++o) {
            tma_load_2d(smem_u32(st + o * kTileBytes), &maps.W[o], kx, i0, fb);
            tma_load_2d(smem_u32(st + (Cfg::kOps + o) * kTileBytes), &maps.L[o], kx, c0, fb);
          }
        }
      }
      // drain: every issued stage must have landed before the CTA may exit
      for (int64_t h = (g > kStages ? g - kStages : 0); h < g; ++h)
        mbar_wait(smem_u32(&full[h % kStages]), (uint32_t)((h / kStages) & 1));
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      // A drain group (one fresh accumulator) holds kStepsPerDrain k-steps,
      // which may lie in one stage or span several; the last group of a tile
      // ends with the tile's last step.
      int64_t g = 0;   // stages consumed
      int64_t dg = 0;  // drain groups started
      bool ok = true;
      for (int64_t x = blockIdx.x; x < a.ntiles && ok; x += gridDim.x) {
        int in_group = 0;  // k-steps issued into the current accumulator
        uint32_t d = 0;
        int buf = 0;
        for (int kb = 0; kb < KB && ok; ++kb, ++g) {
          const int s = (int)(g % kStages);
          const uint32_t ph = (uint32_t)((g / kStages) & 1);
          if (!mbar_wait(smem_u32(&full[s]), ph) || *(volatile int*)&s_fail) {
            atomicExch(&s_fail, 1);
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          unsigned char* st = base + s * kStageBytes;
#pragma unroll
          for (int ks = 0; ks < Cfg::kSteps; ++ks) {
            if (in_group == 0) {
              buf = (int)(dg % kAccBufs);
              const uint32_t aph = (uint32_t)((dg / kAccBufs) & 1);
              if (!mbar_wait(smem_u32(&acc_empty[buf]), aph ^ 1u)) {
                atomicExch(&s_fail, 1);
                ok = false;
                break;
              }
              asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
              d = tmem + (uint32_t)(buf * kBN);
            }
            const uint32_t off = (uint32_t)(ks * 32);  // 32 B per k-step
#pragma unroll
            for (int pidx = 0; pidx < Cfg::kProducts; ++pidx) {
              int ia, ib;
              Cfg::product(pidx, &ia, &ib);
              const uint32_t sa = smem_u32(st + ia * kTileBytes) + off;
              const uint32_t sb = smem_u32(st + (Cfg::kOps + ib) * kTileBytes) + off;
              mma_issue<MODE>(d, sw_desc<Cfg::kRowBytes>(sa), sw_desc<Cfg::kRowBytes>(sb),
                              (in_group == 0 && pidx == 0) ? 0u : 1u);
            }
            ++in_group;
            if (in_group == Cfg::kStepsPerDrain || (kb == KB - 1 && ks == Cfg::kSteps - 1)) {
              mma_commit(smem_u32(&acc_full[buf]));
              ++dg;
              in_group = 0;
            }
          }
          if (!ok) break;
          mma_commit(smem_u32(&empty[s]));
        }
      }
    }
  } else {
    // ---- epilogue: warps 2..9; a thread owns half a row of the tile ----
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int half = (warp - 2) >> 2;
    const int rloc = 32 * quarter + lane;
    int64_t dg = 0;
    bool ok = true;
    const int drains = (KB * Cfg::kSteps + Cfg::kStepsPerDrain - 1) / Cfg::kStepsPerDrain;
    for (int64_t x = blockIdx.x; x < a.ntiles && ok; x += gridDim.x) {
      int64_t tr, tc;
      tile_of(a, x, &tr, &tc);
      const int64_t row = a.r0 + tr * kBM + rloc;
      const int64_t c0 = a.r0 + tc * kBN + half * kEpiCols;
      int64_t cend = c0 + kEpiCols;
      if (cend > a.n) cend = a.n;
      if (!a.full && tr == tc && cend > row + 1) cend = row + 1;
      const int ncol = (row < a.n && cend > c0) ? (int)(cend - c0) : 0;
      // the tile's C values are fetched now and land while the MMAs run, so
      // the read-modify-write at the end of the tile waits on no load
      float cold[kEpiCols];
      {
        const float* rp = a.C + row + c0 * a.ldc;
#pragma unroll
        for (int c = 0; c < kEpiCols; ++c) cold[c] = (c < ncol) ? __ldcg(rp + c * a.ldc) : 0.f;
      }
      float acc[kEpiCols];
#pragma unroll
      for (int c = 0; c < kEpiCols; ++c) acc[c] = 0.f;
      for (int dr = 0; dr < drains; ++dr, ++dg) {
        const int buf = (int)(dg % kAccBufs);
        const uint32_t aph = (uint32_t)((dg / kAccBufs) & 1);
        if (!mbar_wait(smem_u32(&acc_full[buf]), aph) || *(volatile int*)&s_fail) {
          atomicExch(&s_fail, 1);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) +
                               (uint32_t)(buf * kBN + half * kEpiCols);
#pragma unroll
        for (int ch = 0; ch < kEpiCols / 16; ++ch) {
          float v[16];
          tmem_ld16(taddr + (uint32_t)(ch * 16), v);
#pragma unroll
          for (int c = 0; c < 16; ++c) acc[ch * 16 + c] -= v[c];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(smem_u32(&acc_empty[buf]));
      }
      if (!ok) break;
      float* wp = a.C + row + c0 * a.ldc;
#pragma unroll
      for (int c = 0; c < kEpiCols; ++c) {
        if (c < ncol) *wp = cold[c] + acc[c];
        wp += a.ldc;
      }
    }
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Row-major [rows x ldk] operand of `esz`-byte elements, boxes of 128 rows x
// row_bytes bytes, swizzled over row_bytes (128 or 64).
bool make_map(CUtensorMap* m, const void* ptr, int64_t rows, int ldk, int esz, int row_bytes) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldk * (cuuint64_t)esz};
  cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esz), (cuuint32_t)kBM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, esz == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                   2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE,
                   row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int MODE, int V>
cudaError_t launch(float* C, int64_t ldc, int64_t n, int64_t r0, int kdim, void* const* Wops,
                   void* const* Lops, int ldk, bool full, int* err_flag, cudaStream_t s) {
  using Cfg = TcCfg<MODE, V>;
  const int esz = MODE == kSplit3xTf32 ? 4 : 2;
  if (kdim % Cfg::kBK != 0 || kdim <= 0 || kdim > ldk) return cudaErrorInvalidValue;
  if (((int64_t)ldk * esz) % 16 != 0) return cudaErrorInvalidValue;
  const int64_t m = n - r0;
  if (m <= 0) return cudaSuccess;
  if (n > 0x7fffffff) return cudaErrorInvalidValue;
  TcMaps maps;
  for (int o = 0; o < Cfg::kOps; ++o) {
    if (!make_map(&maps.W[o], Wops[o], n, ldk, esz, Cfg::kRowBytes) ||
        !make_map(&maps.L[o], Lops[o], n, ldk, esz, Cfg::kRowBytes))
      return cudaErrorInvalidValue;
  }
  // the shared-memory attribute is set once per device
  static bool attr[64] = {};  // per instantiation
  int dev = 0;
  cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_update_tc<MODE, V>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes<Cfg>());
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  TcArgs a;
  a.C = C;
  a.ldc = ldc;
  a.n = n;
  a.r0 = r0;
  a.kblocks = kdim / Cfg::kBK;
  a.tiles = (m + kBM - 1) / kBM;
  a.ntiles = full ? a.tiles * a.tiles : a.tiles * (a.tiles + 1) / 2;
  a.full = full ? 1 : 0;
  a.err = err_flag;
  DevInfo di;
  cudaError_t e = dev_info(&di);
  if (e != cudaSuccess) return e;
  int64_t grid = di.sm_count;
  if (g_tuning.max_ctas > 0 && grid > g_tuning.max_ctas) grid = g_tuning.max_ctas;
  if (grid > a.ntiles) grid = a.ntiles;
  k_update_tc<MODE, V><<<(unsigned)grid, kThreads, smem_bytes<Cfg>(), s>>>(maps, a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t outer_update_tc(int mode, float* C, int64_t ldc, int64_t n, int64_t r0, int kdim,
                            void* const* Wops, void* const* Lops, int ldk, bool full,
                            int* err_flag, cudaStream_t s) {
  const int v = g_tuning.update_variant;
#define DPP_TC_LAUNCH(M, V) launch<M, V>(C, ldc, n, r0, kdim, Wops, Lops, ldk, full, err_flag, s)
  if (mode == kSplit3xTf32) {
    switch (v) {
      case 1: return DPP_TC_LAUNCH(kSplit3xTf32, 1);
      case 2: return DPP_TC_LAUNCH(kSplit3xTf32, 2);
      case 3: return DPP_TC_LAUNCH(kSplit3xTf32, 3);
      default: return DPP_TC_LAUNCH(kSplit3xTf32, 0);
    }
  }
  if (mode == kSplitBf16x6) {
    return (v & 1) ? DPP_TC_LAUNCH(kSplitBf16x6, 1) : DPP_TC_LAUNCH(kSplitBf16x6, 0);
  }
#undef DPP_TC_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace dpp
