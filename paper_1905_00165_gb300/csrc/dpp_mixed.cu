// Mixed-precision Hermitian (real symmetric) DPP sampler.
//
// Storage: an FP32 copy A32 of the lower triangle of K. Arithmetic:
//   * pivots: a running diagonal kd_i = K_ii - sum_k w_ik l_ik kept in FP64
//     (double-float inside the sequential loop) and formed from the FP32
//     factor entries (w = l d), so a pivot carries no FP32 accumulation error
//     of its own; final pivots and log P(Y) are FP64;
//   * panel solves in FP32 SIMT, trailing updates on tensor cores (BF16x6 or
//     3xTF32 operand splits, FP32 accumulation) or FP32 SIMT;
//   * a decision is exact outside the borderline band and made in FP64 on a
//     recomputed pivot inside it.
// Borderline test: a pivot whose uniform lies within
//   tau_j = c * 2^-22 * sqrt(j + 1) * (K_jj + s_j),   s_j = sum_k |l_jk w_jk|,
// of its threshold is recomputed in FP64 from the original K (the exact
// conditional probability, Props. 3-5) before its decision.
//
// Blocking (two levels): the inner panels (32 wide) of one outer block of
// width NB (<= 256) are decided and solved inside one cooperative launch (see
// the pipeline described at cta0_block); after each outer block one rank-NB
// trailing update is applied to the whole remaining lower triangle, which
// makes the dominant contraction NB deep.
#include <cuda_bf16.h>
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"
#include "dpp_recompute.cuh"

namespace dpp {

Tuning g_settings;
thread_local Tuning g_tuning;

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ inline float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__global__ void __launch_bounds__(256) k_convert(const double* K, int64_t ldk, float* A,
                                                 int64_t lda, int64_t n, double* kd, double* s) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const double* col = K + j * ldk;
    float* dst = A + j * lda;
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) dst[i] = (float)col[i];
    if (threadIdx.x == 0) {
      kd[j] = col[j];
      s[j] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(256) k_export(const float* A, int64_t lda, const double* piv,
                                                double* F, int64_t ldf, int64_t n) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x)
      F[i + j * ldf] = (i == j) ? piv[j] : (double)A[i + j * lda];
  }
}

// One cooperative launch per outer block [p, p + NBp) of the mixed path:
// CTA 0 decides the block's inner panels (warp 0) with its support warps
// preparing each next diagonal block, CTA 1 (the helper) streams the block's
// own rows below that, and CTAs 2.. stream the rows below the block
// (left-looking update, wait, solve), serving FP64 recompute requests while
// they wait. Every CTA from 1 on is a recompute worker.
struct OuterArgs {
  const double* K;
  int64_t ldk;
  float* A;
  int64_t lda, n, p;
  int NBp, NB;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double* piv;
  double* kd;
  double* s;
  float *Wk, *Lk;
  void* Wop[3];  // tensor-core operand splits of W (row-major [n x NB])
  void* Lop[3];  // ... and of L
  int split;     // kSplit3xTf32 or kSplitBf16x6
  float* rdv;    // FP32 reciprocal of each final pivot
  dpp_result* res;
  unsigned epoch0;  // epoch of the first inner panel of this block
  double tol;
  float tau0;
  int64_t wrow0, wrows;  // worker w >= 1 owns rows [wrow0 + (w-1) wrows, ... + wrows)
  RecomputeArgs rc;
};

// control word: the rows of the inner panel with this epoch are final for every
// earlier panel of the block (released before that panel's decisions start)
enum { kCtlRows = 8 };
constexpr int kSwLd = 65;

constexpr int kThreadsOuter = 256;
constexpr size_t kOuterDynSmem = sizeof(float) * kMaxOuterBlock * kPanel;  // staged Lk

// Shared memory of k_outer_mixed, at file scope so that every function sees
// its state space (a shared store can then never be taken to alias a global
// load, and loads are not held back behind stores).
extern __shared__ __align__(16) float g_outer_dyn[];  // staged Lk: [kMaxOuterBlock][kPanel]
__shared__ float g_sW[2 * 32 * kSwLd];
__shared__ float g_stage[kThreadsOuter / 32][kPanel][kPanel + 1];
__shared__ float g_sL[kPanel][kPanel + 1];
__shared__ float g_srd[kPanel];
__shared__ int g_s_ok;

// Copy of N elements by THREADS threads with every load issued before the
// first store, so that the loads are in flight together (a strided loop with
// a runtime count would wait out one load latency per element).
template <int N, int THREADS, class LoadF, class StoreF>
__device__ __forceinline__ void staged_copy(int tid, LoadF ld, StoreF stv) {
  constexpr int kPer = (N + THREADS - 1) / THREADS;
  float v[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e = tid + j * THREADS;
    v[j] = e < N ? ld(e) : 0.f;
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int e = tid + j * THREADS;
    if (e < N) stv(e, v[j]);
  }
}

// A[i, q+c] -= sum_{t < kk} Wk[i, t] Lk[q+c, t] for rows [r_lo, r_hi), c < b,
// restricted to i >= q + c, as a shared-memory tiled product: 64-row tiles,
// 32-deep chunks of W staged k-major in sW (coalesced row loads), L read from
// sLk[t][c] (staged by the caller); each thread owns 2 rows x 4 columns.
__device__ void inner_update(const OuterArgs& a, int64_t q, int b, int kk, int64_t r_lo,
                             int64_t r_hi, int tid) {
  const float* sLk = g_outer_dyn;
  float* sW = g_sW;
  if (kk <= 0 || r_lo >= r_hi) return;
  const int ty = tid / 8, tx = tid % 8;
  const int lr = tid / 8, lf = tid % 8;  // W loader: 8 float4 per row, 2 rows per thread
  const int nchunks = (kk + 31) / 32;
  for (int64_t i0 = r_lo; i0 < r_hi; i0 += 64) {
    float acc[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = 0.f;
    // software pipeline: chunk c+1 is loaded into registers while chunk c is
    // consumed from the other shared buffer
    float4 pre[2];
    auto load = [&](int k0) {
      const int kc = (kk - k0) < 32 ? (kk - k0) : 32;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t i = i0 + lr + 32 * h;
        pre[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < r_hi && 4 * lf < kc)
          pre[h] = __ldcg(reinterpret_cast<const float4*>(a.Wk + i * (int64_t)a.NB + k0 + 4 * lf));
      }
    };
    auto store = [&](float* buf) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = lr + 32 * h;
        buf[(4 * lf + 0) * kSwLd + r] = pre[h].x;
        buf[(4 * lf + 1) * kSwLd + r] = pre[h].y;
        buf[(4 * lf + 2) * kSwLd + r] = pre[h].z;
        buf[(4 * lf + 3) * kSwLd + r] = pre[h].w;
      }
    };
    load(0);
    store(sW);
    __syncthreads();
    for (int c = 0; c < nchunks; ++c) {
      const int k0 = 32 * c;
      const int kc = (kk - k0) < 32 ? (kk - k0) : 32;
      float* cur = sW + (c & 1) * 32 * kSwLd;
      if (c + 1 < nchunks) load(k0 + 32);
      for (int t = 0; t < kc; ++t) {
        const float w0 = cur[t * kSwLd + 2 * ty], w1 = cur[t * kSwLd + 2 * ty + 1];
        const float4 l = *reinterpret_cast<const float4*>(&sLk[(k0 + t) * kPanel + 4 * tx]);
        acc[0][0] = fmaf(w0, l.x, acc[0][0]);
        acc[0][1] = fmaf(w0, l.y, acc[0][1]);
        acc[0][2] = fmaf(w0, l.z, acc[0][2]);
        acc[0][3] = fmaf(w0, l.w, acc[0][3]);
        acc[1][0] = fmaf(w1, l.x, acc[1][0]);
        acc[1][1] = fmaf(w1, l.y, acc[1][1]);
        acc[1][2] = fmaf(w1, l.z, acc[1][2]);
        acc[1][3] = fmaf(w1, l.w, acc[1][3]);
      }
      if (c + 1 < nchunks) store(sW + ((c + 1) & 1) * 32 * kSwLd);
      __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int64_t i = i0 + 2 * ty + rr;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * tx + cc;
        if (i < r_hi && c < b && i >= q + c) a.A[i + (q + c) * a.lda] -= acc[rr][cc];
      }
    }
  }
}

// Stage Lk rows [q, q+b), columns t < kk, into sLk[t][c].
__device__ void stage_lk(const OuterArgs& a, int64_t q, int b, int kk, int tid) {
  float* sLk = g_outer_dyn;
  const int n = kk * kPanel;
  const float* Lk = a.Lk;
  const int64_t NB = a.NB;
  constexpr int kIn = 8;  // loads in flight per thread
  for (int base = tid; base < n; base += kIn * kThreadsOuter) {
    float v[kIn];
#pragma unroll
    for (int j = 0; j < kIn; ++j) {
      const int idx = base + j * kThreadsOuter;
      v[j] = 0.f;
      if (idx < n) {
        const int t = idx % kk, c = idx / kk;
        if (c < b) v[j] = __ldcg(&Lk[(q + c) * NB + t]);
      }
    }
#pragma unroll
    for (int j = 0; j < kIn; ++j) {
      const int idx = base + j * kThreadsOuter;
      if (idx < n) sLk[(idx % kk) * kPanel + idx / kk] = v[j];
    }
  }
}

// Panel solve of rows [r_lo, r_hi) against the factored 32 x 32 block:
// w = a L11^{-T} (FP32), l = w / d; writes L into A (column-major, coalesced),
// folds sum w l into the FP64 running diagonal, and writes W, L and their
// tensor-core splits (TF32 pairs or BF16 triplets) row-major through a
// per-warp shared-memory transpose so each store instruction covers one
// contiguous row segment. All threads iterate together.
__device__ void panel_solve(const OuterArgs& a, int64_t q, int b, int64_t r_lo,
                            int64_t r_hi, int tid) {
  const float (*sL)[kPanel + 1] = g_sL;
  const float* srd = g_srd;
  float (*stage)[kPanel][kPanel + 1] = g_stage;
  const int t0 = (int)(q - a.p);
  const int warp = tid >> 5, lane = tid & 31;
  float* A = a.A;
  const int64_t lda = a.lda;
  for (int64_t base = r_lo; base < r_hi; base += kThreadsOuter) {
    const int64_t i = base + tid;
    const bool valid = i < r_hi;
    float w[kPanel];
#pragma unroll
    for (int k = 0; k < kPanel; ++k) w[k] = (valid && k < b) ? A[i + (q + k) * lda] : 0.f;
#pragma unroll
    for (int k = 1; k < kPanel; ++k) {
      if (k < b) {
#pragma unroll
        for (int t = 0; t < k; ++t) w[k] = fmaf(-w[t], sL[k][t], w[k]);
      }
    }
    float l[kPanel];
    f2 dsum = {0.f, 0.f};
    float ssum = 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
      l[k] = w[k] * srd[k];
      if (k < b) {
        dsum = f2_add_prod(dsum, w[k], l[k]);
        ssum += fabsf(w[k] * l[k]);
        if (valid) A[i + (q + k) * lda] = l[k];
      }
    }
    if (valid) {
      a.kd[i] -= f2_to_double(dsum);
      a.s[i] += (double)ssum;
    }
    // row-major operand rows of this warp: base + 32 warp + rr
    const int64_t wrow0 = base + 32 * warp;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
      for (int k = 0; k < kPanel; ++k) stage[warp][lane][k] = pass == 0 ? w[k] : l[k];
      __syncwarp();
      float* P = pass == 0 ? a.Wk : a.Lk;
      void* const* ops = pass == 0 ? a.Wop : a.Lop;
      for (int rr = 0; rr < 32; ++rr) {
        const int64_t row = wrow0 + rr;
        if (row < r_hi) {
          const float v = stage[warp][rr][lane];
          const int64_t off = row * (int64_t)a.NB + t0 + lane;
          P[off] = v;
          if (a.split == kSplitBf16x6) {
            // three BF16 pieces: v = b0 + b1 + b2 exactly (8 + 8 + 8 bits)
            const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
            const float r1 = v - __bfloat162float(b0);
            const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(b1);
            static_cast<__nv_bfloat16*>(ops[0])[off] = b0;
            static_cast<__nv_bfloat16*>(ops[1])[off] = b1;
            static_cast<__nv_bfloat16*>(ops[2])[off] = __float2bfloat16_rn(r2);
          } else {
            const float h = tf32_rna(v);
            static_cast<float*>(ops[0])[off] = h;
            static_cast<float*>(ops[1])[off] = tf32_rna(v - h);
          }
        }
      }
      __syncwarp();
    }
  }
}

// Per-outer-block bookkeeping kept by CTA 0 (shared memory).
struct BlockLog {
  float dhi[kMaxOuterBlock];
  float dlo[kMaxOuterBlock];
  unsigned char kp[kMaxOuterBlock];
  int border;
  float max_ratio;
  int rc_failed;
};

// Borderline step (rare path, kept out of the unrolled loop): recompute the
// pivot of local index j in FP64 and decide in FP64. The rows of the block
// must be in blk.
struct BorderOut {
  double dfin;  // final FP64 pivot (after -1 on rejection)
  int keep;
  int seq;
};

__device__ __noinline__ BorderOut borderline_step(const OuterArgs& a, float (*blk)[kPanel + 1],
                                                  int b, int64_t q, int j, unsigned epoch, int seq,
                                                  float ph, float pl, double u_j, float tau,
                                                  BlockLog* bl) {
  const int lane = threadIdx.x & 31;
  const double p64 = (double)ph + (double)pl;
  double pe = p64, est = 0.0;
  // the earlier panels' rows, pivots and decisions must be out in global
  // memory before the workers read them
  bool ready = true;
  if (lane == 0) ready = rc_wait_geq(a.rc, &a.rc.ctrl[kCtlRows], epoch);
  ready = __shfl_sync(kFull, ready, 0);
  const bool ok = ready && recompute_leader(a.rc, blk, b, q, j, epoch, &seq, &pe, &est);
  const bool keep = u_j < pe;
  if (lane == 0) {
    bl->border += 1;
    const float ratio = (float)(fabs(pe - p64) / (double)tau);
    if (ratio > bl->max_ratio) bl->max_ratio = ratio;
    if (!ok || est > fabs(u_j - pe)) bl->rc_failed = 1;
  }
  BorderOut o;
  o.dfin = keep ? pe : pe - 1.0;
  o.keep = keep ? 1 : 0;
  o.seq = seq;
  return o;
}

// One decision step of the 32 x 32 diagonal block, local pivot J: lane i
// holds row i of the block as a full symmetric row, the pivot row is
// broadcast by shuffles. The fast chain is unrolled (J known at compile time,
// so the rows stay in registers) and holds no call, which keeps its code
// small enough to run from the instruction cache on its first pass in a
// panel; at the first pivot inside the borderline band it stops (stop = J)
// and the panel is finished by dec_slow.
template <int J>
__device__ __forceinline__ void dec_fast(int b, int lane, float tau0, float (&r)[kPanel], f2& dd,
                                         float& si, float uf, float kf, float sq, bool& mykeep,
                                         int& stop) {
  if (J < b && stop < 0) {
    const float ph = __shfl_sync(kFull, dd.hi, J);
    const float uj = __shfl_sync(kFull, uf, J);
    const float sj = __shfl_sync(kFull, si, J);
    const float kj = __shfl_sync(kFull, kf, J);
    const float sqj = __shfl_sync(kFull, sq, J);
    const float tau = tau0 * sqj * (fabsf(kj) + sj) + 0x1.0p-22f;
    if (fabsf(uj - ph) <= tau) {
      stop = J;
    } else {
      // FP32 comparison of the FP32 uniform with the pivot's high part: u and
      // the double-float pivot in [-1, 2] each lose at most 2^-24 to the
      // rounding (u < 1, |hi| < 2, half an ulp each), and tau >= 2^-22 (its
      // floor), so outside the band the FP64 comparison of u with the pivot
      // gives the same decision
      const bool kp = uj < ph;
      const float df = kp ? ph : ph - 1.0f;
      if (lane == J && !kp) dd = f2_add_f(dd, -1.0f);
      const float rd = 1.0f / df;
      const float wj = r[J];
      const float l = wj * rd;
      const bool act = (lane > J) && (lane < b);
#pragma unroll
      for (int k = J + 1; k < kPanel; ++k) {
        const float pk = __shfl_sync(kFull, r[k], J);
        if (act) r[k] = fmaf(-l, pk, r[k]);
      }
      if (act) {
        r[J] = l;
        dd = f2_sub_prod(dd, wj, l);
        si += fabsf(wj * l);
      }
      if (lane == J) {
        r[J] = df;
        mykeep = kp;
      }
    }
  }
  if constexpr (J + 1 < kPanel)
    dec_fast<J + 1>(b, lane, tau0, r, dd, si, uf, kf, sq, mykeep, stop);
}

// Decision state of warp 0 handed to dec_slow through shared memory (the
// rows of the fast chain must never have their address taken, or they would
// leave the registers).
struct DecState {
  float dd_hi[kPanel], dd_lo[kPanel], si[kPanel];
  unsigned char keep[kPanel];
};

// The rest of the panel from local pivot j0 (a borderline one) on, with a
// runtime step index: the same arithmetic as dec_fast, predicated over all 32
// columns, and one call site for the FP64 recompute of borderline pivots. The
// rows come in and go out through sL (row lane in sL[lane]), the per-lane
// state through ds.
__device__ __noinline__ void dec_slow(const OuterArgs& a, float (*sL)[kPanel + 1], DecState* ds,
                                      BlockLog* bl, int64_t q, unsigned epoch, int b, float tau0,
                                      float uf, float kf, float sq, double u, int& seq, int j0) {
  const int lane = threadIdx.x & 31;
  float r[kPanel];
#pragma unroll
  for (int k = 0; k < kPanel; ++k) r[k] = sL[lane][k];
  f2 dd = make_f2(ds->dd_hi[lane], ds->dd_lo[lane]);
  float si = ds->si[lane];
  bool mykeep = ds->keep[lane] != 0;
  __syncwarp();
#pragma unroll 1
  for (int J = j0; J < b; ++J) {
    const float ph = __shfl_sync(kFull, dd.hi, J);
    const float uj = __shfl_sync(kFull, uf, J);
    const float sj = __shfl_sync(kFull, si, J);
    const float kj = __shfl_sync(kFull, kf, J);
    const float sqj = __shfl_sync(kFull, sq, J);
    const float tau = tau0 * sqj * (fabsf(kj) + sj) + 0x1.0p-22f;
    bool kp;
    float df;
    if (fabsf(uj - ph) <= tau) {
      // rows to shared memory, decisions and FP64 pivots of [q, q + J) to
      // global memory: the recompute reads them
#pragma unroll
      for (int k = 0; k < kPanel; ++k) sL[lane][k] = r[k];
      if (lane < J) {
        a.piv[q + lane] = f2_to_double(dd);
        a.keep[q + lane] = mykeep ? 1 : 0;
      }
      __syncwarp();
      const float pl = __shfl_sync(kFull, dd.lo, J);
      const double uj64 = __shfl_sync(kFull, u, J);
      const BorderOut o = borderline_step(a, sL, b, q, J, epoch, seq, ph, pl, uj64, tau, bl);
      seq = o.seq;
      kp = o.keep != 0;
      df = (float)o.dfin;
      if (lane == J) dd = f2_from_double(o.dfin);
    } else {
      kp = uj < ph;
      df = kp ? ph : ph - 1.0f;
      if (lane == J && !kp) dd = f2_add_f(dd, -1.0f);
    }
    const float rd = 1.0f / df;
    float wj = 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) wj = (k == J) ? r[k] : wj;
    const float l = wj * rd;
    const bool act = (lane > J) && (lane < b);
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
      const float pk = __shfl_sync(kFull, r[k], J);
      if (act && k > J) r[k] = fmaf(-l, pk, r[k]);
    }
#pragma unroll
    for (int k = 0; k < kPanel; ++k)
      if (k == J) r[k] = act ? l : (lane == J ? df : r[k]);
    if (act) {
      dd = f2_sub_prod(dd, wj, l);
      si += fabsf(wj * l);
    }
    if (lane == J) mykeep = kp;
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < kPanel; ++k) sL[lane][k] = r[k];
  ds->dd_hi[lane] = dd.hi;
  ds->dd_lo[lane] = dd.lo;
  ds->si[lane] = si;
  ds->keep[lane] = mykeep ? 1 : 0;
  __syncwarp();
}

// ---- CTA 0 of the outer-block launch ----------------------------------------
//
// The inner panels R_0, R_1, ... of the block (32 rows / columns each) run as
// a pipeline around warp 0, which only makes decisions. With panel k being
// decided:
//   * CTA 1 (the helper) takes the block's rows from R_{k+2} on: it solves
//     them against panel k-1, updates their column block R_k through panel
//     k-1 (left-looking) and raises control word kCtlPre;
//   * warps 1-7 of CTA 0 (the support warps) first write panel k-1 out to
//     global memory and release it (kCtlDone, kCtlRows), then bring the rows
//     of R_{k+1} up to date through panel k-1 (they are the helper's rows
//     through its previous step): solve them against panel k-1, then update
//     their column block R_k and their diagonal block from the stored W and
//     L (left-looking, in 32-wide chunks); once panel k is decided they solve
//     R_{k+1} against it and apply its rank-32 update in shared memory, and
//     hand the result to warp 0.
// Named barriers between warp 0 and the support warps:
//   1  warp 0 arrives when the decisions of a panel are in shared memory;
//   2  the support warps arrive when the inputs of the next panel are;
//   3  support warps only (224 threads).
// Each side arrives on one barrier only after passing the other, so neither
// can arrive twice on a barrier before the other side has passed it.

enum { kCtlPre = 9 };  // control word: the helper's step for the panel with this epoch is done

constexpr int kSupThreads = kThreadsOuter - 32;

__device__ __forceinline__ void nb_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nb_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// CTA 0 working set (shared memory of k_outer_mixed)
struct Cta0Smem {
  // decisions of panel k (warp 0 -> support), double buffered by k & 1
  float L11[2][kPanel][kPanel + 1];  // L (strictly lower) and D (diagonal)
  float rd[2][kPanel];               // FP32 1 / d
  double piv[2][kPanel];             // FP64 final pivots
  unsigned char keep[2][kPanel];
  // inputs of the next panel's decisions (support -> warp 0)
  float blk[kPanel][kPanel + 1];  // symmetric diagonal block
  double kd[kPanel];              // running diagonal (FP64)
  double sj[kPanel];              // borderline scale
  double u[kPanel];               // uniforms
  float kf[kPanel];               // FP32 K_jj
  // prefetched by the support warps while warp 0 decides
  float X[kPanel][kPanel + 1];  // A[R_{k+1}, R_k]
  float Y[kPanel][kPanel + 1];  // A[R_{k+1}, R_{k+1}] (lower)
  double kdP[kPanel];
  double sP[kPanel];
  double uP[kPanel];
  float kfP[kPanel];
  // solve of R_{k+1} against panel k
  float W[kPanel][kPanel + 1];
  float Lr[kPanel][kPanel + 1];
  // 32-wide chunks of the stored W and L (left-looking update), L transposed
  float Wc[kPanel][kPanel + 1];
  __align__(16) float LcT[kPanel][2 * kPanel + 4];
};

__shared__ Cta0Smem g_S0;
__shared__ BlockLog g_bl;

// Column-oriented forward substitution of the rows r = sw, sw + 7, ... of X
// against the factored block of buffer buf (lane = column): w = x L11^{-T},
// l = w / d. Writes S.W, S.Lr and subtracts sum w l from kd (FP64).
__device__ __noinline__ void sup_solve_rows(int buf, int bn, bool prefetched) {
  Cta0Smem& S = g_S0;
  double* kd = prefetched ? S.kdP : S.kd;
  double* sj = prefetched ? S.sP : S.sj;
  const int st = threadIdx.x - 32, lane = threadIdx.x & 31, sw = st >> 5;
  constexpr unsigned kF = 0xffffffffu;
  float w[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const int r = sw + 7 * m;
    w[m] = (r < kPanel) ? S.X[r][lane] : 0.f;
  }
  // a compact loop: this runs once per panel, cold in the instruction cache
#pragma unroll 4
  for (int t = 0; t < kPanel; ++t) {
    const float lt = S.L11[buf][lane][t];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
      const float wt = __shfl_sync(kF, w[m], t);
      if (lane > t) w[m] = fmaf(-wt, lt, w[m]);
    }
  }
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    const int r = sw + 7 * m;
    if (r < kPanel) {
      const bool vr = r < bn;
      const float wv = vr ? w[m] : 0.f;
      const float lv = wv * S.rd[buf][lane];
      S.W[r][lane] = wv;
      S.Lr[r][lane] = lv;
      // sum w l in double-float, sum |w l| in FP32 (FP64 arithmetic is the
      // GPU's slowest pipe; one FP64 subtraction per row remains)
      f2 ds = {__fmul_rn(wv, lv), 0.f};
      ds.lo = __fmaf_rn(wv, lv, -ds.hi);
      float ss = fabsf(wv * lv);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const f2 other = {__shfl_xor_sync(kF, ds.hi, o), __shfl_xor_sync(kF, ds.lo, o)};
        ds = f2_add(ds, other);
        ss += __shfl_xor_sync(kF, ss, o);
      }
      if (lane == 0 && vr) {
        kd[r] -= f2_to_double(ds);
        sj[r] += (double)ss;
      }
    }
  }
}

// Support warps, while panel k (at q) is decided and k + 1 < nP: bring the
// rows of R_{k+1} (bn rows) up to date through panel k - 1 and leave in
// shared memory X = A[R_{k+1}, R_k], Y = A[R_{k+1}, R_{k+1}] (lower), and
// their running diagonals, borderline scales, uniforms and K_jj.
//   1. every global load the step needs is issued at once, into registers
//      (one memory latency instead of one per 32-wide chunk): the rows'
//      block against panel k - 1, the stored W and L of panels 0 .. k - 2,
//      the L rows of R_k for panel k - 1, and the current X and Y;
//   2. the rows are solved against panel k - 1 (shared memory);
//   3. X and Y lose sum_t W[R_{k+1}, t] L[., t] over panels 0 .. k - 1
//      (left-looking), chunk by chunk from registers and shared memory.
constexpr int kMaxPreChunks = kMaxOuterBlock / kPanel - 2;  // panels 0 .. k - 2, k <= 7
constexpr int kPerChunk = (3 * kPanel * kPanel + kSupThreads - 1) / kSupThreads;
constexpr int kPerBlk = (kPanel * kPanel + kSupThreads - 1) / kSupThreads;

__device__ __noinline__ void sup_ready_next(const OuterArgs& a, int k, int64_t q, int bn) {
  Cta0Smem& S = g_S0;
  const int st = threadIdx.x - 32;
  const int64_t p = a.p, qn = q + kPanel, qp = q - kPanel;
  float* A = a.A;
  const int64_t lda = a.lda;
  const int64_t NB = a.NB;
  const int nch = k >= 2 ? k - 1 : 0;  // chunks already in global memory
  const int gi = st >> 2, gc = (st & 3) * 16;
  const bool gemm = st < 4 * kPanel;

  // ---- 1. all loads in flight together ----
  if (st < kPanel) {
    const int i = st;
    const bool vi = i < bn;
    S.kdP[i] = vi ? a.kd[qn + i] : 0.0;
    S.sP[i] = vi ? a.s[qn + i] : 0.0;
    S.uP[i] = vi ? (a.uniforms ? a.uniforms[qn + i]
                               : philox_uniform(a.seed, a.inst, (uint64_t)(qn + i)))
                 : 2.0;
    S.kfP[i] = vi ? (float)a.K[(qn + i) + (qn + i) * a.ldk] : 0.f;
  }
  float x1v[kPerBlk], lrk[kPerBlk];
#pragma unroll
  for (int j = 0; j < kPerBlk; ++j) {
    const int e = st + j * kSupThreads;
    const int i = e % kPanel, c = e / kPanel;
    x1v[j] = (k >= 1 && e < kPanel * kPanel && i < bn) ? __ldcg(&A[(qn + i) + (qp + c) * lda])
                                                       : 0.f;
    const int r = e / kPanel, t = e % kPanel;  // L rows of R_k, panel k - 1
    lrk[j] = (k >= 1 && e < kPanel * kPanel)
                 ? __ldcg(&a.Lk[(q + r) * NB + (k - 1) * kPanel + t]) : 0.f;
  }
  float pre[kMaxPreChunks][kPerChunk];
#pragma unroll
  for (int ch = 0; ch < kMaxPreChunks; ++ch) {
    const int t0 = ch * kPanel;
#pragma unroll
    for (int j = 0; j < kPerChunk; ++j) {
      const int e = st + j * kSupThreads;
      const int r = e / kPanel, t = e % kPanel;  // consecutive threads: one row
      float v = 0.f;
      if (ch < nch && e < 3 * kPanel * kPanel) {
        if (r < kPanel) {
          if (r < bn) v = __ldcg(&a.Wk[(qn + r) * NB + t0 + t]);
        } else if (r < 2 * kPanel) {
          v = __ldcg(&a.Lk[(q + (r - kPanel)) * NB + t0 + t]);
        } else if (r - 2 * kPanel < bn) {
          v = __ldcg(&a.Lk[(qn + (r - 2 * kPanel)) * NB + t0 + t]);
        }
      }
      pre[ch][j] = v;
    }
  }
  float av[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int c = gc + j;
    const bool need = gemm && gi < bn && (c < kPanel || c - kPanel <= gi);
    av[j] = need ? __ldcg(&A[(qn + gi) + ((c < kPanel) ? (q + c) : (qn + c - kPanel)) * lda])
                 : 0.f;
  }

  // ---- 2. the rows against panel k - 1 (its L11 is still in buffer (k-1)&1)
  if (k >= 1) {
#pragma unroll
    for (int j = 0; j < kPerBlk; ++j) {
      const int e = st + j * kSupThreads;
      if (e < kPanel * kPanel) S.X[e % kPanel][e / kPanel] = x1v[j];
    }
    nb_sync(3, kSupThreads);
    sup_solve_rows((k - 1) & 1, bn, true);
    nb_sync(3, kSupThreads);
    for (int e = st; e < kPanel * kPanel; e += kSupThreads) {
      const int i = e / kPanel, c = e % kPanel;  // consecutive threads: one row
      if (i < bn) {
        a.Wk[(qn + i) * NB + (k - 1) * kPanel + c] = S.W[i][c];
        a.Lk[(qn + i) * NB + (k - 1) * kPanel + c] = S.Lr[i][c];
      }
    }
    for (int e = st; e < kPanel * kPanel; e += kSupThreads) {
      const int i = e % kPanel, c = e / kPanel;
      if (i < bn) A[(qn + i) + (qp + c) * lda] = S.Lr[i][c];
    }
  }

  // ---- 3. left-looking update of [X | Y] (Y's upper part is never read):
  // threads st < 128 own row gi and 16 consecutive columns gc.., register
  // blocked; chunk ch < nch comes from registers, the last (panel k - 1)
  // from the solve just done and from lrk
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
  for (int ch = 0; ch <= kMaxPreChunks; ++ch) {
    const bool from_regs = ch < nch;
    const bool last = (k >= 1) && (ch == nch);
    if (from_regs || last) {
      nb_sync(3, kSupThreads);  // the previous chunk's readers are done
      if (from_regs) {
#pragma unroll
        for (int j = 0; j < kPerChunk; ++j) {
          const int e = st + j * kSupThreads;
          if (e < 3 * kPanel * kPanel) {
            const int r = e / kPanel, t = e % kPanel;
            if (r < kPanel) S.Wc[r][t] = pre[ch < kMaxPreChunks ? ch : 0][j];
            else S.LcT[t][r - kPanel] = pre[ch < kMaxPreChunks ? ch : 0][j];
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < kPerBlk; ++j) {
          const int e = st + j * kSupThreads;
          if (e < kPanel * kPanel) {
            const int r = e / kPanel, t = e % kPanel;
            S.Wc[r][t] = S.W[r][t];
            S.LcT[t][r] = lrk[j];
            S.LcT[t][kPanel + r] = S.Lr[r][t];
          }
        }
      }
      nb_sync(3, kSupThreads);
      if (gemm) {
#pragma unroll 4
        for (int t = 0; t < kPanel; ++t) {
          const float w = S.Wc[gi][t];
          const float4* lp = reinterpret_cast<const float4*>(&S.LcT[t][gc]);
#pragma unroll
          for (int v4 = 0; v4 < 4; ++v4) {
            const float4 l = lp[v4];
            acc[4 * v4 + 0] = fmaf(w, l.x, acc[4 * v4 + 0]);
            acc[4 * v4 + 1] = fmaf(w, l.y, acc[4 * v4 + 1]);
            acc[4 * v4 + 2] = fmaf(w, l.z, acc[4 * v4 + 2]);
            acc[4 * v4 + 3] = fmaf(w, l.w, acc[4 * v4 + 3]);
          }
        }
      }
    }
  }
  if (gemm) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int c = gc + j;
      const float v = gi < bn ? av[j] - acc[j] : 0.f;
      if (c < kPanel) S.X[gi][c] = v;
      else S.Y[gi][c - kPanel] = (c - kPanel <= gi) ? v : 0.f;
    }
  }
  nb_sync(3, kSupThreads);
}

// The first panel of the block: its rows as the previous launches left them.
__device__ __noinline__ void sup_load_first(const OuterArgs& a, int b0) {
  Cta0Smem& S = g_S0;
  const int st = threadIdx.x - 32;
  const int64_t p = a.p;
  const float* A = a.A;
  const int64_t lda = a.lda;
  staged_copy<kPanel * kPanel, kSupThreads>(
      st,
      [&](int e) {
        const int i = e % kPanel, c = e / kPanel;
        return (i < b0 && c <= i) ? __ldcg(&A[(p + i) + (p + c) * lda]) : 0.f;
      },
      [&](int e, float v) { S.Y[e % kPanel][e / kPanel] = v; });
  if (st < kPanel) {
    const int i = st;
    const bool vi = i < b0;
    S.kdP[i] = vi ? a.kd[p + i] : 0.0;
    S.sP[i] = vi ? a.s[p + i] : 0.0;
    S.uP[i] = vi ? (a.uniforms ? a.uniforms[p + i]
                               : philox_uniform(a.seed, a.inst, (uint64_t)(p + i)))
                 : 2.0;
    S.kfP[i] = vi ? (float)a.K[(p + i) + (p + i) * a.ldk] : 0.f;
  }
}

// Support warps: the inputs of the next panel's decisions from the prefetched
// blocks. With the previous panel k (buffer buf), solve the rows of R_{k+1}
// (w = x L11^{-T}, l = w / d) and apply the rank-32 update to the diagonal
// block; without (the block's first panel), take the blocks as they are.
__device__ __noinline__ void sup_prepare(int buf, int bn, bool after_panel) {
  Cta0Smem& S = g_S0;
  const int st = threadIdx.x - 32;
  if (after_panel) {
    if (st < kPanel) {
      S.kd[st] = S.kdP[st];
      S.sj[st] = S.sP[st];
    }
    nb_sync(3, kSupThreads);
    sup_solve_rows(buf, bn, false);
    nb_sync(3, kSupThreads);
    // rank-32 update of the lower triangle of the diagonal block
    for (int o = st; o < kPanel * (kPanel + 1) / 2; o += kSupThreads) {
      int i = (int)((sqrtf(8.f * (float)o + 1.f) - 1.f) * 0.5f);
      while (i * (i + 1) / 2 > o) --i;
      while ((i + 1) * (i + 2) / 2 <= o) ++i;
      const int c = o - i * (i + 1) / 2;
      float acc = 0.f;
#pragma unroll 8
      for (int t = 0; t < kPanel; ++t) acc = fmaf(S.W[i][t], S.Lr[c][t], acc);
      const float y = (i < bn) ? S.Y[i][c] - acc : 0.f;
      S.blk[i][c] = y;
      S.blk[c][i] = y;
    }
  } else {
    for (int o = st; o < kPanel * kPanel; o += kSupThreads) {
      const int i = o / kPanel, c = o % kPanel;
      S.blk[i][c] = (c <= i) ? S.Y[i][c] : S.Y[c][i];
    }
    if (st < kPanel) {
      S.kd[st] = S.kdP[st];
      S.sj[st] = S.sP[st];
    }
  }
  if (st < kPanel) {
    S.u[st] = S.uP[st];
    S.kf[st] = S.kfP[st];
  }
  nb_sync(3, kSupThreads);
}

// Support warps: panel k (at q, b rows, buffer buf) and the l rows of R_{k+1}
// (bn rows; bn = 0 for the block's last panel) out to global memory, then
// release both.
__device__ __noinline__ void sup_publish(const OuterArgs& a, int64_t q, int b, int kk, int buf,
                            int bn, unsigned epoch) {
  Cta0Smem& S = g_S0;
  const int st = threadIdx.x - 32;
  float* A = a.A;
  const int64_t lda = a.lda;
  for (int e = st; e < kPanel * kPanel; e += kSupThreads) {
    const int i = e % kPanel, c = e / kPanel;
    if (i < b && c <= i) A[(q + i) + (q + c) * lda] = S.L11[buf][i][c];
    if (i < bn) {
      const int64_t row = q + kPanel + i;
      const float l = S.Lr[i][c];
      A[row + (q + c) * lda] = l;
      a.Lk[row * (int64_t)a.NB + kk + c] = l;
    }
  }
  if (st < kPanel) {
    const int i = st;
    if (i < b) {
      a.piv[q + i] = S.piv[buf][i];
      a.keep[q + i] = S.keep[buf][i];
      a.rdv[q + i] = S.rd[buf][i];
    }
    if (i < bn) {
      a.kd[q + kPanel + i] = S.kd[i];
      a.s[q + kPanel + i] = S.sj[i];
    }
  }
  __threadfence();
  nb_sync(3, kSupThreads);
  if (st == 0) {
    recompute_release_done(a.rc, epoch);
    st_release(&a.rc.ctrl[kCtlRows], epoch + 1);
  }
}

// Warp 0: the decisions of panel k from the inputs in shared memory, results
// back to shared memory (its own register allocation, apart from the rest of
// the launch).
__device__ __noinline__ void w0_decide(const OuterArgs& a, int k, int* seq_io) {
  Cta0Smem& S = g_S0;
  BlockLog& bl = g_bl;
  const int lane = threadIdx.x & 31;
  const int64_t p = a.p;
  const int64_t pend = p + a.NBp;
  const int64_t q = p + (int64_t)kPanel * k;
  const int b = (int)((pend - q) < kPanel ? (pend - q) : kPanel);
  const int kk = (int)(q - p);
  const unsigned epoch = a.epoch0 + (unsigned)k;
  const int buf = k & 1;
  int seq = *seq_io;
  float r[kPanel];
#pragma unroll
  for (int c = 0; c < kPanel; ++c) r[c] = S.blk[lane][c];
  f2 dd = f2_from_double(S.kd[lane]);
  float si = (float)S.sj[lane];
  const double u = S.u[lane];
  const float uf = (float)u, kf = S.kf[lane];
  const float sq = sqrtf((float)(q + lane + 1));
  bool mykeep = false;
  int stop = -1;
  dec_fast<0>(b, lane, a.tau0, r, dd, si, uf, kf, sq, mykeep, stop);
  if (stop >= 0) {
    __shared__ DecState ds;
#pragma unroll
    for (int c = 0; c < kPanel; ++c) S.L11[buf][lane][c] = r[c];
    ds.dd_hi[lane] = dd.hi;
    ds.dd_lo[lane] = dd.lo;
    ds.si[lane] = si;
    ds.keep[lane] = mykeep ? 1 : 0;
    __syncwarp();
    dec_slow(a, S.L11[buf], &ds, &bl, q, epoch, b, a.tau0, uf, kf, sq, u, seq, stop);
#pragma unroll
    for (int c = 0; c < kPanel; ++c) r[c] = S.L11[buf][lane][c];
    dd = make_f2(ds.dd_hi[lane], ds.dd_lo[lane]);
    si = ds.si[lane];
    mykeep = ds.keep[lane] != 0;
    __syncwarp();
  }
#pragma unroll
  for (int c = 0; c < kPanel; ++c) S.L11[buf][lane][c] = r[c];
  if (lane < b) {
    const double d = f2_to_double(dd);
    S.piv[buf][lane] = d;
    S.keep[buf][lane] = mykeep ? 1 : 0;
    S.rd[buf][lane] = 1.0f / __double2float_rn(d);
    bl.dhi[kk + lane] = dd.hi;
    bl.dlo[kk + lane] = dd.lo;
    bl.kp[kk + lane] = mykeep ? 1 : 0;
  } else {
    S.rd[buf][lane] = 1.f;
  }
  __syncwarp();
  *seq_io = seq;
}

__device__ void cta0_block(const OuterArgs& a) {
  Cta0Smem& S = g_S0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p = a.p;
  const int64_t pend = p + a.NBp;
  const int nP = (a.NBp + kPanel - 1) / kPanel;

  if (warp == 0) {
    int seq = 0;
    for (int k = 0; k < nP; ++k) {
      nb_sync(2, kThreadsOuter);  // inputs of panel k are in shared memory
      w0_decide(a, k, &seq);
      nb_arrive(1, kThreadsOuter);  // decisions of panel k are in shared memory
    }
  } else {
    // the block's first panel: its rows as the previous launches left them
    const int b0 = (int)((pend - p) < kPanel ? (pend - p) : kPanel);
    sup_load_first(a, b0);
    nb_sync(3, kSupThreads);
    sup_prepare(0, b0, false);
    if (tid == 32) st_release(&a.rc.ctrl[kCtlRows], a.epoch0);
    nb_arrive(2, kThreadsOuter);
    for (int k = 0; k < nP; ++k) {
      const int64_t q = p + (int64_t)kPanel * k;
      const int b = (int)((pend - q) < kPanel ? (pend - q) : kPanel);
      const int kk = (int)(q - p);
      const unsigned epoch = a.epoch0 + (unsigned)k;
      const int buf = k & 1;
      const bool next = k + 1 < nP;
      const int64_t qn = q + kPanel;
      const int bn = next ? (int)((pend - qn) < kPanel ? (pend - qn) : kPanel) : 0;
      if (k >= 1) {
        // panel k - 1 and the l rows of R_k out to global memory, released
        const int64_t qp = q - kPanel;
        sup_publish(a, qp, kPanel, kk - kPanel, buf ^ 1, b, epoch - 1);
      }
      if (next) {
        // the helper's step for panel k - 1 covered the rows of R_{k+1}
        if (k >= 1 && tid == 32) rc_wait_geq(a.rc, &a.rc.ctrl[kCtlPre], epoch - 1);
        nb_sync(3, kSupThreads);
        sup_ready_next(a, k, q, bn);
      }
      nb_sync(1, kThreadsOuter);  // decisions of panel k
      if (next) {
        sup_prepare(buf, bn, true);
        nb_arrive(2, kThreadsOuter);
      } else {
        sup_publish(a, q, b, kk, buf, 0, epoch);
      }
    }
  }
}

// ---- CTA 1 (the helper): the block's rows from R_{k+2} on ----------------------
__device__ __noinline__ void helper_block(const OuterArgs& a) {
  int* s_ok = &g_s_ok;
  const int tid = threadIdx.x;
  const int64_t p = a.p;
  const int64_t pend = p + a.NBp;
  const float* A = a.A;
  const int64_t lda = a.lda;
  for (int64_t q = p; q < pend; q += kPanel) {
    const int b = (int)((pend - q) < kPanel ? (pend - q) : kPanel);
    const int kk = (int)(q - p);
    const unsigned epoch = a.epoch0 + (unsigned)((q - p) / kPanel);
    const int64_t r2 = q + 2 * kPanel < pend ? q + 2 * kPanel : pend;
    if (kk > 0 && r2 < pend) {
      // panel k - 1 is out (with kCtlDone of k - 1 and the L rows of R_k)
      if (tid == 0) *s_ok = rc_wait_geq(a.rc, &a.rc.ctrl[kCtlRows], epoch) ? 1 : 0;
      __syncthreads();
      if (!*s_ok) return;
      const int64_t qp = q - kPanel;
      for (int idx = tid; idx < kPanel * kPanel; idx += kThreadsOuter) {
        const int i = idx % kPanel, k = idx / kPanel;
        g_sL[i][k] = (k < i) ? __ldcg(&A[(qp + i) + (qp + k) * lda]) : 0.f;
      }
      if (tid < kPanel) g_srd[tid] = __ldcg(&a.rdv[qp + tid]);
      __syncthreads();
      panel_solve(a, qp, kPanel, r2, pend, tid);
      __syncthreads();
      stage_lk(a, q, b, kk, tid);
      __syncthreads();
      inner_update(a, q, b, kk, r2, pend, tid);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release(&a.rc.ctrl[kCtlPre], epoch);
    if (!recompute_follower(a.rc, epoch, s_ok)) return;
  }
}

__global__ void __launch_bounds__(kThreadsOuter, 1) k_outer_mixed(OuterArgs a) {
  BlockLog& bl = g_bl;
  int& s_ok = g_s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t p = a.p, n = a.n;
  const int64_t pend = p + a.NBp;
  float* A = a.A;
  const int64_t lda = a.lda;

  if (blockIdx.x == 0) {
    if (tid == 0) {
      bl.border = 0;
      bl.max_ratio = 0.f;
      bl.rc_failed = 0;
    }
    __syncthreads();
    cta0_block(a);
    __syncthreads();
    // likelihood and bookkeeping of the block (FP64, one pivot per thread)
    double lp = 0.0;
    int kept = 0, oor = 0, bad = 0;
    for (int i = tid; i < a.NBp; i += kThreadsOuter) {
      const double d = (double)bl.dhi[i] + (double)bl.dlo[i];
      const double pre = bl.kp[i] ? d : d + 1.0;
      lp += log(fabs(d));
      kept += bl.kp[i];
      oor += (pre < -a.tol || pre > 1.0 + a.tol) ? 1 : 0;
      bad |= isfinite(d) ? 0 : 1;
    }
    lp = warp_sum(lp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kept += __shfl_xor_sync(kFull, kept, o);
      oor += __shfl_xor_sync(kFull, oor, o);
      bad |= __shfl_xor_sync(kFull, bad, o);
    }
    __shared__ double s_lp[kThreadsOuter / 32];
    __shared__ int s_cnt[3][kThreadsOuter / 32];
    if (lane == 0) {
      s_lp[warp] = lp;
      s_cnt[0][warp] = kept;
      s_cnt[1][warp] = oor;
      s_cnt[2][warp] = bad;
    }
    __syncthreads();
    if (tid == 0) {
      double L = 0.0;
      int K = 0, O = 0, B = 0;
      for (int w = 0; w < kThreadsOuter / 32; ++w) {
        L += s_lp[w];
        K += s_cnt[0][w];
        O += s_cnt[1][w];
        B |= s_cnt[2][w];
      }
      dpp_result* r = a.res;
      r->logp += L;
      if (K) atomicAdd(&r->n_kept, K);
      if (O) {
        atomicAdd(&r->n_out_of_range, O);
        atomicOr(&r->status, DPP_RES_INADMISSIBLE);
      }
      if (B) atomicOr(&r->status, DPP_RES_NONFINITE);
      if (bl.border) {
        atomicAdd(&r->n_borderline, bl.border);
        if ((double)bl.max_ratio > r->max_err_ratio) r->max_err_ratio = (double)bl.max_ratio;
      }
      if (bl.rc_failed) atomicOr(&r->status, DPP_RES_RECOMPUTE);
    }
    return;
  }

  if (blockIdx.x == 1) {
    helper_block(a);
    return;
  }

  // ---- workers: rows below the outer block ----
  const int64_t w = blockIdx.x - 2;
  int64_t r_lo = a.wrow0 + w * a.wrows;
  int64_t r_hi = r_lo + a.wrows;
  if (r_lo > n) r_lo = n;
  if (r_hi > n) r_hi = n;
  for (int64_t q = p; q < pend; q += kPanel) {
    const int b = (int)((pend - q) < kPanel ? (pend - q) : kPanel);
    const int kk = (int)(q - p);
    const unsigned epoch = a.epoch0 + (unsigned)((q - p) / kPanel);
    if (kk > 0 && r_lo < r_hi) {
      if (tid == 0) s_ok = rc_wait_geq(a.rc, &a.rc.ctrl[kCtlRows], epoch) ? 1 : 0;
      __syncthreads();
      if (!s_ok) return;
      stage_lk(a, q, b, kk, tid);
      __syncthreads();
      inner_update(a, q, b, kk, r_lo, r_hi, tid);
    }
    if (!recompute_follower(a.rc, epoch, &s_ok)) return;
    if (r_lo < r_hi) {
      for (int idx = tid; idx < kPanel * kPanel; idx += kThreadsOuter) {
        const int i = idx % kPanel, k = idx / kPanel;
        g_sL[i][k] = (i < b && k < i) ? __ldcg(&A[(q + i) + (q + k) * lda]) : 0.f;
      }
      if (tid < kPanel) g_srd[tid] = tid < b ? __ldcg(&a.rdv[q + tid]) : 1.f;
      __syncthreads();
      panel_solve(a, q, b, r_lo, r_hi, tid);
      __syncthreads();
    }
  }
}

// FP32 SIMT update C[i, c] -= sum_{t < kk} Aop[i * ldk + t] * Bop[c * ldk + t]
// for i in [row0, n), c in [col0, col1); TRI: tiles of the lower triangle of a
// square region (row0 == col0) with i >= c; otherwise a rectangular grid with
// i >= c enforced element-wise (lower part of the diagonal block).
struct F32Args {
  float* C;
  int64_t ldc, row0, n, col0, col1;
  const float* Aop;
  const float* Bop;
  int ldk, kk;
  int64_t tiles_r;
};

constexpr int kT = 64;

template <bool TRI>
__global__ void __launch_bounds__(256) k_f32_update(F32Args u) {
  __shared__ float sA[32][kT + 1];
  __shared__ float sB[32][kT + 1];
  int64_t tr, tc;
  const int64_t x = blockIdx.x;
  if (TRI) {
    tr = (int64_t)((sqrtf(8.f * (float)x + 1.f) - 1.f) * 0.5f);  // FP32 estimate, exact below
    while (tr > 0 && tr * (tr + 1) / 2 > x) --tr;
    while ((tr + 1) * (tr + 2) / 2 <= x) ++tr;
    tc = x - tr * (tr + 1) / 2;
  } else {
    tr = x % u.tiles_r;
    tc = x / u.tiles_r;
  }
  const int64_t i0 = u.row0 + tr * kT, c0 = u.col0 + tc * kT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[p][r] = 0.f;
  for (int k0 = 0; k0 < u.kk; k0 += 32) {
    const int kc = (u.kk - k0) < 32 ? (u.kk - k0) : 32;
    for (int idx = threadIdx.x; idx < 32 * kT; idx += 256) {
      const int t = idx % 32, rr = idx / 32;
      const int64_t i = i0 + rr, c = c0 + rr;
      sA[t][rr] = (t < kc && i < u.n) ? u.Aop[i * u.ldk + k0 + t] : 0.f;
      sB[t][rr] = (t < kc && c < u.col1) ? u.Bop[c * u.ldk + k0 + t] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int t = 0; t < 32; ++t) {
      float ra[4], rb[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) ra[p] = sA[t][tx + 16 * p];
#pragma unroll
      for (int r = 0; r < 4; ++r) rb[r] = sB[t][ty + 16 * r];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[p][r] = fmaf(ra[p], rb[r], acc[p][r]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t c = c0 + ty + 16 * r;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t i = i0 + tx + 16 * p;
      if (i < u.n && c < u.col1 && i >= c) u.C[i + c * u.ldc] -= acc[p][r];
    }
  }
}

template <class K>
int coop_capacity(K kernel, int threads) {
  DevInfo di;
  if (dev_info(&di) != cudaSuccess) return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
    return 1;
  return per_sm > 0 ? per_sm * di.sm_count : 1;
}

struct MixedLayout {
  int64_t ld32;
  int NB;
  float* A32;
  float *Wk, *Lk;
  void* Wop[3];
  void* Lop[3];
  double *kd, *s, *piv;
  float* rdv;
  unsigned* flag;
  int* err;
  RecomputeScratch rs;
};

bool carve(Workspace& ws, int64_t n, int NB, MixedLayout* L) {
  L->NB = NB;
  L->ld32 = ((n + 31) / 32) * 32;
  if (L->ld32 < 32) L->ld32 = 32;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  L->A32 = static_cast<float*>(ws.take(sizeof(float) * (size_t)L->ld32 * nn));
  const size_t ob = sizeof(float) * nn * (size_t)kMaxOuterBlock;
  L->Wk = static_cast<float*>(ws.take(ob));
  L->Lk = static_cast<float*>(ws.take(ob));
  bool ops_ok = true;
  for (int o = 0; o < 3; ++o) {
    L->Wop[o] = ws.take(ob);
    L->Lop[o] = ws.take(ob);
    ops_ok = ops_ok && L->Wop[o] && L->Lop[o];
  }
  L->kd = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->s = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->piv = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->rdv = static_cast<float*>(ws.take(sizeof(float) * nn));
  L->flag = static_cast<unsigned*>(ws.take(256));
  L->err = reinterpret_cast<int*>(L->flag) + 16;
  if (!recompute_carve(ws, n, &L->rs)) return false;
  return L->A32 && L->Wk && L->Lk && ops_ok && L->kd && L->s && L->piv && L->rdv && L->flag;
}

}  // namespace

size_t ws_mixed(int64_t n) {
  Workspace probe;
  probe.base = reinterpret_cast<char*>(256);
  probe.size = ~size_t(0) >> 2;
  MixedLayout L;
  carve(probe, n, kMaxOuterBlock, &L);
  return probe.used + 512;
}

cudaError_t sample_mixed(const DrawArgs& a, Workspace ws) {
  const int64_t n = a.n;
  int NB = g_tuning.outer_block;
  MixedLayout L;
  if (!carve(ws, n, NB, &L)) return cudaErrorInvalidValue;
  cudaError_t e = init_result(a.result, a.stream);
  if (e != cudaSuccess || n == 0) return e;
  if ((e = cudaMemsetAsync(L.flag, 0, 256, a.stream)) != cudaSuccess) return e;
  if ((e = recompute_reset(L.rs, n, a.stream)) != cudaSuccess) return e;
  const double* K = static_cast<const double*>(a.K);
  {
    ProfScope ps(kProfConvert, a.stream, 0.0, 12.0 * (double)n * (double)n / 2.0);
    k_convert<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(K, a.ld, L.A32, L.ld32, n,
                                                                        L.kd, L.s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // cooperative capacity (and the shared-memory attribute), per device
  static int caps[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int& cap = caps[dev];
  if (cap == 0) {
    cudaError_t ea = cudaFuncSetAttribute(k_outer_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kOuterDynSmem);
    if (ea != cudaSuccess) return ea;
    DevInfo di;
    if ((ea = dev_info(&di)) != cudaSuccess) return ea;
    int per_sm = 0;
    ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_outer_mixed, kThreadsOuter,
                                                       kOuterDynSmem);
    if (ea != cudaSuccess) return ea;
    cap = per_sm * di.sm_count;
    if (cap > kMaxCoopCtas) cap = kMaxCoopCtas;
    if (cap < 3) return cudaErrorLaunchOutOfResources;
  }
  unsigned epoch = 1;
  const bool use_tc = g_tuning.update_kernel == 0;
  const int split = a.precision == DPP_PREC_BF16X6 ? kSplitBf16x6 : kSplit3xTf32;
  const int kb_tc = 32;  // k-block of the tensor-core update (both splits)
  for (int64_t p = 0; p < n; p += NB) {
    const int NBp = (int)((n - p) < NB ? (n - p) : NB);
    {
      OuterArgs oa;
      oa.K = K;
      oa.ldk = a.ld;
      oa.A = L.A32;
      oa.lda = L.ld32;
      oa.n = n;
      oa.p = p;
      oa.NBp = NBp;
      oa.NB = NB;
      oa.uniforms = a.uniforms;
      oa.seed = a.seed;
      oa.inst = a.instance;
      oa.keep = a.keep;
      oa.piv = L.piv;
      oa.kd = L.kd;
      oa.s = L.s;
      oa.Wk = L.Wk;
      oa.Lk = L.Lk;
      for (int o = 0; o < 3; ++o) {
        oa.Wop[o] = L.Wop[o];
        oa.Lop[o] = L.Lop[o];
      }
      oa.split = split;
      oa.rdv = L.rdv;
      oa.res = a.result;
      oa.epoch0 = epoch;
      oa.tol = 1e-3;
      oa.tau0 = (float)(g_tuning.tau_safety * 0x1.0p-22);
      // every other SM is a worker: they stream the rows below the block and
      // serve the recomputes (which are bandwidth- and latency-bound)
      const int64_t mw = n - p - NBp;
      int64_t nw = cap - 1;  // CTA 0 decides, CTA 1 helps, the rest stream
      if (g_tuning.max_ctas > 0 && nw + 1 > g_tuning.max_ctas) nw = g_tuning.max_ctas - 1;
      oa.wrow0 = p + NBp;
      const int64_t ntall = nw > 1 ? nw - 1 : 1;  // CTA 1 is the helper
      oa.wrows = (mw + ntall - 1) / ntall;
      if (oa.wrows < 1) oa.wrows = 1;
      oa.rc = recompute_args(L.rs, K, a.ld, L.A32, L.ld32, L.piv, a.keep, n, p, a.result);
      oa.rc.grid = (int)(nw + 1);
      void* args[] = {&oa};
      {
        ProfScope ps(kProfPanel, a.stream);
        e = cudaLaunchCooperativeKernel((const void*)k_outer_mixed, dim3((unsigned)(nw + 1)),
                                        dim3(kThreadsOuter), args, kOuterDynSmem, a.stream);
      }
      if (e != cudaSuccess) return e;
      epoch += (unsigned)((NBp + kPanel - 1) / kPanel);
    }
    const int64_t r0 = p + NBp;
    if (r0 < n) {
      const int64_t m = n - r0;
      const double fl = (double)m * (double)m * (double)NBp;  // lower half of 2 m^2 NB
      if (use_tc && NBp % kb_tc == 0) {
        ProfScope ps(kProfUpdateTc, a.stream, fl, 8.0 * (double)m * (double)m / 2.0);
        e = outer_update_tc(split, L.A32, L.ld32, n, r0, NBp, L.Wop, L.Lop, NB, false, L.err, a.stream);
        if (e != cudaSuccess) return e;
      } else {
        F32Args u;
        u.C = L.A32;
        u.ldc = L.ld32;
        u.row0 = r0;
        u.n = n;
        u.col0 = r0;
        u.col1 = n;
        u.Aop = L.Wk;
        u.Bop = L.Lk;
        u.ldk = NB;
        u.kk = NBp;
        const int64_t T = (m + kT - 1) / kT;
        u.tiles_r = T;
        ProfScope ps(kProfUpdateF32, a.stream, fl, 8.0 * (double)m * (double)m / 2.0);
        k_f32_update<true><<<(unsigned)(T * (T + 1) / 2), 256, 0, a.stream>>>(u);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
    }
  }
  if (a.pivots_user) {
    e = cudaMemcpyAsync(a.pivots_user, L.piv, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                        a.stream);
    if (e != cudaSuccess) return e;
  }
  if (a.factor_out) {
    ProfScope ps(kProfOther, a.stream);
    k_export<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        L.A32, L.ld32, L.piv, static_cast<double*>(a.factor_out), a.ld, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dpp
