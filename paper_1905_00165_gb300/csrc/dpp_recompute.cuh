// FP64 recomputation of a borderline pivot of the mixed-precision sampler.
//
// The pivot of index g given the decisions on P = [0, g) is the conditional
// inclusion probability (Props. 3-5 of arXiv:1905.00165)
//     d_g = K_gg - k^T A^{-1} k,   A = K_P - 1_G,  k = K_{P,g},
// with G the rejected indices. For ANY vector x0, with r = k - A x0,
//     k^T A^{-1} k = k^T x0 + x0^T r + r^T A^{-1} r          (A symmetric)
// so d_g = d1 - r^T A^{-1} r with d1 = K_gg - k^T x0 - x0^T r. We take
//   x0 = L_P^{-T} l,  l = row g of the mixed L   (then x0 ~ A^{-1} k, because
//       L[g,P] D_P L_P^T = K[g,P] in the factorization),
//   r  = k - A x0 in FP64 from the original K,
//   e  = r^T M^{-1} r = sum_c v_c^2 / d_c,  v = L_P^{-1} r  (M = L D L^T ~ A),
// and return d2 = d1 - e. The error of d2 is second order in the mixed
// factorization's backward error; the residual and the dot products are FP64.
//
// Execution: inside the cooperative panel launch. Warp 0 of CTA 0 (the
// leader) posts a request; the worker CTAs 1..G-1 own the 32-row blocks of
// P round-robin and serve it in three steps:
//   R1  x0 = L_P^{-T} l, a wavefront over the blocks from the last one down;
//   R2  r = k - A x0 for the owner's row blocks (FP64, symmetric K read from
//       its lower triangle), with the partial dots k.x0 and x0.r;
//   R3  v = L_P^{-1} r, a wavefront from the first block up, e = sum v^2 / d.
// A wavefront step publishes each value together with the request id in one
// 64-bit word, so a consumer's poll is also its load. The owner of a block
// accumulates the contributions of the blocks it depends on as they appear
// (each warp its share, one warp finishing), and applies the precomputed
// inverse of the block's unit lower diagonal block instead of a serial solve.
// Every wait is bounded; a timeout raises a shared abort flag that ends all
// other waits at once, and DPP_RES_TIMEOUT is reported. Control flow and
// barriers do not depend on an abort, so no CTA can be left waiting on one.
#pragma once

#include "dpp_device.cuh"
#include "dpp_internal.h"

namespace dpp {

// control words (unsigned[32] in the workspace)
enum { kCtlReq = 0, kCtlG = 1, kCtlAck = 2, kCtlDone = 3, kCtlCount = 4, kCtlAbort = 6 };

constexpr int kMaxCoopCtas = 4096;
constexpr unsigned kRcFull = 0xffffffffu;
constexpr int kRcThreads = 256;

struct RecomputeScratch {
  unsigned* ctrl = nullptr;
  unsigned long long* xw = nullptr;  // x0 words: (request id << 32) | FP32 bits
  unsigned long long* vw = nullptr;  // v words
  float* inv = nullptr;              // inverse of each 32 x 32 unit lower diagonal block
  double* r = nullptr;               // FP64 residual
  double* part = nullptr;            // 4 doubles per worker CTA
  int64_t nblk = 0;
};

struct RecomputeArgs {
  unsigned* ctrl;
  unsigned long long* xw;
  unsigned long long* vw;
  float* inv;
  double* r;
  double* part;
  const double* K;
  int64_t ldk;
  float* A;
  int64_t lda;
  const double* piv;
  const uint8_t* keep;
  int64_t n, q;
  int grid;
  dpp_result* res;
  unsigned long long wait_ns;  // limit of every bounded wait of the launch
};

inline bool recompute_carve(Workspace& ws, int64_t n, RecomputeScratch* s) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  s->nblk = (int64_t)(nn + 31) / 32;
  s->ctrl = static_cast<unsigned*>(ws.take(256));
  s->xw = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  s->vw = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  s->inv = static_cast<float*>(ws.take(sizeof(float) * 1024 * (size_t)s->nblk));
  s->r = static_cast<double*>(ws.take(sizeof(double) * nn));
  s->part = static_cast<double*>(ws.take(sizeof(double) * 4 * kMaxCoopCtas));
  return s->ctrl && s->xw && s->vw && s->inv && s->r && s->part;
}

// Request ids start at 256, so zeroed words are never taken for published ones.
inline cudaError_t recompute_reset(const RecomputeScratch& s, int64_t n, cudaStream_t st) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  cudaError_t e = cudaMemsetAsync(s.ctrl, 0, 256, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.xw, 0, sizeof(unsigned long long) * nn, st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(s.vw, 0, sizeof(unsigned long long) * nn, st);
}

inline RecomputeArgs recompute_args(const RecomputeScratch& s, const double* K, int64_t ldk,
                                    float* A, int64_t lda, const double* piv, const uint8_t* keep,
                                    int64_t n, int64_t q, dpp_result* res) {
  RecomputeArgs a;
  a.ctrl = s.ctrl;
  a.xw = s.xw;
  a.vw = s.vw;
  a.inv = s.inv;
  a.r = s.r;
  a.part = s.part;
  a.K = K;
  a.ldk = ldk;
  a.A = A;
  a.lda = lda;
  a.piv = piv;
  a.keep = keep;
  a.n = n;
  a.q = q;
  a.grid = 1;
  a.res = res;
  a.wait_ns = (unsigned long long)g_tuning.wait_ns;
  return a;
}

// ---------------------------------------------------------------------------
// words and bounded waits
// ---------------------------------------------------------------------------
__device__ inline unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ inline void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ inline unsigned long long make_word(unsigned id, float v) {
  return ((unsigned long long)id << 32) | (unsigned long long)__float_as_uint(v);
}

__device__ inline bool word_has(unsigned long long w, unsigned id) {
  return (unsigned)(w >> 32) == id;
}

// Raise the abort flag on timeout; true if the caller must give up.
__device__ inline bool rc_give_up(const RecomputeArgs& a, unsigned long long t0) {
  if (ld_acquire(&a.ctrl[kCtlAbort]) != 0) return true;
  if (global_ns() - t0 > a.wait_ns) {
    atomicExch(&a.ctrl[kCtlAbort], 1u);
    flag_status(a.res, DPP_RES_TIMEOUT);
    return true;
  }
  return false;
}

// Single-thread bounded wait for *flag >= target (abort-aware). The control
// words are polled by every CTA of the launch, so the poll backs off to about
// a microsecond and the abort flag is read only every eighth time, to keep
// the L2 line that holds them from becoming a hot spot.
__device__ inline bool rc_wait_geq(const RecomputeArgs& a, const unsigned* flag, unsigned target) {
  if (ld_acquire(flag) >= target) return true;
  const unsigned long long t0 = global_ns();
  unsigned sleep = 64;
  for (unsigned it = 1;; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if ((it & 7) == 0 && rc_give_up(a, t0)) return false;
    __nanosleep(sleep);
    if (sleep < 1024) sleep <<= 1;
  }
}

// Whole warp: lanes < nvalid wait for word w[lane] to carry `id` and return
// its value (0 for the other lanes). False on abort or timeout.
__device__ inline bool warp_wait_words(const RecomputeArgs& a, const unsigned long long* w,
                                       int nvalid, unsigned id, float* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long v = 0;
  bool mine = lane >= nvalid;
  if (!mine) {
    v = ld_relaxed_u64(w + lane);
    mine = word_has(v, id);
  }
  if (!__all_sync(kRcFull, mine)) {
    // a short pause between polls: every warp of every worker may be waiting
    // here, and unthrottled polling would load the L2 that the residual's
    // streaming reads of K depend on
    const unsigned long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
      __nanosleep(64);
      if (!mine) {
        v = ld_relaxed_u64(w + lane);
        mine = word_has(v, id);
      }
      if (__all_sync(kRcFull, mine)) break;
      const bool bad = (lane == 0 && (it & 7) == 0) ? rc_give_up(a, t0) : false;
      if (__shfl_sync(kRcFull, bad, 0)) {
        *out = 0.f;
        return false;
      }
    }
  }
  *out = (lane < nvalid) ? __uint_as_float((unsigned)v) : 0.f;
  return true;
}

// One thread: the value of word *p once it carries `id` (slow path only when
// the fast check failed).
__device__ inline float word_value_slow(const RecomputeArgs& a, const unsigned long long* p,
                                        unsigned id, bool* live) {
  const unsigned long long t0 = global_ns();
  while (true) {
    const unsigned long long v = ld_relaxed_u64(p);
    if (word_has(v, id)) return __uint_as_float((unsigned)v);
    if (rc_give_up(a, t0)) {
      *live = false;
      return 0.f;
    }
  }
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kRcFull, v, o);
  return v;
}

// Lane c receives sum over the lanes of v[c] (31 shuffles).
__device__ __forceinline__ float transpose_reduce(float (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = up ? v[k] : v[k + h];
      const float keep = up ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(kRcFull, send, h);
    }
  }
  return v[0];
}

// Hand-off of per-warp partial sums of one owned block to warp 0, through a
// double buffer. A warp publishes block i's partial only after warp 0 has
// consumed block i-2 (the buffer's previous user), and warp 0 finishes block
// i only after every warp published it; so no warp runs more than one block
// ahead. Waits are bounded and end early on abort.
struct Handoff {
  float part[2][8][32];
  int ready[8];  // per warp: blocks published
  int cons;      // blocks consumed by warp 0
};

__device__ __forceinline__ bool smem_wait_geq(const RecomputeArgs& a, const volatile int* p,
                                              int target) {
  if (*p >= target) return true;
  const unsigned long long t0 = global_ns();
  while (*p < target) {
    if (rc_give_up(a, t0)) return false;
  }
  return true;
}

// Warp wp != 0: publish its partial (lane-indexed) of owned block i.
__device__ __forceinline__ void handoff_put(const RecomputeArgs& a, Handoff& h, int i, int wp,
                                            float v, bool* live) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  if (lane == 0 && *live) ok = smem_wait_geq(a, &h.cons, i - 1);
  if (!__shfl_sync(kRcFull, ok, 0)) *live = false;
  h.part[i & 1][wp][lane] = v;
  __syncwarp();
  __threadfence_block();
  if (lane == 0) *(volatile int*)&h.ready[wp] = i + 1;
}

// Warp 0: the sum of every warp's partial of owned block i (its own is v).
__device__ __forceinline__ float handoff_take(const RecomputeArgs& a, Handoff& h, int i, float v,
                                              bool* live) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  if (lane >= 1 && lane < 8 && *live) ok = smem_wait_geq(a, &h.ready[lane], i + 1);
  if (!__all_sync(kRcFull, ok)) *live = false;
  __threadfence_block();
  float sum = v;
#pragma unroll
  for (int k = 1; k < 8; ++k) sum += ((volatile float*)h.part[i & 1][k])[lane];
  __syncwarp();
  if (lane == 0) *(volatile int*)&h.cons = i + 1;
  return sum;
}

// Warp 0: the diagonal block of block t (nr rows) into sD and, in z, column
// `lane` of its unit lower inverse; the inverse is also stored row-major.
__device__ __forceinline__ void diag_inverse(const RecomputeArgs& a, int64_t t, int nr,
                                             float (*sD)[33], float (&z)[32]) {
  const int lane = threadIdx.x & 31;
  const float* A = a.A;
  const int64_t r0 = 32 * t;
#pragma unroll
  for (int k = 0; k < 32; ++k)
    sD[lane][k] = (lane < nr && k < lane) ? __ldcg(&A[(r0 + lane) + (r0 + k) * a.lda]) : 0.f;
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < i; ++k) s = fmaf(sD[i][k], z[k], s);
    z[i] = (i == lane) ? 1.f : (i < lane ? 0.f : -s);
  }
  float* dst = a.inv + (size_t)t * 1024;
#pragma unroll
  for (int i = 0; i < 32; ++i) dst[i * 32 + lane] = z[i];
  __syncwarp();
}

// Lane i receives sum over the lanes of v[i] (FP64 version).
__device__ __forceinline__ double transpose_reduce_d(double (&v)[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool up = (lane & h) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const double send = up ? v[k] : v[k + h];
      const double keep = up ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(kRcFull, send, h);
    }
  }
  return v[0];
}

// x0_c for the calling lane (word checked; slow path only if not yet ready).
__device__ __forceinline__ float x0_at(const RecomputeArgs& a, int64_t c, unsigned id, bool* live) {
  const unsigned long long w = ld_relaxed_u64(a.xw + c);
  if (word_has(w, id)) return __uint_as_float((unsigned)w);
  return word_value_slow(a, a.xw + c, id, live);
}

// R2 for the owner's row block t: r_i = k_i - (K_P x0)_i (+ x0_i if i was
// rejected), FP64, K read from its lower triangle only, in 32 x 32 tiles so
// that each warp has 32 independent loads in flight. Warp 0 lane i
// accumulates k_i x0_i and x0_i r_i into kx, xr.
//   part A: tiles of the row slab [32 t, 32 t + nr) x [0, 32 t + nr), lanes =
//           rows (K[i, c], c <= i; in the diagonal tile K[c, i] for c > i);
//   part B: tiles below the diagonal block, K[c, i] for c >= 32 t + 32, lanes
//           = c (coalesced down column i), reduced over the lanes at the end.
static __device__ __noinline__ void residual_block(const RecomputeArgs& a, unsigned id, int64_t g,
                                            int64_t t, int nr, double (*sRedA)[32],
                                            double (*sRedB)[32], bool* live, double* kx,
                                            double* xr) {
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const double* K = a.K;
  const int64_t ldk = a.ldk;
  const int64_t i = 32 * t + lane;
  const bool vi = lane < nr;
  {
    double acc = 0.0;
    for (int64_t m = wp; m <= t; m += 8) {
      const int64_t c0 = 32 * m;
      const int nc = (int)((g - c0) < 32 ? (g - c0) : 32);
      // x0 widened once per lane: the loop below shuffles doubles instead of
      // converting every broadcast value
      const double xl = lane < nc ? (double)x0_at(a, c0 + lane, id, live) : 0.0;
      double kv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const int64_t c = c0 + k;
        kv[k] = (vi && k < nc) ? (c <= i ? K[i + c * ldk] : K[c + i * ldk]) : 0.0;
      }
#pragma unroll
      for (int k = 0; k < 32; ++k) acc = fma(kv[k], __shfl_sync(kRcFull, xl, k), acc);
    }
    sRedA[wp][lane] = acc;
  }
  {
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    const int64_t cb = 32 * t + 32;
    for (int64_t c0 = cb + 32 * wp; c0 < g; c0 += 256) {
      const int64_t c = c0 + lane;
      const bool vc = c < g;
      const double xc = vc ? (double)x0_at(a, c, id, live) : 0.0;
      double kv[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) kv[k] = (vc && k < nr) ? K[c + (32 * t + k) * ldk] : 0.0;
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[k] = fma(kv[k], xc, acc[k]);
    }
    sRedB[wp][lane] = transpose_reduce_d(acc, lane);
  }
  __syncthreads();
  if (wp == 0 && vi) {
    double tot = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += sRedA[k][lane];
#pragma unroll
    for (int k = 0; k < 8; ++k) tot += sRedB[k][lane];
    const double xi = (double)x0_at(a, i, id, live);
    const double ki = K[g + i * ldk];  // K[i, g] from the lower triangle
    double ri = ki - tot;
    if (a.keep[i] == 0) ri += xi;  // (K_P - 1_G) x0 has -x0_i on rejected rows
    a.r[i] = ri;
    *kx = fma(ki, xi, *kx);
    *xr = fma(xi, ri, *xr);
  }
  __syncthreads();
}

// Worker side of one request (all threads of a worker CTA). Returns false on
// abort or timeout (the CTA must then leave the launch).
static __device__ __noinline__ bool recompute_serve(const RecomputeArgs& a, unsigned id) {
  __shared__ float sD[32][33];
  __shared__ Handoff hf;
  __shared__ double sRedA[8][32];
  __shared__ double sRedB[8][32];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t w = blockIdx.x - 1, nw = a.grid - 1;
  const int64_t g = (int64_t)ld_acquire(&a.ctrl[kCtlG]);
  const int64_t nblk = (g + 31) / 32;
  const float* A = a.A;
  const int64_t lda = a.lda;
  bool live = true;
  if (tid < 8) hf.ready[tid] = 0;
  if (tid == 0) hf.cons = 0;
  __syncthreads();

  // ---- R1: x0 = L_P^{-T} l, owned blocks t = w (mod nw), last one first ----
  {
    int i = 0;
    const int64_t tfirst = (w < nblk) ? w + ((nblk - 1 - w) / nw) * nw : -1;
    for (int64_t t = tfirst; t >= 0; t -= nw, ++i) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      float z[32];
      float ell = 0.f;
      if (wp == 0) {
        diag_inverse(a, t, nr, sD, z);
        ell = lane < nr ? __ldcg(&A[g + (32 * t + lane) * lda]) : 0.f;
      }
      // the last source s = t + 1 (warp 0, on the critical path) is loaded
      // transposed (lane = column) so that it needs no reduction over lanes
      float crit[32];
      int ncrit = 0;
      if (wp == 0 && t + 1 < nblk) {
        ncrit = (int)((g - 32 * (t + 1)) < 32 ? (g - 32 * (t + 1)) : 32);
        const float* cp = A + 32 * (t + 1) + (32 * t + lane) * lda;
#pragma unroll
        for (int k = 0; k < 32; ++k) crit[k] = (k < ncrit && lane < nr) ? __ldcg(cp + k) : 0.f;
      }
      // the other sources s = t + 1 + wp + 8 m (s > t + 1), latest-published last
      float acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0.f;
      int64_t s = t + 1 + wp;
      if (s < nblk) s += ((nblk - 1 - s) / 8) * 8;
      for (; s > t + 1 && s < nblk; s -= 8) {
        const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
        float tile[32];
        const float* tp = A + (32 * s + lane) + 32 * t * lda;
#pragma unroll
        for (int c = 0; c < 32; ++c) tile[c] = (lane < ns && c < nr) ? __ldcg(tp + c * lda) : 0.f;
        float xs = 0.f;
        live = __all_sync(kRcFull, live);  // warp-uniform before the collective wait
        if (live && !warp_wait_words(a, a.xw + 32 * s, ns, id, &xs)) live = false;
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fmaf(tile[c], xs, acc[c]);
      }
      float red = transpose_reduce(acc, lane);
      if (wp != 0) {
        handoff_put(a, hf, i, wp, red, &live);
      } else {
        if (ncrit > 0) {
          float xs = 0.f;
          live = __all_sync(kRcFull, live);  // warp-uniform before the collective wait
          if (live && !warp_wait_words(a, a.xw + 32 * (t + 1), ncrit, id, &xs)) live = false;
#pragma unroll
          for (int k = 0; k < 32; ++k) red = fmaf(crit[k], __shfl_sync(kRcFull, xs, k), red);
        }
        const float y = ell - handoff_take(a, hf, i, red, &live);
        // x_t[c] = sum_k inv[k][c] y_k (lane c holds column c of the inverse)
        float x = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) x = fmaf(z[k], __shfl_sync(kRcFull, y, k), x);
        if (lane < nr) st_relaxed_u64(a.xw + 32 * t + lane, make_word(id, x));
      }
    }
  }
  __syncthreads();
  if (tid < 8) hf.ready[tid] = 0;
  if (tid == 0) hf.cons = 0;
  __syncthreads();

  // ---- R2 + R3, owned blocks in increasing order: residual of block t, then
  // v_t = inv(L_tt) (r_t - sum_{s < t} L_ts v_s) ----
  double kx = 0.0, xr = 0.0, es = 0.0;
  {
    int i = 0;
    for (int64_t t = w; t < nblk; t += nw, ++i) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      residual_block(a, id, g, t, nr, sRedA, sRedB, &live, &kx, &xr);
      float invrow[32];
      if (wp == 0) {
        const float* src = a.inv + (size_t)t * 1024 + lane * 32;
#pragma unroll
        for (int c = 0; c < 32; ++c) invrow[c] = src[c];
      }
      // sources s = t - 1 - wp - 8 m, the latest-published (largest) last
      float acc = 0.f;
      const int64_t slast = t - 1 - wp;
      if (slast >= 0) {
        for (int64_t s = slast % 8; s <= slast; s += 8) {
          float tile[32];
          const float* tp = A + (32 * t + lane) + 32 * s * lda;
#pragma unroll
          for (int c = 0; c < 32; ++c) tile[c] = lane < nr ? __ldcg(tp + c * lda) : 0.f;
          float vs = 0.f;
          live = __all_sync(kRcFull, live);  // warp-uniform before the collective wait
          if (live && !warp_wait_words(a, a.vw + 32 * s, 32, id, &vs)) live = false;
#pragma unroll
          for (int c = 0; c < 32; ++c) acc = fmaf(tile[c], __shfl_sync(kRcFull, vs, c), acc);
        }
      }
      if (wp != 0) {
        handoff_put(a, hf, i, wp, acc, &live);
      } else {
        const float sum = handoff_take(a, hf, i, acc, &live);
        const double yd = (lane < nr ? a.r[32 * t + lane] : 0.0) - (double)sum;
        const float y = (float)yd;
        // v_i = sum_{c <= i} inv[i][c] y_c (lane i holds row i of the inverse)
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) v = fmaf(invrow[c], __shfl_sync(kRcFull, y, c), v);
        if (lane < nr) {
          st_relaxed_u64(a.vw + 32 * t + lane, make_word(id, v));
          es += (double)v * (double)v / a.piv[32 * t + lane];
        }
      }
    }
  }
  if (wp == 0) {
    kx = warp_sum(kx);
    xr = warp_sum(xr);
    es = warp_sum(es);
    if (lane == 0) {
      a.part[4 * w + 0] = kx;
      a.part[4 * w + 1] = xr;
      a.part[4 * w + 2] = es;
      __threadfence();
      // the last worker to finish acknowledges the request
      const unsigned done = atomicAdd(&a.ctrl[kCtlCount], 1u) + 1u;
      if (done == (unsigned)nw) {
        atomicExch(&a.ctrl[kCtlCount], 0u);
        __threadfence();
        st_release(&a.ctrl[kCtlAck], id);
      }
    }
  }
  __syncthreads();
  return live && ld_acquire(&a.ctrl[kCtlAbort]) == 0;
}

// Worker CTAs: serve requests until the leader reports the panel's decisions
// done. Returns false (and the CTA must exit) on timeout or abort.
__device__ inline bool recompute_follower(const RecomputeArgs& a, unsigned epoch, int* s_ok) {
  __shared__ unsigned s_cmd, s_id;
  unsigned served = 0;
  while (true) {
    if (threadIdx.x == 0) {
      unsigned cmd = 0, id = 0;
      const unsigned long long t0 = global_ns();
      unsigned sleep = 64;
      for (unsigned it = 1;; ++it) {
        if (ld_acquire(&a.ctrl[kCtlDone]) >= epoch) { cmd = 2; break; }
        const unsigned req = ld_acquire(&a.ctrl[kCtlReq]);
        if (req >= ((epoch << 8) | (served + 1u))) { cmd = 1; id = req; break; }
        if ((it & 7) == 0 && rc_give_up(a, t0)) { cmd = 0; break; }
        __nanosleep(sleep);
        if (sleep < 1024) sleep <<= 1;
      }
      __threadfence();
      s_cmd = cmd;
      s_id = id;
    }
    __syncthreads();
    const unsigned cmd = s_cmd, id = s_id;
    __syncthreads();
    if (cmd == 0) {
      *s_ok = 0;
      return false;
    }
    if (cmd == 2) {
      *s_ok = 1;
      return true;
    }
    if (!recompute_serve(a, id)) {
      *s_ok = 0;
      return false;
    }
    served = id & 0xffu;
  }
}

// Leader (all 32 lanes of warp 0 of CTA 0, inside the decision loop at local
// pivot j). blk holds the diagonal block: rows < j are final rows of L, row j
// carries l = L[g, q:g] in its first j entries. Returns the recomputed
// pivot in *pe and an error estimate in *est (lane-uniform).
__device__ inline bool recompute_leader(const RecomputeArgs& a, float (*blk)[kPanel + 1], int b,
                                        int64_t q, int j, unsigned epoch, int* seq, double* pe,
                                        double* est) {
  const int lane = threadIdx.x & 31;
  const int64_t g = q + j;
  for (int c = 0; c < j; ++c)
    if (lane > c && lane <= j) a.A[(q + lane) + (q + c) * a.lda] = blk[lane][c];
  __threadfence();
  __syncwarp();
  *seq += 1;
  const unsigned id = (epoch << 8) | (unsigned)(*seq);
  bool ok = true;
  if (a.grid < 2) ok = false;
  if (ok && lane == 0) {
    atomicExch(&a.ctrl[kCtlG], (unsigned)g);
    __threadfence();
    st_release(&a.ctrl[kCtlReq], id);
    ok = rc_wait_geq(a, &a.ctrl[kCtlAck], id);
  }
  ok = __shfl_sync(kRcFull, ok, 0);
  double kx = 0.0, xr = 0.0, e = 0.0;
  if (ok && lane == 0) {
    for (int w = 0; w < a.grid - 1; ++w) {
      kx += __ldcg(&a.part[4 * w + 0]);
      xr += __ldcg(&a.part[4 * w + 1]);
      e += __ldcg(&a.part[4 * w + 2]);
    }
  }
  const double kgg = a.K[g + g * a.ldk];
  double d2 = kgg - kx - xr - e;
  double er = fabs(e) * 1e-2 + 1e-12 * (1.0 + fabs(kgg) + fabs(kx));
  d2 = __shfl_sync(kRcFull, d2, 0);
  er = __shfl_sync(kRcFull, er, 0);
  if (ok) {
    *pe = d2;
    *est = er;
  }
  return ok;
}

__device__ inline void recompute_release_done(const RecomputeArgs& a, unsigned epoch) {
  st_release(&a.ctrl[kCtlDone], epoch);
}

}  // namespace dpp
