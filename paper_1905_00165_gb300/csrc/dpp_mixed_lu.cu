// Mixed-precision DPP sampler for a general (non-Hermitian) kernel: the LU
// form of Algorithm 1, blocked as in Algorithm 4.
//
// Factorization kept in an FP32 copy A32 of K (full square, column-major):
//   K_P - 1_G = L D U~,  U~ = D^{-1} U unit upper,  M = U~^T unit lower,
// stored as L strictly below the diagonal, the FP32 pivot on it and U~ (that
// is M^T) strictly above. With W = L D the Schur update of one block of
// columns is  A22 -= L21 U12 = W21 M21^T,  the same C -= W L^T contraction as
// the Hermitian path, over the whole square instead of one triangle.
//
// Arithmetic: as the Hermitian mixed path. A running diagonal
// kd_i = K_ii - sum_k w_ik m_ik in FP64 (double-float inside the decision
// loop) formed from the FP32 factor entries gives each pivot; a pivot whose
// uniform lies within
//   tau_j = c * 2^-22 * sqrt(j + 1) * (|K_jj| + s_j),  s_j = sum_k |w_jk m_jk|,
// of it is recomputed in FP64 from the original K (below) before its
// decision, so every decision is that of the exact chain (Theorem 1).
//
// FP64 recompute of pivot g (Props. 3-5): d_g = K_gg - b^T A^{-1} a with
// A = K_P - 1_G, a = K[P, g], b = K[g, P]^T. For any x0, y0, with
// r = a - A x0 and s = b - A^T y0,
//     b^T A^{-1} a = b^T x0 + y0^T r + s^T A^{-1} r.
// The mixed factors give x0 = M_P^{-T} m (m = row g of M, so x0 ~ A^{-1} a),
// y0 = L_P^{-T} l (l = row g of L), and the last term as
// sum_c (L_P^{-1} r)_c (M_P^{-1} s)_c / d_c, which is second order in the
// factorization's error; residuals and dot products are FP64. The two
// triangular sweeps of each side run as wavefronts over 32-index blocks on
// the worker CTAs, with the protocol and helpers of the Hermitian recompute.
//
// One cooperative launch per outer block [q, q + kb) of at most 256 columns,
// cut into 32-index chunks (32 rows and, for LU, the same 32 columns):
//   CTA 0       : decides each 32-wide panel with all eight warps and
//                 publishes it;
//   CTAs 1..nh  : helpers; own the outer block's later chunks (one each on a
//                 full grid). Before a panel is published they compute their
//                 chunks' left-looking products; after it, they solve them, and
//                 the owner of the next chunk forms the next diagonal block;
//   the rest    : workers; own the chunks beyond the outer block (left-looking
//                 products before the publish as one tall product, solves and
//                 the tensor-core operand splits after it).
// All CTAs from 1 on serve recompute requests while they wait for a panel.
// After each outer block one rank-kb update of the trailing square (LU) or
// triangle (the symmetric instantiation, used by the Hermitian sampler) runs
// on the tensor cores.
#include <cuda_bf16.h>
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"
#include "dpp_recompute.cuh"

namespace dpp {
namespace {

constexpr unsigned kLuFull = 0xffffffffu;
constexpr int kLuThreads = 256;
constexpr int kNB = kMaxOuterBlock;  // row length of the W / M operand buffers

// control words: kCtlChunk + j holds the epoch of the last panel that the
// outer block's chunk j (indices [q + 32 j, q + 32 j + 32)) was solved
// against; once it reaches the epoch of panel j - 1, the chunk's rows are
// final and the buffer Bbuf holds its diagonal block, ready for decisions.
enum { kCtlChunk = 16 };
constexpr int kMaxSlots = 16;  // precomputed chunks per CTA (shared memory)

// Recompute state of the LU form: the Hermitian set (x0 words, v1 words,
// inverses of the L blocks, residual r) plus the second side's.
struct LuRc {
  RecomputeArgs rc;
  unsigned long long* yw;   // y0 words
  unsigned long long* v2w;  // v2 words
  float* inv2;              // inverse of each 32 x 32 unit lower diagonal block of M
  double* s2;               // residual s = b - A^T y0
};

struct LuArgs {
  const double* K;
  int64_t ldk;
  float* A;
  int64_t lda, n, q;
  int kb;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double* piv;
  double* kd;
  double* s;
  float* Wk;  // row-major [n x kNB]: W = L D of the outer block's columns
  float* Mk;  // row-major [n x kNB]: M
  void* Wop[3];
  void* Mop[3];
  int split;
  dpp_result* res;
  unsigned epoch0;
  double tol;
  float tau0;
  float* Bbuf;  // [32 x 32] next diagonal block, row-major
  int nh;       // helper CTAs 1..nh (chunks of the outer block)
  int slots;    // precomputed-chunk slots in shared memory
  int withhold; // fault injection: CTA 0 never publishes a panel
  int no_rows;  // split pipeline: the CTAs beyond the helpers only serve recomputes
  LuRc lr;
};

// ---------------------------------------------------------------------------
// FP64 recompute, LU form
// ---------------------------------------------------------------------------
__device__ inline float word_at(const RecomputeArgs& a, const unsigned long long* words,
                                int64_t c, unsigned id, bool* live) {
  const unsigned long long w = ld_relaxed_u64(words + c);
  if (word_has(w, id)) return __uint_as_float((unsigned)w);
  return word_value_slow(a, words + c, id, live);
}

// F(i, c) is L(i, c) = A[i + c lda] (TRANS false) or M(i, c) = A[c + i lda]
// (TRANS true). Warp 0: column `lane` of the inverse of the unit lower block
// F_tt into z, and the inverse row-major into inv.
template <bool TRANS>
__device__ __forceinline__ void lu_diag_inverse(const RecomputeArgs& a, float* inv, int64_t t,
                                                int nr, float (*sD)[33], float (&z)[32]) {
  const int lane = threadIdx.x & 31;
  const float* A = a.A;
  const int64_t r0 = 32 * t;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float* src = TRANS ? &A[(r0 + k) + (r0 + lane) * a.lda] : &A[(r0 + lane) + (r0 + k) * a.lda];
    sD[lane][k] = (lane < nr && k < lane) ? __ldcg(src) : 0.f;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < i; ++k) s = fmaf(sD[i][k], z[k], s);
    z[i] = (i == lane) ? 1.f : (i < lane ? 0.f : -s);
  }
  float* dst = inv + (size_t)t * 1024;
#pragma unroll
  for (int i = 0; i < 32; ++i) dst[i * 32 + lane] = z[i];
  __syncwarp();
}

// Backward sweep, block t:  x_t = F_tt^{-T} (f_t - sum_{s > t} F_st^T x_s),
// f = row g of F; x published as words. Sources are split over the 8 warps
// (s = t + 1 + wp + 8 m); each loads its tiles in the coalesced orientation.
template <bool TRANS>
__device__ __forceinline__ void lu_r1_block(const RecomputeArgs& a, float* inv,
                                            unsigned long long* words, int64_t g, int64_t nblk,
                                            int64_t t, unsigned id, Handoff& hf, int seqh,
                                            float (*sD)[33], bool* live) {
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const float* A = a.A;
  const int64_t lda = a.lda;
  const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
  float z[32];
  float f = 0.f;
  if (wp == 0) {
    lu_diag_inverse<TRANS>(a, inv, t, nr, sD, z);
    const int64_t c = 32 * t + lane;
    if (lane < nr) f = __ldcg(TRANS ? &A[c + g * lda] : &A[g + c * lda]);
  }
  float red;
  if (TRANS) {
    // lane = column of block t: F(32 s + k, 32 t + lane) = A[(32 t + lane) + (32 s + k) lda]
    float acc = 0.f;
    for (int64_t s = t + 1 + wp + (t + 1 + wp < nblk ? ((nblk - 2 - t - wp) / 8) * 8 : 0);
         s > t && s < nblk; s -= 8) {  // latest-published source last
      const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
      const float* cp = A + (32 * t + lane) + 32 * s * lda;
      float v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = (k < ns && lane < nr) ? __ldcg(cp + k * lda) : 0.f;
      float xs = 0.f;
      *live = __all_sync(kLuFull, *live);  // warp-uniform before the collective wait
      if (*live && !warp_wait_words(a, words + 32 * s, ns, id, &xs)) *live = false;
#pragma unroll
      for (int k = 0; k < 32; ++k) acc = fmaf(v[k], __shfl_sync(kLuFull, xs, k), acc);
    }
    red = acc;
  } else {
    // lane = row of block s: F(32 s + lane, 32 t + c) = A[(32 s + lane) + (32 t + c) lda]
    float acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.f;
    for (int64_t s = t + 1 + wp + (t + 1 + wp < nblk ? ((nblk - 2 - t - wp) / 8) * 8 : 0);
         s > t && s < nblk; s -= 8) {  // latest-published source last
      const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
      const float* tp = A + (32 * s + lane) + 32 * t * lda;
      float tile[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) tile[c] = (lane < ns && c < nr) ? __ldcg(tp + c * lda) : 0.f;
      float xs = 0.f;
      *live = __all_sync(kLuFull, *live);  // warp-uniform before the collective wait
      if (*live && !warp_wait_words(a, words + 32 * s, ns, id, &xs)) *live = false;
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = fmaf(tile[c], xs, acc[c]);
    }
    red = transpose_reduce(acc, lane);
  }
  if (wp != 0) {
    handoff_put(a, hf, seqh, wp, red, live);
  } else {
    const float y = f - handoff_take(a, hf, seqh, red, live);
    float x = 0.f;
#pragma unroll
    for (int k = 0; k < 32; ++k) x = fmaf(z[k], __shfl_sync(kLuFull, y, k), x);
    if (lane < nr) st_relaxed_u64(words + 32 * t + lane, make_word(id, x));
  }
}

// Forward sweep, block t:  v_t = F_tt^{-1} (rhs_t - sum_{s < t} F_ts v_s).
// Returns v for lane i of warp 0 (0 elsewhere).
template <bool TRANS>
__device__ __forceinline__ float lu_r3_block(const RecomputeArgs& a, const float* inv,
                                             unsigned long long* words, const double* rhs,
                                             int64_t g, int64_t t, unsigned id, Handoff& hf,
                                             int seqh, bool* live) {
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const float* A = a.A;
  const int64_t lda = a.lda;
  const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
  float invrow[32];
  if (wp == 0) {
    const float* src = inv + (size_t)t * 1024 + lane * 32;
#pragma unroll
    for (int c = 0; c < 32; ++c) invrow[c] = src[c];
  }
  const int64_t slast = t - 1 - wp;
  float red;
  if (!TRANS) {
    // lane = row of block t: F(32 t + lane, 32 s + c) = A[(32 t + lane) + (32 s + c) lda]
    float acc = 0.f;
    if (slast >= 0) {
      for (int64_t s = slast % 8; s <= slast; s += 8) {
        const float* tp = A + (32 * t + lane) + 32 * s * lda;
        float tile[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) tile[c] = lane < nr ? __ldcg(tp + c * lda) : 0.f;
        float vs = 0.f;
        *live = __all_sync(kLuFull, *live);  // warp-uniform before the collective wait
        if (*live && !warp_wait_words(a, words + 32 * s, 32, id, &vs)) *live = false;
#pragma unroll
        for (int c = 0; c < 32; ++c) acc = fmaf(tile[c], __shfl_sync(kLuFull, vs, c), acc);
      }
    }
    red = acc;
  } else {
    // lane = column of block s: F(32 t + i, 32 s + lane) = A[(32 s + lane) + (32 t + i) lda]
    float acc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) acc[i] = 0.f;
    if (slast >= 0) {
      for (int64_t s = slast % 8; s <= slast; s += 8) {
        const float* tp = A + (32 * s + lane) + 32 * t * lda;
        float tile[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) tile[i] = i < nr ? __ldcg(tp + i * lda) : 0.f;
        float vs = 0.f;
        *live = __all_sync(kLuFull, *live);  // warp-uniform before the collective wait
        if (*live && !warp_wait_words(a, words + 32 * s, 32, id, &vs)) *live = false;
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = fmaf(tile[i], vs, acc[i]);
      }
    }
    red = transpose_reduce(acc, lane);
  }
  float v = 0.f;
  if (wp != 0) {
    handoff_put(a, hf, seqh, wp, red, live);
  } else {
    const float sum = handoff_take(a, hf, seqh, red, live);
    const double yd = (lane < nr ? rhs[32 * t + lane] : 0.0) - (double)sum;
    const float y = (float)yd;
#pragma unroll
    for (int c = 0; c < 32; ++c) v = fmaf(invrow[c], __shfl_sync(kLuFull, y, c), v);
    if (lane < nr) st_relaxed_u64(words + 32 * t + lane, make_word(id, v));
  }
  return v;
}

// Both residuals of the owner's block t (indices i in [32 t, 32 t + nr)):
//   r_i = K[i, g] - sum_{c < g} K[i, c] x0_c  (+ x0_i if i was rejected),
//   s_i = K[g, i] - sum_{c < g} K[c, i] y0_c  (+ y0_i if i was rejected),
// FP64 from the original K; warp 0 lane i accumulates K[g, i] x0_i into bx
// and y0_i r_i into yr. Part r reads rows of K (lane = i), part s columns
// (lane = c, reduced over the lanes at the end); both coalesced.
__device__ __noinline__ void lu_residual(const LuRc& L, unsigned id, int64_t g, int64_t t, int nr,
                                         double (*sRedA)[32], double (*sRedB)[32], bool* live,
                                         double* bx, double* yr) {
  const RecomputeArgs& a = L.rc;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const double* K = a.K;
  const int64_t ldk = a.ldk;
  const int64_t i = 32 * t + lane;
  const bool vi = lane < nr;
  const int64_t nblk = (g + 31) / 32;
  double accA = 0.0;
  double accB[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) accB[k] = 0.0;
  for (int64_t m = wp; m < nblk; m += 8) {
    const int64_t c0 = 32 * m;
    const int nc = (int)((g - c0) < 32 ? (g - c0) : 32);
    const bool vc = lane < nc;
    const float xl = vc ? word_at(a, a.xw, c0 + lane, id, live) : 0.f;
    const float yl = vc ? word_at(a, L.yw, c0 + lane, id, live) : 0.f;
    const double xd = (double)xl;  // widened once: double shuffles below
    double kv[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) kv[k] = (vi && k < nc) ? K[i + (c0 + k) * ldk] : 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k) accA = fma(kv[k], __shfl_sync(kLuFull, xd, k), accA);
#pragma unroll
    for (int k = 0; k < 32; ++k) kv[k] = (vc && k < nr) ? K[(c0 + lane) + (32 * t + k) * ldk] : 0.0;
#pragma unroll
    for (int k = 0; k < 32; ++k) accB[k] = fma(kv[k], (double)yl, accB[k]);
  }
  sRedA[wp][lane] = accA;
  sRedB[wp][lane] = transpose_reduce_d(accB, lane);
  __syncthreads();
  if (wp == 0 && vi) {
    double tr = 0.0, ts = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tr += sRedA[k][lane];
      ts += sRedB[k][lane];
    }
    const double xi = (double)word_at(a, a.xw, i, id, live);
    const double yi = (double)word_at(a, L.yw, i, id, live);
    const double kgi = K[g + i * ldk];
    double ri = K[i + g * ldk] - tr;
    double si = kgi - ts;
    if (a.keep[i] == 0) {  // (K_P - 1_G) has -1 on the rejected diagonal
      ri += xi;
      si += yi;
    }
    a.r[i] = ri;
    L.s2[i] = si;
    *bx = fma(kgi, xi, *bx);
    *yr = fma(yi, ri, *yr);
  }
  __syncthreads();
}

// Worker side of one request (all threads of a worker CTA).
__device__ __noinline__ bool lu_serve(const LuRc& L, unsigned id) {
  const RecomputeArgs& a = L.rc;
  __shared__ float sD[32][33];
  __shared__ Handoff hf;
  __shared__ double sRedA[8][32];
  __shared__ double sRedB[8][32];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t w = blockIdx.x - 1, nw = a.grid - 1;
  const int64_t g = (int64_t)ld_acquire(&a.ctrl[kCtlG]);
  const int64_t nblk = (g + 31) / 32;
  bool live = true;
  if (tid < 8) hf.ready[tid] = 0;
  if (tid == 0) hf.cons = 0;
  __syncthreads();
  {
    // x0 = M_P^{-T} m and y0 = L_P^{-T} l, owned blocks from the last one down
    int seqh = 0;
    const int64_t tfirst = (w < nblk) ? w + ((nblk - 1 - w) / nw) * nw : -1;
    for (int64_t t = tfirst; t >= 0; t -= nw) {
      lu_r1_block<true>(a, L.inv2, a.xw, g, nblk, t, id, hf, seqh++, sD, &live);
      lu_r1_block<false>(a, a.inv, L.yw, g, nblk, t, id, hf, seqh++, sD, &live);
    }
  }
  __syncthreads();
  if (tid < 8) hf.ready[tid] = 0;
  if (tid == 0) hf.cons = 0;
  __syncthreads();
  double bx = 0.0, yr = 0.0, es = 0.0;
  {
    // residuals, then v1 = L_P^{-1} r and v2 = M_P^{-1} s, owned blocks upwards
    int seqh = 0;
    for (int64_t t = w; t < nblk; t += nw) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      lu_residual(L, id, g, t, nr, sRedA, sRedB, &live, &bx, &yr);
      const float v1 = lu_r3_block<false>(a, a.inv, a.vw, a.r, g, t, id, hf, seqh++, &live);
      const float v2 = lu_r3_block<true>(a, L.inv2, L.v2w, L.s2, g, t, id, hf, seqh++, &live);
      if (wp == 0 && lane < nr) es += (double)v1 * (double)v2 / a.piv[32 * t + lane];
    }
  }
  if (wp == 0) {
    bx = warp_sum(bx);
    yr = warp_sum(yr);
    es = warp_sum(es);
    if (lane == 0) {
      a.part[4 * w + 0] = bx;
      a.part[4 * w + 1] = yr;
      a.part[4 * w + 2] = es;
      __threadfence();
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

// CTAs 1..G-1: serve requests until the panel with this epoch is published
// (SYM: the one-sided recompute of the Hermitian form).
template <bool SYM>
__device__ inline bool lu_follower(const LuRc& L, unsigned epoch, int* s_ok, unsigned max_sleep) {
  const RecomputeArgs& a = L.rc;
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
        if (sleep < max_sleep) sleep <<= 1;
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
    if (cmd == 1) {
      if (!(SYM ? recompute_serve(a, id) : lu_serve(L, id))) {
        *s_ok = 0;
        return false;
      }
      served = id & 0xffu;
      continue;
    }
    *s_ok = 1;
    return true;
  }
}

// Bounded wait of one thread with a short poll interval, for the waits on the
// chain of panels (only a few CTAs poll these words).
__device__ inline bool wait_geq_short(const RecomputeArgs& a, const unsigned* flag,
                                      unsigned target) {
  if (ld_acquire(flag) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if ((it & 15) == 0 && rc_give_up(a, t0)) return false;
    __nanosleep(64);
  }
}

// Leader (warp 0 of CTA 0): pivot g recomputed in FP64. The factor entries of
// indices < g must be in global memory. Lane-uniform results.
__device__ inline bool lu_leader(const LuRc& L, int64_t g, unsigned epoch, int* seq, double* pe,
                                 double* est) {
  const RecomputeArgs& a = L.rc;
  const int lane = threadIdx.x & 31;
  __threadfence();
  __syncwarp();
  *seq += 1;
  const unsigned id = (epoch << 8) | (unsigned)(*seq);
  bool ok = a.grid >= 2;
  if (ok && lane == 0) {
    atomicExch(&a.ctrl[kCtlG], (unsigned)g);
    __threadfence();
    st_release(&a.ctrl[kCtlReq], id);
    ok = rc_wait_geq(a, &a.ctrl[kCtlAck], id);
  }
  ok = __shfl_sync(kLuFull, ok, 0);
  double bx = 0.0, yr = 0.0, e = 0.0;
  if (ok && lane == 0) {
    for (int w = 0; w < a.grid - 1; ++w) {
      bx += __ldcg(&a.part[4 * w + 0]);
      yr += __ldcg(&a.part[4 * w + 1]);
      e += __ldcg(&a.part[4 * w + 2]);
    }
  }
  const double kgg = a.K[g + g * a.ldk];
  double d2 = kgg - bx - yr - e;
  double er = fabs(e) * 1e-2 + 1e-12 * (1.0 + fabs(kgg) + fabs(bx) + fabs(yr));
  d2 = __shfl_sync(kLuFull, d2, 0);
  er = __shfl_sync(kLuFull, er, 0);
  if (ok) {
    *pe = d2;
    *est = er;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Panel kernel
// ---------------------------------------------------------------------------
struct LuSmem {
  float d[32];
  float rd[32];
  float L11[32][33];  // L of the current panel's diagonal block (strictly lower)
  float M11[32][33];  // M of the same block (strictly lower)
  // from here on, ten contiguous 32 x 33 tiles; the worker CTAs use them as
  // one staging area (wstage) instead
  float X[32][33];    // chunk rows x panel columns (then W)
  float Z[32][33];    // chunk columns x panel rows, transposed (then M)
  float WA[32][33];   // staged 32-deep slices of the left-looking products
  float MB[32][33];
  float WB[32][33];
  float MA[32][33];
  float Bp[32][33];   // next diagonal block, left-looking part
  float E[3][32][33];
};
// Dynamic shared memory: LuSmem, then `slots` pairs of 32 x 33 tiles (X, Z)
// of chunks whose left-looking part was computed before their panel.
constexpr size_t kTileBytes = sizeof(float) * 32 * 33;
constexpr size_t kLuBaseSmem = (sizeof(LuSmem) + 15) & ~size_t(15);
inline size_t lu_dyn_smem(int slots) { return kLuBaseSmem + (size_t)slots * 2 * kTileBytes; }
extern __shared__ __align__(16) unsigned char g_lu_dyn[];
__device__ __forceinline__ LuSmem& lus() { return *reinterpret_cast<LuSmem*>(g_lu_dyn); }
__device__ __forceinline__ float (*slot_x(int i))[33] {
  return reinterpret_cast<float (*)[33]>(g_lu_dyn + kLuBaseSmem + (size_t)(2 * i) * kTileBytes);
}
__device__ __forceinline__ float (*slot_z(int i))[33] {
  return reinterpret_cast<float (*)[33]>(g_lu_dyn + kLuBaseSmem + (size_t)(2 * i + 1) * kTileBytes);
}
// Worker staging: 128 chunk rows of W and of M, 32 panel rows of M and of W.
__device__ __forceinline__ float (*wstage(int row))[33] { return &lus().X[0] + row; }

// Per-outer-block bookkeeping of CTA 0.
struct LuLog {
  double d[kMaxOuterBlock];
  unsigned char kp[kMaxOuterBlock];
  int border;
  float max_ratio;
  int rc_failed;
};
__shared__ LuLog g_lulog;
__shared__ int g_lu_ok;

__device__ inline float tf32_rna_lu(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Tensor-core operand pieces of v at element off of the split buffers.
__device__ inline void write_split(int split, void* const* ops, int64_t off, float v) {
  if (split == kSplitBf16x6) {
    // three BF16 pieces: v = b0 + b1 + b2 exactly (8 + 8 + 8 bits)
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    static_cast<__nv_bfloat16*>(ops[0])[off] = b0;
    static_cast<__nv_bfloat16*>(ops[1])[off] = b1;
    static_cast<__nv_bfloat16*>(ops[2])[off] = __float2bfloat16_rn(r2);
  } else {
    const float h = tf32_rna_lu(v);
    static_cast<float*>(ops[0])[off] = h;
    static_cast<float*>(ops[1])[off] = tf32_rna_lu(v - h);
  }
}

// The published panel [p, p + b): L11, M11 and the FP32 pivots into shared
// memory (identity beyond b).
template <bool SYM>
__device__ void load_panel(const LuArgs& a, int64_t p, int b) {
  LuSmem& S = lus();
  const float* A = a.A;
  for (int idx = threadIdx.x; idx < 1024; idx += kLuThreads) {
    const int r = idx & 31, c = idx >> 5;
    const float v = (r < b && c < b && r != c && (!SYM || r > c))
                        ? __ldcg(&A[(p + r) + (p + c) * a.lda]) : 0.f;
    S.L11[r][c] = r > c ? v : 0.f;  // L(p + r, p + c)
    if (SYM)
      S.M11[r][c] = r > c ? v : 0.f;  // M = L
    else
      S.M11[c][r] = c > r ? v : 0.f;  // M(p + c, p + r) = A[p + r, p + c]
  }
  if (threadIdx.x < 32) {
    const int c = threadIdx.x;
    const float d = c < b ? (float)__ldcg(&a.piv[p + c]) : 1.f;
    S.d[c] = d;
    S.rd[c] = c < b ? 1.f / d : 0.f;
  }
}

// Chunk [c0, c0 + 32) against panel [p, p + b), left-looking over the first
// D columns of the outer block (the panels already solved):
//   X[r][c] = A[c0 + r, p + c] - sum_{t < D} W[c0 + r, t] M[p + c, t]
//   Z[r][c] = A[p + c, c0 + r] - sum_{t < D} W[p + c, t] M[c0 + r, t]   (Z given)
// Thread (r = lane, c = warp + 8 j) owns 4 + 4 outputs; the W and M rows are
// staged 32 deep in shared memory.
template <bool SYM>
__device__ void chunk_left(const LuArgs& a, int64_t p, int b, int64_t c0, int D, float (*X)[33],
                           float (*Z)[33]) {
  LuSmem& S = lus();
  const int tid = threadIdx.x, r = tid & 31, cg = tid >> 5;
  const bool want_z = Z != nullptr;
  const float* A = a.A;
  const int64_t lda = a.lda;
  const int nc = (int)((a.n - c0) < 32 ? (a.n - c0) : 32);
  float x[4], z[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cg + 8 * j;
    if (SYM && c0 == p) {
      // diagonal block: only its lower triangle is stored
      const int hi = r > c ? r : c, lo = r > c ? c : r;
      x[j] = (r < nc && c < b) ? __ldcg(&A[(p + hi) + (p + lo) * lda]) : 0.f;
    } else {
      x[j] = (r < nc && c < b) ? __ldcg(&A[(c0 + r) + (p + c) * lda]) : 0.f;
    }
    // Z loaded with lanes along the panel rows (contiguous), read back below
    if (want_z) Z[c][r] = (c < nc && r < b) ? __ldcg(&A[(p + r) + (c0 + c) * lda]) : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 4; ++j) z[j] = want_z ? Z[r][cg + 8 * j] : 0.f;
  for (int t0 = 0; t0 < D; t0 += 32) {
    for (int idx = tid; idx < 1024; idx += kLuThreads) {
      const int rr = idx >> 5, tt = idx & 31;
      S.WA[rr][tt] = rr < nc ? __ldcg(&a.Wk[(c0 + rr) * kNB + t0 + tt]) : 0.f;
      S.MB[rr][tt] = rr < b ? __ldcg(&a.Mk[(p + rr) * kNB + t0 + tt]) : 0.f;
      if (want_z) {
        S.WB[rr][tt] = rr < b ? __ldcg(&a.Wk[(p + rr) * kNB + t0 + tt]) : 0.f;
        S.MA[rr][tt] = rr < nc ? __ldcg(&a.Mk[(c0 + rr) * kNB + t0 + tt]) : 0.f;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int tt = 0; tt < 32; ++tt) {
      const float wa = S.WA[r][tt];
      const float ma = want_z ? S.MA[r][tt] : 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = cg + 8 * j;
        x[j] = fmaf(-wa, S.MB[c][tt], x[j]);
        if (want_z) z[j] = fmaf(-ma, S.WB[c][tt], z[j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    X[r][cg + 8 * j] = x[j];
    if (want_z) Z[r][cg + 8 * j] = z[j];
  }
  __syncthreads();
}

// Both triangular solves of a left-looked chunk (X, Z) against the published
// panel, leaving W in X and M in Z; then its running-diagonal terms and the
// stores (L and M into A32, W and M rows into the operand buffers, and the
// tensor-core splits if `splits`).
template <bool SYM>
__device__ void chunk_solve(const LuArgs& a, int64_t p, int b, int64_t c0, float (*X)[33],
                            float (*Z)[33], bool splits) {
  LuSmem& S = lus();
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nc = (int)((a.n - c0) < 32 ? (a.n - c0) : 32);
  const int D = (int)(p - a.q);
  if (wp == 0) {
    // row c0 + lane:  W M11^T = X  (forward over the panel columns)
    float y[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) y[c] = X[lane][c];
#pragma unroll
    for (int c = 1; c < 32; ++c) {
#pragma unroll
      for (int k = 0; k < c; ++k) y[c] = fmaf(-y[k], S.M11[c][k], y[c]);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) X[lane][c] = y[c];
  } else if (!SYM && wp == 1) {
    // column c0 + lane:  L11 u = Z,  M = u / d
    float u[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) u[c] = Z[lane][c];
#pragma unroll
    for (int c = 1; c < 32; ++c) {
#pragma unroll
      for (int k = 0; k < c; ++k) u[c] = fmaf(-S.L11[c][k], u[k], u[c]);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) Z[lane][c] = u[c] * S.rd[c];
  }
  __syncthreads();
  if (SYM) {
    // M = L = W / d
    for (int idx = tid; idx < 1024; idx += kLuThreads) {
      const int c = idx & 31, r = idx >> 5;
      Z[r][c] = X[r][c] * S.rd[c];
    }
    __syncthreads();
  }
  if (wp == 0 && lane < nc) {
    f2 dsum = {0.f, 0.f};
    float ssum = 0.f;
    for (int c = 0; c < b; ++c) {
      const float w = X[lane][c], m = Z[lane][c];
      dsum = f2_add_prod(dsum, w, m);
      ssum += fabsf(w * m);
    }
    a.kd[c0 + lane] -= f2_to_double(dsum);
    a.s[c0 + lane] += (double)ssum;
  }
  float* A = a.A;
  const int64_t lda = a.lda;
  for (int idx = tid; idx < 1024; idx += kLuThreads) {
    {
      // L = W / d, lanes along the chunk rows
      const int r = idx & 31, c = idx >> 5;
      if (r < nc && c < b) A[(c0 + r) + (p + c) * lda] = X[r][c] * S.rd[c];
    }
    {
      // M^T above the diagonal and the operand rows, lanes along the panel
      const int c = idx & 31, r = idx >> 5;
      if (r < nc && c < b) {
        const float m = Z[r][c], w = X[r][c];
        if (!SYM) A[(p + c) + (c0 + r) * lda] = m;
        const int64_t off = (c0 + r) * kNB + D + c;
        a.Wk[off] = w;
        a.Mk[off] = m;
        if (splits) {
          write_split(a.split, a.Wop, off, w);
          write_split(a.split, a.Mop, off, m);
        }
      }
    }
  }
  __syncthreads();
}

// The next diagonal block from its left-looking part (S.Bp) and the chunk's
// just-solved W (in X) and M (in Z) against the current panel, into Bbuf.
__device__ void next_block(const LuArgs& a, float (*X)[33], float (*Z)[33], int b) {
  LuSmem& S = lus();
  const int tid = threadIdx.x, r = tid & 31, cg = tid >> 5;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cg + 8 * j;
    float v = S.Bp[r][c];
    for (int t = 0; t < b; ++t) v = fmaf(-X[r][t], Z[c][t], v);
    a.Bbuf[r * 32 + c] = v;
  }
  __syncthreads();
}

// Left-looking parts of the cnt chunks c_m = c_first + m c_stride (m < cnt)
// against panel [p, p + b) over the first D columns of the outer block, into
// slots 0..cnt-1 (same definitions as chunk_left). The chunks' rows form one
// tall operand: per 32-deep step the panel rows are staged once, then 128
// chunk rows at a time, and each thread accumulates a 4 x 4 block.
template <bool SYM>
__device__ void chunks_left(const LuArgs& a, int64_t p, int b, int D, int64_t c_first,
                            int64_t c_stride, int cnt) {
  const int tid = threadIdx.x;
  const float* A = a.A;
  const int64_t lda = a.lda, n = a.n;
  for (int m = 0; m < cnt; ++m) {
    const int64_t c0 = c_first + m * c_stride;
    const int nc = (int)((n - c0) < 32 ? (n - c0) : 32);
    float (*X)[33] = slot_x(m);
    float (*Z)[33] = slot_z(m);
    for (int idx = tid; idx < 1024; idx += kLuThreads) {
      const int lo = idx & 31, hi = idx >> 5;
      X[lo][hi] = (lo < nc && hi < b) ? __ldcg(&A[(c0 + lo) + (p + hi) * lda]) : 0.f;
      if (!SYM) Z[hi][lo] = (hi < nc && lo < b) ? __ldcg(&A[(p + lo) + (c0 + hi) * lda]) : 0.f;
    }
  }
  __syncthreads();
  float (*WA4)[33] = wstage(0);
  float (*MA4)[33] = wstage(128);
  float (*MB)[33] = wstage(256);
  float (*WB)[33] = wstage(288);
  const int ty = tid >> 3, tx = tid & 7;
  for (int t0 = 0; t0 < D; t0 += 32) {
    for (int idx = tid; idx < 1024; idx += kLuThreads) {
      const int rr = idx >> 5, tt = idx & 31;
      MB[rr][tt] = rr < b ? __ldcg(&a.Mk[(p + rr) * kNB + t0 + tt]) : 0.f;
      if (!SYM) WB[rr][tt] = rr < b ? __ldcg(&a.Wk[(p + rr) * kNB + t0 + tt]) : 0.f;
    }
    for (int m0 = 0; m0 < cnt; m0 += 4) {
      for (int idx = tid; idx < 4096; idx += kLuThreads) {
        const int rr = idx >> 5, tt = idx & 31;
        const int m = m0 + (rr >> 5);
        const int64_t row = c_first + m * c_stride + (rr & 31);
        const bool ok = m < cnt && row < n;
        WA4[rr][tt] = ok ? __ldcg(&a.Wk[row * kNB + t0 + tt]) : 0.f;
        if (!SYM) MA4[rr][tt] = ok ? __ldcg(&a.Mk[row * kNB + t0 + tt]) : 0.f;
      }
      __syncthreads();
      float ax[4][4], az[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) ax[i][j] = az[i][j] = 0.f;
#pragma unroll 4
      for (int tt = 0; tt < 32; ++tt) {
        float wa[4], mb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) wa[i] = WA4[4 * ty + i][tt];
#pragma unroll
        for (int j = 0; j < 4; ++j) mb[j] = MB[4 * tx + j][tt];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) ax[i][j] = fmaf(wa[i], mb[j], ax[i][j]);
        if (!SYM) {
          float ma[4], wb[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) ma[i] = MA4[4 * ty + i][tt];
#pragma unroll
          for (int j = 0; j < 4; ++j) wb[j] = WB[4 * tx + j][tt];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) az[i][j] = fmaf(ma[i], wb[j], az[i][j]);
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = 4 * ty + i, m = m0 + (rr >> 5), r = rr & 31;
        if (m < cnt) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            slot_x(m)[r][4 * tx + j] -= ax[i][j];
            if (!SYM) slot_z(m)[r][4 * tx + j] -= az[i][j];
          }
        }
      }
      __syncthreads();
    }
  }
}

// Solves and stores of the cnt left-looked chunks in slots 0..cnt-1 against
// the published panel (as chunk_solve, one warp per chunk side).
template <bool SYM>
__device__ void chunks_solve(const LuArgs& a, int64_t p, int b, int64_t c_first, int64_t c_stride,
                             int cnt) {
  LuSmem& S = lus();
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t n = a.n;
  const int D = (int)(p - a.q);
  const int ntask = SYM ? cnt : 2 * cnt;
  for (int task = wp; task < ntask; task += kLuThreads / 32) {
    const int m = SYM ? task : task >> 1;
    if (SYM || (task & 1) == 0) {
      float (*X)[33] = slot_x(m);
      float y[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) y[c] = X[lane][c];
#pragma unroll
      for (int c = 1; c < 32; ++c) {
#pragma unroll
        for (int k = 0; k < c; ++k) y[c] = fmaf(-y[k], S.M11[c][k], y[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) X[lane][c] = y[c];
      if (SYM) {
        float (*Z)[33] = slot_z(m);
#pragma unroll
        for (int c = 0; c < 32; ++c) Z[lane][c] = y[c] * S.rd[c];
      }
    } else {
      float (*Z)[33] = slot_z(m);
      float u[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) u[c] = Z[lane][c];
#pragma unroll
      for (int c = 1; c < 32; ++c) {
#pragma unroll
        for (int k = 0; k < c; ++k) u[c] = fmaf(-S.L11[c][k], u[k], u[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) Z[lane][c] = u[c] * S.rd[c];
    }
  }
  __syncthreads();
  // running diagonal: one thread per chunk row
  for (int e = tid; e < 32 * cnt; e += kLuThreads) {
    const int m = e >> 5, r = e & 31;
    const int64_t row = c_first + m * c_stride + r;
    if (row < n) {
      f2 dsum = {0.f, 0.f};
      float ssum = 0.f;
      for (int c = 0; c < b; ++c) {
        const float w = slot_x(m)[r][c], mm = slot_z(m)[r][c];
        dsum = f2_add_prod(dsum, w, mm);
        ssum += fabsf(w * mm);
      }
      a.kd[row] -= f2_to_double(dsum);
      a.s[row] += (double)ssum;
    }
  }
  float* A = a.A;
  const int64_t lda = a.lda;
  for (int m = 0; m < cnt; ++m) {
    const int64_t c0 = c_first + m * c_stride;
    const int nc = (int)((n - c0) < 32 ? (n - c0) : 32);
    float (*X)[33] = slot_x(m);
    float (*Z)[33] = slot_z(m);
    for (int idx = tid; idx < 1024; idx += kLuThreads) {
      {
        const int r = idx & 31, c = idx >> 5;
        if (r < nc && c < b) A[(c0 + r) + (p + c) * lda] = X[r][c] * S.rd[c];
      }
      {
        const int c = idx & 31, r = idx >> 5;
        if (r < nc && c < b) {
          const float mm = Z[r][c], w = X[r][c];
          if (!SYM) A[(p + c) + (c0 + r) * lda] = mm;
          const int64_t off = (c0 + r) * kNB + D + c;
          a.Wk[off] = w;
          a.Mk[off] = mm;
          write_split(a.split, a.Wop, off, w);
          write_split(a.split, a.Mop, off, mm);
        }
      }
    }
  }
  __syncthreads();
}

// Decisions of panel [p, p + b) on the block in S.X, by all 8 warps of CTA 0.
//
// Fast chain: warp w holds columns 4w..4w+3 of every row (lane = row) in
// registers, so the pivot row reaches every warp by shuffles inside the warp;
// row i's running pivot dd (double-float) and the other per-row state live in
// lane i of the warp that owns column i. Step J: the owner of column J
// decides on pivot J in FP32 (exact outside the borderline band, whose floor
// exceeds the rounding of u and of the pivot) and publishes the multipliers
// l_i = A[i][J] / d_J in shared memory (double-buffered); after one barrier
// every warp applies the rank-1 update to its columns. At the first pivot
// inside the band the chain stops, and warp 0 finishes the panel with the
// rolled shared-memory loop, recomputing every band pivot in FP64.
template <bool SYM>
__device__ __noinline__ void lu_decide(const LuArgs& a, int64_t p, int b, unsigned epoch) {
  LuSmem& S = lus();
  LuLog& lg = g_lulog;
  float (*X)[33] = S.X;
  __shared__ float s_l[2][32];
  __shared__ float s_rd[2], s_df[2];
  __shared__ int s_stop[2];
  __shared__ float s_ddh[32], s_ddl[32], s_si[32];
  __shared__ unsigned char s_kp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t i = p + lane;
  const bool vi = lane < b;
  float* A = a.A;
  const int64_t lda = a.lda;
  f2 dd = vi ? f2_from_double(__ldcg(&a.kd[i])) : make_f2(0.f, 0.f);
  float si = vi ? (float)__ldcg(&a.s[i]) : 0.f;
  const float kf = vi ? (float)a.K[i + i * a.ldk] : 0.f;
  const float sq = sqrtf((float)(i + 1));
  const double u = vi ? (a.uniforms ? a.uniforms[i] : philox_uniform(a.seed, a.inst, (uint64_t)i))
                      : 2.0;
  const float uf = (float)u;
  const float tau0 = a.tau0;
  bool mykeep = false;
  int stop = -1;
  float v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) v[j] = (vi && 4 * warp + j < b) ? X[lane][4 * warp + j] : 0.f;
  for (int J = 0; J < b; ++J) {
    const int buf = J & 1;
    if (warp == (J >> 2)) {
      const float ph = __shfl_sync(kLuFull, dd.hi, J);
      const float uj = __shfl_sync(kLuFull, uf, J);
      const float tau = tau0 * __shfl_sync(kLuFull, sq, J) *
                            (fabsf(__shfl_sync(kLuFull, kf, J)) + __shfl_sync(kLuFull, si, J)) +
                        0x1.0p-22f;
      const bool border = fabsf(uj - ph) <= tau;
      if (!border) {
        const bool kp = uj < ph;
        const float df = kp ? ph : ph - 1.0f;
        const float rd = 1.0f / df;
        if (lane == J) {
          if (!kp) dd = f2_add_f(dd, -1.0f);
          mykeep = kp;
        }
        const int jj = J & 3;
        const float colJ = jj == 0 ? v[0] : (jj == 1 ? v[1] : (jj == 2 ? v[2] : v[3]));
        s_l[buf][lane] = colJ * rd;
        if (lane == 0) {
          s_rd[buf] = rd;
          s_df[buf] = df;
        }
      }
      if (lane == 0) s_stop[buf] = border ? 1 : 0;
    }
    __syncthreads();
    if (s_stop[buf]) {
      stop = J;
      break;
    }
    const float l = s_l[buf][lane];
    const float rd = s_rd[buf], df = s_df[buf];
    const bool act = (lane > J) && vi;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * warp + j;
      const float pk = __shfl_sync(kLuFull, v[j], J);  // row J's entry in column c
      float x = v[j];
      if (act && c > J) x = fmaf(-l, pk, x);
      if (act && c == J) x = l;
      if (lane == J && c > J) x = pk * rd;  // M^T entries of row J
      if (lane == J && c == J) x = df;
      v[j] = x;
      if (lane == c && act) {  // row c's running pivot
        dd = f2_sub_prod(dd, l, pk);
        si += fabsf(l * pk);
      }
    }
  }
  // hand the block and the per-row state to warp 0
#pragma unroll
  for (int j = 0; j < 4; ++j) X[lane][4 * warp + j] = v[j];
  if ((lane >> 2) == warp) {
    s_ddh[lane] = dd.hi;
    s_ddl[lane] = dd.lo;
    s_si[lane] = si;
    s_kp[lane] = mykeep ? 1 : 0;
  }
  __syncthreads();
  if (warp != 0) return;
  dd = make_f2(s_ddh[lane], s_ddl[lane]);
  si = s_si[lane];
  mykeep = s_kp[lane] != 0;
  if (stop >= 0) {
    // the pivots decided so far, out to global memory for the recomputes
    if (lane < stop) {
      a.piv[i] = f2_to_double(dd);
      a.keep[i] = mykeep ? 1 : 0;
    }
    int seq = 0;
    for (int J = stop; J < b; ++J) {
      const double ph =
          (double)__shfl_sync(kLuFull, dd.hi, J) + (double)__shfl_sync(kLuFull, dd.lo, J);
      const double uj = __shfl_sync(kLuFull, u, J);
      const float tau = a.tau0 * __shfl_sync(kLuFull, sq, J) *
                            (fabsf(__shfl_sync(kLuFull, kf, J)) + __shfl_sync(kLuFull, si, J)) +
                        0x1.0p-22f;
      double pe = ph;
      if (fabs(uj - ph) <= (double)tau) {
        double est = 0.0;
        bool ok;
        if (SYM) {
          // the Hermitian recompute writes the block's rows itself
          ok = recompute_leader(a.lr.rc, X, b, p, J, epoch, &seq, &pe, &est);
        } else {
          // the factor entries of [p, p + J] so far, out to global memory
          if (lane <= J) {
            for (int c = 0; c <= J; ++c) A[(p + lane) + (p + c) * lda] = X[lane][c];
          }
          ok = lu_leader(a.lr, p + J, epoch, &seq, &pe, &est);
        }
        if (lane == 0) {
          lg.border += 1;
          const float ratio = (float)(fabs(pe - ph) / (double)tau);
          if (ratio > lg.max_ratio) lg.max_ratio = ratio;
          if (!ok || est > fabs(uj - pe)) lg.rc_failed = 1;
        }
        if (!ok) pe = ph;
      }
      const bool kp = uj < pe;
      const double d = kp ? pe : pe - 1.0;
      if (lane == J) {
        dd = f2_from_double(d);
        mykeep = kp;
        a.piv[p + J] = d;
        a.keep[p + J] = kp ? 1 : 0;
      }
      const float df = (float)d;
      const float rdf = 1.f / df;
      if (lane > J && vi) {
        const float l = X[lane][J] * rdf;
        for (int c = J + 1; c < b; ++c) X[lane][c] = fmaf(-l, X[J][c], X[lane][c]);
        const float uji = X[J][lane];  // U(p + J, p + lane), not yet scaled
        dd = f2_sub_prod(dd, l, uji);
        si += fabsf(l * uji);
        X[lane][J] = l;
      }
      __syncwarp();
      if (lane == J) {
        for (int c = J + 1; c < b; ++c) X[J][c] *= rdf;
        X[J][J] = df;
      }
      __syncwarp();
    }
  }
  if (vi) {
    const double d = f2_to_double(dd);
    a.piv[i] = d;
    a.keep[i] = mykeep ? 1 : 0;
    lg.d[p - a.q + lane] = d;
    lg.kp[p - a.q + lane] = mykeep ? 1 : 0;
    const int cend = SYM ? lane + 1 : b;
    for (int c = 0; c < cend; ++c) A[i + (p + c) * lda] = X[lane][c];
  }
  __syncwarp();
}

__device__ __forceinline__ int chunk_owner(int j, int nh) { return 1 + (j - 1) % nh; }

template <bool SYM>
__global__ void __launch_bounds__(kLuThreads, 1) k_lu_outer(LuArgs a) {
  LuSmem& S = lus();
  int& s_ok = g_lu_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = (a.kb + 31) / 32;
  const int64_t q = a.q, qe = q + a.kb;
  const RecomputeArgs& rc = a.lr.rc;
  const int nh = a.nh;

  if (blockIdx.x == 0) {
    // ---- decisions, panel by panel ----
    LuLog& lg = g_lulog;
    if (tid == 0) {
      lg.border = 0;
      lg.max_ratio = 0.f;
      lg.rc_failed = 0;
    }
    __syncthreads();
    bool alive = true;
    for (int k = 0; k < np; ++k) {
      const int64_t p = q + 32 * k;
      const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
      const unsigned epoch = a.epoch0 + (unsigned)k;
      if (k == 0) {
        chunk_left<SYM>(a, p, b, p, 0, S.X, nullptr);
      } else {
        // the chunk's owner has solved it against panel k - 1 and formed the block
        if (tid == 0) s_ok = wait_geq_short(rc, &rc.ctrl[kCtlChunk + k], epoch - 1) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
          alive = false;
          break;
        }
        for (int idx = tid; idx < 1024; idx += kLuThreads) S.X[idx >> 5][idx & 31] = __ldcg(&a.Bbuf[idx]);
        __syncthreads();
      }
      lu_decide<SYM>(a, p, b, epoch);
      __syncthreads();
      if (tid == 0 && !a.withhold) {
        __threadfence();
        st_release(&rc.ctrl[kCtlDone], epoch);
      }
    }
    __syncthreads();
    // likelihood and bookkeeping of the block (FP64)
    double lp = 0.0;
    int kept = 0, oor = 0, bad = 0;
    for (int i = tid; i < a.kb; i += kLuThreads) {
      const double d = lg.d[i];
      const double pre = lg.kp[i] ? d : d + 1.0;
      lp += log(fabs(d));
      kept += lg.kp[i];
      oor += (pre < -a.tol || pre > 1.0 + a.tol) ? 1 : 0;
      bad |= isfinite(d) ? 0 : 1;
    }
    lp = warp_sum(lp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kept += __shfl_xor_sync(kLuFull, kept, o);
      oor += __shfl_xor_sync(kLuFull, oor, o);
      bad |= __shfl_xor_sync(kLuFull, bad, o);
    }
    __shared__ double s_lp[kLuThreads / 32];
    __shared__ int s_cnt[3][kLuThreads / 32];
    if (lane == 0) {
      s_lp[warp] = lp;
      s_cnt[0][warp] = kept;
      s_cnt[1][warp] = oor;
      s_cnt[2][warp] = bad;
    }
    __syncthreads();
    if (tid == 0 && alive) {
      double Ls = 0.0;
      int Kc = 0, O = 0, B = 0;
      for (int w = 0; w < kLuThreads / 32; ++w) {
        Ls += s_lp[w];
        Kc += s_cnt[0][w];
        O += s_cnt[1][w];
        B |= s_cnt[2][w];
      }
      dpp_result* r = a.res;
      r->logp += Ls;
      if (Kc) atomicAdd(&r->n_kept, Kc);
      if (O) {
        atomicAdd(&r->n_out_of_range, O);
        atomicOr(&r->status, DPP_RES_INADMISSIBLE);
      }
      if (B) atomicOr(&r->status, DPP_RES_NONFINITE);
      if (lg.border) {
        atomicAdd(&r->n_borderline, lg.border);
        if ((double)lg.max_ratio > r->max_err_ratio) r->max_err_ratio = (double)lg.max_ratio;
      }
      if (lg.rc_failed) atomicOr(&r->status, DPP_RES_RECOMPUTE);
    }
    return;
  }

  if (blockIdx.x <= nh) {
    // ---- helper h: the outer block's chunks j with owner h, in order ----
    const int h = blockIdx.x;
    for (int k = 0; k < np; ++k) {
      const int64_t p = q + 32 * k;
      const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
      const unsigned epoch = a.epoch0 + (unsigned)k;
      const int D = 32 * k;
      if (k > 0) {
        // the panel's own rows are final through panel k - 1
        if (tid == 0) s_ok = wait_geq_short(rc, &rc.ctrl[kCtlChunk + k], epoch - 1) ? 1 : 0;
        __syncthreads();
        if (!s_ok) return;
      }
      // before the panel is published: the left-looking parts
      int ns = 0;
      for (int j = k + 1; j < np; ++j) {
        if (chunk_owner(j, nh) != h) continue;
        chunk_left<SYM>(a, p, b, q + 32 * j, D, slot_x(ns), SYM ? nullptr : slot_z(ns));
        if (j == k + 1) {
          const int bj = (int)((qe - (q + 32 * j)) < 32 ? (qe - (q + 32 * j)) : 32);
          chunk_left<SYM>(a, q + 32 * j, bj, q + 32 * j, D, S.Bp, nullptr);
        }
        ++ns;
      }
      if (!lu_follower<SYM>(a.lr, epoch, &s_ok, 128)) return;
      load_panel<SYM>(a, p, b);
      __syncthreads();
      ns = 0;
      for (int j = k + 1; j < np; ++j) {
        if (chunk_owner(j, nh) != h) continue;
        chunk_solve<SYM>(a, p, b, q + 32 * j, slot_x(ns), slot_z(ns), false);
        if (j == k + 1) next_block(a, slot_x(ns), slot_z(ns), b);
        if (tid == 0) {
          __threadfence();
          st_release(&rc.ctrl[kCtlChunk + j], epoch);
        }
        ++ns;
      }
      __syncthreads();
    }
    return;
  }

  if (a.no_rows) {
    // split pipeline: the rows below are k_below's; serve each panel's
    // recompute requests until the panel is published
    for (int k = 0; k < np; ++k)
      if (!lu_follower<SYM>(a.lr, a.epoch0 + (unsigned)k, &s_ok, 1024)) return;
    return;
  }
  // ---- workers: chunks beyond the outer block ----
  const int64_t nwk = (int64_t)gridDim.x - nh - 1, w = (int64_t)blockIdx.x - nh - 1;
  const int64_t c_first = qe + 32 * w, c_stride = 32 * nwk;
  const int total = c_first < a.n ? (int)((a.n - 1 - c_first) / c_stride + 1) : 0;
  const int first = total < a.slots ? total : a.slots;
  for (int k = 0; k < np; ++k) {
    const int64_t p = q + 32 * k;
    const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
    const unsigned epoch = a.epoch0 + (unsigned)k;
    const int D = 32 * k;
    if (k > 0) {
      if (tid == 0) s_ok = rc_wait_geq(rc, &rc.ctrl[kCtlChunk + k], epoch - 1) ? 1 : 0;
      __syncthreads();
      if (!s_ok) return;
    }
    chunks_left<SYM>(a, p, b, D, c_first, c_stride, first);
    if (!lu_follower<SYM>(a.lr, epoch, &s_ok, 1024)) return;
    load_panel<SYM>(a, p, b);
    __syncthreads();
    chunks_solve<SYM>(a, p, b, c_first, c_stride, first);
    for (int m0 = first; m0 < total; m0 += a.slots) {
      const int cnt = (total - m0) < a.slots ? (total - m0) : a.slots;
      chunks_left<SYM>(a, p, b, D, c_first + m0 * c_stride, c_stride, cnt);
      chunks_solve<SYM>(a, p, b, c_first + m0 * c_stride, c_stride, cnt);
    }
  }
}

// Split pipeline (DPP_TUNE_PANEL_PIPELINE 3): the panel launch holds only CTA 0
// and the helpers, which factor the outer block's own rows with the decisions;
// afterwards this kernel, on a wide grid, brings every index below the outer
// block through its panels. A CTA takes kBR = 32 indices i and keeps, in shared
// memory, their row segments X[i][c] = A[i, q + c] and (LU) their column
// segments Z[i][c] = A[q + c, i], c < kb, and runs the outer block
// right-looking, panel by panel (p = q + 32 k):
//   solve   W[i, p + c] = X[i][p + c] - sum_{c' < c} W[i, p + c'] M(p + c, p + c')
//           (LU) U[i, p + c] = Z[i][p + c] - sum_{c' < c} L(p + c, p + c') U[i, p + c'],
//           M[i, p + c] = U[i, p + c] / d_{p + c}   (Hermitian: M = L = W / d)
//   update  X[i][j] -= sum_c W[i, p + c] M(q + j, p + c),
//           (LU) Z[i][j] -= sum_c M[i, p + c] W(q + j, p + c),   j beyond the panel,
// with the outer block's own W and M rows (written by the helpers). The sums
// are those of the left-looking worker steps, accumulated panel by panel. At
// the end it stores L (and M^T), the W and M operand rows with their
// tensor-core splits, and subtracts sum_c W M from each running diagonal.
constexpr int kBR = 32;  // indices per CTA of k_below

// row length of the staged panel operands (odd: the transposing fill and the
// product's row reads are both free of bank conflicts)
constexpr int kBelowLdp = kNB + 1;

// (double-buffered panel operands: the next panel's arrive by cp.async while
// this panel's product runs)
inline size_t below_smem(bool sym) {
  const size_t x = sizeof(float) * kBR * (kNB + 1);
  const size_t ps = 2 * sizeof(float) * 32 * kBelowLdp;
  const size_t t = 2 * sizeof(float) * 32 * 33;
  return (sym ? x + ps + t : 2 * (x + ps + t)) + sizeof(float) * (2 * 32 + kNB + 3 * 256);
}


// Substitution of R rows of one side against the panel's 32 x 32 unit lower
// block T (row c, column c' < c), the rows interleaved so that their chains
// overlap: lane c holds column c of every row; step c0 broadcasts the final
// value of column c0 and every later column subtracts its multiple.
template <int R>
__device__ __forceinline__ void below_solve(float* base, int ldx, const int* rows, int D, int b,
                                            const float* T, const float* scale) {
  const int lane = threadIdx.x & 31;
  float x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = lane < b ? base[rows[r] * ldx + D + lane] : 0.f;
  for (int c0 = 0; c0 < b - 1; ++c0) {
    const float t = lane > c0 ? T[lane * 33 + c0] : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float y = __shfl_sync(kLuFull, x[r], c0);
      x[r] = fmaf(-y, t, x[r]);
    }
  }
  const float sc = scale ? scale[lane] : 1.f;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane < b) base[rows[r] * ldx + D + lane] = x[r] * sc;
}

// Panel product of k_below for rows 4 ty .. 4 ty + 3 of the CTA and columns
// C0 + tx + 32 jj (jj < JJ, below kb): X -= W_panel M^T and (LU) Z -= M_panel
// W^T over the panel's 32 columns D .. D + 31. Consecutive lanes touch
// consecutive words, so neither the operand loads nor the updates conflict.
template <bool SYM, int JJ>
__device__ __forceinline__ void below_product(float* X, float* Zs, const float* Ps,
                                              const float* Qs, int ldx, int D, int C0, int kb,
                                              int ty, int tx) {
  float ax[4][JJ], az[SYM ? 1 : 4][SYM ? 1 : JJ];
  bool in[JJ];
#pragma unroll
  for (int jj = 0; jj < JJ; ++jj) in[jj] = C0 + tx + 32 * jj < kb;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj) {
      ax[i][jj] = 0.f;
      if (!SYM) az[i][jj] = 0.f;
    }
#pragma unroll 4
  for (int t = 0; t < 32; ++t) {
    float w[4], m[JJ];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = X[(4 * ty + i) * ldx + D + t];
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj) m[jj] = in[jj] ? Ps[t * kBelowLdp + C0 + tx + 32 * jj] : 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj) ax[i][jj] = fmaf(w[i], m[jj], ax[i][jj]);
    if (!SYM) {
      float mr[4], wq[JJ];
#pragma unroll
      for (int i = 0; i < 4; ++i) mr[i] = Zs[(4 * ty + i) * ldx + D + t];
#pragma unroll
      for (int jj = 0; jj < JJ; ++jj)
        wq[jj] = in[jj] ? Qs[t * kBelowLdp + C0 + tx + 32 * jj] : 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < JJ; ++jj) az[SYM ? 0 : i][SYM ? 0 : jj] =
            fmaf(mr[i], wq[jj], az[SYM ? 0 : i][SYM ? 0 : jj]);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int jj = 0; jj < JJ; ++jj)
      if (in[jj]) {
        const int j = C0 + tx + 32 * jj;
        X[(4 * ty + i) * ldx + j] -= ax[i][jj];
        if (!SYM) Zs[(4 * ty + i) * ldx + j] -= az[SYM ? 0 : i][SYM ? 0 : jj];
      }
}

template <bool SYM>
__global__ void __launch_bounds__(kLuThreads) k_below(LuArgs a) {
  constexpr int ldx = kNB + 1;
  float* X = reinterpret_cast<float*>(g_lu_dyn);   // [kBR][ldx]: A rows, then W
  float* Zs = SYM ? X : X + kBR * ldx;             // [kBR][ldx]: A columns, then M (LU)
  // [2][32][kBelowLdp], panel column t by outer-block index j: M (and, for LU,
  // W) of the outer block's rows, 16-byte aligned rows for vector loads
  float* Ps0 = (SYM ? X : Zs) + kBR * ldx;
  float* Qs0 = SYM ? Ps0 : Ps0 + 2 * 32 * kBelowLdp;
  float* T0 = Qs0 + 2 * 32 * kBelowLdp;            // [2][32][33]: M of the panel's diagonal block
  float* U0 = SYM ? T0 : T0 + 2 * 32 * 33;          // [2][32][33]: L of it (LU)
  float* rdp0 = U0 + 2 * 32 * 33;                  // [2][32]: 1 / d of the panel
  float* rda = rdp0 + 2 * 32;                      // [kNB]: 1 / d of the outer block
  float* red = rda + kNB;                          // [3][8][32]: running-diagonal partials
  const int tid = threadIdx.x, wp = tid >> 5;
  const int kb = a.kb, np = (kb + 31) / 32;
  const int64_t q = a.q, qe = q + kb, n = a.n, lda = a.lda;
  const float* A = a.A;
  float* Aw = a.A;
  const int ty = tid >> 5, tx = tid & 31;  // update: rows 4 ty.., columns 4 tx.. of a 128-wide chunk
  for (int64_t i0 = qe + (int64_t)kBR * blockIdx.x; i0 < n; i0 += (int64_t)kBR * gridDim.x) {
    const int nr = (int)((n - i0) < kBR ? (n - i0) : kBR);
    // the rows (and, for LU, columns) by cp.async: every load in flight at once
    for (int idx = tid; idx < kBR * kb; idx += kLuThreads) {
      const int r = idx % kBR, c = idx / kBR;
      cp_async4(&X[r * ldx + c], r < nr ? &A[(i0 + r) + (q + c) * lda] : A, r < nr);
    }
    if (!SYM) {
      for (int idx = tid; idx < kBR * kb; idx += kLuThreads) {
        const int c = idx % kb, r = idx / kb;
        cp_async4(&Zs[r * ldx + c], r < nr ? &A[(q + c) + (i0 + r) * lda] : A, r < nr);
      }
    }
    cp_async_commit();
    // Panel k's operands (its diagonal block and the M (W) rows of the outer
    // block for the later columns) go to buffer k & 1 by cp.async, issued
    // while panel k - 1's product runs; 1 / d through a register.
    auto issue = [&](int k) {
      const int64_t p = q + 32 * k;
      const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
      const int D = 32 * k, C0 = D + 32, bf = k & 1;
      float* T11 = T0 + bf * 32 * 33;
      float* U11 = U0 + bf * 32 * 33;
      float* Ps = Ps0 + bf * 32 * kBelowLdp;
      float* Qs = Qs0 + bf * 32 * kBelowLdp;
      for (int idx = tid; idx < 1024; idx += kLuThreads) {
        const int rr = idx >> 5, cc = idx & 31;
        const bool in = rr < b && cc < b && rr > cc;
        // M(p + rr, p + cc) (LDL^T: L = M) and, for LU, L(p + rr, p + cc)
        cp_async4(&T11[rr * 33 + cc], in ? (SYM ? &A[(p + rr) + (p + cc) * lda]
                                                 : &A[(p + cc) + (p + rr) * lda]) : A, in);
        if (!SYM) cp_async4(&U11[rr * 33 + cc], in ? &A[(p + rr) + (p + cc) * lda] : A, in);
      }
      const int cnt = C0 < kb ? (kb - C0) * 32 : 0;
      for (int idx = tid; idx < cnt; idx += kLuThreads) {
        const int j = C0 + (idx >> 5), t = idx & 31;
        const int64_t off = (q + j) * (int64_t)kNB + D + t;
        cp_async4(&Ps[t * kBelowLdp + j], t < b ? &a.Mk[off] : a.Mk, t < b);
        if (!SYM) cp_async4(&Qs[t * kBelowLdp + j], t < b ? &a.Wk[off] : a.Wk, t < b);
      }
      cp_async_commit();
      return (tid < 32 && tid < b) ? 1.f / (float)__ldcg(&a.piv[p + tid]) : 0.f;
    };
    float rv = issue(0);
    cp_async_wait_all();
    if (tid < 32) {
      rdp0[tid] = rv;
      rda[tid] = rv;
    }
    __syncthreads();
    for (int k = 0; k < np; ++k) {
      const int64_t p = q + 32 * k;
      const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
      const int D = 32 * k, bf = k & 1;
      const float* T11 = T0 + bf * 32 * 33;
      const float* U11 = U0 + bf * 32 * 33;
      const float* rdp = rdp0 + bf * 32;
      const float* Ps = Ps0 + bf * 32 * kBelowLdp;
      const float* Qs = Qs0 + bf * 32 * kBelowLdp;
      // solves: side 0 (W) and, for LU, side 1 (M = U / d); eight warps
      if (SYM) {
        int rows[4] = {wp, wp + 8, wp + 16, wp + 24};
        below_solve<4>(X, ldx, rows, D, b, T11, nullptr);
      } else if (wp < 4) {
        int rows[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) rows[r] = wp + 4 * r;
        below_solve<8>(X, ldx, rows, D, b, T11, nullptr);
      } else {
        int rows[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) rows[r] = (wp - 4) + 4 * r;
        below_solve<8>(Zs, ldx, rows, D, b, U11, rdp);
      }
      __syncthreads();
      const bool more = k + 1 < np;
      if (more) rv = issue(k + 1);
      const int C0 = D + 32;
      // the product over the columns right of the panel, in one pass: lane tx
      // takes columns C0 + tx + 32 jj, jj < JJ = ceil((kb - C0) / 32)
      switch ((kb - C0 + 31) >> 5) {
        case 1: below_product<SYM, 1>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 2: below_product<SYM, 2>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 3: below_product<SYM, 3>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 4: below_product<SYM, 4>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 5: below_product<SYM, 5>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 6: below_product<SYM, 6>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        case 7: below_product<SYM, 7>(X, Zs, Ps, Qs, ldx, D, C0, kb, ty, tx); break;
        default: break;
      }
      if (more) {
        cp_async_wait_all();
        if (tid < 32) {
          rdp0[(bf ^ 1) * 32 + tid] = rv;
          rda[D + 32 + tid] = rv;
        }
      }
      __syncthreads();
    }
    // stores: L below the outer block (column-major, rows fastest) ...
    for (int idx = tid; idx < kBR * kb; idx += kLuThreads) {
      const int r = idx % kBR, c = idx / kBR;
      if (r < nr) Aw[(i0 + r) + (q + c) * lda] = X[r * ldx + c] * rda[c];
    }
    // ... M^T to the right of it (LU), and the row-major operand rows
    for (int idx = tid; idx < kBR * kb; idx += kLuThreads) {
      const int c = idx % kb, r = idx / kb;
      if (r < nr) {
        const float w = X[r * ldx + c];
        const float m = SYM ? w * rda[c] : Zs[r * ldx + c];
        if (!SYM) Aw[(q + c) + (i0 + r) * lda] = m;
        const int64_t off = (i0 + r) * (int64_t)kNB + c;
        a.Wk[off] = w;
        a.Mk[off] = m;
        write_split(a.split, a.Wop, off, w);
        write_split(a.split, a.Mop, off, m);
      }
    }
    // running diagonal and band scale: lane = index, warp = 32-column slice,
    // then warp 0 adds the eight slices in a fixed order
    {
      const int r = tid & 31, part = tid >> 5;
      f2 dsum = {0.f, 0.f};
      float ssum = 0.f;
      for (int c = 32 * part; c < 32 * part + 32 && c < kb; ++c) {
        const float w = X[r * ldx + c];
        const float m = SYM ? w * rda[c] : Zs[r * ldx + c];
        dsum = f2_add_prod(dsum, w, m);
        ssum += fabsf(w * m);
      }
      red[part * 32 + r] = dsum.hi;
      red[256 + part * 32 + r] = dsum.lo;
      red[512 + part * 32 + r] = ssum;
      __syncthreads();
      if (part == 0) {
        f2 tot = make_f2(red[r], red[256 + r]);
        float st = red[512 + r];
        for (int k = 1; k < 8; ++k) {
          tot = f2_add(tot, make_f2(red[k * 32 + r], red[256 + k * 32 + r]));
          st += red[512 + k * 32 + r];
        }
        if (r < nr) {
          a.kd[i0 + r] -= f2_to_double(tot);
          a.s[i0 + r] += (double)st;
        }
      }
    }
    __syncthreads();
  }
}

// FP32 copy of K (lower: its lower triangle only) and the running diagonal.
__global__ void __launch_bounds__(256) k_convert_full(const double* K, int64_t ldk, float* A,
                                                      int64_t lda, int64_t n, double* kd,
                                                      double* s, int lower) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const double* col = K + j * ldk;
    float* dst = A + j * lda;
    for (int64_t i = (lower ? j : 0) + threadIdx.x; i < n; i += blockDim.x) dst[i] = (float)col[i];
    if (threadIdx.x == 0) {
      kd[j] = col[j];
      s[j] = 0.0;
    }
  }
}

// In-place LU of K - 1_{Y^c} in FP64: L strictly below the diagonal, the
// pivots on it, U = D U~ above it (lower: L and the pivots only, LDL^T).
__global__ void __launch_bounds__(256) k_export_lu(const float* A, int64_t lda, const double* piv,
                                                   double* F, int64_t ldf, int64_t n, int lower) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = (lower ? j : 0) + threadIdx.x; i < n; i += blockDim.x) {
      const double v = (double)A[i + j * lda];
      F[i + j * ldf] = i > j ? v : (i == j ? piv[j] : piv[i] * v);
    }
  }
}

struct LuLayout {
  int64_t ld32;
  float* A32;
  float *Wk, *Mk;
  void* Wop[3];
  void* Mop[3];
  double *kd, *s, *piv;
  unsigned* flag;
  int* err;
  float* Bbuf;
  RecomputeScratch rs;
  unsigned long long *yw, *v2w;
  float* inv2;
  double* s2;
};

bool carve_lu(Workspace& ws, int64_t n, LuLayout* L) {
  L->ld32 = ((n + 31) / 32) * 32;
  if (L->ld32 < 32) L->ld32 = 32;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  L->A32 = static_cast<float*>(ws.take(sizeof(float) * (size_t)L->ld32 * nn));
  const size_t ob = sizeof(float) * nn * (size_t)kNB;
  L->Wk = static_cast<float*>(ws.take(ob));
  L->Mk = static_cast<float*>(ws.take(ob));
  bool ops_ok = true;
  for (int o = 0; o < 3; ++o) {
    L->Wop[o] = ws.take(ob);
    L->Mop[o] = ws.take(ob);
    ops_ok = ops_ok && L->Wop[o] && L->Mop[o];
  }
  L->kd = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->s = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->piv = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->flag = static_cast<unsigned*>(ws.take(256));
  L->err = reinterpret_cast<int*>(L->flag) + 16;
  L->Bbuf = static_cast<float*>(ws.take(sizeof(float) * 1024));
  if (!recompute_carve(ws, n, &L->rs)) return false;
  L->yw = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  L->v2w = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  L->inv2 = static_cast<float*>(ws.take(sizeof(float) * 1024 * (size_t)L->rs.nblk));
  L->s2 = static_cast<double*>(ws.take(sizeof(double) * nn));
  return L->A32 && L->Wk && L->Mk && ops_ok && L->kd && L->s && L->piv && L->flag && L->Bbuf &&
         L->yw &&
         L->v2w && L->inv2 && L->s2;
}

}  // namespace

size_t ws_mixed_lu(int64_t n) {
  Workspace probe;
  probe.base = reinterpret_cast<char*>(256);
  probe.size = ~size_t(0) >> 2;
  LuLayout L;
  carve_lu(probe, n, &L);
  return probe.used + 512;
}

namespace {

template <bool SYM>
cudaError_t sample_chunked(const DrawArgs& a, Workspace ws) {
  const int64_t n = a.n;
  const int NB = g_tuning.outer_block;
  LuLayout L;
  if (!carve_lu(ws, n, &L)) return cudaErrorInvalidValue;
  cudaError_t e = init_result(a.result, a.stream);
  if (e != cudaSuccess || n == 0) return e;
  if ((e = cudaMemsetAsync(L.flag, 0, 256, a.stream)) != cudaSuccess) return e;
  if ((e = recompute_reset(L.rs, n, a.stream)) != cudaSuccess) return e;
  const size_t words = sizeof(unsigned long long) * (size_t)n;
  if ((e = cudaMemsetAsync(L.yw, 0, words, a.stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(L.v2w, 0, words, a.stream)) != cudaSuccess) return e;
  const double* K = static_cast<const double*>(a.K);
  {
    ProfScope ps(kProfConvert, a.stream, 0.0, (SYM ? 6.0 : 12.0) * (double)n * (double)n);
    k_convert_full<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        K, a.ld, L.A32, L.ld32, n, L.kd, L.s, SYM ? 1 : 0);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // cooperative capacity (and the shared-memory attribute), per device
  static int caps[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int& cap = caps[dev];
  if (cap == 0) {
    cudaError_t ea = cudaFuncSetAttribute(k_lu_outer<SYM>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)lu_dyn_smem(kMaxSlots));
    if (ea != cudaSuccess) return ea;
    ea = cudaFuncSetAttribute(k_below<SYM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)below_smem(SYM));
    if (ea != cudaSuccess) return ea;
    DevInfo di;
    if ((ea = dev_info(&di)) != cudaSuccess) return ea;
    int per_sm = 0;
    ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_outer<SYM>, kLuThreads,
                                                       lu_dyn_smem(kMaxSlots));
    if (ea != cudaSuccess) return ea;
    cap = per_sm * di.sm_count;
    if (cap > kMaxCoopCtas) cap = kMaxCoopCtas;
    if (cap < 3) return cudaErrorLaunchOutOfResources;
  }
  int grid = cap;
  if (g_tuning.max_ctas > 0 && grid > g_tuning.max_ctas) grid = g_tuning.max_ctas;
  if (grid < 3) grid = 3;
  // split pipeline: the panel launch is CTA 0 and one helper per chunk of the
  // outer block; the rows below go to k_below on `grid` CTAs
  // (the panel launch keeps the stream's CTA share: the CTAs beyond CTA 0 and
  // the helpers serve the FP64 recomputes)
  const bool split_rows = g_tuning.panel_pipeline == 3;
  const int below_grid = grid;
  if (split_rows && g_tuning.panel_ctas > 0) grid = g_tuning.panel_ctas < cap ? g_tuning.panel_ctas : cap;
  if (split_rows && grid < kMaxOuterBlock / 32) grid = kMaxOuterBlock / 32;
  // CTA 0 decides, CTAs 1..nh own the outer block's chunks, the rest the
  // chunks beyond it; slots hold the chunks a CTA precomputes per panel
  // (one CTA per chunk on a full grid; on a small grid a helper owns
  // several chunks, so that most CTAs stay workers)
  int nh = split_rows ? kMaxOuterBlock / 32 - 1 : (grid - 2) / 8;
  if (nh > kMaxOuterBlock / 32 - 1) nh = kMaxOuterBlock / 32 - 1;
  if (nh < 1) nh = 1;
  const int64_t nwk = split_rows ? below_grid : grid - 1 - nh;
  const int64_t trail = ((n > NB ? n - NB : 0) + 31) / 32;
  int slots = (int)((trail + nwk - 1) / nwk);
  const int hslots = (kMaxOuterBlock / 32 - 1 + nh - 1) / nh;
  if (slots < hslots) slots = hslots;
  if (slots > kMaxSlots) slots = kMaxSlots;
  if (split_rows) slots = hslots;
  const size_t dyn = lu_dyn_smem(slots);
  const int split = a.precision == DPP_PREC_BF16X6 ? kSplitBf16x6 : kSplit3xTf32;
  unsigned epoch = 1;
  for (int64_t q = 0; q < n; q += NB) {
    const int kb = (int)((n - q) < NB ? (n - q) : NB);
    LuArgs la;
    la.K = K;
    la.ldk = a.ld;
    la.A = L.A32;
    la.lda = L.ld32;
    la.n = n;
    la.q = q;
    la.kb = kb;
    la.uniforms = a.uniforms;
    la.seed = a.seed;
    la.inst = a.instance;
    la.keep = a.keep;
    la.piv = L.piv;
    la.kd = L.kd;
    la.s = L.s;
    la.Wk = L.Wk;
    la.Mk = L.Mk;
    for (int o = 0; o < 3; ++o) {
      la.Wop[o] = L.Wop[o];
      la.Mop[o] = L.Mop[o];
    }
    la.split = split;
    la.res = a.result;
    la.epoch0 = epoch;
    la.tol = 1e-3;
    la.tau0 = (float)(g_tuning.tau_safety * 0x1.0p-22);
    la.Bbuf = L.Bbuf;
    la.nh = nh;
    la.slots = slots;
    la.withhold = g_tuning.fault_withhold;
    la.no_rows = split_rows ? 1 : 0;
    la.lr.rc = recompute_args(L.rs, K, a.ld, L.A32, L.ld32, L.piv, a.keep, n, q, a.result);
    la.lr.rc.grid = grid;
    la.lr.yw = L.yw;
    la.lr.v2w = L.v2w;
    la.lr.inv2 = L.inv2;
    la.lr.s2 = L.s2;
    void* args[] = {&la};
    {
      ProfScope ps(kProfPanel, a.stream);
      e = cudaLaunchCooperativeKernel((const void*)k_lu_outer<SYM>, dim3((unsigned)grid),
                                      dim3(kLuThreads), args, dyn, a.stream);
    }
    if (e != cudaSuccess) return e;
    epoch += (unsigned)((kb + 31) / 32);
    const int64_t r0 = q + kb;
    if (split_rows && r0 < n) {
      // the rows below the outer block, through its panels ((n - r0) kb^2
      // flops for the Hermitian form, twice that for LU)
      const double fl = (SYM ? 1.0 : 2.0) * (double)(n - r0) * (double)kb * (double)kb;
      int64_t bg = (n - r0 + kBR - 1) / kBR;
      const int64_t bcap = (int64_t)below_grid * (SYM ? 2 : 1);  // CTAs resident per SM
      if (bg > bcap) bg = bcap;
      ProfScope ps(kProfBelow, a.stream, fl, 0.0);
      k_below<SYM><<<(unsigned)bg, kLuThreads, below_smem(SYM), a.stream>>>(la);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (r0 < n) {
      const int64_t m = n - r0;
      // lower triangle (SYM) or whole square of 2 m^2 kb flops
      const double fl = (SYM ? 1.0 : 2.0) * (double)m * (double)m * (double)kb;
      ProfScope ps(kProfUpdateTc, a.stream, fl, (SYM ? 4.0 : 8.0) * (double)m * (double)m);
      e = outer_update_tc(split, L.A32, L.ld32, n, r0, kb, L.Wop, L.Mop, kNB, !SYM, L.err,
                          a.stream);
      if (e != cudaSuccess) return e;
    }
  }
  if (a.pivots_user) {
    e = cudaMemcpyAsync(a.pivots_user, L.piv, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                        a.stream);
    if (e != cudaSuccess) return e;
  }
  if (a.factor_out) {
    ProfScope ps(kProfOther, a.stream);
    k_export_lu<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        L.A32, L.ld32, L.piv, static_cast<double*>(a.factor_out), a.ld, n, SYM ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t sample_mixed_lu(const DrawArgs& a, Workspace ws) { return sample_chunked<false>(a, ws); }

cudaError_t sample_mixed_chunked(const DrawArgs& a, Workspace ws) {
  return sample_chunked<true>(a, ws);
}

}  // namespace dpp
