// Mixed-precision DPP sampler for a general complex kernel: the LU form of
// Algorithm 1 on complex, non-Hermitian K (the Aztec-diamond kernels of
// Section 1), blocked as in Algorithm 4.
//
// Factorization kept in planar FP32 copies Ar, Ai of K (full square,
// column-major), with the conventions of the real LU path:
//   K_P - 1_G = L D U~,  L unit lower,  U~ = D^{-1} U unit upper,  M = U~^T,
// stored as L strictly below the diagonal, the FP32 pivot on it and U~
// strictly above. With W = L D the Schur update of one outer block is
//   A22 -= W M^T:  Re -= [Wr Wi] [Mr -Mi]^T,  Im -= [Wr Wi] [Mi Mr]^T,
// two real contractions of depth 2 kb over the whole trailing square, each
// run by the tensor-core update of the real paths (no conjugation anywhere:
// LU is bilinear).
//
// Pivots are complex; the decision compares the uniform with Re d_j. A
// running diagonal kd_i = K_ii - sum_k w_ik m_ik (complex FP64 sums of the
// FP32 factor products) gives each pivot; one whose uniform lies within
//   tau_j = c 2^-22 sqrt(j + 1) (|K_jj| + s_j) + 2^-22,  s_j = sum_k |w_jk m_jk|,
// of Re d_j is recomputed in FP64 from the original K before its decision
// (Props. 3-5): with A = K_P - 1_G, a = K[P, g], b = K[g, P]^T and any x0, y0,
// r = a - A x0, s = b - A^T y0,
//     d_g = K_gg - b^T x0 - y0^T r - s^T A^{-1} r,
// x0 = M_P^{-T} m (m = row g of M), y0 = L_P^{-T} l (l = row g of L) and the
// last term as sum_c (L_P^{-1} r)_c (M_P^{-1} s)_c / d_c, second order in the
// factorization's error. The two triangular sweeps of each side run as
// wavefronts over 32-index blocks on the other CTAs of the launch, with the
// protocol of the real recompute; complex values travel as two id-tagged
// words (real, imaginary).
//
// One cooperative launch per outer block [q, q + kb), kb <= 128:
//   CTA 0     : the diagonal block, resident in shared memory, right-looking
//               with a decision before every column; every column of L and
//               row of U~ goes to global memory as soon as it is final (the
//               recompute reads them); then publishes the block;
//   CTAs 1..  : serve recompute requests until the block is published;
//   then all  : 32-index tiles beyond the block: W = A U~^{-1} for their rows
//               and U = L^{-1} A for their columns, 32-wide panels right-
//               looking in shared memory; L, U~, the operand rows with their
//               tensor-core splits and the running diagonal.
// After each outer block the two real contractions update the trailing square.
#include <cuda_bf16.h>
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"
#include "dpp_recompute.cuh"

namespace dpp {
namespace {

constexpr unsigned kXF = 0xffffffffu;
constexpr int kXT = 256;         // threads per CTA
constexpr int kXB = 128;         // columns of one outer block, at most
constexpr int kXLd = 2 * kXB;    // operand row length: [real | imaginary]
constexpr int kXBp = kXB + 1;    // padded row of the shared-memory blocks

struct cf {
  float x, y;
};
__device__ __forceinline__ cf cmk(float x, float y) { return {x, y}; }
__device__ __forceinline__ cf cmul(cf a, cf b) {
  return {fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x)};
}
// acc + a b
__device__ __forceinline__ cf cfma(cf acc, cf a, cf b) {
  return {fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y))};
}
// acc - a b
__device__ __forceinline__ cf cfms(cf acc, cf a, cf b) {
  return {fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y))};
}
__device__ __forceinline__ cf cshfl(cf v, int src) {
  return {__shfl_sync(kXF, v.x, src), __shfl_sync(kXF, v.y, src)};
}
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc + a b, FP64
__device__ __forceinline__ double2 dfma(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 dsub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 dadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double dabs(double2 a) { return hypot(a.x, a.y); }
// 1 / a (scaled so that no intermediate overflows)
__device__ __forceinline__ double2 drecip(double2 a) {
  const double s = fmax(fabs(a.x), fabs(a.y));
  if (s == 0.0) return make_double2(1.0 / 0.0, 0.0);
  const double ar = a.x / s, ai = a.y / s;
  const double den = s * (ar * ar + ai * ai);
  return make_double2(ar / den, -ai / den);
}
__device__ __forceinline__ double2 tod(cf a) { return make_double2((double)a.x, (double)a.y); }
// 1 / a in FP32, scaled so that tiny pivots neither underflow nor overflow
// (the FP64 pipe of this GPU is narrow: per-thread FP64 divisions in the
// decision loop cost more than the rest of a step)
__device__ __forceinline__ cf crecipf(cf a) {
  const float s = fmaxf(fabsf(a.x), fabsf(a.y));
  const float is = __frcp_rn(s);
  const float ar = a.x * is, ai = a.y * is;
  const float den = __frcp_rn(s * fmaf(ar, ar, ai * ai));
  return {ar * den, -ai * den};
}
__device__ __forceinline__ float cabsf_(cf a) { return hypotf(a.x, a.y); }

// ---------------------------------------------------------------------------
// FP64 recompute, complex LU form
// ---------------------------------------------------------------------------
struct XRc {
  RecomputeArgs rc;  // control words, grid, result, wait limit, keep; xw / vw: real words
  const double2* K;  // original K (complex, column-major)
  int64_t ldk;
  const float* Ar;
  const float* Ai;
  int64_t lda;
  const double2* piv;
  unsigned long long* xwi;   // x0 imaginary words
  unsigned long long* yw;    // y0 words
  unsigned long long* ywi;
  unsigned long long* vwi;   // v1 = L^{-1} r imaginary words
  unsigned long long* v2w;   // v2 = M^{-1} s words
  unsigned long long* v2wi;
  float* inv;    // per 32-block: inverse of L_tt, real plane then imaginary (2048 floats)
  float* inv2;   // the same for M_tt
  double2* r;    // residual r = a - A x0
  double2* s2;   // residual s = b - A^T y0
  double* part;  // 8 doubles per worker CTA
};

// F(i, c): L(i, c) = A[i + c lda] (TRANS false) or M(i, c) = A[c + i lda] (TRANS true).
template <bool TRANS>
__device__ __forceinline__ cf ld_f(const XRc& X, int64_t i, int64_t c) {
  const int64_t o = TRANS ? c + i * X.lda : i + c * X.lda;
  return {__ldcg(X.Ar + o), __ldcg(X.Ai + o)};
}

__device__ __forceinline__ float word_f(const RecomputeArgs& a, const unsigned long long* w,
                                        unsigned id, bool* live) {
  const unsigned long long v = ld_relaxed_u64(w);
  return word_has(v, id) ? __uint_as_float((unsigned)v) : word_value_slow(a, w, id, live);
}
__device__ __forceinline__ cf word_c(const RecomputeArgs& a, const unsigned long long* wr,
                                     const unsigned long long* wi, int64_t idx, unsigned id,
                                     bool* live) {
  return {word_f(a, wr + idx, id, live), word_f(a, wi + idx, id, live)};
}

// Whole warp: lanes < nvalid wait for the complex value at words[lane].
__device__ __forceinline__ bool wait_c(const RecomputeArgs& a, const unsigned long long* wr,
                                       const unsigned long long* wi, int nvalid, unsigned id,
                                       cf* out) {
  float x = 0.f, y = 0.f;
  if (!warp_wait_words(a, wr, nvalid, id, &x)) return false;
  if (!warp_wait_words(a, wi, nvalid, id, &y)) return false;
  *out = cmk(x, y);
  return true;
}

// Warp 0: the inverse of the unit lower block F_tt (nr rows), stored
// row-major (real plane, then imaginary); lane c computes column c.
template <bool TRANS>
__device__ __forceinline__ void xl_diag_inverse(const XRc& X, float* inv, int64_t t, int nr,
                                                float (*sDr)[33], float (*sDi)[33]) {
  const int lane = threadIdx.x & 31;
  const int64_t r0 = 32 * t;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const cf v = (lane < nr && k < lane) ? ld_f<TRANS>(X, r0 + lane, r0 + k) : cmk(0.f, 0.f);
    sDr[lane][k] = v.x;
    sDi[lane][k] = v.y;
  }
  __syncwarp();
  cf z[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    cf s = cmk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < i; ++k) s = cfma(s, cmk(sDr[i][k], sDi[i][k]), z[k]);
    z[i] = (i == lane) ? cmk(1.f, 0.f) : (i < lane ? cmk(0.f, 0.f) : cmk(-s.x, -s.y));
  }
  float* dst = inv + (size_t)t * 2048;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    dst[i * 32 + lane] = z[i].x;
    dst[1024 + i * 32 + lane] = z[i].y;
  }
  __syncwarp();
}

// Lane c of a warp receives sum over the lanes of v[c] for the 16 complex
// values v (columns 16 h .. 16 h + 15 of a 32-block; h = c >> 4).
__device__ __forceinline__ cf reduce_halves(const cf (&v0)[16], const cf (&v1)[16], int lane) {
  float a[32], b[32];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    a[k] = v0[k].x;
    a[16 + k] = v0[k].y;
    b[k] = v1[k].x;
    b[16 + k] = v1[k].y;
  }
  // lane L < 16 holds the real sum of column L of its half, lane 16 + L the imaginary
  const float ra = transpose_reduce(a, lane);
  const float rb = transpose_reduce(b, lane);
  const int c = lane & 15;
  const float re0 = __shfl_sync(kXF, ra, c), im0 = __shfl_sync(kXF, ra, 16 + c);
  const float re1 = __shfl_sync(kXF, rb, c), im1 = __shfl_sync(kXF, rb, 16 + c);
  return lane < 16 ? cmk(re0, im0) : cmk(re1, im1);
}

// Backward sweep, block t:  x_t = F_tt^{-T} (f_t - sum_{s > t} F_st^T x_s),
// f = row g of F; x published as words. Sources split over the 8 warps.
template <bool TRANS>
__device__ __forceinline__ void xl_r1_block(const XRc& X, float* inv, unsigned long long* wr,
                                            unsigned long long* wi, int64_t g, int64_t nblk,
                                            int64_t t, unsigned id, Handoff& hr, Handoff& hi,
                                            int seqh, float (*sDr)[33], float (*sDi)[33],
                                            bool* live) {
  const RecomputeArgs& a = X.rc;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
  cf f = cmk(0.f, 0.f);
  if (wp == 0) {
    xl_diag_inverse<TRANS>(X, inv, t, nr, sDr, sDi);
    if (lane < nr) f = ld_f<TRANS>(X, g, 32 * t + lane);
  }
  cf red;
  if (TRANS) {
    // lane = column 32 t + lane: F(32 s + k, 32 t + lane) = A[(32 t + lane) + (32 s + k) lda]
    cf acc = cmk(0.f, 0.f);
    for (int64_t s = t + 1 + wp + (t + 1 + wp < nblk ? ((nblk - 2 - t - wp) / 8) * 8 : 0);
         s > t && s < nblk; s -= 8) {  // latest-published source last
      const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
      cf v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k)
        v[k] = (k < ns && lane < nr) ? ld_f<true>(X, 32 * s + k, 32 * t + lane) : cmk(0.f, 0.f);
      cf xs = cmk(0.f, 0.f);
      *live = __all_sync(kXF, *live);  // warp-uniform before the collective wait
      if (*live && !wait_c(a, wr + 32 * s, wi + 32 * s, ns, id, &xs)) *live = false;
#pragma unroll
      for (int k = 0; k < 32; ++k) acc = cfma(acc, v[k], cshfl(xs, k));
    }
    red = acc;
  } else {
    // lane = row 32 s + lane: F(32 s + lane, 32 t + c) = A[(32 s + lane) + (32 t + c) lda],
    // the 32 columns in two halves (register budget)
    cf acc[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[h][k] = cmk(0.f, 0.f);
    for (int64_t s = t + 1 + wp + (t + 1 + wp < nblk ? ((nblk - 2 - t - wp) / 8) * 8 : 0);
         s > t && s < nblk; s -= 8) {  // latest-published source last
      const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
      cf xs = cmk(0.f, 0.f);
      *live = __all_sync(kXF, *live);  // warp-uniform before the collective wait
      if (*live && !wait_c(a, wr + 32 * s, wi + 32 * s, ns, id, &xs)) *live = false;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        cf tile[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
          tile[k] = (lane < ns && 16 * h + k < nr) ? ld_f<false>(X, 32 * s + lane, 32 * t + 16 * h + k)
                                                 : cmk(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[h][k] = cfma(acc[h][k], tile[k], xs);
      }
    }
    red = reduce_halves(acc[0], acc[1], lane);
  }
  if (wp != 0) {
    handoff_put(a, hr, seqh, wp, red.x, live);
    handoff_put(a, hi, seqh, wp, red.y, live);
  } else {
    const float sr = handoff_take(a, hr, seqh, red.x, live);
    const float si = handoff_take(a, hi, seqh, red.y, live);
    const cf y = cmk(f.x - sr, f.y - si);
    // x_lane = sum_k inv(k, lane) y_k (this lane wrote column lane of inv)
    const float* src = inv + (size_t)t * 2048;
    cf x = cmk(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 32; ++k) x = cfma(x, cmk(src[k * 32 + lane], src[1024 + k * 32 + lane]), cshfl(y, k));
    if (lane < nr) {
      st_relaxed_u64(wr + 32 * t + lane, make_word(id, x.x));
      st_relaxed_u64(wi + 32 * t + lane, make_word(id, x.y));
    }
  }
}

// Forward sweep, block t:  v_t = F_tt^{-1} (rhs_t - sum_{s < t} F_ts v_s).
// Returns v for lane i of warp 0 (0 elsewhere).
template <bool TRANS>
__device__ __forceinline__ cf xl_r3_block(const XRc& X, const float* inv, unsigned long long* wr,
                                          unsigned long long* wi, const double2* rhs, int64_t g,
                                          int64_t t, unsigned id, Handoff& hr, Handoff& hi,
                                          int seqh, bool* live) {
  const RecomputeArgs& a = X.rc;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
  const int64_t slast = t - 1 - wp;
  cf red;
  if (!TRANS) {
    // lane = row 32 t + lane: F(32 t + lane, 32 s + c) = A[(32 t + lane) + (32 s + c) lda]
    cf acc = cmk(0.f, 0.f);
    if (slast >= 0) {
      for (int64_t s = slast % 8; s <= slast; s += 8) {
        cf tile[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
          tile[c] = lane < nr ? ld_f<false>(X, 32 * t + lane, 32 * s + c) : cmk(0.f, 0.f);
        cf vs = cmk(0.f, 0.f);
        *live = __all_sync(kXF, *live);  // warp-uniform before the collective wait
        if (*live && !wait_c(a, wr + 32 * s, wi + 32 * s, 32, id, &vs)) *live = false;
#pragma unroll
        for (int c = 0; c < 32; ++c) acc = cfma(acc, tile[c], cshfl(vs, c));
      }
    }
    red = acc;
  } else {
    // lane = column 32 s + lane: F(32 t + i, 32 s + lane) = A[(32 s + lane) + (32 t + i) lda]
    cf acc[2][16];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int k = 0; k < 16; ++k) acc[h][k] = cmk(0.f, 0.f);
    if (slast >= 0) {
      for (int64_t s = slast % 8; s <= slast; s += 8) {
        cf vs = cmk(0.f, 0.f);
        *live = __all_sync(kXF, *live);  // warp-uniform before the collective wait
        if (*live && !wait_c(a, wr + 32 * s, wi + 32 * s, 32, id, &vs)) *live = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cf tile[16];
#pragma unroll
          for (int i = 0; i < 16; ++i)
            tile[i] = 16 * h + i < nr ? ld_f<true>(X, 32 * t + 16 * h + i, 32 * s + lane)
                                      : cmk(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[h][i] = cfma(acc[h][i], tile[i], vs);
        }
      }
    }
    red = reduce_halves(acc[0], acc[1], lane);
  }
  cf v = cmk(0.f, 0.f);
  if (wp != 0) {
    handoff_put(a, hr, seqh, wp, red.x, live);
    handoff_put(a, hi, seqh, wp, red.y, live);
  } else {
    const float sr = handoff_take(a, hr, seqh, red.x, live);
    const float si = handoff_take(a, hi, seqh, red.y, live);
    const double2 rv = lane < nr ? rhs[32 * t + lane] : make_double2(0.0, 0.0);
    const cf y = cmk((float)(rv.x - (double)sr), (float)(rv.y - (double)si));
    // v_lane = sum_c inv(lane, c) y_c
    const float* src = inv + (size_t)t * 2048 + lane * 32;
#pragma unroll
    for (int c = 0; c < 32; ++c) v = cfma(v, cmk(src[c], src[1024 + c]), cshfl(y, c));
    if (lane < nr) {
      st_relaxed_u64(wr + 32 * t + lane, make_word(id, v.x));
      st_relaxed_u64(wi + 32 * t + lane, make_word(id, v.y));
    }
  }
  return v;
}

// Both residuals of the owner's block t (indices i in [32 t, 32 t + nr)):
//   r_i = K[i, g] - sum_{c < g} K[i, c] x0_c  (+ x0_i if i was rejected),
//   s_i = K[g, i] - sum_{c < g} K[c, i] y0_c  (+ y0_i if i was rejected),
// FP64 from the original K; warp 0 lane i accumulates K[g, i] x0_i into bx
// and y0_i r_i into yr. Part r reads rows of K (lane = i), part s columns
// (lane = c, reduced over the lanes at the end); both coalesced, each in two
// halves of 16 (register budget).
__device__ __noinline__ void xl_residual(const XRc& X, unsigned id, int64_t g, int64_t t, int nr,
                                         double (*sA)[32][2], double (*sB)[32][2], bool* live,
                                         double2* bx, double2* yr) {
  const RecomputeArgs& a = X.rc;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const double2* K = X.K;
  const int64_t ldk = X.ldk;
  const int64_t i = 32 * t + lane;
  const bool vi = lane < nr;
  const int64_t nblk = (g + 31) / 32;
  double2 accA = make_double2(0.0, 0.0);
  for (int64_t m = wp; m < nblk; m += 8) {
    const int64_t c0 = 32 * m;
    const int nc = (int)((g - c0) < 32 ? (g - c0) : 32);
    const cf xl = lane < nc ? word_c(a, a.xw, X.xwi, c0 + lane, id, live) : cmk(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double2 kv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        kv[k] = (vi && 16 * h + k < nc) ? K[i + (c0 + 16 * h + k) * ldk] : make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 16; ++k) accA = dfma(accA, kv[k], tod(cshfl(xl, 16 * h + k)));
    }
  }
  sA[wp][lane][0] = accA.x;
  sA[wp][lane][1] = accA.y;
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    double2 accB[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) accB[k] = make_double2(0.0, 0.0);
    for (int64_t m = wp; m < nblk; m += 8) {
      const int64_t c0 = 32 * m;
      const int nc = (int)((g - c0) < 32 ? (g - c0) : 32);
      const bool vc = lane < nc;
      const double2 yl = vc ? tod(word_c(a, X.yw, X.ywi, c0 + lane, id, live)) : make_double2(0.0, 0.0);
      double2 kv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k)
        kv[k] = (vc && 16 * h + k < nr) ? K[(c0 + lane) + (32 * t + 16 * h + k) * ldk]
                                        : make_double2(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 16; ++k) accB[k] = dfma(accB[k], kv[k], yl);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const double sr = warp_sum(accB[k].x), si = warp_sum(accB[k].y);
      if (lane == 16 * h + k) {
        sB[wp][lane][0] = sr;
        sB[wp][lane][1] = si;
      }
    }
  }
  __syncthreads();
  if (wp == 0 && vi) {
    double2 tr = make_double2(0.0, 0.0), ts = make_double2(0.0, 0.0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tr = dadd(tr, make_double2(sA[k][lane][0], sA[k][lane][1]));
      ts = dadd(ts, make_double2(sB[k][lane][0], sB[k][lane][1]));
    }
    const double2 xi = tod(word_c(a, a.xw, X.xwi, i, id, live));
    const double2 yi = tod(word_c(a, X.yw, X.ywi, i, id, live));
    const double2 kgi = K[g + i * ldk];
    double2 ri = dsub(K[i + g * ldk], tr);
    double2 si = dsub(kgi, ts);
    if (a.keep[i] == 0) {  // (K_P - 1_G) has -1 on the rejected diagonal
      ri = dadd(ri, xi);
      si = dadd(si, yi);
    }
    X.r[i] = ri;
    X.s2[i] = si;
    *bx = dfma(*bx, kgi, xi);
    *yr = dfma(*yr, yi, ri);
  }
  __syncthreads();
}

// Worker side of one request (all threads of a worker CTA).
__device__ __noinline__ bool xl_serve(const XRc& X, unsigned id) {
  const RecomputeArgs& a = X.rc;
  __shared__ float sDr[32][33], sDi[32][33];
  __shared__ Handoff hr, hi;
  __shared__ double sA[8][32][2], sB[8][32][2];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t w = blockIdx.x - 1, nw = a.grid - 1;
  const int64_t g = (int64_t)ld_acquire(&a.ctrl[kCtlG]);
  const int64_t nblk = (g + 31) / 32;
  bool live = true;
  if (tid < 8) {
    hr.ready[tid] = 0;
    hi.ready[tid] = 0;
  }
  if (tid == 0) {
    hr.cons = 0;
    hi.cons = 0;
  }
  __syncthreads();
  {
    // x0 = M_P^{-T} m and y0 = L_P^{-T} l, owned blocks from the last one down
    int seqh = 0;
    const int64_t tfirst = (w < nblk) ? w + ((nblk - 1 - w) / nw) * nw : -1;
    for (int64_t t = tfirst; t >= 0; t -= nw) {
      xl_r1_block<true>(X, X.inv2, a.xw, X.xwi, g, nblk, t, id, hr, hi, seqh++, sDr, sDi, &live);
      xl_r1_block<false>(X, X.inv, X.yw, X.ywi, g, nblk, t, id, hr, hi, seqh++, sDr, sDi, &live);
    }
  }
  __syncthreads();
  if (tid < 8) {
    hr.ready[tid] = 0;
    hi.ready[tid] = 0;
  }
  if (tid == 0) {
    hr.cons = 0;
    hi.cons = 0;
  }
  __syncthreads();
  double2 bx = make_double2(0.0, 0.0), yr = make_double2(0.0, 0.0), es = make_double2(0.0, 0.0);
  {
    // residuals, then v1 = L_P^{-1} r and v2 = M_P^{-1} s, owned blocks upwards
    int seqh = 0;
    for (int64_t t = w; t < nblk; t += nw) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      xl_residual(X, id, g, t, nr, sA, sB, &live, &bx, &yr);
      const cf v1 = xl_r3_block<false>(X, X.inv, a.vw, X.vwi, X.r, g, t, id, hr, hi, seqh++, &live);
      const cf v2 = xl_r3_block<true>(X, X.inv2, X.v2w, X.v2wi, X.s2, g, t, id, hr, hi, seqh++, &live);
      if (wp == 0 && lane < nr) es = dadd(es, dmul(dmul(tod(v1), tod(v2)), drecip(X.piv[32 * t + lane])));
    }
  }
  if (wp == 0) {
    bx.x = warp_sum(bx.x);
    bx.y = warp_sum(bx.y);
    yr.x = warp_sum(yr.x);
    yr.y = warp_sum(yr.y);
    es.x = warp_sum(es.x);
    es.y = warp_sum(es.y);
    if (lane == 0) {
      double* p = X.part + 8 * w;
      p[0] = bx.x;
      p[1] = bx.y;
      p[2] = yr.x;
      p[3] = yr.y;
      p[4] = es.x;
      p[5] = es.y;
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

// CTAs 1..G-1: serve requests until the outer block with this epoch is
// published. False on abort or timeout.
__device__ inline bool xl_follower(const XRc& X, unsigned epoch) {
  const RecomputeArgs& a = X.rc;
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
    if (cmd == 0) return false;
    if (cmd == 2) return true;
    if (!xl_serve(X, id)) return false;
    served = id & 0xffu;
  }
}

// Leader (warp 0 of CTA 0): pivot g recomputed in FP64. The factor entries of
// indices < g must be in global memory. Lane-uniform results.
__device__ inline bool xl_leader(const XRc& X, int64_t g, unsigned epoch, int* seq, double2* pe,
                                 double* est) {
  const RecomputeArgs& a = X.rc;
  const int lane = threadIdx.x & 31;
  __threadfence();
  __syncwarp();
  *seq += 1;
  const unsigned id = (epoch << 8) | (unsigned)(*seq);
  bool ok = a.grid >= 2 && *seq < 256;
  if (ok && lane == 0) {
    atomicExch(&a.ctrl[kCtlG], (unsigned)g);
    __threadfence();
    st_release(&a.ctrl[kCtlReq], id);
    ok = rc_wait_geq(a, &a.ctrl[kCtlAck], id);
  }
  ok = __shfl_sync(kXF, ok, 0);
  double2 bx = make_double2(0.0, 0.0), yr = bx, e = bx;
  if (ok && lane == 0) {
    for (int w = 0; w < a.grid - 1; ++w) {
      const double* p = X.part + 8 * w;
      bx = dadd(bx, make_double2(__ldcg(p + 0), __ldcg(p + 1)));
      yr = dadd(yr, make_double2(__ldcg(p + 2), __ldcg(p + 3)));
      e = dadd(e, make_double2(__ldcg(p + 4), __ldcg(p + 5)));
    }
  }
  const double2 kgg = X.K[g + g * X.ldk];
  double2 d2 = dsub(dsub(dsub(kgg, bx), yr), e);
  double er = dabs(e) * 1e-2 + 1e-12 * (1.0 + dabs(kgg) + dabs(bx) + dabs(yr));
  d2.x = __shfl_sync(kXF, d2.x, 0);
  d2.y = __shfl_sync(kXF, d2.y, 0);
  er = __shfl_sync(kXF, er, 0);
  if (ok) {
    *pe = d2;
    *est = er;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Outer-block kernel
// ---------------------------------------------------------------------------
struct XArgs {
  const double2* K;
  int64_t ldk;
  float* Ar;
  float* Ai;
  int64_t lda, n, q;
  int kb;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double2* piv;
  double2* kd;
  double* s;
  void* Wop[3];   // [Wr | Wi]
  void* M1op[3];  // [Mr | -Mi]
  void* M2op[3];  // [Mi | Mr]
  int split;
  dpp_result* res;
  unsigned epoch;
  double tol;
  float tau0;
  int withhold;  // fault injection: CTA 0 never publishes the block
  XRc xr;
};

extern __shared__ __align__(16) unsigned char g_x_dyn[];

// CTA 0's per-index state of the diagonal block (after the two planes).
// Double-float (FP32 pairs) throughout: the decision loop runs on every
// thread of the CTA, and FP64 instructions issue slowly on this GPU.
struct XDiag {
  double2 pe;                    // a recomputed pivot
  float uh[kXB], ul[kXB];        // uniforms
  float krh[kXB], krl[kXB];      // running pivots, real part
  float kih[kXB], kil[kXB];      // imaginary part
  float ds[kXB];                 // band scales
  float prh[kXB], prl[kXB];      // final pivots
  float pih[kXB], pil[kXB];
  float kabs[kXB];               // |K_jj|
  int kpx;                       // decision after a recompute
  unsigned char kp[kXB];
};
constexpr size_t kXPlane = sizeof(float) * kXB * kXBp;
constexpr size_t kXSmem1 = 2 * kXPlane + ((sizeof(XDiag) + 15) & ~size_t(15));
// tile phase: X, Z planes (32 x kXBp), staged panel operands (32 x kXPc),
// two 32 x 33 diagonal sub-blocks per plane pair, 1 / d of the outer block
constexpr int kXPc = kXB - 32;
constexpr size_t kXSmem2 = sizeof(float) * (4 * 32 * kXBp + 4 * 32 * kXPc + 4 * 32 * 33 + 2 * kXB);
constexpr size_t kXSmem = kXSmem1 > kXSmem2 ? kXSmem1 : kXSmem2;

__device__ inline float tf32_rna_x(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Tensor-core operand pieces of v at element off of the split buffers.
__device__ inline void x_split(int split, void* const* ops, int64_t off, float v) {
  if (split == kSplitBf16x6) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    static_cast<__nv_bfloat16*>(ops[0])[off] = b0;
    static_cast<__nv_bfloat16*>(ops[1])[off] = b1;
    static_cast<__nv_bfloat16*>(ops[2])[off] = __float2bfloat16_rn(r2);
  } else {
    const float h = tf32_rna_x(v);
    static_cast<float*>(ops[0])[off] = h;
    static_cast<float*>(ops[1])[off] = tf32_rna_x(v - h);
  }
}

// CTA 0: the diagonal block [q, q + kb), right-looking in shared memory, a
// decision before every column (FP64 recompute inside the band); every
// column of L, row of U~ and pivot goes to global memory in its step.
__device__ __noinline__ void xl_diag_block(const XArgs& a) {
  float* Br = reinterpret_cast<float*>(g_x_dyn);
  float* Bi = Br + kXB * kXBp;
  XDiag& S = *reinterpret_cast<XDiag*>(g_x_dyn + 2 * kXPlane);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int kb = a.kb;
  const int64_t q = a.q, lda = a.lda;
  float* Ar = a.Ar;
  float* Ai = a.Ai;
  for (int idx = tid; idx < kb * kb; idx += kXT) {
    const int r = idx % kb, c = idx / kb;
    const int64_t o = (q + r) + (q + c) * lda;
    cp_async4(&Br[r * kXBp + c], Ar + o, true);
    cp_async4(&Bi[r * kXBp + c], Ai + o, true);
  }
  cp_async_commit();
  for (int j = tid; j < kb; j += kXT) {
    const int64_t i = q + j;
    // (a given uniform is clamped to +-1e30, which decides like +-infinity
    // against any finite FP32 pivot and keeps the double-float finite)
    double ud = a.uniforms ? a.uniforms[i] : philox_uniform(a.seed, a.inst, (uint64_t)i);
    ud = fmin(fmax(ud, -1e30), 1e30);
    const f2 u = f2_from_double(ud);
    const double2 k = a.kd[i];
    const f2 kr = f2_from_double(k.x), ki = f2_from_double(k.y);
    S.uh[j] = u.hi;
    S.ul[j] = u.lo;
    S.krh[j] = kr.hi;
    S.krl[j] = kr.lo;
    S.kih[j] = ki.hi;
    S.kil[j] = ki.lo;
    S.ds[j] = (float)a.s[i];
    S.kabs[j] = (float)dabs(a.K[i + i * a.ldk]);
  }
  cp_async_wait_all();
  __syncthreads();
  int border = 0, rc_failed = 0, seq = 0;
  float max_ratio = 0.f;
  for (int j = 0; j < kb; ++j) {
    f2 pr = make_f2(S.krh[j], S.krl[j]), pim = make_f2(S.kih[j], S.kil[j]);
    const float uh = S.uh[j], ul = S.ul[j];
    const float tau = a.tau0 * sqrtf((float)(q + j + 1)) * (S.kabs[j] + S.ds[j]) + 0x1.0p-22f;
    // u - Re d in double-float (exact where the two are close); every thread
    // takes the same test on the same shared values
    const float du = (uh - pr.hi) + (ul - pr.lo);
    bool kp = du < 0.f;
    if (fabsf(du) <= tau) {
      // the pivots so far, out to global memory for the recompute
      for (int c = tid; c < j; c += kXT)
        a.piv[q + c] = make_double2(f2_to_double(make_f2(S.prh[c], S.prl[c])),
                                    f2_to_double(make_f2(S.pih[c], S.pil[c])));
      __threadfence();  // with the factor entries stored so far, before the request
      __syncthreads();
      if (wp == 0) {
        const double2 ph = make_double2(f2_to_double(pr), f2_to_double(pim));
        const double ud = (double)uh + (double)ul;
        double2 p2 = ph;
        double est = 0.0;
        const bool ok = xl_leader(a.xr, q + j, a.epoch, &seq, &p2, &est);
        if (lane == 0) {
          S.pe = ok ? p2 : ph;
          S.kpx = ud < (ok ? p2.x : ph.x) ? 1 : 0;
          border += 1;
          const float ratio = (float)(dabs(dsub(p2, ph)) / (double)tau);
          if (ok && ratio > max_ratio) max_ratio = ratio;
          if (!ok || est > fabs(ud - p2.x)) rc_failed = 1;
        }
      }
      __syncthreads();
      pr = f2_from_double(S.pe.x);
      pim = f2_from_double(S.pe.y);
      kp = S.kpx != 0;
    }
    if (!kp) pr = f2_add_f(pr, -1.f);
    const cf rp = crecipf(cmk(pr.hi, pim.hi));
    if (tid == 0) {
      a.keep[q + j] = kp ? 1 : 0;
      S.prh[j] = pr.hi;
      S.prl[j] = pr.lo;
      S.pih[j] = pim.hi;
      S.pil[j] = pim.lo;
      S.kp[j] = kp ? 1 : 0;
      const int64_t o = (q + j) * (1 + lda);
      Ar[o] = pr.hi;
      Ai[o] = pim.hi;
    }
    const int m = kb - j - 1;
    // column j of L and row j of U~ out; the running pivots of the later indices
    for (int t = tid; t < m; t += kXT) {
      const int k = j + 1 + t;
      const cf ujk = cmk(Br[j * kXBp + k], Bi[j * kXBp + k]);        // U(j, k)
      const cf l = cmul(cmk(Br[k * kXBp + j], Bi[k * kXBp + j]), rp);  // L(k, j)
      const cf ut = cmul(ujk, rp);                                    // U~(j, k)
      const int64_t oc = (q + k) + (q + j) * lda, orow = (q + j) + (q + k) * lda;
      Ar[oc] = l.x;
      Ai[oc] = l.y;
      Ar[orow] = ut.x;
      Ai[orow] = ut.y;
      // d_k -= L(k, j) U(j, k), the products formed exactly
      f2 kr = make_f2(S.krh[k], S.krl[k]), ki = make_f2(S.kih[k], S.kil[k]);
      kr = f2_sub_prod(kr, l.x, ujk.x);
      kr = f2_add_prod(kr, l.y, ujk.y);
      ki = f2_sub_prod(ki, l.x, ujk.y);
      ki = f2_sub_prod(ki, l.y, ujk.x);
      S.krh[k] = kr.hi;
      S.krl[k] = kr.lo;
      S.kih[k] = ki.hi;
      S.kil[k] = ki.lo;
      S.ds[k] += cabsf_(l) * cabsf_(ujk);
    }
    // the rest of the block: B[i][k] -= L(i, j) U(j, k), i, k > j; warp w
    // takes rows j + 1 + w + 8 r, lane l the columns j + 1 + l + 32 c (four
    // independent updates per row)
    {
      const int nc = (m + 31) >> 5;
      cf uk[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = j + 1 + lane + 32 * c;
        uk[c] = (c < nc && k < kb) ? cmk(Br[j * kXBp + k], Bi[j * kXBp + k]) : cmk(0.f, 0.f);
      }
#pragma unroll 2
      for (int i = j + 1 + wp; i < kb; i += 8) {
        const cf l = cmul(cmk(Br[i * kXBp + j], Bi[i * kXBp + j]), rp);
        float* br = Br + i * kXBp + j + 1 + lane;
        float* bi = Bi + i * kXBp + j + 1 + lane;
        cf v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          v[c] = (c < nc && j + 1 + lane + 32 * c < kb) ? cmk(br[32 * c], bi[32 * c]) : cmk(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c < nc && j + 1 + lane + 32 * c < kb) {
            const cf w = cfms(v[c], l, uk[c]);
            br[32 * c] = w.x;
            bi[32 * c] = w.y;
          }
        }
      }
    }
    __syncthreads();
  }
  // log P, counts and warnings of the block
  double lp = 0.0;
  int kept = 0, oor = 0, bad = 0;
  for (int j = tid; j < kb; j += kXT) {
    const double2 d = make_double2(f2_to_double(make_f2(S.prh[j], S.prl[j])),
                                   f2_to_double(make_f2(S.pih[j], S.pil[j])));
    a.piv[q + j] = d;
    const double2 pre = S.kp[j] ? d : make_double2(d.x + 1.0, d.y);
    lp += log(dabs(d));
    kept += S.kp[j];
    oor += (pre.x < -a.tol || pre.x > 1.0 + a.tol || fabs(pre.y) > a.tol) ? 1 : 0;
    bad |= (isfinite(d.x) && isfinite(d.y)) ? 0 : 1;
  }
  lp = warp_sum(lp);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kept += __shfl_xor_sync(kXF, kept, o);
    oor += __shfl_xor_sync(kXF, oor, o);
    bad |= __shfl_xor_sync(kXF, bad, o);
  }
  __shared__ double s_lp[kXT / 32];
  __shared__ int s_cnt[3][kXT / 32];
  if (lane == 0) {
    s_lp[wp] = lp;
    s_cnt[0][wp] = kept;
    s_cnt[1][wp] = oor;
    s_cnt[2][wp] = bad;
  }
  __syncthreads();
  if (tid == 0) {
    double Ls = 0.0;
    int Kc = 0, O = 0, B = 0;
    for (int w = 0; w < kXT / 32; ++w) {
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
    if (border) {
      atomicAdd(&r->n_borderline, border);
      if ((double)max_ratio > r->max_err_ratio) r->max_err_ratio = (double)max_ratio;
    }
    if (rc_failed) atomicOr(&r->status, DPP_RES_RECOMPUTE);
  }
}

// Substitution of 8 rows of one side against the unit triangular 32 x 32
// block T (lane c holds column c of every row; T[c * 33 + c0] is the
// coefficient of column c0 in column c, c0 < c), rows interleaved so that
// their chains overlap.
__device__ __forceinline__ void xl_solve8(float* Sr, float* Si, const int (&rows)[8], int D, int b,
                                          const float* Tr, const float* Ti) {
  const int lane = threadIdx.x & 31;
  cf x[8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
    x[r] = lane < b ? cmk(Sr[rows[r] * kXBp + D + lane], Si[rows[r] * kXBp + D + lane])
                    : cmk(0.f, 0.f);
  for (int c0 = 0; c0 < b - 1; ++c0) {
    const cf t = lane > c0 ? cmk(Tr[lane * 33 + c0], Ti[lane * 33 + c0]) : cmk(0.f, 0.f);
#pragma unroll
    for (int r = 0; r < 8; ++r) x[r] = cfms(x[r], cshfl(x[r], c0), t);
  }
  if (lane < b) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      Sr[rows[r] * kXBp + D + lane] = x[r].x;
      Si[rows[r] * kXBp + D + lane] = x[r].y;
    }
  }
}

// All CTAs, once the diagonal block is published: 32-index tiles beyond it.
// Rows: W = A[i, block] U~11^{-1}; columns: U = L11^{-1} A[block, i], M = U / d.
__device__ __noinline__ void xl_tiles(const XArgs& a) {
  float* Xr = reinterpret_cast<float*>(g_x_dyn);
  float* Xi = Xr + 32 * kXBp;
  float* Zr = Xi + 32 * kXBp;
  float* Zi = Zr + 32 * kXBp;
  float* Pr = Zi + 32 * kXBp;  // [32][kXPc]: U~ rows of the panel, later columns
  float* Pi = Pr + 32 * kXPc;
  float* Qr = Pi + 32 * kXPc;  // [32][kXPc]: L columns of the panel, later rows
  float* Qi = Qr + 32 * kXPc;
  float* Tur = Qi + 32 * kXPc;  // [32][33] U~ of the panel's diagonal block (by target column)
  float* Tui = Tur + 32 * 33;
  float* Tlr = Tui + 32 * 33;   // [32][33] L of it (by target row)
  float* Tli = Tlr + 32 * 33;
  float* rdr = Tli + 32 * 33;   // [kXB] 1 / d of the outer block
  float* rdi = rdr + kXB;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int kb = a.kb, np = (kb + 31) / 32;
  const int64_t q = a.q, qe = q + kb, n = a.n, lda = a.lda;
  const float* Ar = a.Ar;
  const float* Ai = a.Ai;
  for (int c = tid; c < kb; c += kXT) {
    const double2 d = a.piv[q + c];
    const cf r = crecipf(cmk((float)d.x, (float)d.y));
    rdr[c] = r.x;
    rdi[c] = r.y;
  }
  const int64_t ntiles = (n - qe + 31) / 32;
  for (int64_t tt = blockIdx.x; tt < ntiles; tt += gridDim.x) {
    const int64_t i0 = qe + 32 * tt;
    const int nr = (int)((n - i0) < 32 ? (n - i0) : 32);
    for (int idx = tid; idx < 32 * kb; idx += kXT) {
      const int r = idx & 31, c = idx >> 5;
      const int64_t o = r < nr ? (i0 + r) + (q + c) * lda : 0;
      cp_async4(&Xr[r * kXBp + c], Ar + o, r < nr);
      cp_async4(&Xi[r * kXBp + c], Ai + o, r < nr);
    }
    for (int idx = tid; idx < 32 * kb; idx += kXT) {
      const int c = idx % kb, r = idx / kb;
      const int64_t o = r < nr ? (q + c) + (i0 + r) * lda : 0;
      cp_async4(&Zr[r * kXBp + c], Ar + o, r < nr);
      cp_async4(&Zi[r * kXBp + c], Ai + o, r < nr);
    }
    cp_async_commit();
    for (int pk = 0; pk < np; ++pk) {
      const int D = 32 * pk;
      const int b = (kb - D) < 32 ? (kb - D) : 32;
      for (int idx = tid; idx < 1024; idx += kXT) {
        const int c = idx >> 5, c0 = idx & 31;
        const bool in = c < b && c0 < c;
        const int64_t ou = in ? (q + D + c0) + (q + D + c) * lda : 0;  // U~(D + c0, D + c)
        const int64_t ol = in ? (q + D + c) + (q + D + c0) * lda : 0;  // L(D + c, D + c0)
        cp_async4(&Tur[c * 33 + c0], Ar + ou, in);
        cp_async4(&Tui[c * 33 + c0], Ai + ou, in);
        cp_async4(&Tlr[c * 33 + c0], Ar + ol, in);
        cp_async4(&Tli[c * 33 + c0], Ai + ol, in);
      }
      cp_async_commit();
      cp_async_wait_all();
      __syncthreads();
      {
        int rows[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) rows[r] = (wp & 3) + 4 * r;
        if (wp < 4)
          xl_solve8(Xr, Xi, rows, D, b, Tur, Tui);
        else
          xl_solve8(Zr, Zi, rows, D, b, Tlr, Tli);
      }
      const int C0 = D + 32;
      const int nc = kb - C0;
      if (nc > 0) {
        for (int idx = tid; idx < 32 * nc; idx += kXT) {
          const int c0 = idx & 31, j = idx >> 5;
          const int64_t o = c0 < b ? (q + D + c0) + (q + C0 + j) * lda : 0;  // U~(D + c0, C0 + j)
          cp_async4(&Pr[c0 * kXPc + j], Ar + o, c0 < b);
          cp_async4(&Pi[c0 * kXPc + j], Ai + o, c0 < b);
        }
        for (int idx = tid; idx < 32 * nc; idx += kXT) {
          const int j = idx % nc, c0 = idx / nc;
          const int64_t o = c0 < b ? (q + C0 + j) + (q + D + c0) * lda : 0;  // L(C0 + j, D + c0)
          cp_async4(&Qr[c0 * kXPc + j], Ar + o, c0 < b);
          cp_async4(&Qi[c0 * kXPc + j], Ai + o, c0 < b);
        }
        cp_async_commit();
        cp_async_wait_all();
      }
      __syncthreads();
      if (nc > 0) {
        // S[r][C0 + j] -= sum_c0 S[r][D + c0] P[c0][j]; rows 4 ty.., columns tx + 32 jj
        // for the ncj 32-column chunks that exist
        const int ty = wp, tx = lane;
        const int ncj = (nc + 31) >> 5;
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
          float* Sr = side ? Zr : Xr;
          float* Si = side ? Zi : Xi;
          const float* Or = side ? Qr : Pr;
          const float* Oi = side ? Qi : Pi;
          cf acc[4][3];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) acc[i][jj] = cmk(0.f, 0.f);
#pragma unroll 2
          for (int c0 = 0; c0 < 32; ++c0) {
            cf w[4], m[3];
#pragma unroll
            for (int i = 0; i < 4; ++i)
              w[i] = cmk(Sr[(4 * ty + i) * kXBp + D + c0], Si[(4 * ty + i) * kXBp + D + c0]);
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              if (jj < ncj) {
                const int j = tx + 32 * jj;
                m[jj] = j < nc ? cmk(Or[c0 * kXPc + j], Oi[c0 * kXPc + j]) : cmk(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[i][jj] = cfma(acc[i][jj], w[i], m[jj]);
              }
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) {
              const int j = tx + 32 * jj;
              if (j < nc) {
                const int o = (4 * ty + i) * kXBp + C0 + j;
                Sr[o] -= acc[i][jj].x;
                Si[o] -= acc[i][jj].y;
              }
            }
        }
      }
      __syncthreads();
    }
    // L below the block (W / d) and U~ right of it (U / d)
    float* Awr = a.Ar;
    float* Awi = a.Ai;
    for (int idx = tid; idx < 32 * kb; idx += kXT) {
      const int r = idx & 31, c = idx >> 5;
      if (r < nr) {
        const cf l = cmul(cmk(Xr[r * kXBp + c], Xi[r * kXBp + c]), cmk(rdr[c], rdi[c]));
        const int64_t o = (i0 + r) + (q + c) * lda;
        Awr[o] = l.x;
        Awi[o] = l.y;
      }
    }
    for (int idx = tid; idx < 32 * kb; idx += kXT) {
      const int c = idx % kb, r = idx / kb;
      if (r < nr) {
        const cf w = cmk(Xr[r * kXBp + c], Xi[r * kXBp + c]);
        const cf mv = cmul(cmk(Zr[r * kXBp + c], Zi[r * kXBp + c]), cmk(rdr[c], rdi[c]));
        const int64_t o = (q + c) + (i0 + r) * lda;
        Awr[o] = mv.x;
        Awi[o] = mv.y;
        const int64_t off = (i0 + r) * (int64_t)kXLd + c;
        x_split(a.split, a.Wop, off, w.x);
        x_split(a.split, a.Wop, off + kb, w.y);
        x_split(a.split, a.M1op, off, mv.x);
        x_split(a.split, a.M1op, off + kb, -mv.y);
        x_split(a.split, a.M2op, off, mv.y);
        x_split(a.split, a.M2op, off + kb, mv.x);
      }
    }
    // running pivots and band scales: eight lanes per index, fixed-order tree
    {
      // (double-float sums of the exact FP32 products; the FP64 pipe is narrow)
      const int r = tid >> 3, part = tid & 7;
      f2 ax = make_f2(0.f, 0.f), ay = make_f2(0.f, 0.f);
      float ssum = 0.f;
      for (int c = part; c < kb; c += 8) {
        const cf w = cmk(Xr[r * kXBp + c], Xi[r * kXBp + c]);
        const cf mv = cmul(cmk(Zr[r * kXBp + c], Zi[r * kXBp + c]), cmk(rdr[c], rdi[c]));
        ax = f2_add_prod(ax, w.x, mv.x);
        ax = f2_add_prod(ax, -w.y, mv.y);
        ay = f2_add_prod(ay, w.x, mv.y);
        ay = f2_add_prod(ay, w.y, mv.x);
        ssum += cabsf_(w) * cabsf_(mv);
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const f2 ox = make_f2(__shfl_down_sync(kXF, ax.hi, o), __shfl_down_sync(kXF, ax.lo, o));
        const f2 oy = make_f2(__shfl_down_sync(kXF, ay.hi, o), __shfl_down_sync(kXF, ay.lo, o));
        const float os = __shfl_down_sync(kXF, ssum, o);
        if (part < o) {
          ax = f2_add(ax, ox);
          ay = f2_add(ay, oy);
          ssum += os;
        }
      }
      if (part == 0 && r < nr) {
        const int64_t i = i0 + r;
        const double2 k = a.kd[i];
        a.kd[i] = make_double2(k.x - f2_to_double(ax), k.y - f2_to_double(ay));
        a.s[i] += (double)ssum;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kXT, 1) k_cxlu_outer(XArgs a) {
  bool go;
  if (blockIdx.x == 0) {
    xl_diag_block(a);
    __syncthreads();
    if (threadIdx.x == 0 && !a.withhold) {
      __threadfence();
      st_release(&a.xr.rc.ctrl[kCtlDone], a.epoch);
    }
    go = a.withhold == 0;
  } else {
    go = xl_follower(a.xr, a.epoch);
  }
  if (!go || a.q + a.kb >= a.n) return;
  __syncthreads();
  xl_tiles(a);
}

// Planar FP32 copy of the whole of K (complex, column-major); running
// pivots K_ii and zero band scales.
__global__ void __launch_bounds__(256) k_convert_cx_full(const double2* K, int64_t ldk, float* Ar,
                                                         float* Ai, int64_t lda, int64_t n,
                                                         double2* kd, double* s) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const double2* col = K + j * ldk;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = col[i];
      Ar[i + j * lda] = (float)v.x;
      Ai[i + j * lda] = (float)v.y;
    }
    if (threadIdx.x == 0) {
      kd[j] = col[j];
      s[j] = 0.0;
    }
  }
}

// LU of K - 1_{Y^c}: L strictly below the diagonal, the FP64 pivots on it,
// U = D U~ above it (complex, interleaved).
__global__ void __launch_bounds__(256) k_export_cx_lu(const float* Ar, const float* Ai, int64_t lda,
                                                      const double2* piv, double2* F, int64_t ldf,
                                                      int64_t n) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = make_double2((double)Ar[i + j * lda], (double)Ai[i + j * lda]);
      F[i + j * ldf] = i > j ? v : (i == j ? piv[j] : dmul(piv[i], v));
    }
  }
}

struct XLayout {
  int64_t ld32;
  float *Ar, *Ai;
  void* Wop[3];
  void* M1op[3];
  void* M2op[3];
  double2 *kd, *piv;
  double* s;
  unsigned* flag;
  int* err;
  unsigned* ctrl;
  unsigned long long* words[8];  // x0, v1 (real, imaginary), x0 im, y0, y0 im, v1 im, v2, v2 im
  float *inv, *inv2;
  double2 *r, *s2;
  double* part;
};

bool carve_cxlu(Workspace& ws, int64_t n, XLayout* L) {
  L->ld32 = ((n + 31) / 32) * 32;
  if (L->ld32 < 32) L->ld32 = 32;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t nblk = (nn + 31) / 32;
  L->Ar = static_cast<float*>(ws.take(sizeof(float) * (size_t)L->ld32 * nn));
  L->Ai = static_cast<float*>(ws.take(sizeof(float) * (size_t)L->ld32 * nn));
  const size_t ob = sizeof(float) * nn * (size_t)kXLd;
  bool ok = L->Ar && L->Ai;
  for (int o = 0; o < 3; ++o) {
    L->Wop[o] = ws.take(ob);
    L->M1op[o] = ws.take(ob);
    L->M2op[o] = ws.take(ob);
    ok = ok && L->Wop[o] && L->M1op[o] && L->M2op[o];
  }
  L->kd = static_cast<double2*>(ws.take(sizeof(double2) * nn));
  L->piv = static_cast<double2*>(ws.take(sizeof(double2) * nn));
  L->s = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->flag = static_cast<unsigned*>(ws.take(256));
  L->err = L->flag ? reinterpret_cast<int*>(L->flag) + 16 : nullptr;
  L->ctrl = static_cast<unsigned*>(ws.take(256));
  for (int k = 0; k < 8; ++k) {
    L->words[k] = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
    ok = ok && L->words[k];
  }
  L->inv = static_cast<float*>(ws.take(sizeof(float) * 2048 * nblk));
  L->inv2 = static_cast<float*>(ws.take(sizeof(float) * 2048 * nblk));
  L->r = static_cast<double2*>(ws.take(sizeof(double2) * nn));
  L->s2 = static_cast<double2*>(ws.take(sizeof(double2) * nn));
  L->part = static_cast<double*>(ws.take(sizeof(double) * 8 * kMaxCoopCtas));
  return ok && L->kd && L->piv && L->s && L->flag && L->ctrl && L->inv && L->inv2 && L->r &&
         L->s2 && L->part;
}

}  // namespace

size_t ws_mixed_cxlu(int64_t n) {
  Workspace probe;
  probe.base = reinterpret_cast<char*>(256);
  probe.size = ~size_t(0) >> 2;
  XLayout L;
  carve_cxlu(probe, n, &L);
  return probe.used + 512;
}

cudaError_t sample_mixed_cxlu(const DrawArgs& a, Workspace ws) {
  const int64_t n = a.n;
  XLayout L;
  if (!carve_cxlu(ws, n, &L)) return cudaErrorInvalidValue;
  cudaError_t e = init_result(a.result, a.stream);
  if (e != cudaSuccess || n == 0) return e;
  if ((e = cudaMemsetAsync(L.flag, 0, 256, a.stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(L.ctrl, 0, 256, a.stream)) != cudaSuccess) return e;
  for (int k = 0; k < 8; ++k) {
    e = cudaMemsetAsync(L.words[k], 0, sizeof(unsigned long long) * (size_t)n, a.stream);
    if (e != cudaSuccess) return e;
  }
  const double2* K = static_cast<const double2*>(a.K);
  {
    ProfScope ps(kProfConvert, a.stream, 0.0, 24.0 * (double)n * (double)n);
    k_convert_cx_full<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        K, a.ld, L.Ar, L.Ai, L.ld32, n, L.kd, L.s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // cooperative capacity (and the shared-memory attribute), per device
  static int caps[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int& cap = caps[dev];
  if (cap == 0) {
    cudaError_t ea = cudaFuncSetAttribute(k_cxlu_outer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kXSmem);
    if (ea != cudaSuccess) return ea;
    DevInfo di;
    if ((ea = dev_info(&di)) != cudaSuccess) return ea;
    int per_sm = 0;
    ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cxlu_outer, kXT, kXSmem);
    if (ea != cudaSuccess) return ea;
    int c = per_sm * di.sm_count;
    if (c > kMaxCoopCtas) c = kMaxCoopCtas;
    if (c < 2) return cudaErrorLaunchOutOfResources;
    cap = c;
  }
  int grid = cap;
  if (g_tuning.max_ctas > 0 && grid > g_tuning.max_ctas) grid = g_tuning.max_ctas;
  if (grid < 2) grid = 2;  // the recompute needs at least one CTA besides the deciding one
  int NB = g_tuning.outer_block;
  if (NB > kXB) NB = kXB;
  NB = (NB / 32) * 32;
  if (NB < 32) NB = 32;
  const int split = a.precision == DPP_PREC_BF16X6 ? kSplitBf16x6 : kSplit3xTf32;
  unsigned epoch = 1;
  for (int64_t q = 0; q < n; q += NB, ++epoch) {
    const int kb = (int)((n - q) < NB ? (n - q) : NB);
    XArgs xa;
    xa.K = K;
    xa.ldk = a.ld;
    xa.Ar = L.Ar;
    xa.Ai = L.Ai;
    xa.lda = L.ld32;
    xa.n = n;
    xa.q = q;
    xa.kb = kb;
    xa.uniforms = a.uniforms;
    xa.seed = a.seed;
    xa.inst = a.instance;
    xa.keep = a.keep;
    xa.piv = L.piv;
    xa.kd = L.kd;
    xa.s = L.s;
    for (int o = 0; o < 3; ++o) {
      xa.Wop[o] = L.Wop[o];
      xa.M1op[o] = L.M1op[o];
      xa.M2op[o] = L.M2op[o];
    }
    xa.split = split;
    xa.res = a.result;
    xa.epoch = epoch;
    xa.tol = 1e-3;
    xa.tau0 = (float)(g_tuning.tau_safety * 0x1.0p-22);
    xa.withhold = g_tuning.fault_withhold;
    RecomputeArgs& rc = xa.xr.rc;
    rc.ctrl = L.ctrl;
    rc.xw = L.words[0];
    rc.vw = L.words[1];
    rc.inv = nullptr;
    rc.r = nullptr;
    rc.part = nullptr;
    rc.K = reinterpret_cast<const double*>(K);
    rc.ldk = a.ld;
    rc.A = L.Ar;
    rc.lda = L.ld32;
    rc.piv = nullptr;
    rc.keep = a.keep;
    rc.n = n;
    rc.q = q;
    rc.grid = grid;
    rc.res = a.result;
    rc.wait_ns = (unsigned long long)g_tuning.wait_ns;
    xa.xr.K = K;
    xa.xr.ldk = a.ld;
    xa.xr.Ar = L.Ar;
    xa.xr.Ai = L.Ai;
    xa.xr.lda = L.ld32;
    xa.xr.piv = L.piv;
    xa.xr.xwi = L.words[2];
    xa.xr.yw = L.words[3];
    xa.xr.ywi = L.words[4];
    xa.xr.vwi = L.words[5];
    xa.xr.v2w = L.words[6];
    xa.xr.v2wi = L.words[7];
    xa.xr.inv = L.inv;
    xa.xr.inv2 = L.inv2;
    xa.xr.r = L.r;
    xa.xr.s2 = L.s2;
    xa.xr.part = L.part;
    void* args[] = {&xa};
    {
      // the tiles' substitutions: 8 (n - q - kb) kb^2 real flops
      const double fl = 8.0 * (double)(n - q - kb) * (double)kb * (double)kb;
      ProfScope ps(kProfPanel, a.stream, fl, 0.0);
      e = cudaLaunchCooperativeKernel((const void*)k_cxlu_outer, dim3((unsigned)grid), dim3(kXT),
                                      args, kXSmem, a.stream);
    }
    if (e != cudaSuccess) return e;
    const int64_t r0 = q + kb;
    if (r0 < n) {
      // two real contractions of depth 2 kb over the trailing square
      const int64_t m = n - r0;
      const double fl = 4.0 * (double)m * (double)m * (double)kb;
      {
        ProfScope ps(kProfUpdateTc, a.stream, fl, 8.0 * (double)m * (double)m);
        e = outer_update_tc(split, L.Ar, L.ld32, n, r0, 2 * kb, L.Wop, L.M1op, kXLd, true, L.err,
                            a.stream);
        if (e != cudaSuccess) return e;
      }
      {
        ProfScope ps(kProfUpdateTc, a.stream, fl, 8.0 * (double)m * (double)m);
        e = outer_update_tc(split, L.Ai, L.ld32, n, r0, 2 * kb, L.Wop, L.M2op, kXLd, true, L.err,
                            a.stream);
        if (e != cudaSuccess) return e;
      }
    }
  }
  if (a.pivots_user) {
    e = cudaMemcpyAsync(a.pivots_user, L.piv, sizeof(double2) * n, cudaMemcpyDeviceToDevice,
                        a.stream);
    if (e != cudaSuccess) return e;
  }
  if (a.factor_out) {
    ProfScope ps(kProfOther, a.stream);
    k_export_cx_lu<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        L.Ar, L.Ai, L.ld32, L.piv, static_cast<double2*>(a.factor_out), a.ld, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dpp
