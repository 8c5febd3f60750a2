// Mixed-precision Hermitian DPP sampler for complex K (LDL^H form of
// Algorithm 1, blocked as in Algorithm 4), on the chunked panel pipeline of
// the real paths (dpp_mixed_lu.cu) in complex arithmetic.
//
// Storage: planar FP32 copies Ar, Ai of the lower triangle of K. With
// W = L D (D real), the Schur update of one block of columns is
//     A22 -= W L^H:   Re -= [Wr Wi] [Lr Li]^T,   Im -= [Wi -Wr] [Lr Li]^T,
// i.e. two real contractions of depth 2 kb, each run by the tensor-core update
// of the real path on the lower triangle. Pivots are real: a running diagonal
// kd_i = Re K_ii - sum_k Re(w_ik conj(l_ik)) in FP64 (double-float inside the
// decision loop), borderline band and FP64 recompute as in the real path:
//   d_g = Re K_gg - Re(k^H x0) - Re(x0^H r) - r^H A^{-1} r,
// A = K_P - 1_G, k = K[P, g], x0 = L_P^{-H} conj(l) (l = row g of L),
// r = k - A x0 in FP64 from K, r^H A^{-1} r ~ sum_c |(L_P^{-1} r)_c|^2 / d_c.
// Complex wavefront values travel as two id-tagged words (real, imaginary).
#include <cuda_bf16.h>
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"
#include "dpp_recompute.cuh"

namespace dpp {
namespace {

constexpr unsigned kCF = 0xffffffffu;
constexpr int kCT = 256;                   // threads per CTA
constexpr int kCNB = kMaxOuterBlock;       // columns of one outer block
constexpr int kCLd = 2 * kCNB;             // [re | im] row length of the operand buffers
constexpr int kCSlots = 7;                 // precomputed chunks per CTA (a lone helper
                                           // owns all 7 later chunks of an outer block)
constexpr int kBpSlot = kCSlots;           // slot of the next diagonal block
enum { kCtlChunkC = 16 };

struct cf {
  float x, y;
};
__device__ __forceinline__ cf mkc(float x, float y) { return {x, y}; }
// acc - a b
__device__ __forceinline__ cf c_sub_mul(cf acc, cf a, cf b) {
  return {fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y))};
}
// acc - a conj(b)
__device__ __forceinline__ cf c_sub_mulc(cf acc, cf a, cf b) {
  return {fmaf(-a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y))};
}
// acc + a b
__device__ __forceinline__ cf c_add_mul(cf acc, cf a, cf b) {
  return {fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y))};
}
// acc + conj(a) b
__device__ __forceinline__ cf c_add_cmul(cf acc, cf a, cf b) {
  return {fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y))};
}
__device__ __forceinline__ cf c_shfl(cf v, int src) {
  return {__shfl_sync(kCF, v.x, src), __shfl_sync(kCF, v.y, src)};
}

// ---------------------------------------------------------------------------
// Recompute state and FP64 recompute (complex, one-sided)
// ---------------------------------------------------------------------------
struct CxRc {
  RecomputeArgs rc;          // ctrl, xw (x0 real words), vw (v real words), part, piv, keep
  const double2* K;          // original K (complex, column-major)
  int64_t ldk;
  const float* Ar;
  const float* Ai;
  int64_t lda;
  unsigned long long* xwi;   // x0 imaginary words
  unsigned long long* vwi;   // v imaginary words
  float* inv;                // per 32-block: inverse of L_tt, real plane then imaginary
  double2* r;                // residual
};

__device__ __forceinline__ cf ld_l(const CxRc& c, int64_t i, int64_t j) {
  const int64_t o = i + j * c.lda;
  return {__ldcg(c.Ar + o), __ldcg(c.Ai + o)};
}

__device__ __forceinline__ cf word_c(const CxRc& c, int64_t idx, unsigned id, bool* live) {
  const RecomputeArgs& a = c.rc;
  const unsigned long long wr = ld_relaxed_u64(a.xw + idx);
  const unsigned long long wi = ld_relaxed_u64(c.xwi + idx);
  const float x = word_has(wr, id) ? __uint_as_float((unsigned)wr) : word_value_slow(a, a.xw + idx, id, live);
  const float y = word_has(wi, id) ? __uint_as_float((unsigned)wi) : word_value_slow(a, c.xwi + idx, id, live);
  return {x, y};
}

// Warp 0: the diagonal block L_tt (nr rows) and, in z, column `lane` of its
// unit lower inverse; the inverse is stored row-major (two planes).
__device__ __forceinline__ void cx_diag_inverse(const CxRc& c, int64_t t, int nr, float (*sDr)[33],
                                                float (*sDi)[33], cf (&z)[32]) {
  const int lane = threadIdx.x & 31;
  const int64_t r0 = 32 * t;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const bool ok = lane < nr && k < lane;
    const cf v = ok ? ld_l(c, r0 + lane, r0 + k) : mkc(0.f, 0.f);
    sDr[lane][k] = v.x;
    sDi[lane][k] = v.y;
  }
  __syncwarp();
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    cf s = mkc(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < i; ++k) s = c_add_mul(s, mkc(sDr[i][k], sDi[i][k]), z[k]);
    z[i] = (i == lane) ? mkc(1.f, 0.f) : (i < lane ? mkc(0.f, 0.f) : mkc(-s.x, -s.y));
  }
  float* dst = c.inv + (size_t)t * 2048;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    dst[i * 32 + lane] = z[i].x;
    dst[1024 + i * 32 + lane] = z[i].y;
  }
  __syncwarp();
}

// Whole warp: lanes < nvalid wait for the complex value at words[lane].
__device__ __forceinline__ bool warp_wait_c(const CxRc& c, const unsigned long long* wr,
                                            const unsigned long long* wi, int nvalid, unsigned id,
                                            cf* out) {
  float x = 0.f, y = 0.f;
  if (!warp_wait_words(c.rc, wr, nvalid, id, &x)) return false;
  if (!warp_wait_words(c.rc, wi, nvalid, id, &y)) return false;
  *out = mkc(x, y);
  return true;
}

__device__ __noinline__ bool cx_serve(const CxRc& c, unsigned id) {
  const RecomputeArgs& a = c.rc;
  __shared__ float sDr[32][33], sDi[32][33];
  __shared__ Handoff hfr, hfi;
  __shared__ double sRA[8][32][2], sRB[8][32][2];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t w = blockIdx.x - 1, nw = a.grid - 1;
  const int64_t g = (int64_t)ld_acquire(&a.ctrl[kCtlG]);
  const int64_t nblk = (g + 31) / 32;
  bool live = true;
  if (tid < 8) {
    hfr.ready[tid] = 0;
    hfi.ready[tid] = 0;
  }
  if (tid == 0) {
    hfr.cons = 0;
    hfi.cons = 0;
  }
  __syncthreads();

  // ---- R1: x0 = L_P^{-H} conj(l), owned blocks from the last one down ----
  {
    int i = 0;
    const int64_t tfirst = (w < nblk) ? w + ((nblk - 1 - w) / nw) * nw : -1;
    for (int64_t t = tfirst; t >= 0; t -= nw, ++i) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      cf z[32];
      cf f = mkc(0.f, 0.f);
      if (wp == 0) {
        cx_diag_inverse(c, t, nr, sDr, sDi, z);
        if (lane < nr) {
          const cf l = ld_l(c, g, 32 * t + lane);
          f = mkc(l.x, -l.y);
        }
      }
      // sources s = t + 1 + wp + 8 m, lane = row of block s:
      // sum_i conj(L(i, 32 t + col)) x_i
      cf acc[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[k] = mkc(0.f, 0.f);
      for (int64_t s = t + 1 + wp + (t + 1 + wp < nblk ? ((nblk - 2 - t - wp) / 8) * 8 : 0);
         s > t && s < nblk; s -= 8) {  // latest-published source last
        const int ns = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
        cf tile[32];
#pragma unroll
        for (int k = 0; k < 32; ++k)
          tile[k] = (lane < ns && k < nr) ? ld_l(c, 32 * s + lane, 32 * t + k) : mkc(0.f, 0.f);
        cf xs = mkc(0.f, 0.f);
        live = __all_sync(kCF, live);  // warp-uniform before the collective wait
        if (live && !warp_wait_c(c, a.xw + 32 * s, c.xwi + 32 * s, ns, id, &xs)) live = false;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = c_add_cmul(acc[k], tile[k], xs);
      }
      float ar[32], ai[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        ar[k] = acc[k].x;
        ai[k] = acc[k].y;
      }
      const float redr = transpose_reduce(ar, lane);
      const float redi = transpose_reduce(ai, lane);
      if (wp != 0) {
        handoff_put(a, hfr, i, wp, redr, &live);
        handoff_put(a, hfi, i, wp, redi, &live);
      } else {
        const float sr = handoff_take(a, hfr, i, redr, &live);
        const float si = handoff_take(a, hfi, i, redi, &live);
        const cf y = mkc(f.x - sr, f.y - si);
        // x_c = sum_k conj(inv[k][c]) y_k
        cf x = mkc(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 32; ++k) x = c_add_cmul(x, z[k], c_shfl(y, k));
        if (lane < nr) {
          st_relaxed_u64(a.xw + 32 * t + lane, make_word(id, x.x));
          st_relaxed_u64(c.xwi + 32 * t + lane, make_word(id, x.y));
        }
      }
    }
  }
  __syncthreads();
  if (tid < 8) {
    hfr.ready[tid] = 0;
    hfi.ready[tid] = 0;
  }
  if (tid == 0) {
    hfr.cons = 0;
    hfi.cons = 0;
  }
  __syncthreads();

  // ---- R2 + R3 per owned block, upwards ----
  double kx = 0.0, xr = 0.0, es = 0.0;
  {
    int i = 0;
    for (int64_t t = w; t < nblk; t += nw, ++i) {
      const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      const int64_t row = 32 * t + lane;
      const bool vi = lane < nr;
      // part A: columns [0, 32 t + nr), lanes = rows of block t
      double2 accA = make_double2(0.0, 0.0);
      for (int64_t m = wp; m <= t; m += 8) {
        const int64_t c0 = 32 * m;
        const int ncol = (int)((g - c0) < 32 ? (g - c0) : 32);
        const cf xl = lane < ncol ? word_c(c, c0 + lane, id, &live) : mkc(0.f, 0.f);
        const double xlr = (double)xl.x, xli = (double)xl.y;  // widened once per lane
        for (int k = 0; k < 32; ++k) {
          const int64_t col = c0 + k;
          double2 kv = make_double2(0.0, 0.0);
          if (vi && k < ncol) {
            if (col <= row) {
              kv = c.K[row + col * c.ldk];
            } else {
              const double2 q = c.K[col + row * c.ldk];
              kv = make_double2(q.x, -q.y);
            }
          }
          const double xr_ = __shfl_sync(kCF, xlr, k), xi_ = __shfl_sync(kCF, xli, k);
          accA.x = fma(kv.x, xr_, fma(-kv.y, xi_, accA.x));
          accA.y = fma(kv.x, xi_, fma(kv.y, xr_, accA.y));
        }
      }
      sRA[wp][lane][0] = accA.x;
      sRA[wp][lane][1] = accA.y;
      // part B: columns >= 32 t + 32, lanes = those columns (rows of K):
      // A(32 t + k, col) = conj(K[col, 32 t + k]); two halves of 16 rows
      for (int half = 0; half < 2; ++half) {
        double br[16], bi[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) br[k] = bi[k] = 0.0;
        for (int64_t c0 = 32 * t + 32 + 32 * wp; c0 < g; c0 += 256) {
          const int64_t col = c0 + lane;
          const bool vc = col < g;
          const cf xc = vc ? word_c(c, col, id, &live) : mkc(0.f, 0.f);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int kk = 16 * half + k;
            double2 q = make_double2(0.0, 0.0);
            if (vc && kk < nr) q = c.K[col + (32 * t + kk) * c.ldk];
            // conj(q) * xc
            br[k] = fma(q.x, (double)xc.x, fma(q.y, (double)xc.y, br[k]));
            bi[k] = fma(q.x, (double)xc.y, fma(-q.y, (double)xc.x, bi[k]));
          }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const double sr = warp_sum(br[k]), sim = warp_sum(bi[k]);
          if (lane == 16 * half + k) {
            sRB[wp][lane][0] = sr;
            sRB[wp][lane][1] = sim;
          }
        }
      }
      __syncthreads();
      if (wp == 0 && vi) {
        double tr = 0.0, ti = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          tr += sRA[k][lane][0] + sRB[k][lane][0];
          ti += sRA[k][lane][1] + sRB[k][lane][1];
        }
        const cf x32 = word_c(c, row, id, &live);
        const double xi_r = (double)x32.x, xi_i = (double)x32.y;
        const double2 kg = c.K[g + row * c.ldk];  // k_i = conj(K[g, i])
        const double ki_r = kg.x, ki_i = -kg.y;
        double rr = ki_r - tr, ri = ki_i - ti;
        if (a.keep[row] == 0) {
          rr += xi_r;
          ri += xi_i;
        }
        c.r[row] = make_double2(rr, ri);
        kx += ki_r * xi_r + ki_i * xi_i;  // Re(conj(k_i) x_i)
        xr += xi_r * rr + xi_i * ri;      // Re(conj(x_i) r_i)
      }
      __syncthreads();
      // R3: v_t = inv_t (r_t - sum_{s < t} L_ts v_s), lanes = rows of block t
      cf invrow[32];
      if (wp == 0) {
        const float* src = c.inv + (size_t)t * 2048 + lane * 32;
#pragma unroll
        for (int k = 0; k < 32; ++k) invrow[k] = mkc(src[k], src[1024 + k]);
      }
      cf acc = mkc(0.f, 0.f);
      const int64_t slast = t - 1 - wp;
      if (slast >= 0) {
        for (int64_t s = slast % 8; s <= slast; s += 8) {
          cf tile[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) tile[k] = vi ? ld_l(c, row, 32 * s + k) : mkc(0.f, 0.f);
          cf vs = mkc(0.f, 0.f);
          live = __all_sync(kCF, live);  // warp-uniform before the collective wait
          if (live && !warp_wait_c(c, a.vw + 32 * s, c.vwi + 32 * s, 32, id, &vs)) live = false;
#pragma unroll
          for (int k = 0; k < 32; ++k) acc = c_add_mul(acc, tile[k], c_shfl(vs, k));
        }
      }
      if (wp != 0) {
        handoff_put(a, hfr, i, wp, acc.x, &live);
        handoff_put(a, hfi, i, wp, acc.y, &live);
      } else {
        const float sr = handoff_take(a, hfr, i, acc.x, &live);
        const float si = handoff_take(a, hfi, i, acc.y, &live);
        const double2 rv = vi ? c.r[row] : make_double2(0.0, 0.0);
        const cf y = mkc((float)(rv.x - (double)sr), (float)(rv.y - (double)si));
        cf v = mkc(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 32; ++k) v = c_add_mul(v, invrow[k], c_shfl(y, k));
        if (vi) {
          st_relaxed_u64(a.vw + row, make_word(id, v.x));
          st_relaxed_u64(c.vwi + row, make_word(id, v.y));
          es += ((double)v.x * v.x + (double)v.y * v.y) / a.piv[row];
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

__device__ inline bool cx_follower(const CxRc& c, unsigned epoch, int* s_ok, unsigned max_sleep) {
  const RecomputeArgs& a = c.rc;
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
      if (!cx_serve(c, id)) {
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

__device__ inline bool cx_wait_short(const RecomputeArgs& a, const unsigned* flag, unsigned target) {
  if (ld_acquire(flag) >= target) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (ld_acquire(flag) >= target) return true;
    if ((it & 15) == 0 && rc_give_up(a, t0)) return false;
    __nanosleep(64);
  }
}

// Leader (warp 0 of CTA 0): pivot g in FP64; the factor rows of indices < g
// must be in global memory. Lane-uniform results.
__device__ inline bool cx_leader(const CxRc& c, int64_t g, unsigned epoch, int* seq, double* pe,
                                 double* est) {
  const RecomputeArgs& a = c.rc;
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
  ok = __shfl_sync(kCF, ok, 0);
  double kx = 0.0, xr = 0.0, e = 0.0;
  if (ok && lane == 0) {
    for (int w = 0; w < a.grid - 1; ++w) {
      kx += __ldcg(&a.part[4 * w + 0]);
      xr += __ldcg(&a.part[4 * w + 1]);
      e += __ldcg(&a.part[4 * w + 2]);
    }
  }
  const double kgg = c.K[g + g * c.ldk].x;
  double d2 = kgg - kx - xr - e;
  double er = fabs(e) * 1e-2 + 1e-12 * (1.0 + fabs(kgg) + fabs(kx) + fabs(xr));
  d2 = __shfl_sync(kCF, d2, 0);
  er = __shfl_sync(kCF, er, 0);
  if (ok) {
    *pe = d2;
    *est = er;
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Panel kernel
// ---------------------------------------------------------------------------
struct CxArgs {
  const double2* K;
  int64_t ldk;
  float* Ar;
  float* Ai;
  int64_t lda, n, q;
  int kb;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double* piv;
  double* kd;
  double* s;
  float* Wf;  // row-major [n x 512]: W = L D of the outer block's kb columns, re at
              // [0, kb), im at [kb, 2 kb)
  float* Lf;  // the same for L
  void* W1[3];  // splits of [Wr | Wi]
  void* W2[3];  // splits of [Wi | -Wr]
  void* Lo[3];  // splits of [Lr | Li]
  int split;
  dpp_result* res;
  unsigned epoch0;
  double tol;
  float tau0;
  float* Bbuf;  // [2 x 32 x 32] next diagonal block (real plane, imaginary plane)
  int nh;
  CxRc cr;
};

constexpr size_t kCTile = sizeof(float) * 32 * 33;
struct CxSmem {
  float d[32], rd[32];
  float Lr[32][33], Li[32][33];  // L of the published panel's diagonal block
  float st[10][32][33];          // staging: W rows (128 x re, im), L panel rows (re, im)
};
constexpr size_t kCxBase = (sizeof(CxSmem) + 15) & ~size_t(15);
// slot i: X (re, im) then Z (re, im); slot kBpSlot holds the next diagonal block
constexpr size_t kCxDyn = kCxBase + (size_t)(kCSlots + 1) * 4 * kCTile;
extern __shared__ __align__(16) unsigned char g_cx_dyn[];
__device__ __forceinline__ CxSmem& cxs() { return *reinterpret_cast<CxSmem*>(g_cx_dyn); }
__device__ __forceinline__ float (*cslot(int i, int plane))[33] {
  return reinterpret_cast<float (*)[33]>(g_cx_dyn + kCxBase + ((size_t)4 * i + plane) * kCTile);
}
__device__ __forceinline__ float (*cstage(int row))[33] { return &cxs().st[0][0] + row; }

struct CxLog {
  double d[kMaxOuterBlock];
  unsigned char kp[kMaxOuterBlock];
  int border;
  float max_ratio;
  int rc_failed;
};
__shared__ CxLog g_cxlog;
__shared__ int g_cx_ok;

__device__ inline float tf32_cx(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ inline void put_split(int split, void* const* ops, int64_t off, float v) {
  if (split == kSplitBf16x6) {
    const __nv_bfloat16 b0 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(b0);
    const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(b1);
    static_cast<__nv_bfloat16*>(ops[0])[off] = b0;
    static_cast<__nv_bfloat16*>(ops[1])[off] = b1;
    static_cast<__nv_bfloat16*>(ops[2])[off] = __float2bfloat16_rn(r2);
  } else {
    const float h = tf32_cx(v);
    static_cast<float*>(ops[0])[off] = h;
    static_cast<float*>(ops[1])[off] = tf32_cx(v - h);
  }
}

// The published panel [p, p + b): L11 and the FP32 pivots.
__device__ void cx_load_panel(const CxArgs& a, int64_t p, int b) {
  CxSmem& S = cxs();
  for (int idx = threadIdx.x; idx < 1024; idx += kCT) {
    const int r = idx & 31, c = idx >> 5;
    const bool ok = r < b && c < r;
    const int64_t o = (p + r) + (p + c) * a.lda;
    S.Lr[r][c] = ok ? __ldcg(&a.Ar[o]) : 0.f;
    S.Li[r][c] = ok ? __ldcg(&a.Ai[o]) : 0.f;
  }
  if (threadIdx.x < 32) {
    const int c = threadIdx.x;
    const float d = c < b ? (float)__ldcg(&a.piv[p + c]) : 1.f;
    S.d[c] = d;
    S.rd[c] = c < b ? 1.f / d : 0.f;
  }
}

// Chunks c_m = c_first + m c_stride (m < cnt) into slots slot0 + m:
//   X[r][c] = A[c_m + r, p + c] - sum_{t < D} W[c_m + r, t] conj(L[p + c, t])
// (for a diagonal block, c_m == p, the upper half mirrored from the lower).
__device__ void cx_chunks_left(const CxArgs& a, int64_t p, int b, int D, int64_t c_first,
                               int64_t c_stride, int cnt, int slot0) {
  const int tid = threadIdx.x;
  const int64_t lda = a.lda, n = a.n;
  for (int m = 0; m < cnt; ++m) {
    const int64_t c0 = c_first + m * c_stride;
    const int nc = (int)((n - c0) < 32 ? (n - c0) : 32);
    float (*Xr)[33] = cslot(slot0 + m, 0);
    float (*Xi)[33] = cslot(slot0 + m, 1);
    for (int idx = tid; idx < 1024; idx += kCT) {
      const int r = idx & 31, c = idx >> 5;
      float vr = 0.f, vi = 0.f;
      if (r < nc && c < b) {
        if (c0 == p && c > r) {
          const int64_t o = (p + c) + (p + r) * lda;
          vr = __ldcg(&a.Ar[o]);
          vi = -__ldcg(&a.Ai[o]);
        } else {
          const int64_t o = (c0 + r) + (p + c) * lda;
          vr = __ldcg(&a.Ar[o]);
          vi = (c0 == p && c == r) ? 0.f : __ldcg(&a.Ai[o]);
        }
      }
      Xr[r][c] = vr;
      Xi[r][c] = vi;
    }
  }
  __syncthreads();
  float (*WAr)[33] = cstage(0);
  float (*WAi)[33] = cstage(128);
  float (*LBr)[33] = cstage(256);
  float (*LBi)[33] = cstage(288);
  const int ty = tid >> 3, tx = tid & 7;
  for (int t0 = 0; t0 < D; t0 += 32) {
    for (int idx = tid; idx < 1024; idx += kCT) {
      const int rr = idx >> 5, tt = idx & 31;
      const bool ok = rr < b;
      LBr[rr][tt] = ok ? __ldcg(&a.Lf[(p + rr) * kCLd + t0 + tt]) : 0.f;
      LBi[rr][tt] = ok ? __ldcg(&a.Lf[(p + rr) * kCLd + a.kb + t0 + tt]) : 0.f;
    }
    for (int m0 = 0; m0 < cnt; m0 += 4) {
      for (int idx = tid; idx < 4096; idx += kCT) {
        const int rr = idx >> 5, tt = idx & 31;
        const int m = m0 + (rr >> 5);
        const int64_t row = c_first + m * c_stride + (rr & 31);
        const bool ok = m < cnt && row < n;
        WAr[rr][tt] = ok ? __ldcg(&a.Wf[row * kCLd + t0 + tt]) : 0.f;
        WAi[rr][tt] = ok ? __ldcg(&a.Wf[row * kCLd + a.kb + t0 + tt]) : 0.f;
      }
      __syncthreads();
      cf acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = mkc(0.f, 0.f);
#pragma unroll 2
      for (int tt = 0; tt < 32; ++tt) {
        cf wa[4], lb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) wa[i] = mkc(WAr[4 * ty + i][tt], WAi[4 * ty + i][tt]);
#pragma unroll
        for (int j = 0; j < 4; ++j) lb[j] = mkc(LBr[4 * tx + j][tt], LBi[4 * tx + j][tt]);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // acc += wa conj(lb)
            acc[i][j].x = fmaf(wa[i].x, lb[j].x, fmaf(wa[i].y, lb[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(wa[i].y, lb[j].x, fmaf(-wa[i].x, lb[j].y, acc[i][j].y));
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int rr = 4 * ty + i, m = m0 + (rr >> 5), r = rr & 31;
        if (m < cnt) {
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            cslot(slot0 + m, 0)[r][4 * tx + j] -= acc[i][j].x;
            cslot(slot0 + m, 1)[r][4 * tx + j] -= acc[i][j].y;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Solves (W L11^H = X, L = W / d) and stores of cnt left-looked chunks in
// slots slot0.. (W stays in X, L goes to Z).
__device__ void cx_chunks_solve(const CxArgs& a, int64_t p, int b, int64_t c_first,
                                int64_t c_stride, int cnt, int slot0, bool splits) {
  CxSmem& S = cxs();
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int64_t n = a.n;
  const int D = (int)(p - a.q);
  for (int m = wp; m < cnt; m += kCT / 32) {
    float (*Xr)[33] = cslot(slot0 + m, 0);
    float (*Xi)[33] = cslot(slot0 + m, 1);
    float (*Zr)[33] = cslot(slot0 + m, 2);
    float (*Zi)[33] = cslot(slot0 + m, 3);
    cf y[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) y[c] = mkc(Xr[lane][c], Xi[lane][c]);
#pragma unroll
    for (int c = 1; c < 32; ++c) {
#pragma unroll
      for (int k = 0; k < c; ++k) y[c] = c_sub_mulc(y[c], y[k], mkc(S.Lr[c][k], S.Li[c][k]));
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      Xr[lane][c] = y[c].x;
      Xi[lane][c] = y[c].y;
      Zr[lane][c] = y[c].x * S.rd[c];
      Zi[lane][c] = y[c].y * S.rd[c];
    }
  }
  __syncthreads();
  for (int e = tid; e < 32 * cnt; e += kCT) {
    const int m = e >> 5, r = e & 31;
    const int64_t row = c_first + m * c_stride + r;
    if (row < n) {
      f2 dsum = {0.f, 0.f};
      float ssum = 0.f;
      for (int c = 0; c < b; ++c) {
        const float wr = cslot(slot0 + m, 0)[r][c], wi = cslot(slot0 + m, 1)[r][c];
        const float lr = cslot(slot0 + m, 2)[r][c], li = cslot(slot0 + m, 3)[r][c];
        // Re(w conj(l)) = wr lr + wi li
        dsum = f2_add_prod(dsum, wr, lr);
        dsum = f2_add_prod(dsum, wi, li);
        ssum += fabsf(wr * lr + wi * li);
      }
      a.kd[row] -= f2_to_double(dsum);
      a.s[row] += (double)ssum;
    }
  }
  const int64_t lda = a.lda;
  for (int m = 0; m < cnt; ++m) {
    const int64_t c0 = c_first + m * c_stride;
    const int nc = (int)((n - c0) < 32 ? (n - c0) : 32);
    for (int idx = tid; idx < 1024; idx += kCT) {
      {
        const int r = idx & 31, c = idx >> 5;
        if (r < nc && c < b) {
          const int64_t o = (c0 + r) + (p + c) * lda;
          a.Ar[o] = cslot(slot0 + m, 2)[r][c];
          a.Ai[o] = cslot(slot0 + m, 3)[r][c];
        }
      }
      {
        const int c = idx & 31, r = idx >> 5;
        if (r < nc && c < b) {
          const float wr = cslot(slot0 + m, 0)[r][c], wi = cslot(slot0 + m, 1)[r][c];
          const float lr = cslot(slot0 + m, 2)[r][c], li = cslot(slot0 + m, 3)[r][c];
          const int64_t off = (c0 + r) * kCLd + D + c;
          a.Wf[off] = wr;
          a.Wf[off + a.kb] = wi;
          a.Lf[off] = lr;
          a.Lf[off + a.kb] = li;
          if (splits) {
            put_split(a.split, a.W1, off, wr);
            put_split(a.split, a.W1, off + a.kb, wi);
            put_split(a.split, a.W2, off, wi);
            put_split(a.split, a.W2, off + a.kb, -wr);
            put_split(a.split, a.Lo, off, lr);
            put_split(a.split, a.Lo, off + a.kb, li);
          }
        }
      }
    }
  }
  __syncthreads();
}

// Next diagonal block: slot kBpSlot (left-looking part) minus the just-solved
// chunk's W conj(L)^T against the current panel, into Bbuf.
__device__ void cx_next_block(const CxArgs& a, int slot, int b) {
  const int tid = threadIdx.x, r = tid & 31, cg = tid >> 5;
  float (*Wr)[33] = cslot(slot, 0);
  float (*Wi)[33] = cslot(slot, 1);
  float (*Lr)[33] = cslot(slot, 2);
  float (*Li)[33] = cslot(slot, 3);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = cg + 8 * j;
    cf v = mkc(cslot(kBpSlot, 0)[r][c], cslot(kBpSlot, 1)[r][c]);
    for (int t = 0; t < b; ++t) v = c_sub_mulc(v, mkc(Wr[r][t], Wi[r][t]), mkc(Lr[c][t], Li[c][t]));
    a.Bbuf[r * 32 + c] = v.x;
    a.Bbuf[1024 + r * 32 + c] = v.y;
  }
  __syncthreads();
}

// Decisions of panel [p, p + b) on the Hermitian block in slot kBpSlot (X
// planes), by all 8 warps of CTA 0 (as in the real chunked pipeline; the
// pivots are real, the multipliers complex).
__device__ __noinline__ void cx_decide(const CxArgs& a, int64_t p, int b, unsigned epoch) {
  CxLog& lg = g_cxlog;
  float (*Xr)[33] = cslot(kBpSlot, 0);
  float (*Xi)[33] = cslot(kBpSlot, 1);
  __shared__ float s_lr[2][32], s_li[2][32];
  __shared__ float s_df[2];
  __shared__ int s_stop[2];
  __shared__ float s_ddh[32], s_ddl[32], s_si[32];
  __shared__ unsigned char s_kp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t i = p + lane;
  const bool vi = lane < b;
  f2 dd = vi ? f2_from_double(__ldcg(&a.kd[i])) : make_f2(0.f, 0.f);
  float si = vi ? (float)__ldcg(&a.s[i]) : 0.f;
  const float kf = vi ? (float)a.K[i + i * a.ldk].x : 0.f;
  const float sq = sqrtf((float)(i + 1));
  const double u = vi ? (a.uniforms ? a.uniforms[i] : philox_uniform(a.seed, a.inst, (uint64_t)i))
                      : 2.0;
  const float uf = (float)u;
  bool mykeep = false;
  int stop = -1;
  cf v[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int c = 4 * warp + j;
    v[j] = (vi && c < b) ? mkc(Xr[lane][c], Xi[lane][c]) : mkc(0.f, 0.f);
  }
  for (int J = 0; J < b; ++J) {
    const int buf = J & 1;
    if (warp == (J >> 2)) {
      const float ph = __shfl_sync(kCF, dd.hi, J);
      const float uj = __shfl_sync(kCF, uf, J);
      const float tau = a.tau0 * __shfl_sync(kCF, sq, J) *
                            (fabsf(__shfl_sync(kCF, kf, J)) + __shfl_sync(kCF, si, J)) +
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
        const cf colJ = jj == 0 ? v[0] : (jj == 1 ? v[1] : (jj == 2 ? v[2] : v[3]));
        s_lr[buf][lane] = colJ.x * rd;
        s_li[buf][lane] = colJ.y * rd;
        if (lane == 0) s_df[buf] = df;
      }
      if (lane == 0) s_stop[buf] = border ? 1 : 0;
    }
    __syncthreads();
    if (s_stop[buf]) {
      stop = J;
      break;
    }
    const cf l = mkc(s_lr[buf][lane], s_li[buf][lane]);
    const float df = s_df[buf];
    const bool act = (lane > J) && vi;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = 4 * warp + j;
      const cf pk = c_shfl(v[j], J);  // row J's entry in column c
      cf x = v[j];
      if (act && c > J) x = c_sub_mul(x, l, pk);
      if (act && c == J) x = l;
      if (lane == J && c == J) x = mkc(df, 0.f);
      v[j] = x;
      if (lane == c && act) {  // row c's running pivot: - Re(l pk)
        dd = f2_sub_prod(dd, l.x, pk.x);
        dd = f2_sub_prod(dd, -l.y, pk.y);
        si += fabsf(l.x * pk.x - l.y * pk.y);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    Xr[lane][4 * warp + j] = v[j].x;
    Xi[lane][4 * warp + j] = v[j].y;
  }
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
  float* Ar = a.Ar;
  float* Ai = a.Ai;
  const int64_t lda = a.lda;
  if (stop >= 0) {
    if (lane < stop) {
      a.piv[i] = f2_to_double(dd);
      a.keep[i] = mykeep ? 1 : 0;
    }
    int seq = 0;
    for (int J = stop; J < b; ++J) {
      const double ph = (double)__shfl_sync(kCF, dd.hi, J) + (double)__shfl_sync(kCF, dd.lo, J);
      const double uj = __shfl_sync(kCF, u, J);
      const float tau = a.tau0 * __shfl_sync(kCF, sq, J) *
                            (fabsf(__shfl_sync(kCF, kf, J)) + __shfl_sync(kCF, si, J)) +
                        0x1.0p-22f;
      double pe = ph;
      if (fabs(uj - ph) <= (double)tau) {
        // rows [p, p + J] of L so far, out to global memory
        if (lane <= J) {
          for (int c = 0; c < lane; ++c) {
            Ar[(p + lane) + (p + c) * lda] = Xr[lane][c];
            Ai[(p + lane) + (p + c) * lda] = Xi[lane][c];
          }
        }
        double est = 0.0;
        const bool ok = cx_leader(a.cr, p + J, epoch, &seq, &pe, &est);
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
        const cf l = mkc(Xr[lane][J] * rdf, Xi[lane][J] * rdf);
        for (int c = J + 1; c < b; ++c) {
          const cf x = c_sub_mul(mkc(Xr[lane][c], Xi[lane][c]), l, mkc(Xr[J][c], Xi[J][c]));
          Xr[lane][c] = x.x;
          Xi[lane][c] = x.y;
        }
        const cf uji = mkc(Xr[J][lane], Xi[J][lane]);
        dd = f2_sub_prod(dd, l.x, uji.x);
        dd = f2_sub_prod(dd, -l.y, uji.y);
        si += fabsf(l.x * uji.x - l.y * uji.y);
        Xr[lane][J] = l.x;
        Xi[lane][J] = l.y;
      }
      __syncwarp();
      if (lane == J) {
        Xr[J][J] = df;
        Xi[J][J] = 0.f;
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
    for (int c = 0; c <= lane; ++c) {
      Ar[i + (p + c) * lda] = Xr[lane][c];
      Ai[i + (p + c) * lda] = c == lane ? 0.f : Xi[lane][c];
    }
  }
  __syncwarp();
}

__device__ __forceinline__ int cx_owner(int j, int nh) { return 1 + (j - 1) % nh; }

__global__ void __launch_bounds__(kCT, 1) k_cx_outer(CxArgs a) {
  int& s_ok = g_cx_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = (a.kb + 31) / 32;
  const int64_t q = a.q, qe = q + a.kb;
  const RecomputeArgs& rc = a.cr.rc;
  const int nh = a.nh;

  if (blockIdx.x == 0) {
    CxLog& lg = g_cxlog;
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
        cx_chunks_left(a, p, b, 0, p, 32, 1, kBpSlot);
      } else {
        if (tid == 0) s_ok = cx_wait_short(rc, &rc.ctrl[kCtlChunkC + k], epoch - 1) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
          alive = false;
          break;
        }
        for (int idx = tid; idx < 1024; idx += kCT) {
          cslot(kBpSlot, 0)[idx >> 5][idx & 31] = __ldcg(&a.Bbuf[idx]);
          cslot(kBpSlot, 1)[idx >> 5][idx & 31] = __ldcg(&a.Bbuf[1024 + idx]);
        }
        __syncthreads();
      }
      cx_decide(a, p, b, epoch);
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        st_release(&rc.ctrl[kCtlDone], epoch);
      }
    }
    __syncthreads();
    double lp = 0.0;
    int kept = 0, oor = 0, bad = 0;
    for (int i = tid; i < a.kb; i += kCT) {
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
      kept += __shfl_xor_sync(kCF, kept, o);
      oor += __shfl_xor_sync(kCF, oor, o);
      bad |= __shfl_xor_sync(kCF, bad, o);
    }
    __shared__ double s_lp[kCT / 32];
    __shared__ int s_cnt[3][kCT / 32];
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
      for (int w = 0; w < kCT / 32; ++w) {
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
    // ---- helper h: the outer block's chunks j with owner h ----
    const int h = blockIdx.x;
    for (int k = 0; k < np; ++k) {
      const int64_t p = q + 32 * k;
      const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
      const unsigned epoch = a.epoch0 + (unsigned)k;
      const int D = 32 * k;
      if (k > 0) {
        if (tid == 0) s_ok = cx_wait_short(rc, &rc.ctrl[kCtlChunkC + k], epoch - 1) ? 1 : 0;
        __syncthreads();
        if (!s_ok) return;
      }
      int ns = 0;
      for (int j = k + 1; j < np; ++j) {
        if (cx_owner(j, nh) != h) continue;
        cx_chunks_left(a, p, b, D, q + 32 * j, 32, 1, ns);
        if (j == k + 1) {
          const int bj = (int)((qe - (q + 32 * j)) < 32 ? (qe - (q + 32 * j)) : 32);
          cx_chunks_left(a, q + 32 * j, bj, D, q + 32 * j, 32, 1, kBpSlot);
        }
        ++ns;
      }
      if (!cx_follower(a.cr, epoch, &s_ok, 128)) return;
      cx_load_panel(a, p, b);
      __syncthreads();
      ns = 0;
      for (int j = k + 1; j < np; ++j) {
        if (cx_owner(j, nh) != h) continue;
        cx_chunks_solve(a, p, b, q + 32 * j, 32, 1, ns, false);
        if (j == k + 1) cx_next_block(a, ns, b);
        if (tid == 0) {
          __threadfence();
          st_release(&rc.ctrl[kCtlChunkC + j], epoch);
        }
        ++ns;
      }
      __syncthreads();
    }
    return;
  }

  // ---- workers: chunks beyond the outer block ----
  const int64_t nwk = (int64_t)gridDim.x - nh - 1, w = (int64_t)blockIdx.x - nh - 1;
  const int64_t c_first = qe + 32 * w, c_stride = 32 * nwk;
  const int total = c_first < a.n ? (int)((a.n - 1 - c_first) / c_stride + 1) : 0;
  const int first = total < kCSlots ? total : kCSlots;
  for (int k = 0; k < np; ++k) {
    const int64_t p = q + 32 * k;
    const int b = (int)((qe - p) < 32 ? (qe - p) : 32);
    const unsigned epoch = a.epoch0 + (unsigned)k;
    const int D = 32 * k;
    if (k > 0) {
      if (tid == 0) s_ok = rc_wait_geq(rc, &rc.ctrl[kCtlChunkC + k], epoch - 1) ? 1 : 0;
      __syncthreads();
      if (!s_ok) return;
    }
    cx_chunks_left(a, p, b, D, c_first, c_stride, first, 0);
    if (!cx_follower(a.cr, epoch, &s_ok, 1024)) return;
    cx_load_panel(a, p, b);
    __syncthreads();
    cx_chunks_solve(a, p, b, c_first, c_stride, first, 0, true);
    for (int m0 = first; m0 < total; m0 += kCSlots) {
      const int cnt = (total - m0) < kCSlots ? (total - m0) : kCSlots;
      cx_chunks_left(a, p, b, D, c_first + m0 * c_stride, c_stride, cnt, 0);
      cx_chunks_solve(a, p, b, c_first + m0 * c_stride, c_stride, cnt, 0, true);
    }
  }
}

// Planar FP32 copy of the lower triangle of complex K, and the running diagonal.
__global__ void __launch_bounds__(256) k_convert_cx(const double2* K, int64_t ldk, float* Ar,
                                                    float* Ai, int64_t lda, int64_t n, double* kd,
                                                    double* s) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    const double2* col = K + j * ldk;
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      const double2 v = col[i];
      Ar[i + j * lda] = (float)v.x;
      Ai[i + j * lda] = (float)v.y;
    }
    if (threadIdx.x == 0) {
      kd[j] = col[j].x;
      s[j] = 0.0;
    }
  }
}

// L (strictly lower, complex) and the pivots on the diagonal, FP64.
__global__ void __launch_bounds__(256) k_export_cx(const float* Ar, const float* Ai, int64_t lda,
                                                   const double* piv, double2* F, int64_t ldf,
                                                   int64_t n) {
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
      F[i + j * ldf] = i == j ? make_double2(piv[j], 0.0)
                              : make_double2((double)Ar[i + j * lda], (double)Ai[i + j * lda]);
    }
  }
}

struct CxLayout {
  int64_t ld32;
  float *Ar, *Ai, *Wf, *Lf;
  void* W1[3];
  void* W2[3];
  void* Lo[3];
  double *kd, *s, *piv;
  unsigned* flag;
  int* err;
  float* Bbuf;
  RecomputeScratch rs;
  unsigned long long *xwi, *vwi;
  float* inv;
  double2* r;
};

bool carve_cx(Workspace& ws, int64_t n, CxLayout* L) {
  L->ld32 = ((n + 31) / 32) * 32;
  if (L->ld32 < 32) L->ld32 = 32;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const size_t mat = sizeof(float) * (size_t)L->ld32 * nn;
  L->Ar = static_cast<float*>(ws.take(mat));
  L->Ai = static_cast<float*>(ws.take(mat));
  const size_t ob = sizeof(float) * nn * (size_t)kCLd;
  L->Wf = static_cast<float*>(ws.take(ob));
  L->Lf = static_cast<float*>(ws.take(ob));
  bool ok = true;
  for (int o = 0; o < 3; ++o) {
    L->W1[o] = ws.take(ob);
    L->W2[o] = ws.take(ob);
    L->Lo[o] = ws.take(ob);
    ok = ok && L->W1[o] && L->W2[o] && L->Lo[o];
  }
  L->kd = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->s = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->piv = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->flag = static_cast<unsigned*>(ws.take(256));
  L->err = reinterpret_cast<int*>(L->flag) + 16;
  L->Bbuf = static_cast<float*>(ws.take(sizeof(float) * 2048));
  if (!recompute_carve(ws, n, &L->rs)) return false;
  L->xwi = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  L->vwi = static_cast<unsigned long long*>(ws.take(sizeof(unsigned long long) * nn));
  L->inv = static_cast<float*>(ws.take(sizeof(float) * 2048 * (size_t)L->rs.nblk));
  L->r = static_cast<double2*>(ws.take(sizeof(double2) * nn));
  return ok && L->Ar && L->Ai && L->Wf && L->Lf && L->kd && L->s && L->piv && L->flag &&
         L->Bbuf && L->xwi && L->vwi && L->inv && L->r;
}

}  // namespace

size_t ws_mixed_cx(int64_t n) {
  Workspace probe;
  probe.base = reinterpret_cast<char*>(256);
  probe.size = ~size_t(0) >> 2;
  CxLayout L;
  carve_cx(probe, n, &L);
  return probe.used + 512;
}

cudaError_t sample_mixed_cx(const DrawArgs& a, Workspace ws) {
  const int64_t n = a.n;
  const int NB = g_tuning.outer_block;
  CxLayout L;
  if (!carve_cx(ws, n, &L)) return cudaErrorInvalidValue;
  cudaError_t e = init_result(a.result, a.stream);
  if (e != cudaSuccess || n == 0) return e;
  if ((e = cudaMemsetAsync(L.flag, 0, 256, a.stream)) != cudaSuccess) return e;
  if ((e = recompute_reset(L.rs, n, a.stream)) != cudaSuccess) return e;
  const size_t words = sizeof(unsigned long long) * (size_t)n;
  if ((e = cudaMemsetAsync(L.xwi, 0, words, a.stream)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(L.vwi, 0, words, a.stream)) != cudaSuccess) return e;
  const double2* K = static_cast<const double2*>(a.K);
  {
    ProfScope ps(kProfConvert, a.stream, 0.0, 12.0 * (double)n * (double)n);
    k_convert_cx<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
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
    cudaError_t ea = cudaFuncSetAttribute(k_cx_outer, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kCxDyn);
    if (ea != cudaSuccess) return ea;
    DevInfo di;
    if ((ea = dev_info(&di)) != cudaSuccess) return ea;
    int per_sm = 0;
    ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cx_outer, kCT, kCxDyn);
    if (ea != cudaSuccess) return ea;
    cap = per_sm * di.sm_count;
    if (cap > kMaxCoopCtas) cap = kMaxCoopCtas;
    if (cap < 3) return cudaErrorLaunchOutOfResources;
  }
  int grid = cap;
  if (g_tuning.max_ctas > 0 && grid > g_tuning.max_ctas) grid = g_tuning.max_ctas;
  if (grid < 3) grid = 3;
  int nh = (grid - 2) / 8;
  if (nh > kMaxOuterBlock / 32 - 1) nh = kMaxOuterBlock / 32 - 1;
  if (nh < 1) nh = 1;
  const int split = a.precision == DPP_PREC_BF16X6 ? kSplitBf16x6 : kSplit3xTf32;
  unsigned epoch = 1;
  for (int64_t q = 0; q < n; q += NB) {
    const int kb = (int)((n - q) < NB ? (n - q) : NB);
    CxArgs ca;
    ca.K = K;
    ca.ldk = a.ld;
    ca.Ar = L.Ar;
    ca.Ai = L.Ai;
    ca.lda = L.ld32;
    ca.n = n;
    ca.q = q;
    ca.kb = kb;
    ca.uniforms = a.uniforms;
    ca.seed = a.seed;
    ca.inst = a.instance;
    ca.keep = a.keep;
    ca.piv = L.piv;
    ca.kd = L.kd;
    ca.s = L.s;
    ca.Wf = L.Wf;
    ca.Lf = L.Lf;
    for (int o = 0; o < 3; ++o) {
      ca.W1[o] = L.W1[o];
      ca.W2[o] = L.W2[o];
      ca.Lo[o] = L.Lo[o];
    }
    ca.split = split;
    ca.res = a.result;
    ca.epoch0 = epoch;
    ca.tol = 1e-3;
    ca.tau0 = (float)(g_tuning.tau_safety * 0x1.0p-22);
    ca.Bbuf = L.Bbuf;
    ca.nh = nh;
    ca.cr.rc = recompute_args(L.rs, nullptr, a.ld, nullptr, L.ld32, L.piv, a.keep, n, q, a.result);
    ca.cr.rc.grid = grid;
    ca.cr.K = K;
    ca.cr.ldk = a.ld;
    ca.cr.Ar = L.Ar;
    ca.cr.Ai = L.Ai;
    ca.cr.lda = L.ld32;
    ca.cr.xwi = L.xwi;
    ca.cr.vwi = L.vwi;
    ca.cr.inv = L.inv;
    ca.cr.r = L.r;
    void* args[] = {&ca};
    {
      ProfScope ps(kProfPanel, a.stream);
      e = cudaLaunchCooperativeKernel((const void*)k_cx_outer, dim3((unsigned)grid), dim3(kCT),
                                      args, kCxDyn, a.stream);
    }
    if (e != cudaSuccess) return e;
    epoch += (unsigned)((kb + 31) / 32);
    const int64_t r0 = q + kb;
    if (r0 < n) {
      // Re -= [Wr Wi][Lr Li]^T and Im -= [Wi -Wr][Lr Li]^T, lower triangle
      const int64_t m = n - r0;
      const double fl = 4.0 * (double)m * (double)m * (double)kb;
      ProfScope ps(kProfUpdateTc, a.stream, fl, 16.0 * (double)m * (double)m);
      e = outer_update_tc(split, L.Ar, L.ld32, n, r0, 2 * kb, L.W1, L.Lo, kCLd, false, L.err,
                          a.stream);
      if (e != cudaSuccess) return e;
      e = outer_update_tc(split, L.Ai, L.ld32, n, r0, 2 * kb, L.W2, L.Lo, kCLd, false, L.err,
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
    k_export_cx<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(
        L.Ar, L.Ai, L.ld32, L.piv, static_cast<double2*>(a.factor_out), a.ld, n);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dpp
