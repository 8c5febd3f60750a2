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
// leader, which holds the diagonal block) posts a request; CTAs 1..G-1 (the
// workers) run the two triangular solves as wavefronts over 32-wide blocks
// with per-block ready flags, the residual as a row-block parallel product,
// and reply with per-CTA partial sums that the leader adds in a fixed order.
// Every wait is bounded; a timeout raises a shared abort flag that ends all
// other waits at once, and DPP_RES_TIMEOUT is reported.
#pragma once

#include "dpp_device.cuh"
#include "dpp_internal.h"

namespace dpp {

// control words (unsigned[32] in the workspace)
enum { kCtlReq = 0, kCtlG = 1, kCtlAck = 2, kCtlDone = 3, kCtlBarCount = 4, kCtlBarGen = 5,
       kCtlAbort = 6, kCtlQ = 7 };

struct RecomputeScratch {
  unsigned* ctrl = nullptr;
  unsigned* flag_x = nullptr;  // per 32-block: x0 block ready (request id)
  unsigned* flag_v = nullptr;  // per 32-block: v block ready
  double* ell = nullptr;
  double* x0 = nullptr;
  double* r = nullptr;
  double* v = nullptr;
  double* part = nullptr;  // 4 doubles per worker CTA
  int64_t nblk = 0;
  int max_workers = 0;
};

struct RecomputeArgs {
  unsigned* ctrl;
  unsigned* flag_x;
  unsigned* flag_v;
  double *ell, *x0, *r, *v, *part;
  const double* K;
  int64_t ldk;
  float* A;
  int64_t lda;
  const double* piv;
  const uint8_t* keep;
  int64_t n, q;
  int grid;
  dpp_result* res;
};

constexpr int kMaxCoopCtas = 4096;

inline bool recompute_carve(Workspace& ws, int64_t n, RecomputeScratch* s) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  s->nblk = (int64_t)(nn + 31) / 32;
  s->max_workers = kMaxCoopCtas;
  s->ctrl = static_cast<unsigned*>(ws.take(256));
  s->flag_x = static_cast<unsigned*>(ws.take(sizeof(unsigned) * (size_t)s->nblk));
  s->flag_v = static_cast<unsigned*>(ws.take(sizeof(unsigned) * (size_t)s->nblk));
  s->ell = static_cast<double*>(ws.take(sizeof(double) * nn));
  s->x0 = static_cast<double*>(ws.take(sizeof(double) * nn));
  s->r = static_cast<double*>(ws.take(sizeof(double) * nn));
  s->v = static_cast<double*>(ws.take(sizeof(double) * nn));
  s->part = static_cast<double*>(ws.take(sizeof(double) * 4 * kMaxCoopCtas));
  return s->ctrl && s->flag_x && s->flag_v && s->ell && s->x0 && s->r && s->v && s->part;
}

inline cudaError_t recompute_reset(const RecomputeScratch& s, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(s.ctrl, 0, 256, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.flag_x, 0, sizeof(unsigned) * (size_t)s.nblk, st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(s.flag_v, 0, sizeof(unsigned) * (size_t)s.nblk, st);
}

inline RecomputeArgs recompute_args(const RecomputeScratch& s, const double* K, int64_t ldk,
                                    float* A, int64_t lda, const double* piv, const uint8_t* keep,
                                    int64_t n, int64_t q, dpp_result* res) {
  RecomputeArgs a;
  a.ctrl = s.ctrl;
  a.flag_x = s.flag_x;
  a.flag_v = s.flag_v;
  a.ell = s.ell;
  a.x0 = s.x0;
  a.r = s.r;
  a.v = s.v;
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
  return a;
}

// ---------------------------------------------------------------------------
// bounded waits that also give up as soon as another CTA raised the abort flag
// ---------------------------------------------------------------------------
__device__ inline bool rc_wait_geq(const RecomputeArgs& a, const unsigned* flag, unsigned target) {
  if (ld_acquire(flag) >= target) return true;
  const unsigned long long t0 = global_ns();
  unsigned sleep = 32;
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (ld_acquire(&a.ctrl[kCtlAbort]) != 0) return false;
    if (global_ns() - t0 > kWaitNs) {
      atomicExch(&a.ctrl[kCtlAbort], 1u);
      flag_status(a.res, DPP_RES_TIMEOUT);
      return false;
    }
    __nanosleep(sleep);
    if (sleep < 256) sleep <<= 1;
  }
}

// Barrier over the worker CTAs (1..grid-1). Returns false on abort/timeout.
__device__ inline bool rc_worker_barrier(const RecomputeArgs& a, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned nw = (unsigned)(a.grid - 1);
    const unsigned g0 = ld_acquire(&a.ctrl[kCtlBarGen]);
    __threadfence();
    const unsigned arrived = atomicAdd(&a.ctrl[kCtlBarCount], 1u) + 1u;
    bool ok = true;
    if (arrived == nw) {
      atomicExch(&a.ctrl[kCtlBarCount], 0u);
      __threadfence();
      st_release(&a.ctrl[kCtlBarGen], g0 + 1u);
    } else {
      ok = rc_wait_geq(a, &a.ctrl[kCtlBarGen], g0 + 1u);
    }
    *s_flag = ok ? 1 : 0;
  }
  __syncthreads();
  return *s_flag != 0;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Worker side of one request (all threads of a worker CTA).
__device__ inline bool recompute_serve(const RecomputeArgs& a, unsigned id) {
  __shared__ float sT[8][32][33];
  __shared__ double spart[8][32];
  __shared__ double sred[4];
  __shared__ int s_flag;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int w = blockIdx.x - 1, nw = a.grid - 1;
  const int64_t g = (int64_t)ld_acquire(&a.ctrl[kCtlG]);
  const int64_t q = (int64_t)ld_acquire(&a.ctrl[kCtlQ]);
  const int64_t nblk = (g + 31) / 32;
  const float* A = a.A;
  const int64_t lda = a.lda;

  // R0: row g of L for the columns before the current panel
  const int64_t qq = q < g ? q : g;
  for (int64_t c = (int64_t)w * blockDim.x + tid; c < qq; c += (int64_t)nw * blockDim.x)
    a.ell[c] = (double)A[g + c * lda];
  if (!rc_worker_barrier(a, &s_flag)) return false;

  // R1: x0 = L_P^{-T} ell (FP32 arithmetic: any x0 is admissible, its residual
  // is computed exactly below), blocks from the last one down (owner t % nw == w)
  {
    int64_t t = nblk - 1;
    if (nblk > 0) t -= ((nblk - 1 - w) % nw + nw) % nw;
    for (; t >= 0; t -= nw) {
      const int nc = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
      float acc = 0.f;
      bool ok = true;
      for (int64_t s = nblk - 1 - wp; s > t; s -= 8) {
        if (lane == 0) ok = rc_wait_geq(a, &a.flag_x[s], id);
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const int nr = (int)((g - 32 * s) < 32 ? (g - 32 * s) : 32);
        float tile[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
          tile[c] = (lane < nr && c < nc) ? __ldcg(&A[(32 * s + lane) + (32 * t + c) * lda]) : 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) sT[wp][c][lane] = tile[c];
        __syncwarp();
        const float xs = (lane < nr) ? (float)__ldcg(&a.x0[32 * s + lane]) : 0.f;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float xi = __shfl_sync(0xffffffffu, xs, i);
          acc = fmaf(sT[wp][lane][i], xi, acc);
        }
        __syncwarp();
      }
      spart[wp][lane] = (double)acc;
      __syncthreads();
      if (ld_acquire(&a.ctrl[kCtlAbort]) != 0) return false;
      if (wp == 0) {
        float y = 0.f;
        if (lane < nc) {
          double yd = a.ell[32 * t + lane];
          for (int k = 0; k < 8; ++k) yd -= spart[k][lane];
          y = (float)yd;
        }
        float tile[32];
#pragma unroll
        for (int c = 0; c < 32; ++c)
          tile[c] = (lane < nc && c < nc) ? __ldcg(&A[(32 * t + lane) + (32 * t + c) * lda]) : 0.f;
#pragma unroll
        for (int c = 0; c < 32; ++c) sT[0][c][lane] = tile[c];
        __syncwarp();
#pragma unroll
        for (int i = 31; i >= 0; --i) {
          const float xi = __shfl_sync(0xffffffffu, y, i);
          if (i < nc && lane < i) y = fmaf(-sT[0][lane][i], xi, y);  // L[32t+i, 32t+lane]
        }
        if (lane < nc) a.x0[32 * t + lane] = (double)y;
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release(&a.flag_x[t], id);
      }
      __syncthreads();
    }
  }
  if (!rc_worker_barrier(a, &s_flag)) return false;

  // R2: r = k - (K_P - 1_G) x0 (FP64), partial dots k.x0 and x0.r
  double kx = 0.0, xr = 0.0;
  for (int64_t t = w; t < nblk; t += nw) {
    const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
    const int64_t i = 32 * t + lane;
    // part A: columns c <= i (lower triangle, contiguous rows per column)
    double accA = 0.0;
    const int64_t cmax = 32 * t + nr;  // exclusive
    for (int64_t c = wp; c < cmax; c += 8) {
      if (lane < nr && c <= i) accA = fma(a.K[i + c * a.ldk], __ldcg(&a.x0[c]), accA);
    }
    spart[wp][lane] = accA;
    __syncthreads();
    // part B: row i's entries right of the diagonal, read down column i
    for (int rr = wp; rr < nr; rr += 8) {
      const int64_t ii = 32 * t + rr;
      double accB = 0.0;
      for (int64_t c = ii + 1 + lane; c < g; c += 32) accB = fma(a.K[c + ii * a.ldk], __ldcg(&a.x0[c]), accB);
      accB = warp_sum(accB);
      if (lane == 0) a.v[ii] = accB;  // stage part B in v (overwritten by R3)
    }
    __syncthreads();
    if (wp == 0 && lane < nr) {
      double tot = __ldcg(&a.v[i]);
      for (int k = 0; k < 8; ++k) tot += spart[k][lane];
      const double xi = __ldcg(&a.x0[i]);
      const double ki = a.K[g + i * a.ldk];  // K[i, g] from the lower triangle
      double ri = ki - tot;
      if (a.keep[i] == 0) ri += xi;  // (K_P - 1_G) x0 has -x0_i on rejected rows
      a.r[i] = ri;
      kx = fma(ki, xi, kx);
      xr = fma(xi, ri, xr);
    }
    __syncthreads();
  }
  if (wp == 0) {
    kx = warp_sum(kx);
    xr = warp_sum(xr);
    if (lane == 0) {
      sred[0] = kx;
      sred[1] = xr;
    }
  }
  if (!rc_worker_barrier(a, &s_flag)) return false;

  // R3: v = L_P^{-1} r (FP32 arithmetic on the small residual), e = sum v^2 / d,
  // blocks from the first one up
  double esum = 0.0;
  for (int64_t t = w; t < nblk; t += nw) {
    const int nr = (int)((g - 32 * t) < 32 ? (g - 32 * t) : 32);
    float acc = 0.f;
    bool ok = true;
    for (int64_t s = wp; s < t; s += 8) {
      if (lane == 0) ok = rc_wait_geq(a, &a.flag_v[s], id);
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      float tile[32];
#pragma unroll
      for (int c = 0; c < 32; ++c)
        tile[c] = (lane < nr) ? __ldcg(&A[(32 * t + lane) + (32 * s + c) * lda]) : 0.f;
      const float vs = (float)__ldcg(&a.v[32 * s + lane]);
#pragma unroll
      for (int c = 0; c < 32; ++c) acc = fmaf(tile[c], __shfl_sync(0xffffffffu, vs, c), acc);
    }
    spart[wp][lane] = (double)acc;
    __syncthreads();
    if (ld_acquire(&a.ctrl[kCtlAbort]) != 0) return false;
    if (wp == 0) {
      float y = 0.f;
      if (lane < nr) {
        double yd = __ldcg(&a.r[32 * t + lane]);
        for (int k = 0; k < 8; ++k) yd -= spart[k][lane];
        y = (float)yd;
      }
      float tile[32];
#pragma unroll
      for (int c = 0; c < 32; ++c)
        tile[c] = (lane < nr && c < nr) ? __ldcg(&A[(32 * t + lane) + (32 * t + c) * lda]) : 0.f;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float vc = __shfl_sync(0xffffffffu, y, c);
        if (c < nr && lane > c && lane < nr) y = fmaf(-tile[c], vc, y);
      }
      if (lane < nr) {
        a.v[32 * t + lane] = (double)y;
        esum += (double)y * (double)y / a.piv[32 * t + lane];
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) st_release(&a.flag_v[t], id);
    }
    __syncthreads();
  }
  if (wp == 0) {
    esum = warp_sum(esum);
    if (lane == 0) {
      a.part[4 * w + 0] = sred[0];
      a.part[4 * w + 1] = sred[1];
      a.part[4 * w + 2] = esum;
    }
  }
  __threadfence();
  if (!rc_worker_barrier(a, &s_flag)) return false;
  if (w == 0 && tid == 0) st_release(&a.ctrl[kCtlAck], id);
  return true;
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
      unsigned sleep = 32;
      while (true) {
        if (ld_acquire(&a.ctrl[kCtlDone]) >= epoch) { cmd = 2; break; }
        const unsigned req = ld_acquire(&a.ctrl[kCtlReq]);
        if (req >= ((epoch << 8) | (served + 1u))) { cmd = 1; id = req; break; }
        if (ld_acquire(&a.ctrl[kCtlAbort]) != 0) { cmd = 0; break; }
        if (global_ns() - t0 > kWaitNs) {
          atomicExch(&a.ctrl[kCtlAbort], 1u);
          flag_status(a.res, DPP_RES_TIMEOUT);
          cmd = 0;
          break;
        }
        __nanosleep(sleep);
        if (sleep < 512) sleep <<= 1;
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
  if (lane < j) a.ell[q + lane] = (double)blk[j][lane];
  __threadfence();
  __syncwarp();
  *seq += 1;
  const unsigned id = (epoch << 8) | (unsigned)(*seq);
  bool ok = true;
  if (a.grid < 2) ok = false;
  if (ok && lane == 0) {
    atomicExch(&a.ctrl[kCtlG], (unsigned)g);
    atomicExch(&a.ctrl[kCtlQ], (unsigned)q);
    __threadfence();
    st_release(&a.ctrl[kCtlReq], id);
    ok = rc_wait_geq(a, &a.ctrl[kCtlAck], id);
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
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
  d2 = __shfl_sync(0xffffffffu, d2, 0);
  er = __shfl_sync(0xffffffffu, er, 0);
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
