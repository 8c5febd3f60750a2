// Batched sampler: many Hermitian (real symmetric) kernels of uneven order in
// one persistent launch.
//
// Each CTA repeatedly takes the next instance from a device work queue (the
// instances ordered by decreasing n, longest-processing-time first) and draws
// its sample alone, left-looking over 32-wide panels (Algorithm 1 in the
// blocked form of Algorithms 3/4, LDL^T specialisation):
//   (a) update the panel's columns from all earlier columns,
//         A[i, q+c] -= sum_{t<q} L[i, t] d_t L[q+c, t]   (FP32, tiled SIMT)
//   (b) the sequential decisions on the 32 x 32 diagonal block (warp 0, FP32
//       with a double-float running diagonal, FP64 pivots; a pivot inside the
//       borderline band is recomputed in FP64 from K by the whole CTA),
//   (c) the panel solve of the rows below (L = W / d, running diagonal).
// Storage: an FP32 working copy per CTA (reused across instances), the FP64
// kernels are only read. Every instance's dpp_result is written on the device.
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kP = 32;         // panel width
// threads per CTA: a template parameter (128 or 256, DPP_TUNE_BATCHED_THREADS)
constexpr int kLd = 65;        // k-major staging tile stride

struct BatchArgs {
  int32_t batch;
  const int64_t* n;
  const double* const* K;
  const int64_t* ld;
  uint64_t seed;
  const uint64_t* instance;
  uint8_t* const* keep;
  const double* const* uniforms;
  double* const* pivots;
  dpp_result* res;
  int64_t n_max, ldw;
  float* work;     // per CTA: ldw x n_max FP32
  double* vec;     // per CTA: 8 x n_max FP64 (kd, s, piv, ell, x0, r, v, spare)
  const int32_t* order;
  unsigned* queue;
  float tau0;
  double tol;
};

// ---------------------------------------------------------------------------
// device-side LPT order: counting sort of the instances by decreasing n
// ---------------------------------------------------------------------------
__global__ void k_order(const int64_t* n, int32_t batch, int64_t n_max, int32_t* counts,
                        int32_t* order) {
  // single CTA: histogram, exclusive scan from the largest n, scatter
  for (int64_t v = threadIdx.x; v <= n_max; v += blockDim.x) counts[v] = 0;
  __syncthreads();
  for (int32_t i = threadIdx.x; i < batch; i += blockDim.x) {
    int64_t v = n[i];
    v = v < 0 ? 0 : (v > n_max ? n_max : v);
    atomicAdd(&counts[v], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t acc = 0;
    for (int64_t v = n_max; v >= 0; --v) {
      const int32_t c = counts[v];
      counts[v] = acc;
      acc += c;
    }
  }
  __syncthreads();
  for (int32_t i = threadIdx.x; i < batch; i += blockDim.x) {
    int64_t v = n[i];
    v = v < 0 ? 0 : (v > n_max ? n_max : v);
    order[atomicAdd(&counts[v], 1)] = i;
  }
}

__device__ inline double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct Inst {
  const double* K;
  int64_t ldk, n;
  float* A;
  int64_t lda;
  double *kd, *s, *piv, *ell, *x0, *r, *v;
  uint8_t* keep;
  const double* u;  // explicit uniforms or NULL (Philox)
  uint64_t seed, inst;
};

// CTA-local FP64 recompute of the pivot of index g (see the exact identity in
// dpp_recompute.cuh): x0 = L_P^{-T} l (FP32 solve), r = k - (K_P - 1_G) x0 in
// FP64, v = L_P^{-1} r, d = K_gg - k.x0 - x0.r - sum v^2/d.
template <int kThreadsB>
__device__ __noinline__ double cta_recompute(const Inst& in, int64_t g) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* A = in.A;
  const int64_t lda = in.lda;
  // l = row g of L (columns < g), in FP64 scratch
  for (int64_t c = tid; c < g; c += kThreadsB) in.ell[c] = (double)A[g + c * lda];
  __syncthreads();
  // x0 = L^{-T} l, backward over 32-blocks: x_blk = l_blk - sum_{i > blk} L[i, c] x_i,
  // then the block's own triangle by warp 0.
  const int64_t nb = (g + kP - 1) / kP;
  for (int64_t t = nb - 1; t >= 0; --t) {
    const int64_t c0 = kP * t;
    const int nc = (int)((g - c0) < kP ? (g - c0) : kP);
    // column c = c0 + (tid % 32); warps split the rows beyond the block
    double part = 0.0;
    const int cc = lane;
    if (cc < nc) {
      for (int64_t i = c0 + kP + warp; i < g; i += kThreadsB / 32)
        part += (double)A[i + (c0 + cc) * lda] * in.x0[i];
    }
    __shared__ double sp[kThreadsB / 32][kP];
    sp[warp][lane] = part;
    __syncthreads();
    if (warp == 0) {
      double y = 0.0;
      if (lane < nc) {
        y = in.ell[c0 + lane];
        for (int w = 0; w < kThreadsB / 32; ++w) y -= sp[w][lane];
      }
      for (int i = nc - 1; i >= 0; --i) {
        const double xi = __shfl_sync(kFull, y, i);
        if (lane < i) y -= (double)A[(c0 + i) + (c0 + lane) * lda] * xi;
      }
      if (lane < nc) in.x0[c0 + lane] = y;
    }
    __syncthreads();
  }
  // r = k - (K_P - 1_G) x0 and the dots, FP64; one row per thread
  double kx = 0.0, xr = 0.0;
  for (int64_t i = tid; i < g; i += kThreadsB) {
    double acc = 0.0;
    for (int64_t c = 0; c <= i; ++c) acc += in.K[i + c * in.ldk] * in.x0[c];
    for (int64_t c = i + 1; c < g; ++c) acc += in.K[c + i * in.ldk] * in.x0[c];
    const double ki = in.K[g + i * in.ldk];
    double ri = ki - acc;
    if (in.keep[i] == 0) ri += in.x0[i];
    in.r[i] = ri;
    kx += ki * in.x0[i];
    xr += in.x0[i] * ri;
  }
  __syncthreads();
  // v = L^{-1} r (forward over 32-blocks), e = sum v^2 / d
  double esum = 0.0;
  for (int64_t t = 0; t < nb; ++t) {
    const int64_t r0 = kP * t;
    const int nr = (int)((g - r0) < kP ? (g - r0) : kP);
    double part = 0.0;
    if (lane < nr) {
      for (int64_t c = warp; c < r0; c += kThreadsB / 32)
        part += (double)A[(r0 + lane) + c * lda] * in.v[c];
    }
    __shared__ double sq[kThreadsB / 32][kP];
    sq[warp][lane] = part;
    __syncthreads();
    if (warp == 0) {
      double y = 0.0;
      if (lane < nr) {
        y = in.r[r0 + lane];
        for (int w = 0; w < kThreadsB / 32; ++w) y -= sq[w][lane];
      }
      for (int c = 0; c < nr; ++c) {
        const double vc = __shfl_sync(kFull, y, c);
        if (lane > c && lane < nr) y -= (double)A[(r0 + lane) + (r0 + c) * lda] * vc;
      }
      if (lane < nr) {
        in.v[r0 + lane] = y;
        esum += y * y / in.piv[r0 + lane];
      }
    }
    __syncthreads();
  }
  // reductions (fixed order)
  kx = warp_sum_d(kx);
  xr = warp_sum_d(xr);
  esum = warp_sum_d(esum);  // nonzero in warp 0 only
  __shared__ double s3[3][kThreadsB / 32];
  if (lane == 0) {
    s3[0][warp] = kx;
    s3[1][warp] = xr;
    s3[2][warp] = esum;
  }
  __syncthreads();
  double K1 = 0.0, X1 = 0.0, E1 = 0.0;
  for (int w = 0; w < kThreadsB / 32; ++w) {
    K1 += s3[0][w];
    X1 += s3[1][w];
    E1 += s3[2][w];
  }
  const double d = in.K[g + g * in.ldk] - K1 - X1 - E1;
  __syncthreads();
  return d;
}

// Left-looking update of panel [q, q+b) for rows [q, n):
// A[i, q+c] -= sum_{t<q} L[i,t] d_t L[q+c,t], tiles of kThreadsB / 4 rows
// (two per thread row ty), 32-deep chunks.
template <int kThreadsB>
__device__ void panel_update(const Inst& in, int64_t q, int b, float* sA, float* sB, int tid) {
  if (q == 0) return;
  constexpr int kTH = kThreadsB / 4;
  const int64_t n = in.n;
  const int ty = tid / 8, tx = tid % 8;
  for (int64_t i0 = q; i0 < n; i0 += kTH) {
    float acc[2][4];
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc[rr][cc] = 0.f;
    for (int64_t k0 = 0; k0 < q; k0 += 32) {
      const int kc = (int)((q - k0) < 32 ? (q - k0) : 32);
      // sA[t][r] = L[i0 + r, k0 + t] (column-major: rows contiguous)
      for (int idx = tid; idx < 32 * kTH; idx += kThreadsB) {
        const int r = idx % kTH, t = idx / kTH;
        const int64_t i = i0 + r;
        sA[t * kLd + r] = (t < kc && i < n) ? in.A[i + (k0 + t) * in.lda] : 0.f;
      }
      // sB[t][c] = d_t L[q + c, k0 + t]
      for (int idx = tid; idx < 32 * 32; idx += kThreadsB) {
        const int c = idx % 32, t = idx / 32;
        sB[t * 33 + c] = (t < kc && c < b)
                             ? (float)in.piv[k0 + t] * in.A[(q + c) + (k0 + t) * in.lda]
                             : 0.f;
      }
      __syncthreads();
      for (int t = 0; t < kc; ++t) {
        const float w0 = sA[t * kLd + 2 * ty], w1 = sA[t * kLd + 2 * ty + 1];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const float l = sB[t * 33 + 4 * tx + cc];
          acc[0][cc] = fmaf(w0, l, acc[0][cc]);
          acc[1][cc] = fmaf(w1, l, acc[1][cc]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int64_t i = i0 + 2 * ty + rr;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int c = 4 * tx + cc;
        if (i < n && c < b && i >= q + c) in.A[i + (q + c) * in.lda] -= acc[rr][cc];
      }
    }
  }
}

template <int kThreadsB>
__global__ void __launch_bounds__(kThreadsB) k_batched(BatchArgs a) {
  __shared__ float sA[32 * kLd];
  __shared__ float sB[32 * 33];
  __shared__ float sL[kP][kP + 1];
  __shared__ float srd[kP];
  __shared__ int s_item;
  __shared__ float s_ddh[kP], s_ddl[kP], s_si[kP];
  __shared__ int s_kp[kP];
  __shared__ int s_pending, s_resume;
  __shared__ double s_pe, s_pold;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* A = a.work + (int64_t)blockIdx.x * a.ldw * a.n_max;
  double* vec = a.vec + (int64_t)blockIdx.x * 8 * a.n_max;

  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= a.batch) break;
    const int32_t idx = a.order[item];
    Inst in;
    in.n = a.n[idx];
    in.K = a.K[idx];
    in.ldk = a.ld[idx];
    in.A = A;
    in.lda = a.ldw;
    in.kd = vec;
    in.s = vec + a.n_max;
    in.piv = vec + 2 * a.n_max;
    in.ell = vec + 3 * a.n_max;
    in.x0 = vec + 4 * a.n_max;
    in.r = vec + 5 * a.n_max;
    in.v = vec + 6 * a.n_max;
    in.keep = a.keep[idx];
    in.u = a.uniforms ? a.uniforms[idx] : nullptr;
    in.seed = a.seed;
    in.inst = a.instance ? a.instance[idx] : (uint64_t)idx;
    dpp_result* res = a.res + idx;
    const int64_t n = in.n;
    if (n <= 0 || n > a.n_max) {
      if (tid == 0) {
        res->status = n > a.n_max ? DPP_RES_NONFINITE : 0;
        res->n_kept = 0;
        res->n_borderline = 0;
        res->n_out_of_range = 0;
        res->logp = 0.0;
        res->max_err_ratio = 0.0;
      }
      continue;
    }
    // FP32 working copy of the lower triangle; FP64 running diagonal
    for (int64_t j = warp; j < n; j += kThreadsB / 32) {
      for (int64_t i = j + lane; i < n; i += 32) A[i + j * in.lda] = (float)in.K[i + j * in.ldk];
      if (lane == 0) {
        in.kd[j] = in.K[j + j * in.ldk];
        in.s[j] = 0.0;
      }
    }
    __syncthreads();
    if (tid == 0) s_resume = 0;
    double lp_acc = 0.0;
    int kept = 0, oor = 0, bad = 0, border = 0;
    float max_ratio = 0.f;
    for (int64_t q = 0; q < n; q += kP) {
      const int b = (int)((n - q) < kP ? (n - q) : kP);
      panel_update<kThreadsB>(in, q, b, sA, sB, tid);
      __syncthreads();
      // decisions (warp 0); a borderline pivot suspends the loop, the whole CTA
      // recomputes it in FP64, and warp 0 resumes at that pivot
      int jstart = 0;
      while (true) {
        if (warp == 0) {
          float r[kP];
          f2 dd;
          float si;
          bool mykeep;
          if (jstart == 0) {
#pragma unroll
            for (int k = 0; k < kP; ++k) {
              float v = 0.f;
              if (lane < b && k < b)
                v = (k <= lane) ? A[(q + lane) + (q + k) * in.lda] : A[(q + k) + (q + lane) * in.lda];
              r[k] = v;
            }
            dd = make_f2(0.f, 0.f);
            si = 0.f;
            if (lane < b) {
              dd = f2_from_double(in.kd[q + lane]);
              si = (float)in.s[q + lane];
            }
            mykeep = false;
          } else {
#pragma unroll
            for (int k = 0; k < kP; ++k) r[k] = sL[lane][k];
            dd = make_f2(s_ddh[lane], s_ddl[lane]);
            si = s_si[lane];
            mykeep = s_kp[lane] != 0;
          }
          double u = 2.0;
          float uf = 2.f, kf = 0.f, sq = 1.f;
          if (lane < b) {
            u = in.u ? in.u[q + lane] : philox_uniform(in.seed, in.inst, (uint64_t)(q + lane));
            uf = (float)u;
            kf = (float)in.K[(q + lane) + (q + lane) * in.ldk];
            sq = sqrtf((float)(q + lane + 1));
          }
          int pending = -1;
#pragma unroll 1
          for (int j = jstart; j < b; ++j) {
            const float ph = __shfl_sync(kFull, dd.hi, j);
            const float uj = __shfl_sync(kFull, uf, j);
            const float sj = __shfl_sync(kFull, si, j);
            const float kj = __shfl_sync(kFull, kf, j);
            const float sqj = __shfl_sync(kFull, sq, j);
            const float tau = a.tau0 * sqj * (fabsf(kj) + sj) + 0x1.0p-22f;
            const bool resumed = (jstart > 0 || s_resume) && j == jstart;
            bool kp;
            float df;
            if (!resumed && fabsf(uj - ph) <= tau) {
              // save the state, publish what the recompute reads, suspend
#pragma unroll
              for (int k = 0; k < kP; ++k) {
                sL[lane][k] = r[k];
                if (lane < b && k < lane && k < j) A[(q + lane) + (q + k) * in.lda] = r[k];
              }
              s_ddh[lane] = dd.hi;
              s_ddl[lane] = dd.lo;
              s_si[lane] = si;
              s_kp[lane] = mykeep ? 1 : 0;
              if (lane < j) {
                in.piv[q + lane] = f2_to_double(dd);
                in.keep[q + lane] = mykeep ? 1 : 0;
              }
              const float pl = __shfl_sync(kFull, dd.lo, j);
              if (lane == 0) s_pold = (double)ph + (double)pl;
              pending = j;
              break;
            }
            if (resumed) {
              const double uj64 = __shfl_sync(kFull, u, j);
              const double pe = s_pe;
              kp = uj64 < pe;
              const double dfin = kp ? pe : pe - 1.0;
              df = (float)dfin;
              if (lane == j) dd = f2_from_double(dfin);
              if (lane == 0) {
                ++border;
                const float ratio = (float)(fabs(pe - s_pold) / (double)tau);
                max_ratio = fmaxf(max_ratio, ratio);
              }
            } else {
              kp = uj < ph;
              df = kp ? ph : ph - 1.0f;
              if (lane == j && !kp) dd = f2_add_f(dd, -1.0f);
            }
            const float rd = 1.0f / df;
            float wj = 0.f;
#pragma unroll
            for (int k = 0; k < kP; ++k) wj = (k == j) ? r[k] : wj;
            const float l = wj * rd;
            const bool act = (lane > j) && (lane < b);
#pragma unroll
            for (int k = 0; k < kP; ++k) {
              const float pk = __shfl_sync(kFull, r[k], j);
              if (act && k > j) r[k] = fmaf(-l, pk, r[k]);
            }
            const float newj = act ? l : df;
#pragma unroll
            for (int k = 0; k < kP; ++k)
              if (k == j && (act || lane == j)) r[k] = newj;
            if (act) {
              dd = f2_sub_prod(dd, wj, l);
              si += fabsf(wj * l);
            }
            if (lane == j) mykeep = kp;
          }
          if (lane == 0) {
            s_pending = pending;
            s_resume = 0;
          }
          if (pending < 0) {
#pragma unroll
            for (int k = 0; k < kP; ++k) {
              sL[lane][k] = r[k];
              if (lane < b && k <= lane) A[(q + lane) + (q + k) * in.lda] = r[k];
            }
            if (lane < b) {
              const double d = f2_to_double(dd);
              const double pre = mykeep ? d : d + 1.0;
              in.piv[q + lane] = d;
              in.keep[q + lane] = mykeep ? 1 : 0;
              srd[lane] = (float)(1.0 / d);
              lp_acc += log(fabs(d));
              kept += mykeep ? 1 : 0;
              oor += (pre < -a.tol || pre > 1.0 + a.tol) ? 1 : 0;
              bad |= isfinite(d) ? 0 : 1;
            } else {
              srd[lane] = 1.f;
            }
          }
        }
        __threadfence_block();
        __syncthreads();
        const int pend = s_pending;
        if (pend < 0) break;
        const double pe = cta_recompute<kThreadsB>(in, q + pend);
        if (tid == 0) {
          s_pe = pe;
          s_resume = 1;
        }
        jstart = pend;
        __syncthreads();
      }
      // panel solve of rows [q+b, n), one row per thread
      for (int64_t i = q + b + tid; i < n; i += kThreadsB) {
        float w[kP];
#pragma unroll
        for (int k = 0; k < kP; ++k) w[k] = (k < b) ? A[i + (q + k) * in.lda] : 0.f;
#pragma unroll
        for (int k = 1; k < kP; ++k)
          if (k < b) {
#pragma unroll
            for (int t = 0; t < k; ++t) w[k] = fmaf(-w[t], sL[k][t], w[k]);
          }
        f2 dsum = {0.f, 0.f};
        float ssum = 0.f;
#pragma unroll
        for (int k = 0; k < kP; ++k) {
          if (k < b) {
            const float l = w[k] * srd[k];
            dsum = f2_add_prod(dsum, w[k], l);
            ssum += fabsf(w[k] * l);
            A[i + (q + k) * in.lda] = l;
          }
        }
        in.kd[i] -= f2_to_double(dsum);
        in.s[i] += (double)ssum;
      }
      __syncthreads();
    }
    // per-instance result
    if (warp == 0) {
      const double lp = warp_sum_d(lp_acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        kept += __shfl_xor_sync(kFull, kept, o);
        oor += __shfl_xor_sync(kFull, oor, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
      }
      if (lane == 0) {
        res->status = (oor ? DPP_RES_INADMISSIBLE : 0) | (bad ? DPP_RES_NONFINITE : 0);
        res->n_kept = kept;
        res->n_borderline = border;
        res->n_out_of_range = oor;
        res->logp = lp;
        res->max_err_ratio = (double)max_ratio;
      }
      if (a.pivots && a.pivots[idx])
        for (int64_t j = lane; j < n; j += 32) a.pivots[idx][j] = in.piv[j];
    }
    __syncthreads();
  }
}

}  // namespace

size_t ws_batched_per_cta(int64_t n_max) {
  const int64_t ldw = ((n_max + 31) / 32) * 32;
  return align256(sizeof(float) * (size_t)ldw * (size_t)n_max) +
         align256(sizeof(double) * 8 * (size_t)n_max);
}

size_t ws_batched(int32_t batch, int64_t n_max, int ctas) {
  return align256(sizeof(int32_t) * (size_t)(batch > 0 ? batch : 1)) +
         align256(sizeof(int32_t) * (size_t)(n_max + 1)) + 256 +
         (size_t)ctas * ws_batched_per_cta(n_max) + 1024;
}

int batched_default_ctas() {
  DevInfo di;
  if (dev_info(&di) != cudaSuccess || di.sm_count <= 0) return 2 * 152;
  return 2 * di.sm_count;
}

cudaError_t sample_batched(const BatchedArgs& b, Workspace ws) {
  cudaError_t e;
  const int64_t n_max = b.n_max;
  const int64_t ldw = ((n_max + 31) / 32) * 32;
  int32_t* order = static_cast<int32_t*>(ws.take(sizeof(int32_t) * (size_t)(b.batch > 0 ? b.batch : 1)));
  int32_t* counts = static_cast<int32_t*>(ws.take(sizeof(int32_t) * (size_t)(n_max + 1)));
  unsigned* queue = static_cast<unsigned*>(ws.take(256));
  if (!order || !counts || !queue) return cudaErrorInvalidValue;
  // CTAs that fit in the remaining workspace (at most two per SM)
  const size_t per = ws_batched_per_cta(n_max);
  const size_t left = ws.size - ((ws.used + 255) & ~size_t(255));
  int64_t ctas = (int64_t)(left / (per + 256));
  const int64_t cap = batched_default_ctas();
  if (ctas > cap) ctas = cap;
  if (ctas > b.batch) ctas = b.batch;
  if (ctas < 1) return cudaErrorInvalidValue;
  float* work = static_cast<float*>(ws.take(sizeof(float) * (size_t)ldw * (size_t)n_max * (size_t)ctas));
  double* vec = static_cast<double*>(ws.take(sizeof(double) * 8 * (size_t)n_max * (size_t)ctas));
  if (!work || !vec) return cudaErrorInvalidValue;
  if ((e = cudaMemsetAsync(queue, 0, 256, b.stream)) != cudaSuccess) return e;
  {
    ProfScope ps(kProfOther, b.stream);
    k_order<<<1, 1024, 0, b.stream>>>(b.n, b.batch, n_max, counts, order);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  BatchArgs a;
  a.batch = b.batch;
  a.n = b.n;
  a.K = b.K;
  a.ld = b.ld;
  a.seed = b.seed;
  a.instance = b.instance;
  a.keep = b.keep;
  a.uniforms = b.uniforms;
  a.pivots = b.pivots;
  a.res = b.results;
  a.n_max = n_max;
  a.ldw = ldw;
  a.work = work;
  a.vec = vec;
  a.order = order;
  a.queue = queue;
  a.tau0 = (float)(g_tuning.tau_safety * 0x1.0p-22);
  a.tol = 1e-3;
  {
    ProfScope ps(kProfBatched, b.stream, b.flops, 0.0);
    if (g_tuning.batched_threads == 256)
      k_batched<256><<<(unsigned)ctas, 256, 0, b.stream>>>(a);
    else
      k_batched<128><<<(unsigned)ctas, 128, 0, b.stream>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dpp
