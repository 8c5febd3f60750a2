// Elementary (projection) DPP sampler: Algorithm 2 / Theorem 2 of
// arXiv:1905.00165. For a marginal kernel K that is an orthogonal projection of
// rank k, k steps of left-looking, diagonally pivoted Cholesky in which each
// pivot index is drawn from the remaining diagonal d (probability d_t / (k - j)
// at step j) give a sample of DPP(K) of size k, with P(Y) the product of the
// squared pivots. Cost O(n k^2).
//
// One cooperative launch per draw. The n positions (the order of the paper's
// symmetric swaps) are split into contiguous ranges, one per CTA. Step j:
//   A  each CTA sums max(d, 0) over its positions >= j;            barrier
//   B  every CTA forms the same running sums of those partials (fixed order)
//      and finds the CTA whose range holds the position t at which the
//      running sum first exceeds u_j S (S the total); that CTA scans its range,
//      swaps positions j and t of the permutation, and writes the pivot
//      sqrt(d_sel) of the selected index sel;                       barrier
//   C  every CTA, for its positions > j (index i), forms the new column entry
//        F[i][j] = (K[i, sel] - sum_{s<j} F[i][s] F[sel][s]) / pivot
//      (one warp per index, the row of F contiguous), subtracts F[i][j]^2 from
//      d_i, and then sums max(d, 0) for step j + 1 (phase A without a barrier:
//      the ranges do not change).
// Factor columns are kept by ORIGINAL index (F is n x k, row-major), so the
// swaps move one permutation entry instead of matrix rows. Both barriers are
// bounded: a barrier that waits longer than the wait limit raises an abort
// word that ends every CTA, and DPP_RES_TIMEOUT is reported.
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

constexpr int kEThreads = 256;
constexpr unsigned kEFull = 0xffffffffu;

struct ElemArgs {
  const double* K;
  int64_t n, ld, k;
  const double* uniforms;
  uint64_t seed, inst;
  int64_t* sample;   // k, selection order (output)
  uint8_t* keep;     // n or nullptr (output)
  double* chol;      // k x k column-major or nullptr (output)
  dpp_result* res;
  double* d;         // n: remaining diagonal, by original index
  int32_t* perm;     // n: original index at each position
  double* F;         // n x k row-major: factor columns by original index
  double* part;      // per CTA: partial sum of max(d, 0)
  int32_t* lastpos;  // per CTA: last position with d > 0 (or -1)
  double* piv;       // k pivots (square roots)
  unsigned* ctrl;    // [0] barrier count, [1] generation, [2] abort, [3] selected index
  int64_t chunk;     // positions per CTA
  unsigned long long wait_ns;
};

enum { kBarCount = 0, kBarGen = 1, kAbort = 2, kSel = 3 };

// Bounded grid barrier (all CTAs are co-resident: cooperative launch).
__device__ bool elem_barrier(const ElemArgs& a) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = ld_acquire(&a.ctrl[kAbort]) == 0;
    if (ok) {
      const unsigned g = ld_acquire(&a.ctrl[kBarGen]);
      __threadfence();
      if (atomicAdd(&a.ctrl[kBarCount], 1u) == gridDim.x - 1) {
        atomicExch(&a.ctrl[kBarCount], 0u);
        __threadfence();
        st_release(&a.ctrl[kBarGen], g + 1u);
      } else {
        const unsigned long long t0 = global_ns();
        unsigned sleep = 32;
        while (ld_acquire(&a.ctrl[kBarGen]) == g) {
          if (ld_acquire(&a.ctrl[kAbort]) != 0) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > a.wait_ns) {
            atomicExch(&a.ctrl[kAbort], 1u);
            flag_status(a.res, DPP_RES_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(sleep);
          if (sleep < 256) sleep <<= 1;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kEFull, v, o);
  if (lane == 0) red[wp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kEThreads / 32; ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

// Phase A for step j: this CTA's partial of max(d, 0) over positions >= j.
__device__ void elem_partial(const ElemArgs& a, int64_t j, double* red) {
  const int64_t lo = (int64_t)blockIdx.x * a.chunk;
  int64_t hi = lo + a.chunk;
  if (hi > a.n) hi = a.n;
  const int64_t p0 = lo > j ? lo : j;
  double v = 0.0;
  int last = -1;
  for (int64_t p = p0 + threadIdx.x; p < hi; p += kEThreads) {
    const double dp = __ldcg(&a.d[__ldcg(&a.perm[p])]);
    if (dp > 0.0) {
      v += dp;
      last = (int)p;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(kEFull, last, o));
  __shared__ int s_last[kEThreads / 32];
  if ((threadIdx.x & 31) == 0) s_last[threadIdx.x >> 5] = last;
  const double t = block_sum(v, red);
  if (threadIdx.x == 0) {
    int m = -1;
    for (int w = 0; w < kEThreads / 32; ++w) m = max(m, s_last[w]);
    a.part[blockIdx.x] = t;
    a.lastpos[blockIdx.x] = m;
  }
}

constexpr int kEMaxCtas = 1024;   // partials staged in shared memory
constexpr int kEMaxChunk = 2048;  // positions per CTA (the owner's staged range)

__global__ void __launch_bounds__(kEThreads) k_elementary(ElemArgs a) {
  __shared__ double red[kEThreads / 32];
  __shared__ double s_part[kEMaxCtas];
  __shared__ int s_lastp[kEMaxCtas];
  __shared__ double s_d[kEMaxChunk];
  __shared__ int s_owner;
  __shared__ double s_acc, s_target;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t n = a.n, k = a.k;
  const int64_t lo = (int64_t)blockIdx.x * a.chunk;
  int64_t hi = lo + a.chunk;
  if (hi > n) hi = n;
  // d = diag(K), identity permutation (by position ranges)
  for (int64_t p = lo + threadIdx.x; p < hi; p += kEThreads) {
    a.d[p] = a.K[p + p * a.ld];
    a.perm[p] = (int32_t)p;
    if (a.keep) a.keep[p] = 0;
  }
  if (!elem_barrier(a)) return;
  elem_partial(a, 0, red);
  double lp = 0.0;  // CTA 0's thread 0 accumulates log P
  for (int64_t j = 0; j < k; ++j) {
    if (!elem_barrier(a)) return;
    // ---- B: the position t (all CTAs agree on the CTA that holds it) ----
    // the partials are staged in shared memory by all threads (independent
    // loads), then thread 0 forms the running sums in CTA order
    for (unsigned b = threadIdx.x; b < gridDim.x; b += kEThreads) {
      s_part[b] = __ldcg(&a.part[b]);
      s_lastp[b] = __ldcg(&a.lastpos[b]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double S = 0.0;
      for (unsigned b = 0; b < gridDim.x; ++b) S += s_part[b];
      const double u = a.uniforms ? a.uniforms[j] : philox_uniform(a.seed, a.inst, (uint64_t)j);
      const double target = u * S;
      double acc = 0.0;
      int owner = -1;
      for (unsigned b = 0; b < gridDim.x; ++b) {
        const double pb = s_part[b];
        if (acc + pb > target && pb > 0.0) {
          owner = (int)b;
          break;
        }
        acc += pb;
      }
      if (owner < 0) {  // rounding left the target at the end: last positive position
        int best = -1;
        for (unsigned b = 0; b < gridDim.x; ++b) best = max(best, s_lastp[b]);
        owner = best >= 0 ? (int)(best / a.chunk) : (int)(j / a.chunk);
        acc = -1.0;  // marks "take the last positive position"
      }
      s_owner = owner;
      s_acc = acc;
      s_target = target;
    }
    __syncthreads();
    if ((int)blockIdx.x == s_owner) {
      // the owner's remaining diagonal, staged by all threads, scanned in order
      const int64_t p0 = lo > j ? lo : j;
      for (int64_t p = p0 + threadIdx.x; p < hi; p += kEThreads)
        s_d[p - p0] = __ldcg(&a.d[__ldcg(&a.perm[p])]);
      __syncthreads();
      if (threadIdx.x == 0) {
        const int owner = s_owner;
        const double target = s_target;
        int64_t t = -1;
        if (s_acc >= 0.0) {
          double run = s_acc;
          for (int64_t p = p0; p < hi; ++p) {
            const double dp = s_d[p - p0];
            if (dp > 0.0) {
              run += dp;
              if (run > target) {
                t = p;
                break;
              }
            }
          }
        }
        if (t < 0) {
          const int lp_owner = s_lastp[owner];
          t = lp_owner >= 0 ? lp_owner : j;
        }
        const int32_t pj = __ldcg(&a.perm[j]), pt = __ldcg(&a.perm[t]);
        a.perm[j] = pt;
        a.perm[t] = pj;
        const double dsel = __ldcg(&a.d[pt]);
        const double piv = sqrt(dsel > 0.0 ? dsel : 0.0);
        if (!(dsel > 0.0)) flag_status(a.res, isfinite(dsel) ? DPP_RES_INADMISSIBLE : DPP_RES_NONFINITE);
        a.F[(int64_t)pt * k + j] = piv;
        a.piv[j] = piv;
        atomicExch(&a.ctrl[kSel], (unsigned)pt);
        __threadfence();
      }
    }
    __syncthreads();
    if (!elem_barrier(a)) return;
    const int64_t sel = (int64_t)ld_acquire(&a.ctrl[kSel]);
    const double piv = __ldcg(&a.piv[j]);
    if (blockIdx.x == 0 && threadIdx.x == 0) lp += 2.0 * log(piv);
    if (j == k - 1) break;
    // ---- C: column j for this CTA's positions > j, then phase A of j + 1 ----
    // four lanes per index (eight indices per warp at once), so the latency
    // chain of one index (permutation, K entry and factor row, reduction,
    // diagonal) overlaps with the other indices'
    const double* Fs = a.F + sel * k;
    const int grp = threadIdx.x >> 2, gl = threadIdx.x & 3;
    const int64_t p0 = lo > j + 1 ? lo : j + 1;
    // (the loop bound is the warp's, so every lane reaches the shuffles)
    for (int64_t pb = p0 + (grp & ~7); pb < hi; pb += kEThreads / 4) {
      const int64_t p = pb + (grp & 7);
      const bool act = p < hi;
      const int64_t i = act ? __ldcg(&a.perm[p]) : 0;
      const double* Fi = a.F + i * k;
      const double kis = (act && gl == 0) ? a.K[i + sel * a.ld] : 0.0;
      double dot = 0.0, dot2 = 0.0;
      if (act) {
        int64_t s2 = gl;
#pragma unroll 4
        for (; s2 + 4 < j; s2 += 8) {
          dot = fma(__ldcg(&Fi[s2]), __ldcg(&Fs[s2]), dot);
          dot2 = fma(__ldcg(&Fi[s2 + 4]), __ldcg(&Fs[s2 + 4]), dot2);
        }
        if (s2 < j) dot = fma(__ldcg(&Fi[s2]), __ldcg(&Fs[s2]), dot);
      }
      dot += dot2;
      dot += __shfl_xor_sync(kEFull, dot, 2);
      dot += __shfl_xor_sync(kEFull, dot, 1);
      if (act && gl == 0) {
        const double c = (kis - dot) / piv;
        a.F[i * k + j] = c;
        a.d[i] = __ldcg(&a.d[i]) - c * c;
      }
    }
    __syncthreads();
    elem_partial(a, j + 1, red);
  }
  // ---- outputs (positions 0..k-1 hold the sample in selection order) ----
  if (!elem_barrier(a)) return;
  const int64_t gtid = (int64_t)blockIdx.x * kEThreads + threadIdx.x;
  const int64_t gsz = (int64_t)gridDim.x * kEThreads;
  for (int64_t jj = gtid; jj < k; jj += gsz) {
    const int32_t idx = __ldcg(&a.perm[jj]);
    a.sample[jj] = idx;
    if (a.keep) a.keep[idx] = 1;
  }
  if (a.chol) {
    for (int64_t e = gtid; e < k * k; e += gsz) {
      const int64_t i = e % k, c = e / k;
      a.chol[e] = i >= c ? __ldcg(&a.F[(int64_t)__ldcg(&a.perm[i]) * k + c]) : 0.0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.res->logp = lp;
    a.res->n_kept = (int32_t)k;
  }
}

}  // namespace

size_t ws_elementary(int64_t n, int64_t k) {
  const size_t nn = (size_t)(n > 0 ? n : 1), kk = (size_t)(k > 0 ? k : 1);
  return align256(sizeof(double) * nn) + align256(sizeof(int32_t) * nn) +
         align256(sizeof(double) * nn * kk) + align256(sizeof(double) * 4096) +
         align256(sizeof(int32_t) * 4096) + align256(sizeof(double) * kk) + 256 + 256;
}

cudaError_t sample_elementary(const double* K, int64_t n, int64_t ld, int64_t k, uint64_t seed,
                              uint64_t instance, const double* uniforms, int64_t* sample,
                              uint8_t* keep, double* chol, dpp_result* result, Workspace ws,
                              cudaStream_t s) {
  ElemArgs a;
  a.K = K;
  a.n = n;
  a.ld = ld;
  a.k = k;
  a.uniforms = uniforms;
  a.seed = seed;
  a.inst = instance;
  a.sample = sample;
  a.keep = keep;
  a.chol = chol;
  a.res = result;
  const size_t nn = (size_t)(n > 0 ? n : 1), kk = (size_t)(k > 0 ? k : 1);
  a.d = static_cast<double*>(ws.take(sizeof(double) * nn));
  a.perm = static_cast<int32_t*>(ws.take(sizeof(int32_t) * nn));
  a.F = static_cast<double*>(ws.take(sizeof(double) * nn * kk));
  a.part = static_cast<double*>(ws.take(sizeof(double) * 4096));
  a.lastpos = static_cast<int32_t*>(ws.take(sizeof(int32_t) * 4096));
  a.piv = static_cast<double*>(ws.take(sizeof(double) * kk));
  a.ctrl = static_cast<unsigned*>(ws.take(256));
  if (!a.d || !a.perm || !a.F || !a.part || !a.lastpos || !a.piv || !a.ctrl)
    return cudaErrorInvalidValue;
  a.wait_ns = (unsigned long long)g_tuning.wait_ns;
  cudaError_t e = init_result(result, s);
  if (e != cudaSuccess || n == 0) return e;
  if (k == 0) {
    if (keep) return cudaMemsetAsync(keep, 0, (size_t)n, s);
    return cudaSuccess;
  }
  if ((e = cudaMemsetAsync(a.ctrl, 0, 256, s)) != cudaSuccess) return e;
  // one CTA per SM at most (cooperative), at least 32 positions per CTA
  static int caps[64] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (caps[dev] == 0) {
    DevInfo di;
    if ((e = dev_info(&di)) != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_elementary, kEThreads, 0);
    if (e != cudaSuccess) return e;
    caps[dev] = per_sm >= 1 ? di.sm_count : 1;
  }
  int64_t grid = caps[dev];
  if (g_tuning.max_ctas > 0 && grid > g_tuning.max_ctas) grid = g_tuning.max_ctas;
  int64_t by_n = (n + 31) / 32;
  if (grid > by_n) grid = by_n;
  if (grid > kEMaxCtas) grid = kEMaxCtas;
  const int64_t min_grid = (n + kEMaxChunk - 1) / kEMaxChunk;
  if (grid < min_grid) grid = min_grid;
  if (grid < 1) grid = 1;
  if (grid > caps[dev] || grid > kEMaxCtas) return cudaErrorInvalidValue;  // n too large
  a.chunk = (n + grid - 1) / grid;
  grid = (n + a.chunk - 1) / a.chunk;  // every CTA owns at least one position
  void* args[] = {&a};
  const double fl = (double)n * (double)k * (double)k;  // ~n k^2 multiply-adds
  ProfScope ps(kProfElementary, s, fl, 0.0);
  return cudaLaunchCooperativeKernel((const void*)k_elementary, dim3((unsigned)grid),
                                     dim3(kEThreads), args, 0, s);
}

}  // namespace dpp
