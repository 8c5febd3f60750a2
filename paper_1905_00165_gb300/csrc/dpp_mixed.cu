// Mixed-precision Hermitian (real symmetric) DPP sampler.
//
// Storage: an FP32 copy A32 of the lower triangle of K. Arithmetic:
//   * pivots: a running diagonal kd_i = K_ii - sum_k w_ik l_ik kept in FP64
//     (double-float inside the sequential loop) and formed from the FP32
//     factor entries (w = l d), so a pivot carries no FP32 accumulation error
//     of its own; final pivots and log P(Y) are FP64;
//   * panel solves in FP32 SIMT, trailing updates on tensor cores (3xTF32,
//     FP32 accumulate) or FP32 SIMT;
//   * a decision is exact outside the borderline band and made in FP64 on a
//     recomputed pivot inside it.
// Borderline test: a pivot whose uniform lies within
//   tau_j = c * 2^-22 * sqrt(j + 1) * (K_jj + s_j),   s_j = sum_k |l_jk w_jk|,
// of its threshold is recomputed in FP64 from the original K (the exact
// conditional probability, Props. 3-5) before its decision.
//
// Blocking (two levels): a 32-wide inner panel carries the sequential
// decisions (one warp) and the panel solve (all CTAs, one cooperative launch);
// the inner panels of one outer block of width NB (<= 256) are updated
// left-looking from the previous inner panels of the same outer block; after
// each outer block one rank-NB trailing update is applied to the whole
// remaining lower triangle, which makes the dominant contraction NB deep.
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"
#include "dpp_recompute.cuh"

namespace dpp {

Tuning g_tuning;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kUEff = 0x1.0p-22;

__device__ inline float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct MixedPanelArgs {
  const double* K;
  int64_t ldk;
  float* A;
  int64_t lda, n, q, p;
  int b, NB;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double* piv;
  double* kd;
  double* s;
  float *Wk, *Lk, *Wh, *Wl, *Lh, *Ll;
  dpp_result* res;
  unsigned* flag;
  unsigned epoch;
  double tol, tau_c;
  RecomputeArgs rc;
};

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

// Panel of the mixed path: decisions on the 32 x 32 diagonal block (CTA 0,
// warp 0), then the FP32 panel solve for every row below (all CTAs).
//
// The decision loop runs in FP32 (FP64 instructions cost ~64 cycles per warp
// on this part, and the loop is a strict sequential chain): the running
// diagonal is a double-float (~48 bits), the Bernoulli test u < d and the
// borderline test |u - d| <= tau are evaluated in FP32 with tau widened by the
// FP32 rounding of u and d (2^-22 absolute). Outside the band the FP32 test
// and the FP64 test cannot disagree; inside it the pivot is recomputed in FP64
// from K and decided in FP64. Final pivots and log|d| are then formed in FP64,
// once per panel, in parallel over the lanes.
__global__ void __launch_bounds__(kPanelThreads) k_panel_mixed(MixedPanelArgs a) {
  __shared__ float blk[kPanel][kPanel + 1];
  __shared__ float srd[kPanel];
  __shared__ int s_ok;
  float* A = a.A;
  const int b = a.b;
  const int64_t q = a.q, lda = a.lda;

  if (blockIdx.x == 0) {
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      float v = 0.f;
      if (i < b && k < b) v = (k <= i) ? A[(q + i) + (q + k) * lda] : A[(q + k) + (q + i) * lda];
      blk[i][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double u = 2.0;
      float uf = 2.f, si = 0.f, kf = 0.f;
      f2 dd = {0.f, 0.f};
      if (lane < b) {
        u = a.uniforms ? a.uniforms[q + lane] : philox_uniform(a.seed, a.inst, (uint64_t)(q + lane));
        uf = (float)u;
        dd = f2_from_double(a.kd[q + lane]);
        si = (float)a.s[q + lane];
        kf = (float)a.K[(q + lane) + (q + lane) * a.ldk];
      }
      const float tau0 = (float)(a.tau_c * kUEff);
      int border = 0, seq = 0;
      float max_ratio = 0.f;
      bool rc_failed = false;
      bool mykeep = false;
      for (int j = 0; j < b; ++j) {
        const float ph = __shfl_sync(kFull, dd.hi, j);
        const float uj = __shfl_sync(kFull, uf, j);
        const float sj = __shfl_sync(kFull, si, j);
        const float kj = __shfl_sync(kFull, kf, j);
        const float tau = tau0 * sqrtf((float)(q + j + 1)) * (fabsf(kj) + sj) + 0x1.0p-22f;
        bool kp;
        float df;
        if (fabsf(uj - ph) <= tau) {
          // Borderline: recompute d_j in FP64 from K with the worker CTAs and
          // decide in FP64.
          const double p64 = f2_to_double(make_f2(ph, __shfl_sync(kFull, dd.lo, j)));
          if (lane < j) a.piv[q + lane] = f2_to_double(dd);
          double pe = p64, est = 0.0;
          const bool ok = recompute_leader(a.rc, blk, b, j, a.epoch, &seq, &pe, &est);
          const double ujd = __shfl_sync(kFull, u, j);
          kp = ujd < pe;
          const double dfin = kp ? pe : pe - 1.0;
          df = (float)dfin;
          if (lane == j) dd = f2_from_double(dfin);
          ++border;
          const float ratio = (float)(fabs(pe - p64) / (double)tau);
          max_ratio = fmaxf(max_ratio, ratio);
          if (!ok || est > fabs(ujd - pe)) rc_failed = true;
        } else {
          kp = uj < ph;
          df = kp ? ph : ph - 1.0f;
          if (lane == j && !kp) dd = f2_add_f(dd, -1.0f);
        }
        const float rd = 1.0f / df;
        __syncwarp();
        if (lane > j && lane < b) {
          const float w = blk[lane][j];
          const float l = w * rd;
          for (int k = j + 1; k < b; ++k) blk[lane][k] = fmaf(-l, blk[j][k], blk[lane][k]);
          blk[lane][j] = l;
          dd = f2_sub_prod(dd, w, l);
          si += fabsf(w * l);
        }
        if (lane == j) mykeep = kp;
        if (lane == 0) {
          blk[j][j] = df;
          a.keep[q + j] = kp ? 1 : 0;
        }
        __syncwarp();
      }
      // final pivots (FP64), likelihood and bookkeeping, one lane per row
      double lp = 0.0;
      int kept = 0, oor = 0, bad = 0;
      if (lane < b) {
        const double d = f2_to_double(dd);
        const double pre = mykeep ? d : d + 1.0;
        a.piv[q + lane] = d;
        srd[lane] = (float)(1.0 / d);
        lp = log(fabs(d));
        kept = mykeep ? 1 : 0;
        oor = (pre < -a.tol || pre > 1.0 + a.tol) ? 1 : 0;
        bad = isfinite(d) ? 0 : 1;
      } else {
        srd[lane] = 1.f;
      }
      lp = warp_sum(lp);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        kept += __shfl_xor_sync(kFull, kept, o);
        oor += __shfl_xor_sync(kFull, oor, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
      }
      if (lane == 0) {
        dpp_result* r = a.res;
        r->logp += lp;
        if (kept) atomicAdd(&r->n_kept, kept);
        if (oor) {
          atomicAdd(&r->n_out_of_range, oor);
          atomicOr(&r->status, DPP_RES_INADMISSIBLE);
        }
        if (bad) atomicOr(&r->status, DPP_RES_NONFINITE);
        if (border) {
          atomicAdd(&r->n_borderline, border);
          if ((double)max_ratio > r->max_err_ratio) r->max_err_ratio = (double)max_ratio;
        }
        if (rc_failed) atomicOr(&r->status, DPP_RES_RECOMPUTE);
      }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k <= i) A[(q + i) + (q + k) * lda] = blk[i][k];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) recompute_release_done(a.rc, a.epoch);
  } else {
    // Serve recompute requests until CTA 0 reports the decisions done.
    if (!recompute_follower(a.rc, a.epoch, &s_ok)) return;
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k < i) blk[i][k] = __ldcg(&A[(q + i) + (q + k) * lda]);
    }
    if (threadIdx.x < kPanel) {
      const double d = threadIdx.x < b ? __ldcg(&a.piv[q + threadIdx.x]) : 1.0;
      srd[threadIdx.x] = (float)(1.0 / d);
    }
    __syncthreads();
  }

  // Panel solve for rows below the block (FP32): w = a L11^{-T}, l = w / d.
  const int64_t m = a.n - q - b;
  const int t0 = (int)(q - a.p);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q + b + r;
    float w[kPanel];
#pragma unroll
    for (int k = 0; k < kPanel; ++k) w[k] = (k < b) ? A[i + (q + k) * lda] : 0.f;
#pragma unroll
    for (int k = 1; k < kPanel; ++k) {
      if (k < b) {
#pragma unroll
        for (int t = 0; t < k; ++t) w[k] = fmaf(-w[t], blk[k][t], w[k]);
      }
    }
    float l[kPanel];
    f2 dsum = {0.f, 0.f};
    float ssum = 0.f;
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
      if (k < b) {
        l[k] = w[k] * srd[k];
        dsum = f2_add_prod(dsum, w[k], l[k]);
        ssum += fabsf(w[k] * l[k]);
        A[i + (q + k) * lda] = l[k];
      } else {
        l[k] = 0.f;
        w[k] = 0.f;
      }
    }
    a.kd[i] -= f2_to_double(dsum);
    a.s[i] += (double)ssum;
    const int64_t off = i * (int64_t)a.NB + t0;
    float4* wk = reinterpret_cast<float4*>(a.Wk + off);
    float4* lk = reinterpret_cast<float4*>(a.Lk + off);
    float4* wh = reinterpret_cast<float4*>(a.Wh + off);
    float4* wlo = reinterpret_cast<float4*>(a.Wl + off);
    float4* lh = reinterpret_cast<float4*>(a.Lh + off);
    float4* llo = reinterpret_cast<float4*>(a.Ll + off);
#pragma unroll
    for (int v = 0; v < kPanel / 4; ++v) {
      float4 W4 = make_float4(w[4 * v], w[4 * v + 1], w[4 * v + 2], w[4 * v + 3]);
      float4 L4 = make_float4(l[4 * v], l[4 * v + 1], l[4 * v + 2], l[4 * v + 3]);
      float4 WH = make_float4(tf32_rna(W4.x), tf32_rna(W4.y), tf32_rna(W4.z), tf32_rna(W4.w));
      float4 LH = make_float4(tf32_rna(L4.x), tf32_rna(L4.y), tf32_rna(L4.z), tf32_rna(L4.w));
      float4 WL = make_float4(tf32_rna(W4.x - WH.x), tf32_rna(W4.y - WH.y), tf32_rna(W4.z - WH.z),
                              tf32_rna(W4.w - WH.w));
      float4 LL = make_float4(tf32_rna(L4.x - LH.x), tf32_rna(L4.y - LH.y), tf32_rna(L4.z - LH.z),
                              tf32_rna(L4.w - LH.w));
      wk[v] = W4;
      lk[v] = L4;
      wh[v] = WH;
      wlo[v] = WL;
      lh[v] = LH;
      llo[v] = LL;
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
    tr = (int64_t)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while (tr * (tr + 1) / 2 > x) --tr;
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
  float *Wk, *Lk, *Wh, *Wl, *Lh, *Ll;
  double *kd, *s, *piv;
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
  L->Wh = static_cast<float*>(ws.take(ob));
  L->Wl = static_cast<float*>(ws.take(ob));
  L->Lh = static_cast<float*>(ws.take(ob));
  L->Ll = static_cast<float*>(ws.take(ob));
  L->kd = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->s = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->piv = static_cast<double*>(ws.take(sizeof(double) * nn));
  L->flag = static_cast<unsigned*>(ws.take(256));
  L->err = reinterpret_cast<int*>(L->flag) + 16;
  if (!recompute_carve(ws, n, &L->rs)) return false;
  return L->A32 && L->Wk && L->Lk && L->Wh && L->Wl && L->Lh && L->Ll && L->kd && L->s &&
         L->piv && L->flag;
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
  if ((e = recompute_reset(L.rs, a.stream)) != cudaSuccess) return e;
  const double* K = static_cast<const double*>(a.K);
  {
    ProfScope ps(kProfConvert, a.stream, 0.0, 12.0 * (double)n * (double)n / 2.0);
    k_convert<<<(unsigned)(n < 65535 ? n : 65535), 256, 0, a.stream>>>(K, a.ld, L.A32, L.ld32, n,
                                                                        L.kd, L.s);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  static int cap = 0;
  if (cap == 0) cap = coop_capacity(k_panel_mixed, kPanelThreads);
  unsigned epoch = 1;
  const bool use_tc = g_tuning.update_kernel == 0;
  for (int64_t p = 0; p < n; p += NB) {
    const int NBp = (int)((n - p) < NB ? (n - p) : NB);
    for (int64_t q = p; q < p + NBp; q += kPanel, ++epoch) {
      const int b = (int)((n - q) < kPanel ? (n - q) : kPanel);
      if (q > p) {
        // left-looking inner update of columns [q, q+b) from [p, q)
        F32Args u;
        u.C = L.A32;
        u.ldc = L.ld32;
        u.row0 = q;
        u.n = n;
        u.col0 = q;
        u.col1 = q + b;
        u.Aop = L.Wk;
        u.Bop = L.Lk;
        u.ldk = NB;
        u.kk = (int)(q - p);
        u.tiles_r = (n - q + kT - 1) / kT;
        const double fl = 2.0 * (double)(n - q) * (double)b * (double)u.kk;
        ProfScope ps(kProfUpdateF32, a.stream, fl, 0.0);
        k_f32_update<false><<<(unsigned)u.tiles_r, 256, 0, a.stream>>>(u);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      MixedPanelArgs pa;
      pa.K = K;
      pa.ldk = a.ld;
      pa.A = L.A32;
      pa.lda = L.ld32;
      pa.n = n;
      pa.q = q;
      pa.p = p;
      pa.b = b;
      pa.NB = NB;
      pa.uniforms = a.uniforms;
      pa.seed = a.seed;
      pa.inst = a.instance;
      pa.keep = a.keep;
      pa.piv = L.piv;
      pa.kd = L.kd;
      pa.s = L.s;
      pa.Wk = L.Wk;
      pa.Lk = L.Lk;
      pa.Wh = L.Wh;
      pa.Wl = L.Wl;
      pa.Lh = L.Lh;
      pa.Ll = L.Ll;
      pa.res = a.result;
      pa.flag = L.flag;
      pa.epoch = epoch;
      pa.tol = 1e-3;
      pa.tau_c = g_tuning.tau_safety;
      pa.rc = recompute_args(L.rs, K, a.ld, L.A32, L.ld32, L.piv, a.keep, n, q, a.result);
      // at least two CTAs: CTA 0 decides, the others serve FP64 recomputes
      int64_t g = (n - q - b + 63) / 64;
      if (g < 2) g = 2;
      if (g > cap) g = cap;
      pa.rc.grid = (int)g;
      void* args[] = {&pa};
      {
        ProfScope ps(kProfPanel, a.stream);
        e = cudaLaunchCooperativeKernel((const void*)k_panel_mixed, dim3((unsigned)g),
                                        dim3(kPanelThreads), args, 0, a.stream);
      }
      if (e != cudaSuccess) return e;
    }
    const int64_t r0 = p + NBp;
    if (r0 < n) {
      const int64_t m = n - r0;
      const double fl = (double)m * (double)m * (double)NBp;  // lower half of 2 m^2 NB
      if (use_tc && NBp % 32 == 0) {
        ProfScope ps(kProfUpdateTc, a.stream, fl, 8.0 * (double)m * (double)m / 2.0);
        e = outer_update_tc(L.A32, L.ld32, n, r0, NBp, L.Wh, L.Wl, L.Lh, L.Ll, NB, L.err, a.stream);
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
