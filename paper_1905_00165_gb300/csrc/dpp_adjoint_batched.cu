// Adjoint of log P(Y_i) for a batch of real symmetric kernels in ONE
// persistent launch:
//
//   log P(Y) = log|det(K - 1_{Y^c})|  (Theorem 1)   =>   dK = g (K - 1_{Y^c})^{-1}
//
// Each CTA takes the next instance from a device counter over the instances
// sorted by decreasing n (longest first), and does the whole instance in
// FP64 with 32 x 32 tiles staged in shared memory:
//   1. A = K - 1_{Y^c} (lower triangle) in the instance's dK buffer, and its
//      blocked LDL^T in place (the decisions are the given sample, so no
//      uniforms: each pivot is taken as it comes);
//   2. the inverses of the 32 x 32 unit lower diagonal blocks of L;
//   3. Z = L^{-1}, block row by block row:  Z_IJ = L_II^{-1} (delta_IJ - sum_K L_IK Z_KJ);
//   4. A^{-1} = Z^T D^{-1} Z on the lower tiles (k >= max(i, j)), times g,
//      written to both triangles of dK.
// GB300's FP64 rate is a small fraction of its FP32 rate, so the work is
// FP64-compute-bound; one instance per CTA keeps every SM busy without any
// inter-CTA synchronisation. The adjoint may instead run in FP32 (the working
// matrix then lives in the scratch, the result is widened to FP64 in dK): the
// same steps at the FP32 rate, with FP32 rounding in the factor and inverse.
//
// The same launch converts L-ensembles to marginal kernels (mode kLEnsemble):
// with A = L + I (positive definite for positive semi-definite L) in step 1
// and  K = I - A^{-1} = L (L + I)^{-1}  written in step 4.
#include <algorithm>
#include <vector>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

constexpr int kAT = 256;  // threads per CTA

enum { kAdjoint = 0, kLEnsemble = 1 };

struct AdjDesc {
  const double* K;      // K (adjoint) or L (L-ensemble), lower triangle read
  const uint8_t* keep;  // adjoint only
  const double* g;      // adjoint only
  double* dK;           // output: g A^{-1} (adjoint) or I - A^{-1} (L-ensemble)
  int64_t n, ld, ldd;
  int mode;
};

struct AdjArgs {
  const AdjDesc* desc;  // sorted by decreasing n
  int32_t batch;
  unsigned* counter;
  void* scratch;        // per CTA (elements of the working type): Z [ldz x ldz],
                        // W [ldz x 32], Linv [nt x 1024], d [ldz], and for FP32
                        // the working matrix [ldz x ldz]
  int64_t per_cta;      // elements per CTA
  int64_t ldz;          // n_max rounded up to 32
};

__shared__ unsigned s_inst;

__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct AdjTiles {
  T a[32][33];
  T b[32][33];
  T c[32][33];
};

// acc[j] (thread: row r = lane, column cg + 8 j) += sum_t s_a[r][t] s_b[cg + 8 j][t]
template <typename T>
__device__ __forceinline__ void tile_abT(const AdjTiles<T>& S, T (&acc)[4]) {
  const int r = threadIdx.x & 31, cg = threadIdx.x >> 5;
#pragma unroll 8
  for (int t = 0; t < 32; ++t) {
    const T a = S.a[r][t];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] = tfma(a, S.b[cg + 8 * j][t], acc[j]);
  }
}

template <typename T>
__device__ void adjoint_one(const AdjArgs& a, const AdjDesc& d, T* scr, AdjTiles<T>& S) {
  auto& s_a = S.a;
  auto& s_b = S.b;
  auto& s_c = S.c;
  constexpr bool kF64 = sizeof(T) == 8;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  const int r = lane, cg = wp;
  const int64_t n = d.n, ldz = a.ldz;
  const int nt = (int)((n + 31) / 32);
  T* Z = scr;
  T* Wb = Z + ldz * ldz;
  T* Linv = Wb + ldz * 32;
  T* dv = Linv + (int64_t)nt * 1024;
  // the working matrix: dK itself in FP64, a scratch matrix in FP32
  T* A = kF64 ? reinterpret_cast<T*>(d.dK) : dv + ldz + 32;
  const int64_t ldd = kF64 ? d.ldd : ldz;

  // ---- 1. A = K - 1_{Y^c} (adjoint) or L + I (L-ensemble), lower triangle ----
  const bool lens = d.mode == kLEnsemble;
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = j + tid; i < n; i += kAT) {
      double v = d.K[i + j * d.ld];
      if (i == j) {
        if (lens) v += 1.0;
        else if (d.keep[i] == 0) v -= 1.0;
      }
      A[i + j * ldd] = (T)v;
    }
  }
  __syncthreads();

  // ---- blocked LDL^T, right-looking ----
  for (int P = 0; P < nt; ++P) {
    const int64_t p = 32 * (int64_t)P;
    const int b = (int)((n - p) < 32 ? (n - p) : 32);
    // (a) diagonal block, one row per lane of warp 0, mirrored to full
    for (int idx = tid; idx < 1024; idx += kAT) {
      const int i = idx & 31, c = idx >> 5;
      T v = 0;
      if (i < b && c < b) v = i >= c ? A[(p + i) + (p + c) * ldd] : A[(p + c) + (p + i) * ldd];
      s_a[i][c] = v;
    }
    __syncthreads();
    if (wp == 0) {
      for (int J = 0; J < b; ++J) {
        const T dj = s_a[J][J];
        if (lane > J && lane < b) {
          const T l = s_a[lane][J] / dj;
          for (int c = J + 1; c < b; ++c) s_a[lane][c] = tfma(-l, s_a[J][c], s_a[lane][c]);
          s_a[lane][J] = l;
        }
        __syncwarp();
      }
      if (lane < b) {
        dv[p + lane] = s_a[lane][lane];
        for (int c = 0; c <= lane; ++c) A[(p + lane) + (p + c) * ldd] = s_a[lane][c];
      }
    }
    __syncthreads();
    // (b) rows below: W L11^T = A[i, p:p+b], L = W / d
    for (int64_t i = p + b + tid; i < n; i += kAT) {
      T w[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) w[c] = c < b ? A[i + (p + c) * ldd] : (T)0;
#pragma unroll
      for (int c = 1; c < 32; ++c) {
#pragma unroll
        for (int k = 0; k < c; ++k) w[c] = tfma(-w[k], s_a[c][k], w[c]);
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < b) {
          Wb[i * 32 + c] = w[c];
          A[i + (p + c) * ldd] = w[c] / dv[p + c];
        }
      }
    }
    __syncthreads();
    // (c) trailing update of the lower tiles: A_IJ -= W_I L_J^T
    for (int I = P + 1; I < nt; ++I) {
      for (int J = P + 1; J <= I; ++J) {
        for (int idx = tid; idx < 1024; idx += kAT) {
          const int rr = idx >> 5, t = idx & 31;
          const int64_t ri = 32 * (int64_t)I + rr, rj = 32 * (int64_t)J + rr;
          s_a[rr][t] = (ri < n && t < b) ? Wb[ri * 32 + t] : (T)0;
          s_b[rr][t] = (rj < n && t < b) ? A[rj + (p + t) * ldd] : (T)0;
        }
        __syncthreads();
        T acc[4] = {0, 0, 0, 0};
        tile_abT(S, acc);
        const int64_t i = 32 * (int64_t)I + r;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int64_t c = 32 * (int64_t)J + cg + 8 * j;
          if (i < n && c <= i) A[i + c * ldd] -= acc[j];
        }
        __syncthreads();
      }
    }
  }

  // ---- 2. inverses of the unit lower diagonal blocks (one warp each) ----
  for (int I = wp; I < nt; I += kAT / 32) {
    const int64_t p = 32 * (int64_t)I;
    const int b = (int)((n - p) < 32 ? (n - p) : 32);
    T z[32];  // column `lane` of the inverse
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      T s = 0;
      if (i > lane && i < b) {
#pragma unroll
        for (int k = 0; k < i; ++k)
          if (k >= lane) s = tfma(A[(p + i) + (p + k) * ldd], z[k], s);
      }
      z[i] = (i == lane) ? (T)1 : (i < lane || i >= b ? (T)0 : -s);
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) Linv[(int64_t)I * 1024 + i * 32 + lane] = z[i];
  }
  __syncthreads();

  // ---- 3. Z = L^{-1}, block rows in order ----
  for (int I = 0; I < nt; ++I) {
    for (int J = 0; J <= I; ++J) {
      T acc[4] = {0, 0, 0, 0};
      // T = sum_{K=J}^{I-1} L_IK Z_KJ   (acc holds T[r][c] with c = cg + 8 j)
      for (int K = J; K < I; ++K) {
        for (int idx = tid; idx < 1024; idx += kAT) {
          const int rr = idx >> 5, t = idx & 31;
          const int64_t ri = 32 * (int64_t)I + rr, ck = 32 * (int64_t)K + t;
          s_a[rr][t] = (ri < n && ck < n) ? A[ri + ck * ldd] : (T)0;
          // s_b[c][t] = Z[K*32 + t][J*32 + c]
          const int64_t zr = 32 * (int64_t)K + t, zc = 32 * (int64_t)J + rr;
          s_b[rr][t] = (zr < n && zc < n) ? Z[zr + zc * ldz] : (T)0;
        }
        __syncthreads();
        tile_abT(S, acc);
        __syncthreads();
      }
      // Z_IJ = Linv_I (delta_IJ - T)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = cg + 8 * j;
        s_c[c][r] = (I == J ? (r == c ? (T)1 : (T)0) : (T)0) - acc[j];  // transposed: s_c[c][t]
      }
      for (int idx = tid; idx < 1024; idx += kAT) {
        const int rr = idx >> 5, t = idx & 31;
        s_a[rr][t] = Linv[(int64_t)I * 1024 + rr * 32 + t];
      }
      __syncthreads();
      T z[4] = {0, 0, 0, 0};
#pragma unroll 8
      for (int t = 0; t < 32; ++t) {
        const T la = s_a[r][t];
#pragma unroll
        for (int j = 0; j < 4; ++j) z[j] = tfma(la, s_c[cg + 8 * j][t], z[j]);
      }
      const int64_t i = 32 * (int64_t)I + r;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t c = 32 * (int64_t)J + cg + 8 * j;
        if (i < n && c < n) Z[i + c * ldz] = z[j];
      }
      __syncthreads();
    }
  }

  // ---- 4. dK = g Z^T D^{-1} Z (or K = I - Z^T D^{-1} Z), lower tiles mirrored ----
  const T g = lens ? (T)-1 : (T)*d.g;
  for (int I = 0; I < nt; ++I) {
    for (int J = 0; J <= I; ++J) {
      T acc[4] = {0, 0, 0, 0};
      for (int K = I; K < nt; ++K) {
        for (int idx = tid; idx < 1024; idx += kAT) {
          const int rr = idx >> 5, t = idx & 31;
          const int64_t k = 32 * (int64_t)K + t;
          const int64_t ci = 32 * (int64_t)I + rr, cj = 32 * (int64_t)J + rr;
          // s_a[r][t] = Z[k][I*32 + r] / d_k ; s_b[c][t] = Z[k][J*32 + c]
          s_a[rr][t] = (k < n && ci < n) ? Z[k + ci * ldz] / dv[k] : (T)0;
          s_b[rr][t] = (k < n && cj < n) ? Z[k + cj * ldz] : (T)0;
        }
        __syncthreads();
        tile_abT(S, acc);
        __syncthreads();
      }
      const int64_t i = 32 * (int64_t)I + r;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int64_t c = 32 * (int64_t)J + cg + 8 * j;
        if (i < n && c <= i) {
          const double v = (double)(g * acc[j]) + ((lens && i == c) ? 1.0 : 0.0);
          d.dK[i + c * d.ldd] = v;
          d.dK[c + i * d.ldd] = v;
        }
      }
    }
  }
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kAT, 1) k_adjoint_batched(AdjArgs a) {
  __shared__ AdjTiles<T> S;
  T* scr = static_cast<T*>(a.scratch) + (int64_t)blockIdx.x * a.per_cta;
  while (true) {
    if (threadIdx.x == 0) s_inst = atomicAdd(a.counter, 1u);
    __syncthreads();
    const unsigned inst = s_inst;
    __syncthreads();
    if (inst >= (unsigned)a.batch) return;
    const AdjDesc d = a.desc[inst];
    if (d.n > 0) adjoint_one<T>(a, d, scr, S);
  }
}

inline int64_t adj_ldz(int64_t n_max) { return ((n_max + 31) / 32) * 32; }

// elements of the working type per CTA (FP32: also the working matrix)
inline int64_t adj_per_cta(int64_t n_max, bool fp32) {
  const int64_t ldz = adj_ldz(n_max > 0 ? n_max : 1);
  return ldz * ldz + ldz * 32 + (ldz / 32) * 1024 + ldz + 32 + (fp32 ? ldz * ldz : 0);
}
inline size_t adj_per_cta_bytes(int64_t n_max, bool fp32) {
  return (fp32 ? sizeof(float) : sizeof(double)) * (size_t)adj_per_cta(n_max, fp32);
}

inline size_t adj_header(int32_t batch) {
  return align256(sizeof(AdjDesc) * (size_t)(batch > 0 ? batch : 1)) + 256;
}

}  // namespace

size_t ws_adjoint_batched(int32_t batch, int64_t n_max, int ctas) {
  // (either precision: the FP64 layout is the larger)
  const size_t a = adj_per_cta_bytes(n_max, false), b = adj_per_cta_bytes(n_max, true);
  return adj_header(batch) + (a > b ? a : b) * (size_t)ctas + 256;
}

int adjoint_batched_ctas() {
  DevInfo di;
  if (dev_info(&di) != cudaSuccess || di.sm_count <= 0) return 1;
  int c = di.sm_count;
  if (g_tuning.max_ctas > 0 && c > g_tuning.max_ctas) c = g_tuning.max_ctas;
  return c;
}

cudaError_t adjoint_batched(int32_t batch, const int64_t* n, const double* const* K,
                            const int64_t* ld, const uint8_t* const* keep,
                            const double* const* g, double* const* dK, const int64_t* ld_dk,
                            int64_t n_max, bool fp32, Workspace ws, cudaStream_t s) {
  // descriptors, longest instance first
  std::vector<AdjDesc> h((size_t)batch);
  std::vector<int32_t> order((size_t)batch);
  for (int32_t i = 0; i < batch; ++i) order[(size_t)i] = i;
  std::sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return n[x] > n[y]; });
  for (int32_t k = 0; k < batch; ++k) {
    const int32_t i = order[(size_t)k];
    h[(size_t)k] = AdjDesc{K[i], keep ? keep[i] : nullptr, g ? g[i] : nullptr, dK[i],
                           n[i], ld[i], ld_dk[i], keep ? kAdjoint : kLEnsemble};
  }
  char* base = ws.base;
  AdjDesc* desc = reinterpret_cast<AdjDesc*>(base);
  unsigned* counter = reinterpret_cast<unsigned*>(base + adj_header(batch) - 256);
  const size_t used = adj_header(batch);
  const bool f32 = fp32 && keep != nullptr;  // the L-ensemble conversion stays FP64
  const int64_t per = adj_per_cta(n_max, f32);
  int ctas = adjoint_batched_ctas();
  const int64_t room = (int64_t)((ws.size - used) / adj_per_cta_bytes(n_max, f32));
  if (room < ctas) ctas = (int)room;
  if (ctas < 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemcpyAsync(desc, h.data(), sizeof(AdjDesc) * (size_t)batch,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  AdjArgs a;
  a.desc = desc;
  a.batch = batch;
  a.counter = counter;
  a.scratch = base + used;
  a.per_cta = per;
  a.ldz = adj_ldz(n_max > 0 ? n_max : 1);
  {
    ProfScope ps(keep ? kProfAdjoint : kProfLEnsemble, s);
    if (f32)
      k_adjoint_batched<float><<<(unsigned)ctas, kAT, 0, s>>>(a);
    else
      k_adjoint_batched<double><<<(unsigned)ctas, kAT, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace dpp
