// Adjoint of the log-likelihood of a fixed sample:
//
//   log P(Y) = log|det(K - 1_{Y^c})|  (Theorem 1)   =>   dK = g (K - 1_{Y^c})^{-H}
//
// (d log|det A| = Re tr(A^{-1} dA); in the complex-gradient convention the
// gradient is A^{-H}). The factors of A = K - 1_{Y^c} are recomputed by the
// sampler's own kernels with every decision forced to the given sample
// (uniforms -inf / +inf), then
//   LDL^H:  Z = L^{-1},  A^{-1} = Z^H D^{-1} Z
//   LU   :  Z = L^{-1},  V = U^{-1},  A^{-1} = V Z
// with the triangular inverses computed by blocked solves on the identity and
// the products restricted to the k-range where both triangular factors are
// nonzero (k >= max(i, j)). Everything runs in FP64 (real or complex).
#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

constexpr int kB = 32;   // triangular block
constexpr int kGT = 64;  // GEMM tile

template <class T>
__global__ void k_forced_uniforms(const uint8_t* keep, int64_t n, double* u) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    u[j] = keep[j] ? -1e300 : 1e300;
}

template <class T>
__global__ void k_identity(T* B, int64_t ldb, int64_t n) {
  using S = Sc<T>;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      B[i + j * ldb] = (i == j) ? S::from_real(1.0) : S::zero();
}

// Solve with the diagonal block T[k0:k0+nb, k0:k0+nb] of F for columns
// [c_lo, c_hi) of B, rows [k0, k0+nb):
//   LOWER_UNIT : X = L_kk^{-1} B_k     (forward, unit diagonal)
//   UPPER      : X = U_kk^{-1} B_k     (backward, diagonal from F)
template <class T, bool LOWER_UNIT>
__global__ void __launch_bounds__(256) k_trsm_block(const T* F, int64_t ldf, T* B, int64_t ldb,
                                                    int64_t k0, int nb, int64_t c_lo,
                                                    int64_t c_hi) {
  using S = Sc<T>;
  __shared__ T sT[kB][kB + 1];
  for (int idx = threadIdx.x; idx < kB * kB; idx += blockDim.x) {
    const int i = idx % kB, k = idx / kB;
    sT[i][k] = (i < nb && k < nb) ? F[(k0 + i) + (k0 + k) * ldf] : S::zero();
  }
  __syncthreads();
  for (int64_t c = c_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < c_hi;
       c += (int64_t)gridDim.x * blockDim.x) {
    T x[kB];
#pragma unroll
    for (int r = 0; r < kB; ++r) x[r] = (r < nb) ? B[(k0 + r) + c * ldb] : S::zero();
    if (LOWER_UNIT) {
#pragma unroll
      for (int r = 1; r < kB; ++r)
#pragma unroll
        for (int t = 0; t < r; ++t) x[r] = S::fnms(x[r], sT[r][t], x[t]);
    } else {
#pragma unroll
      for (int r = kB - 1; r >= 0; --r) {
        if (r < nb) {
#pragma unroll
          for (int t = r + 1; t < kB; ++t)
            if (t < nb) x[r] = S::fnms(x[r], sT[r][t], x[t]);
          x[r] = S::div(x[r], sT[r][r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < kB; ++r)
      if (r < nb) B[(k0 + r) + c * ldb] = x[r];
  }
}

// Generic tiled GEMM on a rectangle of C:
//   C[i, j] = (SUB ? C[i, j] - s : s),  s = sum_{k in [klo, khi)} opA(i, k) B[k, j]
// opA(i, k) = A[i + k lda] (CONJ_A false) or conj(A[k + i lda]) (CONJ_A true).
// KFROM_TILE: klo = max(klo, tile's first row, tile's first column) (products
// of triangular factors). LOWER_TILES: only tiles with tr >= tc of a square
// region (row_lo == col_lo).
struct GemmArgs {
  void* C;
  int64_t ldc;
  const void* A;
  int64_t lda;
  const void* B;
  int64_t ldb;
  int64_t row_lo, row_hi, col_lo, col_hi, klo, khi;
  int64_t tiles_r;
};

template <class T, bool CONJ_A, bool SUB, bool KFROM_TILE, bool LOWER_TILES>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs g) {
  using S = Sc<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);  // [32][kGT + 1] (k-major)
  T* sB = sA + 32 * (kGT + 1);             // [32][kGT + 1]
  int64_t tr, tc;
  const int64_t x = blockIdx.x;
  if (LOWER_TILES) {
    tr = (int64_t)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while (tr * (tr + 1) / 2 > x) --tr;
    while ((tr + 1) * (tr + 2) / 2 <= x) ++tr;
    tc = x - tr * (tr + 1) / 2;
  } else {
    tr = x % g.tiles_r;
    tc = x / g.tiles_r;
  }
  const int64_t i0 = g.row_lo + tr * kGT, j0 = g.col_lo + tc * kGT;
  int64_t klo = g.klo;
  if (KFROM_TILE) {
    klo = klo > i0 ? klo : i0;
    klo = klo > j0 ? klo : j0;
  }
  const T* A = static_cast<const T*>(g.A);
  const T* B = static_cast<const T*>(g.B);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[p][r] = S::zero();
  for (int64_t k0 = klo; k0 < g.khi; k0 += 32) {
    for (int idx = threadIdx.x; idx < 32 * kGT; idx += 256) {
      int kk, ii;
      if (CONJ_A) {
        kk = idx % 32;
        ii = idx / 32;
      } else {
        ii = idx % kGT;
        kk = idx / kGT;
      }
      const int64_t i = i0 + ii, k = k0 + kk;
      T v = S::zero();
      if (i < g.row_hi && k < g.khi) v = CONJ_A ? S::conj(A[k + i * g.lda]) : A[i + k * g.lda];
      sA[kk * (kGT + 1) + ii] = v;
    }
    for (int idx = threadIdx.x; idx < 32 * kGT; idx += 256) {
      const int kk = idx % 32, jj = idx / 32;
      const int64_t j = j0 + jj, k = k0 + kk;
      sB[kk * (kGT + 1) + jj] = (j < g.col_hi && k < g.khi) ? B[k + j * g.ldb] : S::zero();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      T ra[4], rb[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) ra[p] = sA[kk * (kGT + 1) + tx + 16 * p];
#pragma unroll
      for (int r = 0; r < 4; ++r) rb[r] = sB[kk * (kGT + 1) + ty + 16 * r];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[p][r] = S::fnms(acc[p][r], ra[p], rb[r]);  // acc = -sum
    }
    __syncthreads();
  }
  T* C = static_cast<T*>(g.C);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t j = j0 + ty + 16 * r;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t i = i0 + tx + 16 * p;
      if (i < g.row_hi && j < g.col_hi) {
        T* dst = &C[i + j * g.ldc];
        *dst = SUB ? S::add(*dst, acc[p][r]) : S::sub(S::zero(), acc[p][r]);
      }
    }
  }
}

// W[i, j] = Z[i, j] / d_i  (rows scaled by the inverse pivots)
template <class T>
__global__ void k_scale_rows(const T* Z, int64_t ldz, const double* piv, T* W, int64_t ldw,
                             int64_t n) {
  using S = Sc<T>;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x)
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
      W[i + j * ldw] = S::div_real(Z[i + j * ldz], piv[i]);
}

// dK = g X^H for a full X; HERM_LOWER: X given in its lower triangle only
// (X Hermitian), so dK = g X (mirrored).
template <class T, bool HERM_LOWER>
__global__ void k_finish(const T* X, int64_t ldx, const double* g, T* dK, int64_t ldd,
                         int64_t n) {
  using S = Sc<T>;
  const double s = *g;
  for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      T v;
      if (HERM_LOWER) {
        v = (i >= j) ? X[i + j * ldx] : S::conj(X[j + i * ldx]);
      } else {
        v = S::conj(X[j + i * ldx]);  // (X^H)_{ij}
      }
      dK[i + j * ldd] = S::mul(S::from_real(s), v);
    }
  }
}

template <class T, bool CONJ_A, bool SUB, bool KFT, bool LT>
cudaError_t gemm(const GemmArgs& g0, cudaStream_t s) {
  GemmArgs g = g0;
  const int64_t rows = g.row_hi - g.row_lo, cols = g.col_hi - g.col_lo;
  if (rows <= 0 || cols <= 0 || g.khi <= g.klo) return cudaSuccess;
  g.tiles_r = (rows + kGT - 1) / kGT;
  const int64_t tc = (cols + kGT - 1) / kGT;
  const int64_t nt = LT ? g.tiles_r * (g.tiles_r + 1) / 2 : g.tiles_r * tc;
  const size_t smem = sizeof(T) * 2 * 32 * (kGT + 1);
  auto k = k_gemm<T, CONJ_A, SUB, KFT, LT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const double cf = Sc<T>::cplx ? 8.0 : 2.0;
  ProfScope ps(kProfOther, s, cf * (double)rows * (double)cols * (double)(g.khi - g.klo), 0.0);
  k<<<(unsigned)nt, 256, smem, s>>>(g);
  return cudaGetLastError();
}

// Z := L^{-1} (unit lower part of F), Z initialised to the identity.
template <class T>
cudaError_t invert_unit_lower(const T* F, int64_t ldf, T* Z, int64_t n, cudaStream_t s) {
  cudaError_t e;
  for (int64_t k0 = 0; k0 < n; k0 += kB) {
    const int nb = (int)((n - k0) < kB ? (n - k0) : kB);
    const int64_t c_hi = k0 + nb;  // columns beyond are still identity-free zeros
    {
      ProfScope ps(kProfOther, s);
      int64_t gdim = (c_hi + 255) / 256;
      k_trsm_block<T, true><<<(unsigned)gdim, 256, 0, s>>>(F, ldf, Z, n, k0, nb, 0, c_hi);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmArgs g;
    g.C = Z;
    g.ldc = n;
    g.A = F;
    g.lda = ldf;
    g.B = Z;
    g.ldb = n;
    g.row_lo = k0 + nb;
    g.row_hi = n;
    g.col_lo = 0;
    g.col_hi = c_hi;
    g.klo = k0;
    g.khi = k0 + nb;
    if ((e = gemm<T, false, true, false, false>(g, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// V := U^{-1} (upper part of F incl. diagonal), V initialised to the identity.
template <class T>
cudaError_t invert_upper(const T* F, int64_t ldf, T* V, int64_t n, cudaStream_t s) {
  cudaError_t e;
  const int64_t nblk = (n + kB - 1) / kB;
  for (int64_t b = nblk - 1; b >= 0; --b) {
    const int64_t k0 = b * kB;
    const int nb = (int)((n - k0) < kB ? (n - k0) : kB);
    {
      ProfScope ps(kProfOther, s);
      int64_t gdim = (n - k0 + 255) / 256;
      k_trsm_block<T, false><<<(unsigned)gdim, 256, 0, s>>>(F, ldf, V, n, k0, nb, k0, n);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmArgs g;
    g.C = V;
    g.ldc = n;
    g.A = F;
    g.lda = ldf;
    g.B = V;
    g.ldb = n;
    g.row_lo = 0;
    g.row_hi = k0;
    g.col_lo = k0;
    g.col_hi = n;
    g.klo = k0;
    g.khi = k0 + nb;
    if ((e = gemm<T, false, true, false, false>(g, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class T>
cudaError_t run_backward(const void* K, int64_t n, int64_t ld, int32_t dtype, bool herm,
                         const uint8_t* keep, const double* grad, void* dK, int64_t ld_dk,
                         Workspace ws, cudaStream_t s) {
  const size_t esz = sizeof(T);
  const size_t nn = (size_t)n * (size_t)n;
  T* F = static_cast<T*>(ws.take(esz * nn));
  T* Z = static_cast<T*>(ws.take(esz * nn));
  T* X = static_cast<T*>(ws.take(esz * nn));
  double* u = static_cast<double*>(ws.take(sizeof(double) * (size_t)n));
  double* piv = static_cast<double*>(ws.take(sizeof(double) * 2 * (size_t)n));
  uint8_t* kept = static_cast<uint8_t*>(ws.take((size_t)n));
  dpp_result* res = static_cast<dpp_result*>(ws.take(sizeof(dpp_result)));
  if (!F || !Z || !X || !u || !piv || !kept || !res) return cudaErrorInvalidValue;
  Workspace inner;
  inner.base = ws.base + ws.used;
  inner.size = ws.size - ws.used;
  cudaError_t e;
  {
    ProfScope ps(kProfOther, s);
    k_forced_uniforms<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keep, n, u);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // 1. factors of K - 1_{Y^c}: the sampler with every decision forced
  DrawArgs a;
  a.K = K;
  a.n = n;
  a.ld = ld;
  a.dtype = dtype;
  a.precision = DPP_PREC_FP64;
  a.seed = 0;
  a.instance = 0;
  a.uniforms = u;
  a.keep = kept;
  a.factor_out = nullptr;
  a.pivots_user = piv;
  a.result = res;
  a.stream = s;
  // factor into F (ld = n) through factor_out semantics
  if ((e = cudaMemcpy2DAsync(F, n * esz, K, ld * esz, n * esz, n, cudaMemcpyDeviceToDevice, s)) !=
      cudaSuccess)
    return e;
  a.K = F;
  a.ld = n;
  a.factor_out = F;
  if ((e = sample_fp64(a, herm, inner)) != cudaSuccess) return e;
  // 2. Z = L^{-1}
  {
    ProfScope ps(kProfOther, s);
    k_identity<T><<<(unsigned)(n < 65535 ? n : 65535), 256, 0, s>>>(Z, n, n);
  }
  if ((e = invert_unit_lower<T>(F, n, Z, n, s)) != cudaSuccess) return e;
  if (herm) {
    // 3. W = D^{-1} Z (into X), then lower triangle of A^{-1} = Z^H W into F
    {
      ProfScope ps(kProfOther, s);
      k_scale_rows<T><<<(unsigned)(n < 65535 ? n : 65535), 256, 0, s>>>(Z, n, piv, X, n, n);
    }
    GemmArgs g;
    g.C = F;
    g.ldc = n;
    g.A = Z;
    g.lda = n;
    g.B = X;
    g.ldb = n;
    g.row_lo = 0;
    g.row_hi = n;
    g.col_lo = 0;
    g.col_hi = n;
    g.klo = 0;
    g.khi = n;
    if ((e = gemm<T, true, false, true, true>(g, s)) != cudaSuccess) return e;
    ProfScope ps(kProfOther, s);
    k_finish<T, true><<<(unsigned)(n < 65535 ? n : 65535), 256, 0, s>>>(
        F, n, grad, static_cast<T*>(dK), ld_dk, n);
  } else {
    // 3. V = U^{-1} (into X), A^{-1} = V Z (into F... F still holds U: use dK's
    //    workspace copy) — compute into the u/piv-free buffer X2 = F after V is formed
    {
      ProfScope ps(kProfOther, s);
      k_identity<T><<<(unsigned)(n < 65535 ? n : 65535), 256, 0, s>>>(X, n, n);
    }
    if ((e = invert_upper<T>(F, n, X, n, s)) != cudaSuccess) return e;
    GemmArgs g;
    g.C = F;  // U no longer needed
    g.ldc = n;
    g.A = X;
    g.lda = n;
    g.B = Z;
    g.ldb = n;
    g.row_lo = 0;
    g.row_hi = n;
    g.col_lo = 0;
    g.col_hi = n;
    g.klo = 0;
    g.khi = n;
    if ((e = gemm<T, false, false, true, false>(g, s)) != cudaSuccess) return e;
    ProfScope ps(kProfOther, s);
    k_finish<T, false><<<(unsigned)(n < 65535 ? n : 65535), 256, 0, s>>>(
        F, n, grad, static_cast<T*>(dK), ld_dk, n);
  }
  return cudaGetLastError();
}

}  // namespace

size_t ws_backward(int64_t n, int32_t dtype, bool hermitian) {
  const size_t esz = dtype == DPP_C128 ? 16 : 8;
  const size_t nn = (size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1);
  size_t b = 3 * align256(esz * nn) + 2 * align256(sizeof(double) * 2 * (size_t)(n + 1)) +
             align256((size_t)n + 1) + align256(sizeof(dpp_result));
  b += ws_fp64(n, dtype, hermitian, false);
  return b + 1024;
}

cudaError_t logprob_backward(const void* K, int64_t n, int64_t ld, int32_t dtype, bool hermitian,
                             const uint8_t* keep, const double* grad, void* dK, int64_t ld_dk,
                             Workspace ws, cudaStream_t stream) {
  if (dtype == DPP_C128)
    return run_backward<cdouble>(K, n, ld, dtype, hermitian, keep, grad, dK, ld_dk, ws, stream);
  return run_backward<double>(K, n, ld, dtype, hermitian, keep, grad, dK, ld_dk, ws, stream);
}

}  // namespace dpp
