// FP64 blocked DPP samplers (real and complex; Hermitian LDL^H and general LU).
//
// Algorithm 4 of arXiv:1905.00165 (the blocked form of Algorithm 1): for each
// kPanel-wide diagonal block J1 = [q, q+b)
//   a1  factor A[J1,J1] with the sequential Bernoulli decisions (one warp, one
//       row of the block per lane, the block in shared memory);
//   a2  solve the panels against it (Algorithm 3's two triangular solves):
//         LDL^H: W = A21 L11^{-H},  L21 = W D1^{-1}
//         LU   : L21 = A21 U11^{-1}, U12 = L11^{-1} A12;
//   a3  Schur update of the trailing block:
//         LDL^H: A22 -= W L21^H (lower triangle),  LU: A22 -= L21 U12.
// a1 and a2 run in one cooperative launch: CTA 0 makes the decisions, then
// releases a device flag on which every other CTA waits (bounded) before the
// row/column solves. a3 is a tiled SIMT DFMA kernel (GB300's FP64 rate is a
// small fraction of its FP32/tensor rates, so FP64 is compute-bound at any
// reasonable tile size).
#include <math.h>

#include "dpp_device.cuh"
#include "dpp_internal.h"
#include "dpp_profile.h"

namespace dpp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTile = 64;  // trailing-update tile (rows and columns)

struct PanelArgs {
  void* A;
  int64_t lda, n, q;
  int b;
  const double* uniforms;
  uint64_t seed, inst;
  uint8_t* keep;
  double* piv;  // final pivots: n doubles (real) or 2n (complex LU: re, im)
  dpp_result* res;
  void* W;  // LDL^H only: W = L21 D1, column-major, ldw
  int64_t ldw;
  unsigned* flag;
  unsigned epoch;
  double tol;
  unsigned long long wait_ns;  // limit of the other CTAs' wait for the release
  int withhold;                // fault injection: CTA 0 never releases the panel
};

template <class T>
__device__ inline T ldcg(const T* p);
template <>
__device__ inline double ldcg<double>(const double* p) { return __ldcg(p); }
template <>
__device__ inline cdouble ldcg<cdouble>(const cdouble* p) {
  const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Lane-0 bookkeeping of one decision (Theorem 1: the factor contributed to
// P(Y) is |d| after the decision).
struct DecisionLog {
  double lp = 0.0;
  int kept = 0, oor = 0, bad = 0;
  __device__ void add(double p_re, bool finite, bool kp, double absd, double tol) {
    if (!finite) bad = 1;
    if (p_re < -tol || p_re > 1.0 + tol) ++oor;
    kept += kp ? 1 : 0;
    lp += log(absd);
  }
  __device__ void flush(dpp_result* r) const {
    r->logp += lp;  // panels are stream-ordered: plain update is race-free
    if (kept) atomicAdd(&r->n_kept, kept);
    if (oor) {
      atomicAdd(&r->n_out_of_range, oor);
      atomicOr(&r->status, DPP_RES_INADMISSIBLE);
    }
    if (bad) atomicOr(&r->status, DPP_RES_NONFINITE);
  }
};

// Non-zero CTAs wait for CTA 0's release of this panel's epoch.
__device__ inline bool panel_wait(const PanelArgs& a, int* s_ok) {
  if (threadIdx.x == 0) {
    const bool ok = wait_geq(a.flag, a.epoch, a.wait_ns);
    if (!ok) flag_status(a.res, DPP_RES_TIMEOUT);
    *s_ok = ok ? 1 : 0;
    __threadfence();
  }
  __syncthreads();
  return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Hermitian (LDL^H) panel: decisions + W/L21 solve.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kPanelThreads) k_panel_herm(PanelArgs a) {
  using S = Sc<T>;
  __shared__ T blk[kPanel][kPanel + 1];
  __shared__ double sd[kPanel];
  __shared__ int s_ok;
  T* A = static_cast<T*>(a.A);
  const int b = a.b;
  const int64_t q = a.q, lda = a.lda;

  if (blockIdx.x == 0) {
    // Full Hermitian copy of the diagonal block (lower triangle read).
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      T v = S::zero();
      if (i < b && k < b)
        v = (k <= i) ? A[(q + i) + (q + k) * lda] : S::conj(A[(q + k) + (q + i) * lda]);
      blk[i][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double u = 0.0;
      if (lane < b)
        u = a.uniforms ? a.uniforms[q + lane] : philox_uniform(a.seed, a.inst, (uint64_t)(q + lane));
      DecisionLog log;
      for (int j = 0; j < b; ++j) {
        const double p = S::re(blk[j][j]);
        const double uj = __shfl_sync(kFull, u, j);
        const bool kp = uj < p;                 // Bernoulli(p): keep j
        const double d = kp ? p : p - 1.0;      // exclusion subtracts 1 (Prop. 4)
        __syncwarp();
        if (lane > j && lane < b) {
          // Row `lane` of the rank-1 Schur update (Prop. 3/4): the pivot row
          // j is read from its stored (mirrored) entries.
          const T l = S::div_real(blk[lane][j], d);
          for (int k = j + 1; k < b; ++k) blk[lane][k] = S::fnms(blk[lane][k], l, blk[j][k]);
          blk[lane][j] = l;
        }
        if (lane == 0) {
          blk[j][j] = S::from_real(d);
          log.add(p, isfinite(p), kp, fabs(d), a.tol);
          a.keep[q + j] = kp ? 1 : 0;
          a.piv[q + j] = d;
        }
        __syncwarp();
      }
      if (lane == 0) log.flush(a.res);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k <= i) A[(q + i) + (q + k) * lda] = blk[i][k];
    }
    if (threadIdx.x < kPanel) sd[threadIdx.x] = threadIdx.x < b ? S::re(blk[threadIdx.x][threadIdx.x]) : 1.0;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && !a.withhold) st_release(a.flag, a.epoch);
  } else {
    if (!panel_wait(a, &s_ok)) return;
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k < i) blk[i][k] = ldcg(&A[(q + i) + (q + k) * lda]);
    }
    if (threadIdx.x < kPanel) sd[threadIdx.x] = threadIdx.x < b ? __ldcg(&a.piv[q + threadIdx.x]) : 1.0;
    __syncthreads();
  }

  // a2: rows below the block. Row i: a = w L11^H  ->  w_k = a_k - sum_{t<k} w_t conj(L_kt).
  T* W = static_cast<T*>(a.W);
  const int64_t m = a.n - q - b;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < m;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = q + b + r;
    T w[kPanel];
#pragma unroll
    for (int k = 0; k < kPanel; ++k) w[k] = (k < b) ? A[i + (q + k) * lda] : S::zero();
#pragma unroll
    for (int k = 1; k < kPanel; ++k) {
      if (k < b) {
#pragma unroll
        for (int t = 0; t < k; ++t) w[k] = S::fnms_conj(w[k], w[t], blk[k][t]);
      }
    }
#pragma unroll
    for (int k = 0; k < kPanel; ++k) {
      if (k < b) {
        W[i + k * a.ldw] = w[k];
        A[i + (q + k) * lda] = S::div_real(w[k], sd[k]);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// General (LU) panel: decisions + L21 and U12 solves.
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kPanelThreads) k_panel_lu(PanelArgs a) {
  using S = Sc<T>;
  __shared__ T blk[kPanel][kPanel + 1];
  __shared__ int s_ok;
  T* A = static_cast<T*>(a.A);
  const int b = a.b;
  const int64_t q = a.q, lda = a.lda;

  if (blockIdx.x == 0) {
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      blk[i][k] = (i < b && k < b) ? A[(q + i) + (q + k) * lda] : S::zero();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double u = 0.0;
      if (lane < b)
        u = a.uniforms ? a.uniforms[q + lane] : philox_uniform(a.seed, a.inst, (uint64_t)(q + lane));
      DecisionLog log;
      for (int j = 0; j < b; ++j) {
        T d = blk[j][j];
        const double p = S::re(d);
        const double uj = __shfl_sync(kFull, u, j);
        const bool kp = uj < p;
        if (!kp) d = S::sub(d, S::from_real(1.0));
        __syncwarp();
        if (lane > j && lane < b) {
          const T l = S::div(blk[lane][j], d);
          for (int k = j + 1; k < b; ++k) blk[lane][k] = S::fnms(blk[lane][k], l, blk[j][k]);
          blk[lane][j] = l;
        }
        if (lane == 0) {
          blk[j][j] = d;
          log.add(p, S::finite(d), kp, S::absv(d), a.tol);
          a.keep[q + j] = kp ? 1 : 0;
          if (Sc<T>::cplx) {
            a.piv[2 * (q + j)] = S::re(d);
            a.piv[2 * (q + j) + 1] = S::im(d);
          } else {
            a.piv[q + j] = S::re(d);
          }
        }
        __syncwarp();
      }
      if (lane == 0) log.flush(a.res);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k < b) A[(q + i) + (q + k) * lda] = blk[i][k];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && !a.withhold) st_release(a.flag, a.epoch);
  } else {
    if (!panel_wait(a, &s_ok)) return;
    for (int idx = threadIdx.x; idx < kPanel * kPanel; idx += blockDim.x) {
      const int i = idx % kPanel, k = idx / kPanel;
      if (i < b && k < b) blk[i][k] = ldcg(&A[(q + i) + (q + k) * lda]);
    }
    __syncthreads();
  }

  const int64_t m = a.n - q - b;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < 2 * m;
       it += (int64_t)gridDim.x * blockDim.x) {
    T x[kPanel];
    if (it < m) {
      // L21 row: x U11 = a  ->  x_k = (a_k - sum_{t<k} x_t U_tk) / U_kk
      const int64_t i = q + b + it;
#pragma unroll
      for (int k = 0; k < kPanel; ++k) x[k] = (k < b) ? A[i + (q + k) * lda] : S::zero();
#pragma unroll
      for (int k = 0; k < kPanel; ++k) {
        if (k < b) {
#pragma unroll
          for (int t = 0; t < k; ++t) x[k] = S::fnms(x[k], x[t], blk[t][k]);
          x[k] = S::div(x[k], blk[k][k]);
        }
      }
#pragma unroll
      for (int k = 0; k < kPanel; ++k)
        if (k < b) A[i + (q + k) * lda] = x[k];
    } else {
      // U12 column: L11 y = a  ->  y_k = a_k - sum_{t<k} L_kt y_t
      const int64_t c = q + b + (it - m);
#pragma unroll
      for (int k = 0; k < kPanel; ++k) x[k] = (k < b) ? A[(q + k) + c * lda] : S::zero();
#pragma unroll
      for (int k = 1; k < kPanel; ++k) {
        if (k < b) {
#pragma unroll
          for (int t = 0; t < k; ++t) x[k] = S::fnms(x[k], blk[k][t], x[t]);
        }
      }
#pragma unroll
      for (int k = 0; k < kPanel; ++k)
        if (k < b) A[(q + k) + c * lda] = x[k];
    }
  }
}

// ---------------------------------------------------------------------------
// Trailing Schur update (a3), SIMT DFMA, 64 x 64 tiles, 256 threads (4 x 4
// outputs per thread). HERM: C -= W L^H on the lower triangle, where
// Aop(i,k) = W[i + k ldw] and Bop(k,c) = conj(L[c + k ldl]). LU: C -= L21 U12
// with Aop(i,k) = A[i + (q+k) lda], Bop(k,c) = A[(q+k) + c lda].
// ---------------------------------------------------------------------------
struct UpdArgs {
  void* C;
  int64_t ldc, r0, n;
  const void* Aop;
  int64_t lda_op;
  const void* Bop;
  int64_t ldb_op;
  int b;
  int64_t tiles;
};

template <class T, bool HERM>
__global__ void __launch_bounds__(256) k_update(UpdArgs u) {
  using S = Sc<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sA = reinterpret_cast<T*>(smem_raw);  // [kPanel][kTile]
  T* sB = sA + kPanel * kTile;             // [kPanel][kTile + 1]
  int64_t tr, tc;
  const int64_t x = blockIdx.x;
  if (HERM) {
    tr = (int64_t)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while (tr * (tr + 1) / 2 > x) --tr;
    while ((tr + 1) * (tr + 2) / 2 <= x) ++tr;
    tc = x - tr * (tr + 1) / 2;
  } else {
    tr = x % u.tiles;
    tc = x / u.tiles;
  }
  const int64_t i0 = u.r0 + tr * kTile, c0 = u.r0 + tc * kTile;
  const int b = u.b;
  const T* Aop = static_cast<const T*>(u.Aop);
  const T* Bop = static_cast<const T*>(u.Bop);
  for (int idx = threadIdx.x; idx < b * kTile; idx += blockDim.x) {
    const int k = idx / kTile, ii = idx % kTile;
    const int64_t i = i0 + ii;
    sA[k * kTile + ii] = (i < u.n) ? Aop[i + k * u.lda_op] : S::zero();
  }
  if (HERM) {
    for (int idx = threadIdx.x; idx < b * kTile; idx += blockDim.x) {
      const int k = idx / kTile, cc = idx % kTile;
      const int64_t c = c0 + cc;
      sB[k * (kTile + 1) + cc] = (c < u.n) ? S::conj(Bop[c + k * u.ldb_op]) : S::zero();
    }
  } else {
    for (int idx = threadIdx.x; idx < b * kTile; idx += blockDim.x) {
      const int k = idx % b, cc = idx / b;
      const int64_t c = c0 + cc;
      sB[k * (kTile + 1) + cc] = (c < u.n) ? Bop[k + c * u.ldb_op] : S::zero();
    }
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[p][r] = S::zero();
  for (int k = 0; k < b; ++k) {
    T ra[4], rb[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) ra[p] = sA[k * kTile + tx + 16 * p];
#pragma unroll
    for (int r = 0; r < 4; ++r) rb[r] = sB[k * (kTile + 1) + ty + 16 * r];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[p][r] = S::fnms(acc[p][r], ra[p], rb[r]);
  }
  T* C = static_cast<T*>(u.C);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t c = c0 + ty + 16 * r;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t i = i0 + tx + 16 * p;
      if (i < u.n && c < u.n && (!HERM || i >= c)) {
        T* dst = &C[i + c * u.ldc];
        *dst = S::add(*dst, acc[p][r]);
      }
    }
  }
}

__global__ void k_init_result(dpp_result* r) {
  r->status = 0;
  r->n_kept = 0;
  r->n_borderline = 0;
  r->n_out_of_range = 0;
  r->logp = 0.0;
  r->max_err_ratio = 0.0;
}

__global__ void k_uniforms(uint64_t seed, uint64_t inst, int64_t n, double* out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = philox_uniform(seed, inst, (uint64_t)j);
}

__global__ void k_fill(double value, int64_t n, double* out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = value;
}

template <class K>
int coop_capacity(K kernel, int threads, size_t smem) {
  DevInfo di;
  if (dev_info(&di) != cudaSuccess) return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
    return 1;
  return per_sm > 0 ? per_sm * di.sm_count : 1;
}

template <class T>
cudaError_t run_fp64(const DrawArgs& a, bool herm, Workspace ws) {
  const int64_t n = a.n;
  const size_t esz = sizeof(T);
  T* A;
  int64_t lda;
  if (a.factor_out) {
    A = static_cast<T*>(a.factor_out);
    lda = a.ld;
  } else {
    A = static_cast<T*>(ws.take(esz * (size_t)n * (size_t)n));
    lda = n;
  }
  T* W = herm ? static_cast<T*>(ws.take(esz * (size_t)n * kPanel)) : nullptr;
  double* piv = static_cast<double*>(ws.take(sizeof(double) * 2 * (size_t)n));
  unsigned* flag = static_cast<unsigned*>(ws.take(256));
  if (n > 0 && (!A || !piv || !flag || (herm && !W))) return cudaErrorInvalidValue;
  cudaError_t e = init_result(a.result, a.stream);
  if (e != cudaSuccess || n == 0) return e;
  if ((e = cudaMemsetAsync(flag, 0, sizeof(unsigned), a.stream)) != cudaSuccess) return e;
  if ((const void*)A != a.K) {
    e = cudaMemcpy2DAsync(A, lda * esz, a.K, a.ld * esz, n * esz, n, cudaMemcpyDeviceToDevice,
                          a.stream);
    if (e != cudaSuccess) return e;
  }
  auto panel = herm ? k_panel_herm<T> : k_panel_lu<T>;
  // cooperative capacity of the panel kernel, per device and form
  static int caps[64][2] = {};
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  int& cap = caps[dev][herm ? 0 : 1];
  if (cap == 0) cap = coop_capacity(panel, kPanelThreads, 0);
  const size_t upd_smem = esz * (size_t)kPanel * (2 * kTile + 1);
  auto upd = herm ? k_update<T, true> : k_update<T, false>;
  if ((e = cudaFuncSetAttribute(upd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem)) !=
      cudaSuccess)
    return e;
  unsigned epoch = 1;
  for (int64_t q = 0; q < n; q += kPanel, ++epoch) {
    const int b = (int)((n - q) < kPanel ? (n - q) : kPanel);
    const int64_t m = n - q - b;
    PanelArgs pa;
    pa.A = A;
    pa.lda = lda;
    pa.n = n;
    pa.q = q;
    pa.b = b;
    pa.uniforms = a.uniforms;
    pa.seed = a.seed;
    pa.inst = a.instance;
    pa.keep = a.keep;
    pa.piv = piv;
    pa.res = a.result;
    pa.W = W;
    pa.ldw = n;
    pa.flag = flag;
    pa.epoch = epoch;
    pa.tol = 1e-6;
    pa.wait_ns = (unsigned long long)g_tuning.wait_ns;
    pa.withhold = g_tuning.fault_withhold;
    const int64_t items = herm ? m : 2 * m;
    int64_t g = (items + kPanelThreads - 1) / kPanelThreads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    void* args[] = {&pa};
    {
      ProfScope ps(kProfPanel, a.stream);
      e = cudaLaunchCooperativeKernel((const void*)panel, dim3((unsigned)g), dim3(kPanelThreads),
                                      args, 0, a.stream);
    }
    if (e != cudaSuccess) return e;
    if (m > 0) {
      UpdArgs ua;
      ua.C = A;
      ua.ldc = lda;
      ua.r0 = q + b;
      ua.n = n;
      ua.b = b;
      ua.tiles = (m + kTile - 1) / kTile;
      if (herm) {
        ua.Aop = W;  // absolute row index into W
        ua.lda_op = n;
        ua.Bop = A + q * lda;       // L columns [q, q+b)
        ua.ldb_op = lda;
      } else {
        ua.Aop = A + q * lda;       // L21 columns
        ua.lda_op = lda;
        ua.Bop = A + q;             // U12 rows [q, q+b): Bop(k,c) = A[(q+k) + c lda]
        ua.ldb_op = lda;
      }
      const int64_t nt = herm ? ua.tiles * (ua.tiles + 1) / 2 : ua.tiles * ua.tiles;
      // algorithmic work: m^2 b real multiply-adds pairs (LDL^H lower half) or
      // 2 m^2 b (LU); complex multiplies cost 4x
      const double cf = Sc<T>::cplx ? 4.0 : 1.0;
      const double fl = cf * (herm ? 1.0 : 2.0) * (double)m * (double)m * (double)b;
      const double by = (double)esz * (herm ? 1.0 : 2.0) * (double)m * (double)m;
      {
        ProfScope ps(kProfUpdateFp64, a.stream, fl, by);
        upd<<<(unsigned)nt, 256, upd_smem, a.stream>>>(ua);
      }
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  if (a.pivots_user) {
    const size_t pb = sizeof(double) * (size_t)n * ((!herm && Sc<T>::cplx) ? 2 : 1);
    e = cudaMemcpyAsync(a.pivots_user, piv, pb, cudaMemcpyDeviceToDevice, a.stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t init_result(dpp_result* r, cudaStream_t s) {
  ProfScope ps(kProfOther, s);
  k_init_result<<<1, 1, 0, s>>>(r);
  return cudaGetLastError();
}

cudaError_t fill_constant(double value, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  ProfScope ps(kProfOther, s);
  k_fill<<<(unsigned)g, 256, 0, s>>>(value, n, out);
  return cudaGetLastError();
}

cudaError_t fill_uniforms(uint64_t seed, uint64_t instance, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int64_t g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  ProfScope ps(kProfOther, s);
  k_uniforms<<<(unsigned)g, 256, 0, s>>>(seed, instance, n, out);
  return cudaGetLastError();
}

size_t ws_fp64(int64_t n, int32_t dtype, bool hermitian, bool own_matrix) {
  const size_t esz = dtype == DPP_C128 ? 16 : 8;
  size_t b = 0;
  if (own_matrix) b += align256(esz * (size_t)n * (size_t)n);
  if (hermitian) b += align256(esz * (size_t)n * kPanel);
  b += align256(sizeof(double) * 2 * (size_t)n);
  b += 256;
  return b + 256;
}

cudaError_t sample_fp64(const DrawArgs& a, bool hermitian, Workspace ws) {
  if (a.dtype == DPP_C128) return run_fp64<cdouble>(a, hermitian, ws);
  return run_fp64<double>(a, hermitian, ws);
}

}  // namespace dpp
