// C ABI of the sampler library: argument validation, workspace carving and
// dispatch to the FP64 / mixed-precision / adjoint implementations.
#include <stdio.h>
#include <string.h>

#include <string>

#include "dpp.h"
#include "dpp_internal.h"

namespace dpp {

static thread_local std::string g_last_error;

static dpp_status fail(dpp_status s, const char* msg) {
  g_last_error = msg;
  return s;
}

static dpp_status fail_cuda(cudaError_t e, const char* where) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  g_last_error = buf;
  return DPP_ERR_CUDA;
}

void clear_last_error() { g_last_error.clear(); }

dpp_status set_last_error(dpp_status s, const char* msg) { return fail(s, msg); }

dpp_status set_last_cuda_error(cudaError_t e, const char* where) { return fail_cuda(e, where); }

cudaError_t dev_info(DevInfo* out) {
  static thread_local DevInfo cache[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (cache[dev].device != dev) {
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cache[dev].device = dev;
    cache[dev].sm_count = sms;
  }
  *out = cache[dev];
  return cudaSuccess;
}

static bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Validation shared by the two samplers.
static dpp_status check_draw(const void* K, int64_t n, int64_t ld, int32_t dtype,
                             uint8_t* keep, void* factor_out, dpp_result* result,
                             void* workspace, size_t ws_bytes, size_t ws_need) {
  if (n < 0) return fail(DPP_ERR_INVALID_ARG, "n must be >= 0");
  if (n > (int64_t)0x7fffffff) return fail(DPP_ERR_INVALID_ARG, "n too large");
  if (ld < (n > 1 ? n : 1)) return fail(DPP_ERR_INVALID_ARG, "ld must be >= max(1, n)");
  if (dtype != DPP_R64 && dtype != DPP_C128) return fail(DPP_ERR_INVALID_ARG, "unknown dtype");
  if (!result) return fail(DPP_ERR_INVALID_ARG, "result must not be NULL");
  if (n > 0 && (!K || !keep)) return fail(DPP_ERR_INVALID_ARG, "K and keep must not be NULL");
  const size_t esz = dtype == DPP_C128 ? 16 : 8;
  if (n > 0 && !aligned(K, esz)) return fail(DPP_ERR_INVALID_ARG, "K misaligned");
  if (factor_out && !aligned(factor_out, esz))
    return fail(DPP_ERR_INVALID_ARG, "factor_out misaligned");
  if (!aligned(result, 8)) return fail(DPP_ERR_INVALID_ARG, "result misaligned");
  if (ws_need == 0) return fail(DPP_ERR_UNSUPPORTED, "unsupported dtype/precision combination");
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < ws_need) return fail(DPP_ERR_WORKSPACE, "workspace too small");
  return DPP_OK;
}

}  // namespace dpp

using namespace dpp;

extern "C" {

int32_t dpp_abi_version(void) { return DPP_ABI_VERSION; }

const char* dpp_last_error(void) { return g_last_error.c_str(); }

size_t dpp_workspace_size(int32_t op, int64_t n, int32_t dtype, int32_t precision,
                          int32_t hermitian) {
  if (n < 0 || (dtype != DPP_R64 && dtype != DPP_C128)) return 0;
  switch (op) {
    case DPP_OP_SAMPLE_HERMITIAN:
      if (precision == DPP_PREC_FP64) return ws_fp64(n, dtype, true, true);
      if ((precision == DPP_PREC_3XTF32 || precision == DPP_PREC_BF16X6) && dtype == DPP_R64) {
        // either panel pipeline may run
        const size_t a = ws_mixed(n), b = ws_mixed_lu(n);
        return a > b ? a : b;
      }
      if ((precision == DPP_PREC_3XTF32 || precision == DPP_PREC_BF16X6) && dtype == DPP_C128)
        return ws_mixed_cx(n);
      return 0;
    case DPP_OP_SAMPLE_LU:
      if (precision == DPP_PREC_FP64) return ws_fp64(n, dtype, false, true);
      if ((precision == DPP_PREC_3XTF32 || precision == DPP_PREC_BF16X6) && dtype == DPP_R64)
        return ws_mixed_lu(n);
      if ((precision == DPP_PREC_3XTF32 || precision == DPP_PREC_BF16X6) && dtype == DPP_C128)
        return ws_mixed_cxlu(n);
      return 0;
    case DPP_OP_LOGPROB_BACKWARD:
      if (precision == DPP_PREC_FP64) return ws_backward(n, dtype, hermitian != 0);
      return 0;
    case DPP_OP_GREEDY_HERMITIAN:
    case DPP_OP_GREEDY_LU: {
      // the sampler's workspace behind n doubles of decision thresholds
      const size_t w = dpp_workspace_size(op == DPP_OP_GREEDY_HERMITIAN ? DPP_OP_SAMPLE_HERMITIAN
                                                                        : DPP_OP_SAMPLE_LU,
                                          n, dtype, precision, hermitian);
      return w ? w + align256(sizeof(double) * (size_t)(n > 0 ? n : 1)) : 0;
    }
    default:
      return 0;
  }
}

static dpp_status sample_common(bool hermitian, const void* K, int64_t n, int64_t ld,
                                int32_t dtype, int32_t precision, uint64_t seed,
                                uint64_t instance, const double* uniforms, uint8_t* keep,
                                void* factor_out, double* pivots, dpp_result* result,
                                void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  const size_t need = dpp_workspace_size(hermitian ? DPP_OP_SAMPLE_HERMITIAN : DPP_OP_SAMPLE_LU,
                                         n, dtype, precision, hermitian);
  dpp_status st = check_draw(K, n, ld, dtype, keep, factor_out, result, workspace, ws_bytes, need);
  if (st != DPP_OK) return st;
  begin_call(hermitian ? DPP_OP_SAMPLE_HERMITIAN : DPP_OP_SAMPLE_LU, n, dtype, precision);
  DrawArgs a;
  a.K = K;
  a.n = n;
  a.ld = ld;
  a.dtype = dtype;
  a.precision = precision;
  a.seed = seed;
  a.instance = instance;
  a.uniforms = uniforms;
  a.keep = keep;
  a.factor_out = factor_out;
  a.pivots_user = pivots;
  a.result = result;
  a.stream = static_cast<cudaStream_t>(stream);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = ws_bytes;
  cudaError_t e;
  if (precision == DPP_PREC_FP64) {
    e = sample_fp64(a, hermitian, ws);
  } else {
    if (factor_out == K && factor_out) {
      // the mixed path reads K in FP64 for recomputes: it must stay intact
      return fail(DPP_ERR_INVALID_ARG, "mixed precision cannot factor in place (factor_out == K)");
    }
    if (!hermitian && dtype == DPP_C128)
      e = sample_mixed_cxlu(a, ws);
    else if (!hermitian)
      e = sample_mixed_lu(a, ws);
    else if (dtype == DPP_C128)
      e = sample_mixed_cx(a, ws);
    else if (g_tuning.update_kernel == 0 &&
             (g_tuning.panel_pipeline >= 2 ||
              (g_tuning.panel_pipeline == 0 && (g_tuning.max_ctas == 0 || g_tuning.max_ctas >= 96))))
      e = sample_mixed_chunked(a, ws);
    else
      e = sample_mixed(a, ws);
  }
  if (e != cudaSuccess) return fail_cuda(e, hermitian ? "dpp_sample_hermitian" : "dpp_sample_lu");
  return DPP_OK;
}

dpp_status dpp_sample_hermitian(const void* K, int64_t n, int64_t ld, int32_t dtype,
                                int32_t precision, uint64_t seed, uint64_t instance,
                                const double* uniforms, uint8_t* keep, void* factor_out,
                                double* pivots, dpp_result* result, void* workspace,
                                size_t workspace_bytes, void* stream) {
  return sample_common(true, K, n, ld, dtype, precision, seed, instance, uniforms, keep,
                       factor_out, pivots, result, workspace, workspace_bytes, stream);
}

dpp_status dpp_sample_lu(const void* K, int64_t n, int64_t ld, int32_t dtype, int32_t precision,
                         uint64_t seed, uint64_t instance, const double* uniforms, uint8_t* keep,
                         void* factor_out, double* pivots, dpp_result* result, void* workspace,
                         size_t workspace_bytes, void* stream) {
  return sample_common(false, K, n, ld, dtype, precision, seed, instance, uniforms, keep,
                       factor_out, pivots, result, workspace, workspace_bytes, stream);
}

// Greedy maximum-likelihood draw: the sampler's decision "keep j iff
// u_j < Re d_j" with every threshold u_j = 1/2 is "keep j iff Re d_j > 1/2, a
// tie rejects". The thresholds live in the first bytes of the workspace.
static dpp_status greedy_common(bool hermitian, const void* K, int64_t n, int64_t ld,
                                int32_t dtype, int32_t precision, uint8_t* keep,
                                void* factor_out, double* pivots, dpp_result* result,
                                void* workspace, size_t ws_bytes, void* stream) {
  g_last_error.clear();
  const size_t need = dpp_workspace_size(hermitian ? DPP_OP_GREEDY_HERMITIAN : DPP_OP_GREEDY_LU,
                                         n, dtype, precision, hermitian);
  dpp_status st = check_draw(K, n, ld, dtype, keep, factor_out, result, workspace, ws_bytes, need);
  if (st != DPP_OK) return st;
  if (precision != DPP_PREC_FP64 && factor_out && factor_out == K)
    return fail(DPP_ERR_INVALID_ARG, "mixed precision cannot factor in place (factor_out == K)");
  const size_t ub = align256(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* half = static_cast<double*>(workspace);
  cudaError_t e = fill_constant(0.5, n, half, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_greedy: thresholds");
  return sample_common(hermitian, K, n, ld, dtype, precision, 0, 0, half, keep, factor_out,
                       pivots, result, static_cast<char*>(workspace) + ub, ws_bytes - ub, stream);
}

dpp_status dpp_greedy_hermitian(const void* K, int64_t n, int64_t ld, int32_t dtype,
                                int32_t precision, uint8_t* keep, void* factor_out,
                                double* pivots, dpp_result* result, void* workspace,
                                size_t workspace_bytes, void* stream) {
  return greedy_common(true, K, n, ld, dtype, precision, keep, factor_out, pivots, result,
                       workspace, workspace_bytes, stream);
}

dpp_status dpp_greedy_lu(const void* K, int64_t n, int64_t ld, int32_t dtype, int32_t precision,
                         uint8_t* keep, void* factor_out, double* pivots, dpp_result* result,
                         void* workspace, size_t workspace_bytes, void* stream) {
  return greedy_common(false, K, n, ld, dtype, precision, keep, factor_out, pivots, result,
                       workspace, workspace_bytes, stream);
}

size_t dpp_elementary_workspace_size(int64_t n, int64_t k) {
  if (n < 0 || k < 0 || k > n || n > (int64_t)0x7fffffff) return 0;
  return ws_elementary(n, k);
}

dpp_status dpp_sample_elementary(const double* K, int64_t n, int64_t ld, int64_t k, uint64_t seed,
                                 uint64_t instance, const double* uniforms, int64_t* sample,
                                 uint8_t* keep, double* chol, dpp_result* result, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  g_last_error.clear();
  if (n < 0 || n > (int64_t)0x7fffffff) return fail(DPP_ERR_INVALID_ARG, "bad n");
  if (k < 0 || k > n) return fail(DPP_ERR_INVALID_ARG, "k must be in [0, n]");
  if (ld < (n > 1 ? n : 1)) return fail(DPP_ERR_INVALID_ARG, "ld must be >= max(1, n)");
  if (!result || !aligned(result, 8)) return fail(DPP_ERR_INVALID_ARG, "result NULL or misaligned");
  if (n > 0 && (!K || !aligned(K, 8))) return fail(DPP_ERR_INVALID_ARG, "K NULL or misaligned");
  if (k > 0 && (!sample || !aligned(sample, 8)))
    return fail(DPP_ERR_INVALID_ARG, "sample NULL or misaligned");
  if (chol && !aligned(chol, 8)) return fail(DPP_ERR_INVALID_ARG, "chol misaligned");
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  if (workspace_bytes < ws_elementary(n, k)) return fail(DPP_ERR_WORKSPACE, "workspace too small");
  begin_call(DPP_OP_SAMPLE_HERMITIAN, n, DPP_R64, DPP_PREC_FP64);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = workspace_bytes;
  cudaError_t e = sample_elementary(K, n, ld, k, seed, instance, uniforms, sample, keep, chol,
                                    result, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_sample_elementary");
  return DPP_OK;
}

size_t dpp_batched_workspace_size(int32_t batch, int64_t n_max, int32_t precision) {
  if (batch < 0 || n_max < 0 || precision != DPP_PREC_FP32) return 0;
  return ws_batched(batch, n_max, batched_default_ctas());
}

dpp_status dpp_sample_batched(int32_t batch, const int64_t* n, const double* const* K,
                              const int64_t* ld, int64_t n_max, int32_t precision, uint64_t seed,
                              const uint64_t* instance, uint8_t* const* keep,
                              const double* const* uniforms, double* const* pivots,
                              dpp_result* results, void* workspace, size_t workspace_bytes,
                              void* stream) {
  g_last_error.clear();
  if (precision != DPP_PREC_FP32)
    return fail(DPP_ERR_UNSUPPORTED, "dpp_sample_batched supports DPP_PREC_FP32 only");
  if (batch < 0 || n_max < 0 || n_max > (1 << 20))
    return fail(DPP_ERR_INVALID_ARG, "bad batch or n_max");
  if (batch == 0) return DPP_OK;
  if (!n || !K || !ld || !keep || !results)
    return fail(DPP_ERR_INVALID_ARG, "n, K, ld, keep and results must not be NULL");
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  const size_t minimal = ws_batched(batch, n_max, 1);
  if (workspace_bytes < minimal) return fail(DPP_ERR_WORKSPACE, "workspace too small");
  begin_call(kOpBatched, n_max, DPP_R64, precision);
  BatchedArgs b;
  b.batch = batch;
  b.n = n;
  b.K = K;
  b.ld = ld;
  b.n_max = n_max;
  b.seed = seed;
  b.instance = instance;
  b.keep = keep;
  b.uniforms = uniforms;
  b.pivots = pivots;
  b.results = results;
  b.flops = 0.0;
  b.stream = static_cast<cudaStream_t>(stream);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = workspace_bytes;
  cudaError_t e = sample_batched(b, ws);
  if (e != cudaSuccess) return fail_cuda(e, "dpp_sample_batched");
  return DPP_OK;
}

dpp_status dpp_logprob_backward(const void* K, int64_t n, int64_t ld, int32_t dtype,
                                int32_t precision, int32_t hermitian, const uint8_t* keep,
                                const double* grad_logp, void* dK, int64_t ld_dk,
                                void* workspace, size_t workspace_bytes, void* stream) {
  g_last_error.clear();
  if (precision != DPP_PREC_FP64)
    return fail(DPP_ERR_UNSUPPORTED, "dpp_logprob_backward supports DPP_PREC_FP64 only");
  if (n < 0 || ld < (n > 1 ? n : 1) || ld_dk < (n > 1 ? n : 1))
    return fail(DPP_ERR_INVALID_ARG, "bad n / ld / ld_dk");
  if (dtype != DPP_R64 && dtype != DPP_C128) return fail(DPP_ERR_INVALID_ARG, "unknown dtype");
  if (n > 0 && (!K || !keep || !grad_logp || !dK))
    return fail(DPP_ERR_INVALID_ARG, "K, keep, grad_logp and dK must not be NULL");
  const size_t need = dpp_workspace_size(DPP_OP_LOGPROB_BACKWARD, n, dtype, precision, hermitian);
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  if (workspace_bytes < need) return fail(DPP_ERR_WORKSPACE, "workspace too small");
  if (n == 0) return DPP_OK;
  begin_call(DPP_OP_LOGPROB_BACKWARD, n, dtype, precision);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = workspace_bytes;
  cudaError_t e = logprob_backward(K, n, ld, dtype, hermitian != 0, keep, grad_logp, dK, ld_dk,
                                   ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_logprob_backward");
  return DPP_OK;
}

static dpp_status backward_batched_common(int32_t batch, const int64_t* n, const void* const* K,
                                          const int64_t* ld, const uint8_t* const* keep,
                                          const double* const* grad_logp, void* const* dK,
                                          const int64_t* ld_dk, bool fp32, void* workspace,
                                          size_t workspace_bytes, void* stream) {
  g_last_error.clear();
  if (batch < 0) return fail(DPP_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return DPP_OK;
  if (!n || !K || !ld || !keep || !grad_logp || !dK || !ld_dk)
    return fail(DPP_ERR_INVALID_ARG, "the per-instance host arrays must not be NULL");
  int64_t n_max = 0;
  for (int32_t i = 0; i < batch; ++i) {
    if (n[i] < 0 || ld[i] < (n[i] > 1 ? n[i] : 1) || ld_dk[i] < (n[i] > 1 ? n[i] : 1))
      return fail(DPP_ERR_INVALID_ARG, "bad n / ld / ld_dk of an instance");
    if (n[i] > 0 && (!K[i] || !keep[i] || !grad_logp[i] || !dK[i]))
      return fail(DPP_ERR_INVALID_ARG, "NULL pointer of a non-empty instance");
    if (n[i] > n_max) n_max = n[i];
  }
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  if (workspace_bytes < ws_adjoint_batched(batch, n_max, 1))
    return fail(DPP_ERR_WORKSPACE, "workspace too small for one CTA of the batched adjoint");
  // one persistent launch over all instances, on as many CTAs as the workspace holds
  begin_call(DPP_OP_LOGPROB_BACKWARD, n_max, DPP_R64, fp32 ? DPP_PREC_FP32 : DPP_PREC_FP64);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = workspace_bytes;
  cudaError_t e = adjoint_batched(batch, n, reinterpret_cast<const double* const*>(K), ld, keep,
                                  grad_logp, reinterpret_cast<double* const*>(dK), ld_dk, n_max,
                                  fp32, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_logprob_backward_batched");
  return DPP_OK;
}

dpp_status dpp_logprob_backward_batched(int32_t batch, const int64_t* n, const void* const* K,
                                        const int64_t* ld, const uint8_t* const* keep,
                                        const double* const* grad_logp, void* const* dK,
                                        const int64_t* ld_dk, void* workspace,
                                        size_t workspace_bytes, void* stream) {
  return backward_batched_common(batch, n, K, ld, keep, grad_logp, dK, ld_dk, false, workspace,
                                 workspace_bytes, stream);
}

dpp_status dpp_logprob_backward_batched_fp32(int32_t batch, const int64_t* n,
                                             const void* const* K, const int64_t* ld,
                                             const uint8_t* const* keep,
                                             const double* const* grad_logp, void* const* dK,
                                             const int64_t* ld_dk, void* workspace,
                                             size_t workspace_bytes, void* stream) {
  return backward_batched_common(batch, n, K, ld, keep, grad_logp, dK, ld_dk, true, workspace,
                                 workspace_bytes, stream);
}

dpp_status dpp_lensemble_to_marginal_batched(int32_t batch, const int64_t* n,
                                             const double* const* L, const int64_t* ld,
                                             double* const* K, const int64_t* ld_k,
                                             void* workspace, size_t workspace_bytes,
                                             void* stream) {
  g_last_error.clear();
  if (batch < 0) return fail(DPP_ERR_INVALID_ARG, "batch must be >= 0");
  if (batch == 0) return DPP_OK;
  if (!n || !L || !ld || !K || !ld_k)
    return fail(DPP_ERR_INVALID_ARG, "the per-instance host arrays must not be NULL");
  int64_t n_max = 0;
  for (int32_t i = 0; i < batch; ++i) {
    if (n[i] < 0 || ld[i] < (n[i] > 1 ? n[i] : 1) || ld_k[i] < (n[i] > 1 ? n[i] : 1))
      return fail(DPP_ERR_INVALID_ARG, "bad n / ld / ld_k of an instance");
    if (n[i] > 0 && (!L[i] || !K[i])) return fail(DPP_ERR_INVALID_ARG, "NULL pointer of a non-empty instance");
    if (n[i] > n_max) n_max = n[i];
  }
  if (n_max > 4096) return fail(DPP_ERR_INVALID_ARG, "n above 4096 (one CTA per instance)");
  if (!workspace || !aligned(workspace, 256))
    return fail(DPP_ERR_WORKSPACE, "workspace must be non-NULL and 256-byte aligned");
  if (workspace_bytes < ws_adjoint_batched(batch, n_max, 1))
    return fail(DPP_ERR_WORKSPACE, "workspace too small for one CTA");
  begin_call(DPP_OP_LOGPROB_BACKWARD, n_max, DPP_R64, DPP_PREC_FP64);
  Workspace ws;
  ws.base = static_cast<char*>(workspace);
  ws.size = workspace_bytes;
  cudaError_t e = adjoint_batched(batch, n, L, ld, nullptr, nullptr, K, ld_k, n_max, false, ws,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_lensemble_to_marginal_batched");
  return DPP_OK;
}

size_t dpp_logprob_backward_batched_workspace(int32_t batch, int64_t n_max) {
  if (batch < 0 || n_max < 0) return 0;
  begin_call(DPP_OP_LOGPROB_BACKWARD, n_max, DPP_R64, DPP_PREC_FP64);
  return ws_adjoint_batched(batch, n_max, adjoint_batched_ctas());
}

dpp_status dpp_set_tuning(int32_t key, double value) {
  g_last_error.clear();
  switch (key) {
    case DPP_TUNE_TAU_SAFETY:
      if (!(value > 0.0 && value < 1e6)) return fail(DPP_ERR_INVALID_ARG, "tau safety out of range");
      g_settings.tau_safety = value;
      return DPP_OK;
    case DPP_TUNE_OUTER_BLOCK: {
      const int v = (int)value;
      if ((double)v != value || v < 32 || v > kMaxOuterBlock || v % 32 != 0)
        return fail(DPP_ERR_INVALID_ARG, "outer block must be a multiple of 32 in [32, 256]");
      g_settings.outer_block = v;
      return DPP_OK;
    }
    case DPP_TUNE_UPDATE_KERNEL:
      if (value != 0.0 && value != 1.0) return fail(DPP_ERR_INVALID_ARG, "update kernel is 0 or 1");
      g_settings.update_kernel = (int)value;
      return DPP_OK;
    case DPP_TUNE_MAX_CTAS: {
      const int v = (int)value;
      if ((double)v != value || (v != 0 && v < 8) || v > 4096)
        return fail(DPP_ERR_INVALID_ARG, "max CTAs must be 0 or in [8, 4096]");
      g_settings.max_ctas = v;
      return DPP_OK;
    }
    case DPP_TUNE_PANEL_PIPELINE:
      if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0)
        return fail(DPP_ERR_INVALID_ARG, "panel pipeline is 0, 1, 2 or 3");
      g_settings.panel_pipeline = (int)value;
      return DPP_OK;
    case DPP_TUNE_WAIT_NS:
      if (!(value >= 1e5 && value <= 6e10))
        return fail(DPP_ERR_INVALID_ARG, "wait limit must be in [1e5, 6e10] ns");
      g_settings.wait_ns = value;
      return DPP_OK;
    case DPP_TUNE_FAULT_WITHHOLD:
      if (value != 0.0 && value != 1.0) return fail(DPP_ERR_INVALID_ARG, "fault withhold is 0 or 1");
      g_settings.fault_withhold = (int)value;
      return DPP_OK;
    case DPP_TUNE_USE_CACHE:
      if (value != 0.0 && value != 1.0) return fail(DPP_ERR_INVALID_ARG, "use cache is 0 or 1");
      g_settings.use_cache = (int)value;
      return DPP_OK;
    case DPP_TUNE_UPDATE_VARIANT: {
      const int v = (int)value;
      if ((double)v != value || v < 0 || v > 3)
        return fail(DPP_ERR_INVALID_ARG, "update variant is 0, 1, 2 or 3");
      g_settings.update_variant = v;
      return DPP_OK;
    }
    case DPP_TUNE_BATCHED_THREADS: {
      const int v = (int)value;
      if ((double)v != value || (v != 128 && v != 256))
        return fail(DPP_ERR_INVALID_ARG, "batched threads are 128 or 256");
      g_settings.batched_threads = v;
      return DPP_OK;
    }
    case DPP_TUNE_PANEL_CTAS: {
      const int v = (int)value;
      if ((double)v != value || (v != 0 && (v < 8 || v > 4096)))
        return fail(DPP_ERR_INVALID_ARG, "panel CTAs must be 0 or in [8, 4096]");
      g_settings.panel_ctas = v;
      return DPP_OK;
    }
    default:
      return fail(DPP_ERR_INVALID_ARG, "unknown tuning key");
  }
}

double dpp_get_tuning(int32_t key) {
  switch (key) {
    case DPP_TUNE_TAU_SAFETY: return g_settings.tau_safety;
    case DPP_TUNE_OUTER_BLOCK: return (double)g_settings.outer_block;
    case DPP_TUNE_UPDATE_KERNEL: return (double)g_settings.update_kernel;
    case DPP_TUNE_MAX_CTAS: return (double)g_settings.max_ctas;
    case DPP_TUNE_PANEL_PIPELINE: return (double)g_settings.panel_pipeline;
    case DPP_TUNE_WAIT_NS: return g_settings.wait_ns;
    case DPP_TUNE_FAULT_WITHHOLD: return (double)g_settings.fault_withhold;
    case DPP_TUNE_USE_CACHE: return (double)g_settings.use_cache;
    case DPP_TUNE_UPDATE_VARIANT: return (double)g_settings.update_variant;
    case DPP_TUNE_PANEL_CTAS: return (double)g_settings.panel_ctas;
    case DPP_TUNE_BATCHED_THREADS: return (double)g_settings.batched_threads;
    default: return -1.0;
  }
}

dpp_status dpp_uniforms(uint64_t seed, uint64_t instance, int64_t n, double* out, void* stream) {
  g_last_error.clear();
  if (n < 0) return fail(DPP_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && !out) return fail(DPP_ERR_INVALID_ARG, "out must not be NULL");
  cudaError_t e = fill_uniforms(seed, instance, n, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail_cuda(e, "dpp_uniforms");
  return DPP_OK;
}

}  // extern "C"
