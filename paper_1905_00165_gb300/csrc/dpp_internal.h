// Host-side internal interface between the C ABI (dpp_api.cu) and the kernel
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "dpp.h"

namespace dpp {

// Inner panel width of the sequential decisions: one warp owns the
// kPanel x kPanel diagonal block (one row per lane).
constexpr int kPanel = 32;
// Threads per CTA of the panel kernels.
constexpr int kPanelThreads = 256;

struct Workspace {
  char* base = nullptr;
  size_t size = 0;
  size_t used = 0;
  // Carve `bytes` (256-byte aligned); returns nullptr when out of space.
  void* take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    if (off + bytes > size) return nullptr;
    used = off + bytes;
    return base + off;
  }
};

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Per-device properties cached on first use.
struct DevInfo {
  int device = -1;
  int sm_count = 0;
};
cudaError_t dev_info(DevInfo* out);

// Thread-local error text read back by dpp_last_error (dpp_api.cu).
void clear_last_error();
dpp_status set_last_error(dpp_status s, const char* msg);
dpp_status set_last_cuda_error(cudaError_t e, const char* where);

// Common arguments of one draw.
struct DrawArgs {
  const void* K;
  int64_t n, ld;
  int32_t dtype;
  int32_t precision;
  uint64_t seed, instance;
  const double* uniforms;
  uint8_t* keep;
  void* factor_out;
  double* pivots_user;
  dpp_result* result;
  cudaStream_t stream;
};

// FP64 samplers (dpp_fp64.cu).
size_t ws_fp64(int64_t n, int32_t dtype, bool hermitian, bool own_matrix);
cudaError_t sample_fp64(const DrawArgs& a, bool hermitian, Workspace ws);

// Process-wide tuning knobs (dpp_set_tuning).
struct Tuning {
  double tau_safety = 8.0;  // c in the borderline bound
  int outer_block = 256;    // mixed path: columns contracted per trailing update
  int update_kernel = 0;    // 0 = tcgen05, 1 = SIMT FP32
  int update_variant = 0;   // tcgen05 update: operand ring and drain interval (0..3)
  int max_ctas = 0;         // mixed path: CTAs per launch (0 = one per SM)
  int panel_pipeline = 0;   // mixed Hermitian path: 0 = auto, 1 = single helper, 2 = chunked
  double wait_ns = 2e9;     // limit of the bounded device waits (ns)
  int fault_withhold = 0;   // fault injection: the deciding CTA never releases a panel
  int use_cache = 1;        // apply the autotuner's entry for a call's key
  int panel_ctas = 0;       // split pipeline: CTAs of the decision launch (0 = cap)
  int batched_threads = 128;  // batched sampler: threads per CTA (128 or 256)
};
// The process-wide settings (dpp_set_tuning), and the settings of the call in
// progress on this host thread: every entry point starts with begin_call,
// which copies the former into the latter and applies the autotuner's cached
// entry for the call's key (dpp_tune.cu).
extern Tuning g_settings;
extern thread_local Tuning g_tuning;
void begin_call(int32_t op, int64_t n, int32_t dtype, int32_t precision);
constexpr int32_t kOpBatched = 5;  // key of dpp_sample_batched in the tuning cache
constexpr int kMaxOuterBlock = 256;

// Mixed-precision Hermitian sampler (dpp_mixed.cu).
size_t ws_mixed(int64_t n);
cudaError_t sample_mixed(const DrawArgs& a, Workspace ws);

// Mixed-precision general (LU) sampler, and the Hermitian sampler on the same
// chunked panel pipeline (dpp_mixed_lu.cu).
size_t ws_mixed_lu(int64_t n);
cudaError_t sample_mixed_lu(const DrawArgs& a, Workspace ws);
cudaError_t sample_mixed_chunked(const DrawArgs& a, Workspace ws);

// Mixed-precision Hermitian sampler for complex K (dpp_mixed_cplx.cu).
size_t ws_mixed_cx(int64_t n);
cudaError_t sample_mixed_cx(const DrawArgs& a, Workspace ws);

// Mixed-precision LU sampler for complex, non-Hermitian K (dpp_mixed_cxlu.cu).
size_t ws_mixed_cxlu(int64_t n);
cudaError_t sample_mixed_cxlu(const DrawArgs& a, Workspace ws);

// Operand splits of the tensor-core trailing update.
enum { kSplit3xTf32 = 0, kSplitBf16x6 = 1 };

// Trailing update C -= W L^T on the lower triangle (full = false) or the whole
// square (full = true) of rows/cols [r0, n) of the FP32 column-major C (ldc),
// on tcgen05 tensor cores (dpp_tc.cu). The W and L
// operands are given as splits in row-major [n x ldk] buffers (first kdim
// columns used): two TF32 pieces (fp32 storage) for kSplit3xTf32, three BF16
// pieces for kSplitBf16x6. kdim must be a multiple of the k-block (32 / 64);
// ldk * element size must be a multiple of 16; buffers 16-byte aligned.
cudaError_t outer_update_tc(int mode, float* C, int64_t ldc, int64_t n, int64_t r0, int kdim,
                            void* const* Wops, void* const* Lops, int ldk, bool full,
                            int* err_flag, cudaStream_t s);

// Batched sampler (dpp_batched.cu).
struct BatchedArgs {
  int32_t batch;
  const int64_t* n;
  const double* const* K;
  const int64_t* ld;
  int64_t n_max;
  uint64_t seed;
  const uint64_t* instance;
  uint8_t* const* keep;
  const double* const* uniforms;
  double* const* pivots;
  dpp_result* results;
  double flops;  // algorithmic flops (profiling only; 0 if unknown)
  cudaStream_t stream;
};
size_t ws_batched(int32_t batch, int64_t n_max, int ctas);
size_t ws_batched_per_cta(int64_t n_max);
int batched_default_ctas();
cudaError_t sample_batched(const BatchedArgs& b, Workspace ws);

// Elementary (projection) sampler, Algorithm 2 (dpp_elementary.cu).
size_t ws_elementary(int64_t n, int64_t k);
cudaError_t sample_elementary(const double* K, int64_t n, int64_t ld, int64_t k, uint64_t seed,
                              uint64_t instance, const double* uniforms, int64_t* sample,
                              uint8_t* keep, double* chol, dpp_result* result, Workspace ws,
                              cudaStream_t s);

// Adjoint (dpp_backward.cu).
size_t ws_backward(int64_t n, int32_t dtype, bool hermitian);
cudaError_t logprob_backward(const void* K, int64_t n, int64_t ld, int32_t dtype,
                             bool hermitian, const uint8_t* keep,
                             const double* grad, void* dK, int64_t ld_dk,
                             Workspace ws, cudaStream_t stream);

// Batched adjoint in one persistent launch (dpp_adjoint_batched.cu).
size_t ws_adjoint_batched(int32_t batch, int64_t n_max, int ctas);
int adjoint_batched_ctas();
cudaError_t adjoint_batched(int32_t batch, const int64_t* n, const double* const* K,
                            const int64_t* ld, const uint8_t* const* keep,
                            const double* const* g, double* const* dK, const int64_t* ld_dk,
                            int64_t n_max, bool fp32, Workspace ws, cudaStream_t s);

// Result initialisation and uniform generation (dpp_fp64.cu).
cudaError_t init_result(dpp_result* r, cudaStream_t s);
cudaError_t fill_uniforms(uint64_t seed, uint64_t instance, int64_t n, double* out,
                          cudaStream_t s);
cudaError_t fill_constant(double value, int64_t n, double* out, cudaStream_t s);

}  // namespace dpp
