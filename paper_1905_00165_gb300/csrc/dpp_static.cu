// Allocation-free entry point: the FP64 Hermitian sampler (Algorithm 1 in its
// LDL^H form, blocked as in Algorithm 4) with its scratch held in one
// file-scope device array instead of a caller-supplied workspace. It has no
// counterpart in the paper; it serves callers that cannot allocate device
// memory at the moment they sample (a serving loop whose memory was planned
// once at start-up, where a cudaMalloc would synchronise the device or could
// fail under memory pressure, and plain C callers that own only K and the
// outputs and have no allocator to get a workspace from).
//
// Scratch layout (carved in this order, 256-byte aligned, as the workspace of
// dpp_sample_hermitian with a caller-held factor): the n x 32 panel of
// D-scaled rows (W), 2n pivot doubles, one 256-byte flag block. Nothing in it
// has to start at zero: the call clears the panel flag word on its stream
// before the first kernel, and every other word is written before it is read.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress, which may load this
// module onto the device. Later calls look it up again whenever their stream
// is not capturing (a device reset reloads the module, and the array may then
// live at another address); a call inside a stream capture uses the address
// of the device's last call.
//
// Concurrency: every call on one device uses the same array, so two calls in
// flight at the same time on one device (two streams, or two host threads
// without ordering between their streams) race on it. Calls must be ordered,
// e.g. issued on one stream.
#include <stdio.h>

#include <mutex>

#include "dpp.h"
#include "dpp_internal.h"

namespace dpp {
namespace {

constexpr size_t kStaticScratchBytes = DPP_STATIC_SCRATCH_BYTES;
static_assert(kStaticScratchBytes % 256 == 0, "scratch size must be a multiple of 256");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device: looked up on
// every call whose stream is not capturing, else the device's cached one.
cudaError_t static_scratch(cudaStream_t stream, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(stream, &cs)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev] || cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    if (!p || ((uintptr_t)p & 255)) return cudaErrorInvalidDevicePointer;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

bool aligned_to(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace
}  // namespace dpp

using namespace dpp;

extern "C" {

dpp_status dpp_sample_hermitian_static(const void* K, int64_t n, int64_t ld, int32_t dtype,
                                       uint64_t seed, uint64_t instance, const double* uniforms,
                                       uint8_t* keep, void* factor_out, double* pivots,
                                       dpp_result* result, void* stream) {
  clear_last_error();
  if (n < 0) return set_last_error(DPP_ERR_INVALID_ARG, "n must be >= 0");
  if (ld < (n > 1 ? n : 1)) return set_last_error(DPP_ERR_INVALID_ARG, "ld must be >= max(1, n)");
  if (dtype != DPP_R64 && dtype != DPP_C128)
    return set_last_error(DPP_ERR_INVALID_ARG, "unknown dtype");
  if (!result) return set_last_error(DPP_ERR_INVALID_ARG, "result must not be NULL");
  if (n > 0 && (!K || !keep || !factor_out))
    return set_last_error(DPP_ERR_INVALID_ARG,
                          "K, keep and factor_out must not be NULL (the factor is written to "
                          "caller memory; factor_out may equal K)");
  const size_t esz = dtype == DPP_C128 ? 16 : 8;
  if (n > 0 && (!aligned_to(K, esz) || !aligned_to(factor_out, esz)))
    return set_last_error(DPP_ERR_INVALID_ARG, "K or factor_out misaligned");
  if (!aligned_to(result, 8)) return set_last_error(DPP_ERR_INVALID_ARG, "result misaligned");
  const size_t need = ws_fp64(n, dtype, true, false);
  if (need > kStaticScratchBytes) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "n = %lld needs %zu bytes of static scratch; the limit is %zu bytes "
             "(real n <= %d, complex n <= %d)",
             (long long)n, need, kStaticScratchBytes, DPP_STATIC_MAX_N_R64,
             DPP_STATIC_MAX_N_C128);
    return set_last_error(DPP_ERR_WORKSPACE, buf);
  }
  void* scratch = nullptr;
  cudaError_t e = static_scratch(static_cast<cudaStream_t>(stream), &scratch);
  if (e != cudaSuccess) return set_last_cuda_error(e, "dpp_sample_hermitian_static: scratch set-up");
  begin_call(DPP_OP_SAMPLE_HERMITIAN, n, dtype, DPP_PREC_FP64);
  DrawArgs a;
  a.K = K;
  a.n = n;
  a.ld = ld;
  a.dtype = dtype;
  a.precision = DPP_PREC_FP64;
  a.seed = seed;
  a.instance = instance;
  a.uniforms = uniforms;
  a.keep = keep;
  a.factor_out = factor_out;
  a.pivots_user = pivots;
  a.result = result;
  a.stream = static_cast<cudaStream_t>(stream);
  Workspace ws;
  ws.base = static_cast<char*>(scratch);
  ws.size = kStaticScratchBytes;
  e = sample_fp64(a, true, ws);
  if (e != cudaSuccess) return set_last_cuda_error(e, "dpp_sample_hermitian_static");
  return DPP_OK;
}

}  // extern "C"
