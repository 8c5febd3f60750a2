// Device-side building blocks shared by the sampler kernels: scalar traits
// for real/complex FP64 and FP32, the Philox4x32-10 uniform, bounded waits on
// device flags and the per-draw result record.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dpp.h"

namespace dpp {

// ---------------------------------------------------------------------------
// Scalars
// ---------------------------------------------------------------------------
struct cdouble {
  double re, im;
};

__host__ __device__ inline cdouble mk(double r, double i) { return {r, i}; }

template <class T>
struct Sc;

template <>
struct Sc<double> {
  static constexpr bool cplx = false;
  __device__ static inline double zero() { return 0.0; }
  __device__ static inline double from_real(double r) { return r; }
  __device__ static inline double re(double a) { return a; }
  __device__ static inline double im(double) { return 0.0; }
  __device__ static inline double conj(double a) { return a; }
  __device__ static inline double add(double a, double b) { return a + b; }
  __device__ static inline double sub(double a, double b) { return a - b; }
  __device__ static inline double mul(double a, double b) { return a * b; }
  // a - b * c
  __device__ static inline double fnms(double a, double b, double c) { return fma(-b, c, a); }
  // a - b * conj(c)
  __device__ static inline double fnms_conj(double a, double b, double c) { return fma(-b, c, a); }
  __device__ static inline double div_real(double a, double d) { return a / d; }
  __device__ static inline double div(double a, double b) { return a / b; }
  __device__ static inline double abs2(double a) { return a * a; }
  __device__ static inline double absv(double a) { return fabs(a); }
  __device__ static inline bool finite(double a) { return isfinite(a); }
};

template <>
struct Sc<cdouble> {
  static constexpr bool cplx = true;
  __device__ static inline cdouble zero() { return {0.0, 0.0}; }
  __device__ static inline cdouble from_real(double r) { return {r, 0.0}; }
  __device__ static inline double re(cdouble a) { return a.re; }
  __device__ static inline double im(cdouble a) { return a.im; }
  __device__ static inline cdouble conj(cdouble a) { return {a.re, -a.im}; }
  __device__ static inline cdouble add(cdouble a, cdouble b) { return {a.re + b.re, a.im + b.im}; }
  __device__ static inline cdouble sub(cdouble a, cdouble b) { return {a.re - b.re, a.im - b.im}; }
  __device__ static inline cdouble mul(cdouble a, cdouble b) {
    return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
  }
  __device__ static inline cdouble fnms(cdouble a, cdouble b, cdouble c) {
    // a - b*c
    double r = fma(-b.re, c.re, a.re);
    r = fma(b.im, c.im, r);
    double i = fma(-b.re, c.im, a.im);
    i = fma(-b.im, c.re, i);
    return {r, i};
  }
  __device__ static inline cdouble fnms_conj(cdouble a, cdouble b, cdouble c) {
    // a - b*conj(c)
    double r = fma(-b.re, c.re, a.re);
    r = fma(-b.im, c.im, r);
    double i = fma(b.re, c.im, a.im);
    i = fma(-b.im, c.re, i);
    return {r, i};
  }
  __device__ static inline cdouble div_real(cdouble a, double d) { return {a.re / d, a.im / d}; }
  __device__ static inline cdouble div(cdouble a, cdouble b) {
    // Smith's algorithm (scaled complex division)
    if (fabs(b.re) >= fabs(b.im)) {
      double r = b.im / b.re, den = b.re + b.im * r;
      return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    } else {
      double r = b.re / b.im, den = b.re * r + b.im;
      return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
    }
  }
  __device__ static inline double abs2(cdouble a) { return a.re * a.re + a.im * a.im; }
  __device__ static inline double absv(cdouble a) { return hypot(a.re, a.im); }
  __device__ static inline bool finite(cdouble a) { return isfinite(a.re) && isfinite(a.im); }
};

// ---------------------------------------------------------------------------
// Double-float ("df64") values: an unevaluated sum hi + lo of two floats with
// about 48 significant bits, built from the error-free transformations TwoSum
// (Knuth) and TwoProduct-by-FMA (Dekker / Ogita-Rump-Oishi). Used where an
// FP64 accumulation would otherwise sit on a latency-critical FP32 path.
// Every operation uses explicit _rn intrinsics so no contraction can break
// the transformations.
// ---------------------------------------------------------------------------
struct f2 {
  float hi, lo;
};

__device__ inline f2 make_f2(float hi, float lo) { return {hi, lo}; }

__device__ inline f2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ inline f2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ inline f2 f2_from_double(double x) {
  const float hi = __double2float_rn(x);
  return {hi, __double2float_rn(x - (double)hi)};
}

__device__ inline double f2_to_double(f2 a) { return (double)a.hi + (double)a.lo; }

// a + c (c a float)
__device__ inline f2 f2_add_f(f2 a, float c) {
  const f2 s = two_sum(a.hi, c);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// a - w * l with the product formed exactly (w * l = p + pe)
__device__ inline f2 f2_sub_prod(f2 a, float w, float l) {
  const float p = __fmul_rn(w, l);
  const float pe = __fmaf_rn(w, l, -p);
  const f2 s = two_sum(a.hi, -p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, pe)));
}

// a + b (both double-float)
__device__ inline f2 f2_add(f2 a, f2 b) {
  const f2 s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// a + w * l
__device__ inline f2 f2_add_prod(f2 a, float w, float l) {
  const float p = __fmul_rn(w, l);
  const float pe = __fmaf_rn(w, l, -p);
  const f2 s = two_sum(a.hi, p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, pe)));
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
// multiply/xor bijection with a Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__device__ inline void philox4x32_10(uint32_t& x0, uint32_t& x1, uint32_t& x2,
                                     uint32_t& x3, uint32_t k0, uint32_t k1) {
  const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
  const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hA = __umulhi(kMulA, x0), lA = kMulA * x0;
    const uint32_t hB = __umulhi(kMulB, x2), lB = kMulB * x2;
    const uint32_t y0 = hB ^ x1 ^ k0;
    const uint32_t y2 = hA ^ x3 ^ k1;
    x0 = y0;
    x1 = lB;
    x2 = y2;
    x3 = lA;
    k0 += kWeylA;
    k1 += kWeylB;
  }
}

// u_j in (0,1) with 53 random bits, counter (j, instance), key = seed.
__device__ inline double philox_uniform(uint64_t seed, uint64_t instance, uint64_t j) {
  uint32_t x0 = (uint32_t)j, x1 = (uint32_t)instance, x2 = (uint32_t)(instance >> 32), x3 = 0u;
  philox4x32_10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint64_t bits = ((uint64_t)x0 << 21) | (uint64_t)(x1 >> 11);
  return ((double)bits + 0.5) * 0x1.0p-53;
}

// ---------------------------------------------------------------------------
// Bounded waits. Every spin in this library gives up after a limit of
// wall-clock time (device %globaltimer), reports DPP_RES_TIMEOUT and returns.
// The waits between the CTAs of the panel launches take their limit from the
// launch arguments (DPP_TUNE_WAIT_NS, 2 s by default); the tensor-core
// update's pipeline waits use the fixed kWaitNs.
// ---------------------------------------------------------------------------
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s

__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ inline unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ inline void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin (one thread) until *flag >= target. Returns false after limit_ns.
__device__ inline bool wait_geq(const unsigned* flag, unsigned target,
                                unsigned long long limit_ns) {
  if (ld_acquire(flag) >= target) return true;
  const unsigned long long t0 = global_ns();
  unsigned sleep = 32;
  while (true) {
    if (ld_acquire(flag) >= target) return true;
    if (global_ns() - t0 > limit_ns) return false;
    __nanosleep(sleep);
    if (sleep < 1024) sleep <<= 1;
  }
}

// Asynchronous 4-byte global -> shared copies (cp.async): every copy of a
// staging loop is in flight at once instead of one dependent load at a time.
// A copy with valid == false writes zero and reads nothing (gmem must still be
// a valid address).
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem),
               "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Status word that any kernel may OR bits into.
__device__ inline void flag_status(dpp_result* r, int bits) { atomicOr(&r->status, bits); }

}  // namespace dpp
