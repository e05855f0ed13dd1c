// Division of 32-bit unsigned integers by a run-time invariant divisor with one
// multiply-high, two shifts and two adds (Granlund & Montgomery, "Division by Invariant
// Integers using Multiplication", PLDI 1994, Figure 4.1, the N+1-bit multiplier case).
//
// This replaces the `%` and `/` of the paper's reindexing (Algorithm 4), which Section 1
// identifies as what makes reindexing slower than tuple iteration: the divisor (a tensor
// extent) is fixed for a whole launch, so its magic multiplier is computed once on the
// host and each decode step costs a few integer instructions.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define TRIOT_HD __host__ __device__ __forceinline__
#else
#define TRIOT_HD inline
#endif

namespace triot {

struct FastDiv {
  uint32_t d;    // divisor, 1 <= d < 2^31
  uint32_t m;    // magic multiplier m' = floor(2^32 * (2^l - d) / d) + 1
  uint8_t s1;    // min(l, 1)
  uint8_t s2;    // max(l - 1, 0)
  uint8_t pad[2];
};

// l = ceil(log2(d)); the paper's axes never need divisors >= 2^31.
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{};
  f.d = d;
  uint32_t l = 0;
  while (l < 32 && (uint64_t(1) << l) < d) ++l;
  const uint64_t two32 = uint64_t(1) << 32;
  f.m = uint32_t((two32 * ((uint64_t(1) << l) - d)) / d + 1);
  f.s1 = uint8_t(l < 1 ? l : 1);
  f.s2 = uint8_t(l > 1 ? l - 1 : 0);
  return f;
}

TRIOT_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  return __umulhi(a, b);
#else
  return uint32_t((uint64_t(a) * uint64_t(b)) >> 32);
#endif
}

// q = n / d for every 0 <= n < 2^32.
TRIOT_HD uint32_t fdiv(uint32_t n, const FastDiv& f) {
  const uint32_t t = mulhi32(f.m, n);
  return (t + ((n - t) >> f.s1)) >> f.s2;
}

// q = n / d, r = n % d.
TRIOT_HD uint32_t fdivmod(uint32_t n, const FastDiv& f, uint32_t& r) {
  const uint32_t q = fdiv(n, f);
  r = n - q * f.d;
  return q;
}

}  // namespace triot
