// Signed 128-bit fixed-point helpers for exact (order-independent) sums of f64 values.
#pragma once

namespace triot {

__device__ __forceinline__ __int128 shr_arith(__int128 v, int sh) {
  if (sh <= 0) return v;
  if (sh >= 127) return v < 0 ? (__int128)-1 : (__int128)0;
  return v >> sh;
}
__device__ __forceinline__ __int128 scale_shift(__int128 v, int sh) {  // v * 2^sh
  if (sh >= 0) return v << sh;
  return shr_arith(v, -sh);
}

__device__ __forceinline__ double i128_to_double(__int128 v) {
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)(-(v + 1)) + 1u : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  const double d = fma(__ull2double_rn(hi), 0x1p64, __ull2double_rn(lo));
  return neg ? -d : d;
}

// v * 2^k rounded to f64 (nearest, ties to even) with 64-bit integer operations; the FP64
// pipe of this GPU is narrow, so it is used only where the result leaves the normal range
__device__ __forceinline__ double fixed_to_double(__int128 v, int k) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 u = neg ? (unsigned __int128)0 - (unsigned __int128)v : (unsigned __int128)v;
  const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
  // t: the top 64 significant bits (leading bit at 63); sticky: any bit below them
  unsigned long long t;
  bool sticky;
  int e;  // exponent of the leading bit
  if (hi == 0) {
    const int lz = __clzll((long long)lo);
    t = lo << lz;
    sticky = false;
    e = 63 - lz + k;
  } else {
    const int lz = __clzll((long long)hi);
    t = lz ? (hi << lz) | (lo >> (64 - lz)) : hi;
    sticky = lz ? (lo << lz) != 0 : lo != 0;
    e = 127 - lz + k;
  }
  if (e < -1022 || e > 1023) {
    const int k1 = k / 2, k2 = k - k1;
    return i128_to_double(v) * __longlong_as_double((long long)(k1 + 1023) << 52) *
           __longlong_as_double((long long)(k2 + 1023) << 52);
  }
  unsigned long long mant = t >> 11;  // 53 bits
  const unsigned r = (unsigned)(t & 0x7FFull);
  if (r > 0x400u || (r == 0x400u && (sticky || (mant & 1ull)))) ++mant;
  // mant in [2^52, 2^53]; a carry to 2^53 moves into the exponent field by itself
  const unsigned long long bits =
      ((unsigned long long)(e + 1022) << 52) + mant + (neg ? 0x8000000000000000ull : 0ull);
  return __longlong_as_double((long long)bits);
}

// acc += a * b exactly (the 128-bit product from the low and high 64-bit halves)
__device__ __forceinline__ void mac128(__int128& acc, long long a, long long b) {
  const unsigned long long lo = (unsigned long long)a * (unsigned long long)b;
  const long long hi = __mul64hi(a, b);
  acc += (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// acc += a * t exactly for |a| < 2^95 (the product stays inside 128 bits)
__device__ __forceinline__ void mac128x32(__int128& acc, __int128 a, uint32_t t) {
  const unsigned long long lo = (unsigned long long)a;
  const long long hi = (long long)(a >> 64);
  const unsigned long long plo = lo * (unsigned long long)t;
  const unsigned long long phi = __umul64hi(lo, (unsigned long long)t) + (unsigned long long)(hi * (long long)t);
  acc += (__int128)(((unsigned __int128)phi << 64) | plo);
}

// acc += a * t exactly for 0 <= t < 2^31 (two 32x32 -> 64-bit products)
__device__ __forceinline__ void mac64x32(__int128& acc, long long a, uint32_t t) {
  const unsigned long long p0 = (unsigned long long)(uint32_t)a * (unsigned long long)t;
  const long long p1 = (long long)(int)(a >> 32) * (long long)t;
  acc += (__int128)p0 + ((__int128)p1 << 32);
}

__device__ __forceinline__ long long shr64(long long v, int d) {
  return d >= 63 ? (v < 0 ? -1ll : 0ll) : (v >> d);
}

// one lane's column of a lane-major shared-memory array (STRIDE threads): element i of
// this lane
template <typename T, int STRIDE>
struct LaneCol {
  T* p;
  __device__ __forceinline__ T& operator[](int i) const { return p[i * STRIDE]; }
};

}  // namespace triot
