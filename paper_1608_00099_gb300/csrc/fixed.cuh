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

}  // namespace triot
