// Device helpers shared by the float-accumulating block moment kernels (moment_blk32.cu,
// moment_wb.cu): element conversion, staged-copy waits and the warps' compensated totals.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "sync.cuh"

namespace triot {

// element i (0 .. 16/sizeof(T) - 1) of a 16-byte piece, and one element of global memory,
// as f32 (exact for every storage type)
template <typename T> struct FPiece;
template <> struct FPiece<float> {
  __device__ static float get(const uint4& v, int i) {
    return __uint_as_float(i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w);
  }
  __device__ static float ld(const float* p, long long i) { return __ldcs(p + i); }
};
template <> struct FPiece<__nv_bfloat16> {
  __device__ static float get(const uint4& v, int i) {
    const unsigned w = (i >> 1) == 0 ? v.x : (i >> 1) == 1 ? v.y : (i >> 1) == 2 ? v.z : v.w;
    return __uint_as_float((i & 1) ? (w & 0xFFFF0000u) : (w << 16));
  }
  __device__ static float ld(const __nv_bfloat16* p, long long i) {
    return __uint_as_float((unsigned)__ldcs(reinterpret_cast<const unsigned short*>(p) + i) << 16);
  }
};
template <> struct FPiece<__half> {
  __device__ static float get(const uint4& v, int i) {
    const unsigned w = (i >> 1) == 0 ? v.x : (i >> 1) == 1 ? v.y : (i >> 1) == 2 ? v.z : v.w;
    return __half2float(__ushort_as_half((unsigned short)((i & 1) ? (w >> 16) : (w & 0xFFFFu))));
  }
  __device__ static float ld(const __half* p, long long i) {
    return __half2float(__ushort_as_half(__ldcs(reinterpret_cast<const unsigned short*>(p) + i)));
  }
};

// 16-byte cp.async; bytes past src_bytes are zero-filled
__device__ __forceinline__ void fm_cp16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes)
               : "memory");
}

// bounded wait for the phase of parity `par` of the mbarrier at shared address `bar`; on
// time-out the sticky flag is set (lane 0) and the caller goes on, so the kernel ends
__device__ __forceinline__ void fm_wait(unsigned bar, unsigned par, int lane, int* flag) {
  if (!mbar_wait_bounded(bar, par, kWaitLimit) && lane == 0) atomicExch(flag, 1);
}

// one window sum of every lane into the warp's total: f32 xor tree (a fixed order), then a
// compensated (Knuth two-sum) pair kept by lane 0
__device__ __forceinline__ void fm_warp_add(float v, float* ts, float* te, int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) {
    const float a = *ts, t = a + v, bp = t - a;
    *te += (a - (t - bp)) + (v - bp);
    *ts = t;
  }
}

// the CTA's partial of component c: its warps' compensated totals added in f64 (a non-finite
// total carries no meaningful compensation: inf - inf there is NaN)
template <int NW>
__device__ __forceinline__ double fm_cta_total(const float (*tot)[2][kMaxRank + 1], int c) {
  double acc = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) {
    const float ts = tot[w][0][c], te = tot[w][1][c];
    acc += isfinite(ts) ? (double)ts + (double)te : (double)ts;
  }
  return acc;
}

}  // namespace triot
