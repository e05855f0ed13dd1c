// Exact, order-independent combine of the moment kernels' per-CTA partial sums.
#include "common.cuh"
#include "fixed.cuh"
#include "kernels.h"

namespace triot {

// ====================================================================== combine (K3b)
//
// One CTA per effective component.  The block partials of that component are summed
// exactly: each f64 is converted to an integer in units of 2^(Emax-1075-56), Emax the
// largest exponent among them, and the integers are added (order-independent).  One
// rounding to f64 at the end.  Non-finite partials fall back to an ordered f64 sum.
// CTA 0 also zero-fills the outputs of axes dropped by canonicalisation (extent 1).
constexpr int kCombineThreads = 256;
constexpr int kCombineFrac = 56;

__global__ void __launch_bounds__(kCombineThreads) combine_kernel(
    const __grid_constant__ CombineGeom g, const double* __restrict__ partial,
    double* __restrict__ out) {
  __shared__ unsigned s_emax[kCombineThreads / 32];
  __shared__ int s_bad[kCombineThreads / 32];
  __shared__ unsigned long long s_lo[kCombineThreads / 32], s_hi[kCombineThreads / 32];
  // launched as a programmatic dependent of the moment kernel: its launch is prepared while
  // that kernel runs, and this wait returns once the kernel has finished and its partials
  // are visible (a plain launch returns at once)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int c = blockIdx.x;
  const int stride = g.D + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (c == 0) {
    for (int k = threadIdx.x; k < g.rank; k += blockDim.x) {
      bool covered = false;
      for (int a = 0; a < g.D; ++a) covered |= (g.orig[a] == k);
      if (!covered) out[k] = 0.0;
    }
  }
  // the first kCache partials of each thread stay in registers between the two passes
  // (every launch with at most kCache * kCombineThreads partials reads them once)
  constexpr int kCache = 4;
  unsigned long long cb[kCache];
  unsigned emax = 0;
  int bad = 0;
  auto scan = [&](unsigned long long b) {
    const unsigned e = (unsigned)((b >> 52) & 0x7FF);
    if (e == 0x7FF) bad = 1;
    else emax = e > emax ? e : emax;
  };
#pragma unroll
  for (int r = 0; r < kCache; ++r) {
    const int k = threadIdx.x + r * kCombineThreads;
    cb[r] = k < g.nparts ? (unsigned long long)__double_as_longlong(partial[(long long)k * stride + c]) : 0ull;
    scan(cb[r]);
  }
  for (int k = threadIdx.x + kCache * kCombineThreads; k < g.nparts; k += kCombineThreads)
    scan((unsigned long long)__double_as_longlong(partial[(long long)k * stride + c]));
  emax = __reduce_max_sync(0xffffffffu, emax);
  bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
  if (lane == 0) { s_emax[warp] = emax; s_bad[warp] = bad; }
  __syncthreads();
  emax = 0; bad = 0;
  for (int w = 0; w < kCombineThreads / 32; ++w) { emax = s_emax[w] > emax ? s_emax[w] : emax; bad |= s_bad[w]; }
  const int outidx = (c < g.D) ? g.orig[c] : g.rank;
  if (bad) {
    if (threadIdx.x == 0) {
      double acc = 0.0;
      for (int k = 0; k < g.nparts; ++k) acc += partial[(long long)k * stride + c];
      out[outidx] = acc;
    }
    return;
  }
  const int E = emax ? (int)emax : 1;
  __int128 acc = 0;
  auto add = [&](unsigned long long b) {
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    const int sh = kCombineFrac - (E - (e ? e : 1));
    __int128 v = scale_shift((__int128)m, sh);
    acc += (b >> 63) ? -v : v;
  };
#pragma unroll
  for (int r = 0; r < kCache; ++r) add(cb[r]);  // absent partials are +0 and add nothing
  for (int k = threadIdx.x + kCache * kCombineThreads; k < g.nparts; k += kCombineThreads)
    add((unsigned long long)__double_as_longlong(partial[(long long)k * stride + c]));
  unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)((unsigned __int128)acc >> 64);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
    const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
    const unsigned __int128 sum = (((unsigned __int128)hi << 64) | lo) + (((unsigned __int128)ohi << 64) | olo);
    lo = (unsigned long long)sum;
    hi = (unsigned long long)(sum >> 64);
  }
  if (lane == 0) { s_lo[warp] = lo; s_hi[warp] = hi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned __int128 tot = 0;
    for (int w = 0; w < kCombineThreads / 32; ++w) tot += ((unsigned __int128)s_hi[w] << 64) | s_lo[w];
    // one rounding to f64 with integer operations (the FP64 pipe of this GPU is narrow)
    out[outidx] = fixed_to_double((__int128)tot, E - 1075 - kCombineFrac);
  }
}

const void* combine_kernel_ptr() { return reinterpret_cast<const void*>(&combine_kernel); }

}  // namespace triot
