// Naive multidimensional convolution (Algorithms 14 and 15; Section 3, benchmark 4):
//   out[t] = sum over tuples u of a's shape with t - u a tuple of b's shape of a[u] * b[t - u]
// for every tuple t of the result shape a.shape + b.shape - 1.  The paper scatters each
// product a[u] b[v] into out[u + v]; here each output gathers its own products
// (output-stationary: no atomics, every output written once): one warp per output, the
// lanes splitting the outermost axis of the box of contributing u, a fixed-order warp sum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {

struct ConvGeom {
  int D;
  long long sa[kMaxRank], sb[kMaxRank], sr[kMaxRank];  // extents of a, b and the result
  long long n_out;
};

namespace {

constexpr int kConvWarps = 8;

__global__ void __launch_bounds__(kConvWarps * 32) conv_kernel(const __grid_constant__ ConvGeom g,
                                                                const double* __restrict__ a,
                                                                const double* __restrict__ b,
                                                                double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long gw = (long long)blockIdx.x * kConvWarps + (threadIdx.x >> 5);
  const long long tw = (long long)gridDim.x * kConvWarps;
  const int D = g.D;
  long long t[kMaxRank], lo[kMaxRank], hi[kMaxRank], u[kMaxRank];
  for (long long k = gw; k < g.n_out; k += tw) {
    // the output's tuple (Algorithm 4) and the box of u with 0 <= u < sa, 0 <= t - u < sb
    long long rem = k;
    bool empty = false;
    for (int i = D - 1; i >= 0; --i) {
      const long long q = i > 0 ? rem / g.sr[i] : 0;
      t[i] = i > 0 ? rem - q * g.sr[i] : rem;
      rem = q;
      lo[i] = t[i] >= g.sb[i] ? t[i] - g.sb[i] + 1 : 0;
      hi[i] = t[i] < g.sa[i] - 1 ? t[i] : g.sa[i] - 1;
      empty = empty || lo[i] > hi[i];
    }
    double acc = 0.0;
    if (!empty) {
      // lane takes u_0 = lo_0 + lane, lo_0 + lane + 32, ...; the other axes in order
      for (long long u0 = lo[0] + lane; u0 <= hi[0]; u0 += 32) {
        u[0] = u0;
        for (int i = 1; i < D; ++i) u[i] = lo[i];
        while (true) {
          // Horner (Algorithm 2) for u in a and t - u in b, then the innermost axis
          long long ia = 0, ib = 0;
          for (int i = 0; i < D; ++i) {
            ia = ia * g.sa[i] + u[i];
            ib = ib * g.sb[i] + (t[i] - u[i]);
          }
          const long long n = hi[D - 1] - u[D - 1] + 1;
          if (D == 1) {
            acc = __dadd_rn(acc, __dmul_rn(a[ia], b[ib]));
            break;
          }
          for (long long j = 0; j < n; ++j) acc = __dadd_rn(acc, __dmul_rn(a[ia + j], b[ib - j]));
          // advance_tuple (Algorithm 3) over axes D-2 .. 1 of the box
          int i = D - 2;
          for (; i >= 1; --i) {
            if (++u[i] <= hi[i]) break;
            u[i] = lo[i];
          }
          if (i < 1) break;
        }
      }
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[k] = acc;
  }
}

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" int triot_convolve(int rank, const int64_t* ashape, const void* a, const int64_t* bshape,
                              const void* b, void* out, int dtype, void* stream) {
  char buf[256];
  if (dtype != TRIOT_F64) return fail(TRIOT_ERR_DTYPE, "convolution is f64 only");
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    return fail(TRIOT_ERR_RANK, buf);
  }
  if (!ashape || !bshape) return fail(TRIOT_ERR_NULL, "a shape pointer is NULL");
  ConvGeom g = ConvGeom();
  g.D = rank;
  g.n_out = 1;
  int64_t na = 1, nb = 1;
  for (int i = 0; i < rank; ++i) {
    if (ashape[i] < 0 || bshape[i] < 0) {
      snprintf(buf, sizeof buf, "negative extent on axis %d", i);
      return fail(TRIOT_ERR_SHAPE, buf);
    }
    if (ashape[i] >= (int64_t(1) << 31) || bshape[i] >= (int64_t(1) << 31))
      return fail(TRIOT_ERR_SHAPE, "extents must be < 2^31");
    g.sa[i] = ashape[i];
    g.sb[i] = bshape[i];
    g.sr[i] = std::max<int64_t>(0, ashape[i] + bshape[i] - 1);
    if (g.sr[i] && g.n_out > INT64_MAX / g.sr[i]) return fail(TRIOT_ERR_SHAPE, "element count overflows int64");
    g.n_out *= g.sr[i];
    na *= ashape[i];
    nb *= bshape[i];
  }
  if (g.n_out == 0) return ok();
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if ((na > 0 && !a) || (nb > 0 && !b)) return fail(TRIOT_ERR_NULL, "a or b is NULL");
  if ((a && overlaps_bytes(out, size_t(g.n_out) * 8, a, size_t(na) * 8)) ||
      (b && overlaps_bytes(out, size_t(g.n_out) * 8, b, size_t(nb) * 8)))
    return fail(TRIOT_ERR_ALIAS, "out overlaps an input");
  DeviceInfo dev;
  int st = device_info(dev);
  if (st) return st;
  const long long warps_needed = g.n_out;
  const long long grid = std::max(1ll, std::min<long long>((warps_needed + kConvWarps - 1) / kConvWarps,
                                                           (long long)dev.sms * 8));
  const double* ap = static_cast<const double*>(a ? a : out);
  const double* bp = static_cast<const double*>(b ? b : out);
  double* op = static_cast<double*>(out);
  void* args[] = {(void*)&g, (void*)&ap, (void*)&bp, (void*)&op};
  cudaError_t e = cudaLaunchKernel((const void*)conv_kernel, dim3((unsigned)grid), dim3(kConvWarps * 32), args, 0,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "convolution kernel launch");
  return ok();
}
