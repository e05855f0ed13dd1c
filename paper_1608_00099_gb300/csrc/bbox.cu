// The nonzero bounding box of a product of tensors (Section 2: with the tuple visible to
// the operation, the bounding box of the nonzero entries of the element-wise product of two
// tensors is a simple reduction over the tuples).
//
// Over the intersection I of the shapes, a tuple t counts when every factor x_k[t] is
// nonzero (the support of the product as real functions: IEEE comparison with zero, so NaN
// and infinities count, +0 and -0 do not, and nothing is rounded).  The result per axis is
// the least and greatest t_i over the counted tuples, and their number.
//
// Kernels: for rows of 32 elements or more, warps take rows of I (all axes but the
// innermost) in a strided order; a row's
// tuple is decoded once (Algorithm 4 with magic-number division) into each tensor's row
// offset, and the lanes test the row's elements (coalesced along the innermost axis), each
// lane keeping the least and greatest inner digit and a count.  A row with a counted
// element (a warp vote) updates the outer axes' least and greatest digits with the row's
// digits.  Per CTA the warps' boxes are merged (min / max / sum, exact and independent of
// order) into a workspace slot; a one-CTA combine merges the slots and writes the result in
// the caller's axis order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {
namespace {

constexpr int kBoxWarps = 8;
constexpr int kBoxMaxTensors = 4;

struct BoxGeom {
  int D;                                  // rank of the canonical I (unit axes dropped), >= 1
  int n;                                  // tensors
  int rank;                               // caller's rank
  int rows32;                             // rows < 2^32
  long long rows;                         // product of the extents of axes 0 .. D-2
  long long L;                            // extent of the innermost axis
  long long ext[kMaxRank];
  FastDiv div[kMaxRank];
  long long stride[kBoxMaxTensors][kMaxRank];  // element strides of every tensor on I's axes
  const void* x[kBoxMaxTensors];
  int orig[kMaxRank];                     // caller's axis of each canonical axis
};

// nonzero test on the bit pattern (sign bit ignored): exact for every format
template <typename B>
__device__ __forceinline__ bool nz_bits(B b) {
  return (B)(b << 1) != (B)0;
}

template <typename B, int N>
__global__ void __launch_bounds__(kBoxWarps * 32) bbox_kernel(const __grid_constant__ BoxGeom g,
                                                             long long* __restrict__ slots) {
  __shared__ unsigned s_lo[kBoxWarps][kMaxRank], s_hi[kBoxWarps][kMaxRank];
  __shared__ unsigned long long s_cnt[kBoxWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBoxWarps + warp;
  const long long W = (long long)gridDim.x * kBoxWarps;
  const int D = g.D;
  unsigned lo[kMaxRank], hi[kMaxRank];    // outer axes 0 .. D-2 (warp-uniform)
  for (int a = 0; a + 1 < D; ++a) {
    lo[a] = 0xFFFFFFFFu;
    hi[a] = 0u;
  }
  unsigned ilo = 0xFFFFFFFFu, ihi = 0u;   // innermost axis (per lane)
  unsigned long long cnt = 0;
  const B* X[N];
#pragma unroll
  for (int k = 0; k < N; ++k) X[k] = static_cast<const B*>(g.x[k]);
  for (long long r = gw; r < g.rows; r += W) {
    // the row's digits (innermost outer axis first) and each tensor's row offset
    unsigned dig[kMaxRank];
    long long off[N];
#pragma unroll
    for (int k = 0; k < N; ++k) off[k] = 0;
    if (g.rows32) {
      uint32_t q = (uint32_t)r;
      for (int a = D - 2; a >= 0; --a) {
        uint32_t d = q;
        if (a > 0) {
          const uint32_t q1 = fdiv(q, g.div[a]);
          d = q - q1 * g.div[a].d;
          q = q1;
        }
        dig[a] = d;
#pragma unroll
        for (int k = 0; k < N; ++k) off[k] += (long long)d * g.stride[k][a];
      }
    } else {
      long long q = r;
      for (int a = D - 2; a >= 0; --a) {
        long long d = q;
        if (a > 0) {
          d = q % g.ext[a];
          q /= g.ext[a];
        }
        dig[a] = (unsigned)d;
#pragma unroll
        for (int k = 0; k < N; ++k) off[k] += d * g.stride[k][a];
      }
    }
    unsigned rowcnt = 0;
    for (long long j = lane; j < g.L; j += 32) {
      bool all = true;
#pragma unroll
      for (int k = 0; k < N; ++k) all = all && nz_bits(__ldg(X[k] + off[k] + j * g.stride[k][D - 1]));
      if (all) {
        ilo = min(ilo, (unsigned)j);
        ihi = max(ihi, (unsigned)j);
        ++rowcnt;
      }
    }
    cnt += rowcnt;
    if (__any_sync(0xffffffffu, rowcnt != 0)) {
      for (int a = 0; a + 1 < D; ++a) {
        lo[a] = min(lo[a], dig[a]);
        hi[a] = max(hi[a], dig[a]);
      }
    }
  }
  // warp: innermost axis and count reduced over the lanes; outer axes are uniform already
  ilo = __reduce_min_sync(0xffffffffu, ilo);
  ihi = __reduce_max_sync(0xffffffffu, ihi);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
    for (int a = 0; a + 1 < D; ++a) {
      s_lo[warp][a] = lo[a];
      s_hi[warp][a] = hi[a];
    }
    s_lo[warp][D - 1] = ilo;
    s_hi[warp][D - 1] = ihi;
    s_cnt[warp] = cnt;
  }
  __syncthreads();
  // slot layout: [lo_0, hi_0, .., lo_{D-1}, hi_{D-1}, count] (lo = INT64_MAX, hi = -1 when
  // the CTA counted nothing)
  long long* slot = slots + (long long)blockIdx.x * (2 * D + 1);
  if (threadIdx.x < D) {
    const int a = threadIdx.x;
    unsigned l = 0xFFFFFFFFu, h = 0u;
    unsigned long long c = 0;
    for (int w = 0; w < kBoxWarps; ++w) {
      if (s_cnt[w] == 0) continue;
      l = min(l, s_lo[w][a]);
      h = max(h, s_hi[w][a]);
      c += s_cnt[w];
    }
    slot[2 * a] = c ? (long long)l : LLONG_MAX;
    slot[2 * a + 1] = c ? (long long)h : -1;
  }
  if (threadIdx.x == 0) {
    unsigned long long c = 0;
    for (int w = 0; w < kBoxWarps; ++w) c += s_cnt[w];
    slot[2 * D] = (long long)c;
  }
}

// Short rows (fewer than 32 elements): a warp takes 32 consecutive rows at a time, one per
// lane, so that each load instruction of the warp reads neighbouring rows (a contiguous
// stretch of every tensor).  Each lane decodes its row (magic-number division) and tests the
// row's elements; the outer axes' least and greatest digits over the group's counted rows
// come from one warp min / max per axis, so the per-lane bookkeeping stays in registers.
template <typename B, int N>
__global__ void __launch_bounds__(kBoxWarps * 32) bbox_rows_kernel(const __grid_constant__ BoxGeom g,
                                                                  long long* __restrict__ slots) {
  __shared__ unsigned s_lo[kBoxWarps][kMaxRank], s_hi[kBoxWarps][kMaxRank];
  __shared__ unsigned long long s_cnt[kBoxWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBoxWarps + warp;
  const long long W = (long long)gridDim.x * kBoxWarps;
  const int D = g.D;  // >= 2 here (a short innermost axis and at least one outer axis)
  unsigned lo[kMaxRank], hi[kMaxRank];  // outer axes (warp-uniform), registers
#pragma unroll
  for (int a = 0; a < kMaxRank; ++a) {
    lo[a] = 0xFFFFFFFFu;
    hi[a] = 0u;
  }
  unsigned ilo = 0xFFFFFFFFu, ihi = 0u;
  unsigned long long cnt = 0;
  const B* X[N];
#pragma unroll
  for (int k = 0; k < N; ++k) X[k] = static_cast<const B*>(g.x[k]);
  const long long ngroups = (g.rows + 31) / 32;
  for (long long grp = gw; grp < ngroups; grp += W) {
    const long long r = grp * 32 + lane;
    const bool valid = r < g.rows;
    unsigned dig[kMaxRank];
    long long off[N];
#pragma unroll
    for (int k = 0; k < N; ++k) off[k] = 0;
    {
      uint32_t q = valid ? (uint32_t)r : 0u;  // rows < 2^32 for this kernel
#pragma unroll
      for (int a = kMaxRank - 1; a >= 0; --a) {
        dig[a] = 0;
        if (a + 1 < D) {
          uint32_t d = q;
          if (a > 0) {
            const uint32_t q1 = fdiv(q, g.div[a]);
            d = q - q1 * g.div[a].d;
            q = q1;
          }
          dig[a] = d;
#pragma unroll
          for (int k = 0; k < N; ++k) off[k] += (long long)d * g.stride[k][a];
        }
      }
    }
    unsigned rowcnt = 0;
    if (valid) {
      // eight elements of every factor loaded before any is tested (no short-circuit: the
      // loads of one batch are all in flight together)
      for (int j0 = 0; j0 < (int)g.L; j0 += 8) {
        B v[N][8];
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
#pragma unroll
          for (int k = 0; k < N; ++k)
            v[k][jj] = j0 + jj < (int)g.L ? __ldg(X[k] + off[k] + (j0 + jj) * g.stride[k][D - 1]) : (B)0;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
          bool all = j0 + jj < (int)g.L;
#pragma unroll
          for (int k = 0; k < N; ++k) all = all & nz_bits(v[k][jj]);
          if (all) {
            ilo = min(ilo, (unsigned)(j0 + jj));
            ihi = max(ihi, (unsigned)(j0 + jj));
            ++rowcnt;
          }
        }
      }
    }
    cnt += rowcnt;
    if (__any_sync(0xffffffffu, rowcnt != 0)) {
#pragma unroll
      for (int a = 0; a < kMaxRank; ++a) {
        if (a + 1 >= D) break;
        lo[a] = min(lo[a], __reduce_min_sync(0xffffffffu, rowcnt ? dig[a] : 0xFFFFFFFFu));
        hi[a] = max(hi[a], __reduce_max_sync(0xffffffffu, rowcnt ? dig[a] : 0u));
      }
    }
  }
  ilo = __reduce_min_sync(0xffffffffu, ilo);
  ihi = __reduce_max_sync(0xffffffffu, ihi);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < kMaxRank; ++a) {
      if (a + 1 >= D) break;
      s_lo[warp][a] = lo[a];
      s_hi[warp][a] = hi[a];
    }
    s_lo[warp][D - 1] = ilo;
    s_hi[warp][D - 1] = ihi;
    s_cnt[warp] = cnt;
  }
  __syncthreads();
  long long* slot = slots + (long long)blockIdx.x * (2 * D + 1);
  if (threadIdx.x < D) {
    const int a = threadIdx.x;
    unsigned l = 0xFFFFFFFFu, h = 0u;
    unsigned long long c = 0;
    for (int w = 0; w < kBoxWarps; ++w) {
      if (s_cnt[w] == 0) continue;
      l = min(l, s_lo[w][a]);
      h = max(h, s_hi[w][a]);
      c += s_cnt[w];
    }
    slot[2 * a] = c ? (long long)l : LLONG_MAX;
    slot[2 * a + 1] = c ? (long long)h : -1;
  }
  if (threadIdx.x == 0) {
    unsigned long long c = 0;
    for (int w = 0; w < kBoxWarps; ++w) c += s_cnt[w];
    slot[2 * D] = (long long)c;
  }
}

// merge the CTAs' slots; write [lo_0, hi_0, .., count] in the caller's axis order (axes of
// extent 1 in I: 0 .. 0 when anything counted); nothing counted: lo 0, hi -1 everywhere
__global__ void __launch_bounds__(256) bbox_combine_kernel(const __grid_constant__ BoxGeom g, int nslots,
                                                           const long long* __restrict__ slots,
                                                           long long* __restrict__ out) {
  __shared__ long long s_lo[kMaxRank], s_hi[kMaxRank];
  __shared__ unsigned long long s_cnt;
  const int D = g.D;
  if (threadIdx.x == 0) {
    unsigned long long c = 0;
    for (int k = 0; k < nslots; ++k) c += (unsigned long long)slots[(long long)k * (2 * D + 1) + 2 * D];
    s_cnt = c;
  }
  if (threadIdx.x < D) {
    long long l = LLONG_MAX, h = -1;
    for (int k = 0; k < nslots; ++k) {
      const long long* sl = slots + (long long)k * (2 * D + 1);
      l = min(l, sl[2 * threadIdx.x]);
      h = max(h, sl[2 * threadIdx.x + 1]);
    }
    s_lo[threadIdx.x] = l;
    s_hi[threadIdx.x] = h;
  }
  __syncthreads();
  const bool any = s_cnt != 0;
  for (int i = threadIdx.x; i < g.rank; i += blockDim.x) {
    long long l = 0, h = any ? 0 : -1;  // an axis of extent 1 in I
    for (int a = 0; a < D; ++a)
      if (g.orig[a] == i) {
        l = any ? s_lo[a] : 0;
        h = any ? s_hi[a] : -1;
      }
    out[2 * i] = l;
    out[2 * i + 1] = h;
  }
  if (threadIdx.x == 0) out[2 * g.rank] = (long long)s_cnt;
}

template <typename B>
const void* pick_bbox(int n, bool short_rows) {
  if (short_rows) {
    switch (n) {
      case 1: return reinterpret_cast<const void*>(&bbox_rows_kernel<B, 1>);
      case 2: return reinterpret_cast<const void*>(&bbox_rows_kernel<B, 2>);
      case 3: return reinterpret_cast<const void*>(&bbox_rows_kernel<B, 3>);
      default: return reinterpret_cast<const void*>(&bbox_rows_kernel<B, 4>);
    }
  }
  switch (n) {
    case 1: return reinterpret_cast<const void*>(&bbox_kernel<B, 1>);
    case 2: return reinterpret_cast<const void*>(&bbox_kernel<B, 2>);
    case 3: return reinterpret_cast<const void*>(&bbox_kernel<B, 3>);
    default: return reinterpret_cast<const void*>(&bbox_kernel<B, 4>);
  }
}

bool mul_overflows_box(int64_t a, int64_t b) { return a != 0 && b > INT64_MAX / a; }

struct BoxLaunch {
  BoxGeom g;
  int grid = 0;
  bool empty = false;
  bool short_rows = false;
};

int plan_bbox(int rank, int n, const int64_t* const* shapes, int dtype, const void* const* ptrs, BoxLaunch& L) {
  char buf[256];
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    return fail(TRIOT_ERR_RANK, buf);
  }
  if (n < 1 || n > kBoxMaxTensors) {
    snprintf(buf, sizeof buf, "ntensors %d outside [1, %d]", n, kBoxMaxTensors);
    return fail(TRIOT_ERR_ARG, buf);
  }
  if (!shapes) return fail(TRIOT_ERR_NULL, "shapes is NULL");
  int64_t I[kMaxRank];
  for (int k = 0; k < n; ++k) {
    if (!shapes[k]) return fail(TRIOT_ERR_NULL, "a shape pointer is NULL");
    for (int i = 0; i < rank; ++i) {
      const int64_t e = shapes[k][i];
      if (e < 0) {
        snprintf(buf, sizeof buf, "negative extent on axis %d of tensor %d", i, k);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      if (e >= (int64_t(1) << 31)) {
        snprintf(buf, sizeof buf, "extent %lld on axis %d of tensor %d must be < 2^31", (long long)e, i, k);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      I[i] = k == 0 ? e : std::min(I[i], e);
    }
  }
  int64_t st[kBoxMaxTensors][kMaxRank];
  for (int k = 0; k < n; ++k) {
    int64_t s = 1;
    for (int i = rank - 1; i >= 0; --i) {
      st[k][i] = s;
      const int64_t e = shapes[k][i] > 0 ? shapes[k][i] : 1;
      if (mul_overflows_box(s, e)) return fail(TRIOT_ERR_SHAPE, "element count overflows int64");
      s *= e;
    }
  }
  int64_t total = 1;
  for (int i = 0; i < rank; ++i) total *= I[i];
  L = BoxLaunch();
  BoxGeom& g = L.g;
  g.rank = rank;
  g.n = n;
  int D = 0;
  for (int i = 0; i < rank; ++i) {
    if (I[i] == 1) continue;
    g.ext[D] = I[i];
    for (int k = 0; k < n; ++k) g.stride[k][D] = st[k][i];
    g.orig[D] = i;
    ++D;
  }
  if (D == 0) {  // a single element: one axis of extent 1 (reported through orig = -1)
    g.ext[0] = 1;
    for (int k = 0; k < n; ++k) g.stride[k][0] = 0;
    g.orig[0] = -1;
    D = 1;
  }
  g.D = D;
  for (int a = 0; a < D; ++a) g.div[a] = make_fastdiv((uint32_t)std::max<int64_t>(1, g.ext[a]));
  g.L = g.ext[D - 1];
  g.rows = 1;
  for (int a = 0; a + 1 < D; ++a) g.rows *= g.ext[a];
  g.rows32 = g.rows < (1ll << 32);
  for (int k = 0; k < n; ++k) g.x[k] = ptrs ? ptrs[k] : nullptr;
  L.empty = total == 0;
  DeviceInfo dev;
  int s = device_info(dev);
  if (s) return s;
  // short rows: a warp per group of 32 rows; long rows: a warp per row
  L.short_rows = g.D >= 2 && g.L < 32 && g.rows32;
  const long long want = L.short_rows ? (g.rows + 32 * kBoxWarps - 1) / (32 * kBoxWarps)
                                      : (g.rows + kBoxWarps - 1) / kBoxWarps;
  L.grid = L.empty ? 1 : (int)std::max(1ll, std::min(want, (long long)dev.sms * 8));
  return TRIOT_OK;
}

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" {

int triot_nonzero_bbox_workspace_size(int rank, int ntensors, const int64_t* const* shapes, int dtype,
                                      size_t* bytes) {
  if (!bytes) return fail(TRIOT_ERR_NULL, "bytes is NULL");
  BoxLaunch L;
  const int st = plan_bbox(rank, ntensors, shapes, dtype, nullptr, L);
  if (st) return st;
  *bytes = (size_t)L.grid * (2 * L.g.D + 1) * sizeof(long long);
  return ok();
}

int triot_nonzero_bbox(int rank, int ntensors, const int64_t* const* shapes, const void* const* tensors,
                       int dtype, int64_t* out, void* workspace, size_t workspace_bytes, void* stream) {
  BoxLaunch L;
  int st = plan_bbox(rank, ntensors, shapes, dtype, tensors, L);
  if (st) return st;
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if (!tensors) return fail(TRIOT_ERR_NULL, "tensors is NULL");
  if (!L.empty)
    for (int k = 0; k < ntensors; ++k)
      if (!tensors[k]) return fail(TRIOT_ERR_NULL, "a tensor pointer is NULL");
  const size_t need = (size_t)L.grid * (2 * L.g.D + 1) * sizeof(long long);
  if (!workspace || workspace_bytes < need) return fail(TRIOT_ERR_WORKSPACE, "workspace is NULL or too small");
  if (reinterpret_cast<uintptr_t>(workspace) % 16) return fail(TRIOT_ERR_WORKSPACE, "workspace is not 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  long long* slots = static_cast<long long*>(workspace);
  int nslots = L.grid;
  cudaError_t e;
  if (L.empty) {
    nslots = 0;
  } else {
    const int es = dtype_size(dtype);
    const void* fn = es == 8 ? pick_bbox<unsigned long long>(ntensors, L.short_rows)
                     : es == 4 ? pick_bbox<unsigned>(ntensors, L.short_rows)
                               : pick_bbox<unsigned short>(ntensors, L.short_rows);
    void* args[] = {(void*)&L.g, (void*)&slots};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(kBoxWarps * 32), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "bounding box kernel launch");
  }
  const long long* cslots = slots;
  void* cargs[] = {(void*)&L.g, (void*)&nslots, (void*)&cslots, (void*)&out};
  e = cudaLaunchKernel(reinterpret_cast<const void*>(&bbox_combine_kernel), dim3(1), dim3(256), cargs, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "bounding box combine launch");
  return ok();
}

}  // extern "C"
