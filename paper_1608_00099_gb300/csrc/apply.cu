// Elementwise apply over three tensors of different shapes (Section 3, benchmark 3):
//   x[t] <- x[t] + y[t] * x[t] - z[t]   for every tuple t of x's shape,
// each tensor addressed with its own shape; y and z contain x's shape.  This is
// Algorithm 9's apply over several tensors with a fixed operation.
//
// The iteration runs over x's canonical shape (unit axes dropped, axes contiguous in all
// three tensors merged).  A CTA takes a tile of whole rows (or one segment of a long row),
// decodes each row's tuple once (Algorithm 4 with magic division) into the rows' offsets in
// y and z (Horner with their strides), and then streams the tile in slots of one 16-byte x
// vector (or one element when x's rows are not whole vectors), two slots per thread in
// flight: x is dense, so its index is the flat index.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {

struct ApplyGeom {
  int nouter;                 // outer axes (innermost first below)
  int rows32;
  FastDiv div[kMaxRank];
  long long ext[kMaxRank];
  long long sy[kMaxRank], sz[kMaxRank];
  long long L;                // row length
  long long syi, szi;         // y and z strides along the row
  long long rows;
  long long rows_per_tile;    // >= 1 whole rows per tile, or 1 with segs > 1
  long long segs;             // segments per row
  long long seg_len;
  long long ntiles;
  FastDiv Ldiv;               // divisor L (rows_per_tile > 1 only; L < 2^31)
  int vec;                    // x elements per 16-byte access (1: element accesses)
};

namespace {

constexpr int kApplyThreads = 256;
constexpr int kApplyTileRows = 512;  // row-table entries per tile (shared memory)

template <typename T> struct Arith;
template <> struct Arith<double> {
  __device__ static double run(double x, double y, double z) {
    return __dsub_rn(__dadd_rn(x, __dmul_rn(y, x)), z);
  }
};
template <> struct Arith<float> {
  __device__ static float run(float x, float y, float z) {
    return __fsub_rn(__fadd_rn(x, __fmul_rn(y, x)), z);
  }
};
template <> struct Arith<__nv_bfloat16> {
  __device__ static __nv_bfloat16 run(__nv_bfloat16 x, __nv_bfloat16 y, __nv_bfloat16 z) {
    const float xf = __bfloat162float(x), yf = __bfloat162float(y), zf = __bfloat162float(z);
    return __float2bfloat16_rn(__fsub_rn(__fadd_rn(xf, __fmul_rn(yf, xf)), zf));
  }
};
template <> struct Arith<__half> {
  __device__ static __half run(__half x, __half y, __half z) {
    const float xf = __half2float(x), yf = __half2float(y), zf = __half2float(z);
    return __float2half_rn(__fsub_rn(__fadd_rn(xf, __fmul_rn(yf, xf)), zf));
  }
};

template <typename T, int V>
__device__ __forceinline__ void apply_slots(const ApplyGeom& g, T* __restrict__ x, const T* __restrict__ y,
                                            const T* __restrict__ z, const long long* s_oy,
                                            const long long* s_oz, long long xbase, long long col0,
                                            long long nrows, long long E) {
  const long long nslot = E / V;
  auto slot_row = [&](long long sidx, long long& q, long long& c) {
    const long long e = sidx * V;
    if (nrows > 1) {
      uint32_t cc;
      q = fdivmod((uint32_t)e, g.Ldiv, cc);
      c = cc;
    } else {
      q = 0;
      c = e;
    }
  };
  auto load_slot = [&](long long sidx, long long q, long long c, T (&xv)[V], T (&yv)[V], T (&zv)[V]) {
    const long long xi = xbase + sidx * V;
    const long long oy = s_oy[q] + (col0 + c) * g.syi, oz = s_oz[q] + (col0 + c) * g.szi;
    if constexpr (V > 1) {
      const uint4 w = __ldcs(reinterpret_cast<const uint4*>(x + xi));
      memcpy(xv, &w, 16);
    } else {
      xv[0] = x[xi];
    }
#pragma unroll
    for (int i = 0; i < V; ++i) {
      yv[i] = __ldg(y + oy + i * g.syi);
      zv[i] = __ldg(z + oz + i * g.szi);
    }
  };
  auto store_slot = [&](long long sidx, T (&xv)[V], const T (&yv)[V], const T (&zv)[V]) {
#pragma unroll
    for (int i = 0; i < V; ++i) xv[i] = Arith<T>::run(xv[i], yv[i], zv[i]);
    const long long xi = xbase + sidx * V;
    if constexpr (V > 1) {
      uint4 w;
      memcpy(&w, xv, 16);
      __stcs(reinterpret_cast<uint4*>(x + xi), w);
    } else {
      x[xi] = xv[0];
    }
  };
  for (long long s0 = threadIdx.x; s0 < nslot; s0 += 2 * (long long)blockDim.x) {
    const long long s1 = s0 + blockDim.x;
    const bool two = s1 < nslot;
    long long q0, c0, q1 = 0, c1 = 0;
    slot_row(s0, q0, c0);
    if (two) slot_row(s1, q1, c1);
    T xa[V], ya[V], za[V], xb[V], yb[V], zb[V];
    load_slot(s0, q0, c0, xa, ya, za);
    if (two) load_slot(s1, q1, c1, xb, yb, zb);
    store_slot(s0, xa, ya, za);
    if (two) store_slot(s1, xb, yb, zb);
  }
}

template <typename T, int NOUT>
__global__ void __launch_bounds__(kApplyThreads) apply_kernel(const __grid_constant__ ApplyGeom g,
                                                               T* __restrict__ x,
                                                               const T* __restrict__ y,
                                                               const T* __restrict__ z) {
  __shared__ long long s_oy[kApplyTileRows], s_oz[kApplyTileRows];
  for (long long tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
    long long row0, nrows, col0, E;
    if (g.segs > 1) {
      row0 = tile / g.segs;
      col0 = (tile - row0 * g.segs) * g.seg_len;
      nrows = 1;
      E = g.L - col0 < g.seg_len ? g.L - col0 : g.seg_len;
    } else {
      row0 = tile * g.rows_per_tile;
      nrows = g.rows - row0 < g.rows_per_tile ? g.rows - row0 : g.rows_per_tile;
      col0 = 0;
      E = nrows * g.L;
    }
    __syncthreads();  // the previous tile's table is no longer read
    for (long long q = threadIdx.x; q < nrows; q += blockDim.x) {
      const long long r = row0 + q;
      long long oy = 0, oz = 0;
      if (g.rows32) {
        uint32_t rem = (uint32_t)r;
#pragma unroll
        for (int k = 0; k < NOUT; ++k) {
          uint32_t t;
          if (k + 1 < NOUT) {
            const uint32_t qq = fdiv(rem, g.div[k]);
            t = rem - qq * g.div[k].d;
            rem = qq;
          } else {
            t = rem;
          }
          oy += (long long)t * g.sy[k];
          oz += (long long)t * g.sz[k];
        }
      } else {
        long long rem = r;
#pragma unroll
        for (int k = 0; k < NOUT; ++k) {
          long long t;
          if (k + 1 < NOUT) {
            const long long qq = rem / g.ext[k];
            t = rem - qq * g.ext[k];
            rem = qq;
          } else {
            t = rem;
          }
          oy += t * g.sy[k];
          oz += t * g.sz[k];
        }
      }
      s_oy[q] = oy;
      s_oz[q] = oz;
    }
    __syncthreads();
    const long long xbase = row0 * g.L + col0;
    // slots of V consecutive x elements (V = 1, or one 16-byte vector when every row of x
    // is a whole number of aligned vectors); y and z are read element by element.  Two
    // slots per thread are loaded before either is computed, so six loads are in flight.
    if (g.vec > 1)
      apply_slots<T, 16 / sizeof(T)>(g, x, y, z, s_oy, s_oz, xbase, col0, nrows, E);
    else
      apply_slots<T, 1>(g, x, y, z, s_oy, s_oz, xbase, col0, nrows, E);
  }
}

template <typename T, int... N>
const void* pick(int nout, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&apply_kernel<T, N>)...};
  return table[nout];
}

const void* apply_kernel_ptr(int dtype, int nout) {
  if (nout < 0 || nout >= kMaxRank) return nullptr;
  auto seq = std::make_integer_sequence<int, kMaxRank>{};
  switch (dtype) {
    case DT_F64: return pick<double>(nout, seq);
    case DT_F32: return pick<float>(nout, seq);
    case DT_BF16: return pick<__nv_bfloat16>(nout, seq);
    case DT_F16: return pick<__half>(nout, seq);
  }
  return nullptr;
}

bool mul_overflows(int64_t a, int64_t b) { return a != 0 && b > INT64_MAX / a; }

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" int triot_apply(int op, int rank, const int64_t* xshape, void* x, const int64_t* yshape,
                           const void* y, const int64_t* zshape, const void* z, int dtype,
                           void* stream) {
  char buf[256];
  if (op != TRIOT_APPLY_XPYXMZ) return fail(TRIOT_ERR_ARG, "unknown apply operation");
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    return fail(TRIOT_ERR_RANK, buf);
  }
  if (!xshape || !yshape || !zshape) return fail(TRIOT_ERR_NULL, "a shape pointer is NULL");
  int64_t nx = 1, ny = 1, nz = 1;
  for (int i = 0; i < rank; ++i) {
    if (xshape[i] < 0 || yshape[i] < 0 || zshape[i] < 0) {
      snprintf(buf, sizeof buf, "negative extent on axis %d", i);
      return fail(TRIOT_ERR_SHAPE, buf);
    }
    if (xshape[i] > yshape[i] || xshape[i] > zshape[i]) {
      snprintf(buf, sizeof buf, "x extent %lld exceeds y or z on axis %d", (long long)xshape[i], i);
      return fail(TRIOT_ERR_SHAPE, buf);
    }
    if (mul_overflows(nx, xshape[i]) || mul_overflows(ny, yshape[i]) || mul_overflows(nz, zshape[i]))
      return fail(TRIOT_ERR_SHAPE, "element count overflows int64");
    nx *= xshape[i];
    ny *= yshape[i];
    nz *= zshape[i];
  }
  if (nx == 0) return ok();
  if (!x || !y || !z) return fail(TRIOT_ERR_NULL, "a tensor pointer is NULL");
  const int es = dtype_size(dtype);
  if (overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es) || overlaps_bytes(x, size_t(nx) * es, z, size_t(nz) * es))
    return fail(TRIOT_ERR_ALIAS, "x overlaps y or z");
  // canonical form over x's shape: unit axes dropped, axes contiguous in all three merged
  int64_t sx[kMaxRank], sy[kMaxRank], sz[kMaxRank];
  {
    int64_t a = 1, b = 1, c = 1;
    for (int i = rank - 1; i >= 0; --i) {
      sx[i] = a; sy[i] = b; sz[i] = c;
      a *= std::max<int64_t>(1, xshape[i]);
      b *= std::max<int64_t>(1, yshape[i]);
      c *= std::max<int64_t>(1, zshape[i]);
    }
  }
  int64_t ext[kMaxRank], cy[kMaxRank], cz[kMaxRank], cx[kMaxRank];
  int D = 0;
  for (int i = 0; i < rank; ++i) {
    if (xshape[i] == 1) continue;
    if (D > 0) {
      const int j = D - 1;
      if (cx[j] == sx[i] * xshape[i] && cy[j] == sy[i] * xshape[i] && cz[j] == sz[i] * xshape[i] &&
          !mul_overflows(ext[j], xshape[i])) {
        ext[j] *= xshape[i];
        cx[j] = sx[i];
        cy[j] = sy[i];
        cz[j] = sz[i];
        continue;
      }
    }
    ext[D] = xshape[i];
    cx[D] = sx[i];
    cy[D] = sy[i];
    cz[D] = sz[i];
    ++D;
  }
  if (D == 0) {
    ext[0] = 1;
    cx[0] = cy[0] = cz[0] = 1;
    D = 1;
  }
  ApplyGeom g = ApplyGeom();
  g.nouter = D - 1;
  g.L = ext[D - 1];
  g.syi = cy[D - 1];
  g.szi = cz[D - 1];
  g.rows = nx / g.L;
  for (int k = 0; k < g.nouter; ++k) {
    const int a = D - 2 - k;
    g.ext[k] = ext[a];
    g.sy[k] = cy[a];
    g.sz[k] = cz[a];
    g.div[k] = make_fastdiv(ext[a] < 0xFFFFFFFFll ? (uint32_t)ext[a] : 1u);
  }
  g.rows32 = g.rows <= 0xFFFFFFFFll;
  DeviceInfo dev;
  int st = device_info(dev);
  if (st) return st;
  // x vectors when every row of x is a whole number of aligned 16-byte vectors
  const int vw = 16 / es;
  g.vec = ((reinterpret_cast<uintptr_t>(x) % 16) == 0 && g.L % vw == 0) ? vw : 1;
  // tiles of up to 8192 elements, smaller for small problems so that every SM gets four
  long long target = 8192;
  target = std::max<long long>(256, std::min(target, (nx + 4ll * dev.sms - 1) / (4ll * dev.sms)));
  if (g.L <= target && g.L < (1ll << 31)) {
    g.rows_per_tile = std::max(1ll, std::min<long long>(kApplyTileRows, target / g.L));
    g.segs = 1;
    g.seg_len = g.L;
    g.ntiles = (g.rows + g.rows_per_tile - 1) / g.rows_per_tile;
    g.Ldiv = make_fastdiv((uint32_t)g.L);
    if (g.rows_per_tile * g.L >= (1ll << 32)) return fail(TRIOT_ERR_ARG, "internal: tile too large");
  } else {
    g.rows_per_tile = 1;
    g.seg_len = (target + g.vec - 1) / g.vec * g.vec;  // segments start on a vector
    g.segs = (g.L + g.seg_len - 1) / g.seg_len;
    g.ntiles = g.rows * g.segs;
  }
  const void* fn = apply_kernel_ptr(dtype, g.nouter);
  if (!fn) return fail(TRIOT_ERR_RANK, "no kernel for this effective rank");
  const long long grid = std::max(1ll, std::min<long long>(g.ntiles, (long long)dev.sms * 8));
  void* args[] = {(void*)&g, (void*)&x, (void*)&y, (void*)&z};
  cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kApplyThreads), args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "apply kernel launch");
  return ok();
}
