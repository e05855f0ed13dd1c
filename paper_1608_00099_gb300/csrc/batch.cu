// Batched pipeline: thousands of independent (x, y) pairs of uneven rank and shape, each
// embedded (x into a zero-padded y), multiplied (y[t] *= x[t] over x's shape) and reduced
// to its tuple-weighted moment, in one persistent launch driven by a device work list
// and replayed from a CUDA graph.  Section 4 suggests partitioning independent work
// across processors with per-processor pre-results combined afterwards; here a tile of a
// pair is the unit of work and each tile writes its moment pre-result to a fixed slot.
//
// Fused mode: a tile reads x once and writes y once.  The value written is
// x[t] * x[t] inside x's shape and +0 outside, which is exactly embed followed by the
// in-place product (the product of a tile reads only what that tile wrote), and the
// tile's moment pre-result is accumulated from the same registers.
// Phased mode: the same kernel runs three times (embed, product, moment) for comparison.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/triot.h"
#include "internal.h"
#include "fixed.cuh"
#include "rows.cuh"

namespace triot {

constexpr int kWarpRows = 256;         // rows one warp tile decodes (warp-private table)
constexpr int kBatchWarps = 8;         // warps per CTA
constexpr int kBatchThreads = 32 * kBatchWarps;

enum { BM_FUSED = 0, BM_EMBED = 1, BM_PRODUCT = 2, BM_MOMENT = 3 };

struct PairDev {
  int D;                          // rank
  int rows_per_tile;              // rows per warp tile (multi-row tiles)
  int packed;                     // the outer digits of a row fit one 64-bit word
  int pad_;
  long long rows;                 // rows of y (product of its outer extents)
  long long inner;                // y's inner extent
  long long xinner;               // x's inner extent
  long long segs;                 // segments per row (>= 1)
  long long seg_len;
  long long tile_begin;           // first global tile of the pair
  long long ntiles;
  const void* x;
  void* y;
  double* out;
  FastDiv div[kMaxRank];          // y's outer extents, innermost first
  FastDiv inner_div;
  long long xstride[kMaxRank];    // x's strides for the outer axes, innermost first
  unsigned xext[kMaxRank];        // x's outer extents, innermost first
  unsigned char dshift[kMaxRank]; // bit offset of outer digit k in the packed word
  unsigned char dbits[kMaxRank];  // bits of outer digit k
  // x-driven tiles (rows of x) for the fused, embed and product passes
  int xrows_per_tile;
  int pad2_;
  long long xrows;                // rows of x (product of its outer extents)
  long long xsegs;                // segments per x row (>= 1)
  long long xseg_len;
  long long xtile_begin;          // first global x tile of the pair
  long long xntiles;
  FastDiv xdiv[kMaxRank];         // x's outer extents, innermost first
  long long ystride[kMaxRank];    // y's strides for the outer axes, innermost first
  // zero-fill tiles of y
  long long ny;                   // elements of y
  long long fill_begin;
  long long fill_ntiles;
};

constexpr long long kFillTileBytes = 16384;

__device__ int g_triot_device_flag = 0;

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type to_acc(T v) { return (typename AccOf<T>::type)v; }
template <>
__device__ __forceinline__ float to_acc<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_acc<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T zero_of() { return T(0); }
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() { return __ushort_as_bfloat16(0); }
template <> __device__ __forceinline__ __half zero_of<__half>() { return __ushort_as_half(0); }

// Persistent warps; warp w owns the contiguous tile range [T w / W, T (w+1) / W).  A warp
// tile is up to kWarpRows whole rows of one pair's y (or one segment of a long row).  No
// CTA-wide synchronisation.  Phase A, one lane per row: decode the row's tuple (Alg 4 with
// magic division), its x offset, and -- for the moment -- the row's mass and inner-index
// weighted mass, which are pushed onto the outer axes with the row's digits (so the
// per-element work carries no tuple arithmetic).  Phase B, lanes over elements: coalesced
// writes of y.  Moment pre-results are kept in registers while consecutive tiles belong
// to the same pair and written once per run to the run's first tile slot (the run's other
// slots get zeros), so the per-pair combine reads a dense slot range.
template <typename T, int MAXD>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(
    const PairDev* __restrict__ pairs, const int* __restrict__ tile_pair, long long ntiles,
    int npairs, int mode, double* __restrict__ slots) {
  using Acc = typename AccOf<T>::type;
  constexpr int NV = MAXD + 1;  // moment slots: up to MAXD axes + the mass
  __shared__ __align__(16) PairDev s_pd[kBatchWarps];
  __shared__ long long s_xoff[kBatchWarps][kWarpRows];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBatchWarps + warp;
  const long long tw = (long long)gridDim.x * kBatchWarps;
  const long long t_begin = ntiles * gw / tw, t_end = ntiles * (gw + 1) / tw;
  PairDev& pd = s_pd[warp];
  long long* xoff = s_xoff[warp];
  const bool do_moment = (mode == BM_FUSED || mode == BM_MOMENT);
  int cur = -1;
  long long run_first = -1;  // first tile of the current run of one pair
  int D = 1, nout = 0;
  Acc acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = Acc(0);

  // reduce the run's pre-result over the warp and store it (axis order, mass at index D)
  auto flush_run = [&]() {
    if (!do_moment || run_first < 0) return;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      Acc v = acc[i];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      int axis;
      if (i == MAXD) axis = D;
      else if (i == MAXD - 1) axis = D - 1;
      else axis = (i < nout) ? D - 2 - i : -1;
      if (lane == 0 && axis >= 0) slots[run_first * NV + axis] = (double)v;
      acc[i] = Acc(0);
    }
  };

  for (long long tile = t_begin; tile < t_end; ++tile) {
    const int pi = tile_pair[tile];
    if (pi < 0 || pi >= npairs) {  // corrupted work list: flag it and skip the tile
      if (lane == 0) atomicExch(&g_triot_device_flag, 1);
      continue;
    }
    if (pi != cur) {
      flush_run();
      __syncwarp();
      const int* src = reinterpret_cast<const int*>(pairs + pi);
      int* dst = reinterpret_cast<int*>(&pd);
      for (int w = lane; w < int(sizeof(PairDev) / sizeof(int)); w += 32) dst[w] = src[w];
      __syncwarp();
      cur = pi;
      run_first = tile;
      D = pd.D;
      nout = D - 1;
    } else if (do_moment && lane <= D) {
      slots[tile * NV + lane] = 0.0;  // folded into the run's first slot
    }
    const long long lt = tile - pd.tile_begin;
    const long long inner = pd.inner, xinner = pd.xinner;
    const T* __restrict__ X = static_cast<const T*>(pd.x);
    T* __restrict__ Y = static_cast<T*>(pd.y);
    const bool multi = pd.segs == 1;
    long long row0, nrows, col0, E;
    if (multi) {
      row0 = lt * pd.rows_per_tile;
      nrows = pd.rows - row0 < pd.rows_per_tile ? pd.rows - row0 : pd.rows_per_tile;
      col0 = 0;
      E = nrows * inner;
    } else {
      row0 = lt / pd.segs;
      col0 = (lt - row0 * pd.segs) * pd.seg_len;
      nrows = 1;
      E = inner - col0 < pd.seg_len ? inner - col0 : pd.seg_len;
    }
    // ---- phase A: one lane per row
    unsigned dgt[MAXD];  // digits of this lane's last decoded row (segment tiles: row0)
    for (int q = lane; q < nrows; q += 32) {
      uint32_t rem = (uint32_t)(row0 + q);
      long long xo = 0;
      bool inside = true;
#pragma unroll
      for (int k = 0; k < MAXD; ++k) {
        dgt[k] = 0;
        if (k < nout) {
          uint32_t t;
          if (k + 1 < nout) {
            const uint32_t qq = fdiv(rem, pd.div[k]);
            t = rem - qq * pd.div[k].d;
            rem = qq;
          } else {
            t = rem;
          }
          dgt[k] = t;
          xo += (long long)t * pd.xstride[k];
          inside = inside && (t < pd.xext[k]);
        }
      }
      xoff[q] = inside ? xo : -1;
      if (do_moment && multi) {
        // the row's mass and inner-weighted mass (FUSED: x^2 over x's row; MOMENT: y's row)
        Acc m = Acc(0), w = Acc(0), cf = Acc(0);
        if (mode == BM_FUSED) {
          if (inside) {
            for (long long c = 0; c < xinner; ++c) {
              const T xv = X[xo + c];
              const Acc v = to_acc<T>(mul_rn(xv, xv));
              m += v;
              w += cf * v;
              cf += Acc(1);
            }
          }
        } else {
          const T* yr = Y + (row0 + q) * inner;
          for (long long c = 0; c < inner; ++c) {
            const Acc v = to_acc<T>(yr[c]);
            m += v;
            w += cf * v;
            cf += Acc(1);
          }
        }
        if (m != Acc(0) || w != Acc(0)) {
#pragma unroll
          for (int k = 0; k < MAXD; ++k)
            if (k < nout) acc[k] += (Acc)dgt[k] * m;  // axis D-2-k
          acc[MAXD - 1] += w;
          acc[MAXD] += m;
        }
      }
    }
    __syncwarp();
    // ---- phase B: lanes over elements (coalesced)
    const long long ybase = row0 * inner + col0;
    Acc sm = Acc(0), sw = Acc(0);                  // segment tiles: moment per element
    Acc cf = (Acc)(col0 + lane);
    for (long long e = lane; e < E; e += 32, cf += Acc(32)) {
      long long q, c;
      if (multi) {
        uint32_t cc;
        q = fdivmod((uint32_t)e, pd.inner_div, cc);
        c = cc;
      } else {
        q = 0;
        c = col0 + e;
      }
      const long long xo = xoff[q];
      const bool inside = xo >= 0 && c < xinner;
      if (mode == BM_FUSED) {
        T o = zero_of<T>();
        if (inside) {
          const T xv = X[xo + c];
          o = mul_rn(xv, xv);
        }
        Y[ybase + e] = o;
        if (!multi) { const Acc v = to_acc<T>(o); sm += v; sw += cf * v; }
      } else if (mode == BM_EMBED) {
        Y[ybase + e] = inside ? X[xo + c] : zero_of<T>();
      } else if (mode == BM_PRODUCT) {
        if (inside) Y[ybase + e] = mul_rn(Y[ybase + e], X[xo + c]);
      } else if (!multi) {
        const Acc v = to_acc<T>(Y[ybase + e]);
        sm += v;
        sw += cf * v;
      }
    }
    if (do_moment && !multi) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        sm += __shfl_xor_sync(0xffffffffu, sm, off);
        sw += __shfl_xor_sync(0xffffffffu, sw, off);
      }
      if (lane == 0) {  // lane 0 decoded the segment's row in phase A
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nout) acc[k] += (Acc)dgt[k] * sm;
        acc[MAXD - 1] += sw;
        acc[MAXD] += sm;
      }
    }
    __syncwarp();
  }
  flush_run();
}

// Zero fill of every pair's y (the pad of the embed): a tile is 16 KB of one y buffer,
// written with 128-bit stores where the buffer is 16-byte aligned.
__global__ void __launch_bounds__(256) batch_fill_kernel(const PairDev* __restrict__ pairs,
                                                         const int* __restrict__ fill_pair,
                                                         long long ntiles, int npairs, int es) {
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pi = fill_pair[tile];
    if (pi < 0 || pi >= npairs) {
      if (threadIdx.x == 0) atomicExch(&g_triot_device_flag, 1);
      continue;
    }
    const PairDev* pd = pairs + pi;
    unsigned char* y = static_cast<unsigned char*>(pd->y);
    const long long bytes = pd->ny * es;
    const long long b0 = (tile - pd->fill_begin) * kFillTileBytes;
    const long long b1 = b0 + kFillTileBytes < bytes ? b0 + kFillTileBytes : bytes;
    long long tail = b0;
    if ((reinterpret_cast<uintptr_t>(y) & 15) == 0) {
      const long long v1 = b1 / 16;
      uint4* yv = reinterpret_cast<uint4*>(y);
      for (long long v = b0 / 16 + threadIdx.x; v < v1; v += blockDim.x) yv[v] = make_uint4(0u, 0u, 0u, 0u);
      tail = v1 * 16 > b0 ? v1 * 16 : b0;
    }
    for (long long b = tail + (long long)threadIdx.x * es; b < b1; b += (long long)blockDim.x * es) {
      if (es == 8) *reinterpret_cast<unsigned long long*>(y + b) = 0ull;
      else if (es == 4) *reinterpret_cast<unsigned*>(y + b) = 0u;
      else *reinterpret_cast<unsigned short*>(y + b) = (unsigned short)0;
    }
  }
}

// x-driven pass over the rows of x (x rows map one to one onto the inside rows of y).
// One lane per x row: decode the row's tuple, read the contiguous x row, write its image
// into y (fused: x*x, the embed followed by the product; embed: x; product: y*x) and, in
// the fused pass, accumulate the row's mass and inner-weighted mass, pushed onto the outer
// axes with the row's digits.  Rows longer than a tile are split into segments that the
// whole warp streams.
template <typename T, int MAXD>
__global__ void __launch_bounds__(kBatchThreads) batch_x_kernel(
    const PairDev* __restrict__ pairs, const int* __restrict__ xtile_pair, long long ntiles,
    int npairs, int mode, double* __restrict__ slots) {
  using Acc = typename AccOf<T>::type;
  constexpr int NV = MAXD + 1;
  __shared__ __align__(16) PairDev s_pd[kBatchWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBatchWarps + warp;
  const long long tw = (long long)gridDim.x * kBatchWarps;
  const long long t_begin = ntiles * gw / tw, t_end = ntiles * (gw + 1) / tw;
  PairDev& pd = s_pd[warp];
  const bool do_moment = (mode == BM_FUSED);
  int cur = -1;
  long long run_first = -1;
  int D = 1, nout = 0;
  Acc acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) acc[i] = Acc(0);
  // pair constants, copied to registers at each pair change
  const T* X = nullptr;
  T* Y = nullptr;
  long long xinner = 0, xrows = 0, xsegs = 1, xseg_len = 0, xtb = 0;
  int xrpt = 1;

  auto flush_run = [&]() {
    if (!do_moment || run_first < 0) return;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      Acc v = acc[i];
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      int axis;
      if (i == MAXD) axis = D;
      else if (i == MAXD - 1) axis = D - 1;
      else axis = (i < nout) ? D - 2 - i : -1;
      if (lane == 0 && axis >= 0) slots[run_first * NV + axis] = (double)v;
      acc[i] = Acc(0);
    }
  };
  // tuple digits (innermost first), y offset of an x row
  auto decode = [&](long long r, unsigned (&dg)[MAXD]) -> long long {
    uint32_t rem = (uint32_t)r;
    long long yo = 0;
#pragma unroll
    for (int k = 0; k < MAXD; ++k) {
      dg[k] = 0;
      if (k < nout) {
        uint32_t t;
        if (k + 1 < nout) {
          const uint32_t qq = fdiv(rem, pd.xdiv[k]);
          t = rem - qq * pd.xdiv[k].d;
          rem = qq;
        } else {
          t = rem;
        }
        dg[k] = t;
        yo += (long long)t * pd.ystride[k];
      }
    }
    return yo;
  };

  for (long long tile = t_begin; tile < t_end; ++tile) {
    const int pi = xtile_pair[tile];
    if (pi < 0 || pi >= npairs) {
      if (lane == 0) atomicExch(&g_triot_device_flag, 1);
      continue;
    }
    if (pi != cur) {
      flush_run();
      __syncwarp();
      const int* src = reinterpret_cast<const int*>(pairs + pi);
      int* dst = reinterpret_cast<int*>(&pd);
      for (int w = lane; w < int(sizeof(PairDev) / sizeof(int)); w += 32) dst[w] = src[w];
      __syncwarp();
      cur = pi;
      run_first = tile;
      D = pd.D;
      nout = D - 1;
      X = static_cast<const T*>(pd.x);
      Y = static_cast<T*>(pd.y);
      xinner = pd.xinner;
      xrows = pd.xrows;
      xsegs = pd.xsegs;
      xseg_len = pd.xseg_len;
      xtb = pd.xtile_begin;
      xrpt = pd.xrows_per_tile;
    } else if (do_moment && lane <= D) {
      slots[tile * NV + lane] = 0.0;  // folded into the run's first slot
    }
    const long long lt = tile - xtb;
    unsigned dg[MAXD];
    if (xsegs == 1) {
      const long long row0 = lt * xrpt;
      const long long nrows = xrows - row0 < xrpt ? xrows - row0 : xrpt;
      for (long long q = lane; q < nrows; q += 32) {
        const long long r = row0 + q;
        const long long yo = decode(r, dg);
        const T* xr = X + r * xinner;
        T* yr = Y + yo;
        Acc m = Acc(0), w = Acc(0), cf = Acc(0);
        for (long long c = 0; c < xinner; ++c) {
          const T xv = xr[c];
          if (mode == BM_FUSED) {
            const T o = mul_rn(xv, xv);
            yr[c] = o;
            const Acc v = to_acc<T>(o);
            m += v;
            w += cf * v;
            cf += Acc(1);
          } else if (mode == BM_EMBED) {
            yr[c] = xv;
          } else {
            yr[c] = mul_rn(yr[c], xv);
          }
        }
        if (do_moment) {
#pragma unroll
          for (int k = 0; k < MAXD; ++k)
            if (k < nout) acc[k] += (Acc)dg[k] * m;  // axis D-2-k
          acc[MAXD - 1] += w;
          acc[MAXD] += m;
        }
      }
    } else {
      // one segment of a long x row, streamed by the whole warp
      const long long r = lt / xsegs;
      const long long col0 = (lt - r * xsegs) * xseg_len;
      const long long n = xinner - col0 < xseg_len ? xinner - col0 : xseg_len;
      const long long yo = decode(r, dg);
      const T* xr = X + r * xinner + col0;
      T* yr = Y + yo + col0;
      Acc m = Acc(0), w = Acc(0), cf = (Acc)(col0 + lane);
      for (long long c = lane; c < n; c += 32, cf += Acc(32)) {
        const T xv = xr[c];
        if (mode == BM_FUSED) {
          const T o = mul_rn(xv, xv);
          yr[c] = o;
          const Acc v = to_acc<T>(o);
          m += v;
          w += cf * v;
        } else if (mode == BM_EMBED) {
          yr[c] = xv;
        } else {
          yr[c] = mul_rn(yr[c], xv);
        }
      }
      if (do_moment) {
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
          m += __shfl_xor_sync(0xffffffffu, m, off);
          w += __shfl_xor_sync(0xffffffffu, w, off);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < MAXD; ++k)
            if (k < nout) acc[k] += (Acc)dg[k] * m;
          acc[MAXD - 1] += w;
          acc[MAXD] += m;
        }
      }
    }
    __syncwarp();
  }
  flush_run();
}

// Exact per-pair combine of the tiles' moment pre-results (as combine_kernel, per pair).
template <int MAXD>
__global__ void __launch_bounds__(256) batch_combine_kernel(const PairDev* __restrict__ pairs,
                                                            const double* __restrict__ slots,
                                                            int xtiles) {
  constexpr int NV = MAXD + 1;
  const PairDev& pd = pairs[blockIdx.x];
  const long long tb = xtiles ? pd.xtile_begin : pd.tile_begin;
  const long long nt = xtiles ? pd.xntiles : pd.ntiles;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int comp = warp; comp <= pd.D; comp += blockDim.x / 32) {
    unsigned emax = 0;
    int bad = 0;
    for (long long k = lane; k < nt; k += 32) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(slots[(tb + k) * NV + comp]);
      const unsigned e = (unsigned)((b >> 52) & 0x7FF);
      if (e == 0x7FF) bad = 1;
      else emax = e > emax ? e : emax;
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    double result;
    if (bad) {
      double acc = 0.0;
      if (lane == 0)
        for (long long k = 0; k < nt; ++k) acc += slots[(tb + k) * NV + comp];
      result = acc;
    } else {
      const int E = emax ? (int)emax : 1;
      __int128 acc = 0;
      for (long long k = lane; k < nt; k += 32) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(slots[(tb + k) * NV + comp]);
        const int e = (int)((b >> 52) & 0x7FF);
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
        const __int128 v = scale_shift((__int128)m, 56 - (E - (e ? e : 1)));
        acc += (b >> 63) ? -v : v;
      }
      unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)((unsigned __int128)acc >> 64);
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
        const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
        const unsigned __int128 sum = (((unsigned __int128)hi << 64) | lo) + (((unsigned __int128)ohi << 64) | olo);
        lo = (unsigned long long)sum;
        hi = (unsigned long long)(sum >> 64);
      }
      const __int128 tot = (__int128)(((unsigned __int128)hi << 64) | lo);
      result = (emax == 0 && tot == 0) ? 0.0 : ldexp(i128_to_double(tot), E - 1075 - 56);
    }
    if (lane == 0) pd.out[comp] = result;
  }
}

// ====================================================================== host side

struct triot_plan_impl {
  int dtype = 0, mode = 0, maxd = 0, npairs = 0;
  long long ntiles = 0, nxtiles = 0, nfill = 0;
  int grid = 0, xgrid = 0, fgrid = 0;
  std::vector<triot_batch_desc> descs;     // host copy for the plain per-pair launches
  PairDev* d_pairs = nullptr;
  int* d_tile_pair = nullptr;              // y-row tiles (phased moment)
  int* d_xtile_pair = nullptr;             // x-row tiles (fused, embed, product)
  int* d_fill_pair = nullptr;              // zero-fill tiles
  double* d_slots = nullptr;
  void* d_ws = nullptr;                    // moment workspace of the plain launches
  size_t ws_bytes = 0;
  size_t dev_bytes = 0;
  int tile_elems = 0, ctas_per_sm = 0;     // geometry in force
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace {

template <typename T, int... M>
const void* batch_ptr_t(int maxd) {
  switch (maxd) {
    case 4: return reinterpret_cast<const void*>(&batch_kernel<T, 4>);
    case 8: return reinterpret_cast<const void*>(&batch_kernel<T, 8>);
    case 12: return reinterpret_cast<const void*>(&batch_kernel<T, 12>);
    case 16: return reinterpret_cast<const void*>(&batch_kernel<T, 16>);
    default: return reinterpret_cast<const void*>(&batch_kernel<T, 24>);
  }
}

const void* batch_ptr(int dtype, int maxd) {
  switch (dtype) {
    case DT_F64: return batch_ptr_t<double>(maxd);
    case DT_F32: return batch_ptr_t<float>(maxd);
    case DT_BF16: return batch_ptr_t<__nv_bfloat16>(maxd);
    default: return batch_ptr_t<__half>(maxd);
  }
}

template <typename T>
const void* batch_x_ptr_t(int maxd) {
  switch (maxd) {
    case 4: return reinterpret_cast<const void*>(&batch_x_kernel<T, 4>);
    case 8: return reinterpret_cast<const void*>(&batch_x_kernel<T, 8>);
    case 12: return reinterpret_cast<const void*>(&batch_x_kernel<T, 12>);
    case 16: return reinterpret_cast<const void*>(&batch_x_kernel<T, 16>);
    default: return reinterpret_cast<const void*>(&batch_x_kernel<T, 24>);
  }
}

const void* batch_x_ptr(int dtype, int maxd) {
  switch (dtype) {
    case DT_F64: return batch_x_ptr_t<double>(maxd);
    case DT_F32: return batch_x_ptr_t<float>(maxd);
    case DT_BF16: return batch_x_ptr_t<__nv_bfloat16>(maxd);
    default: return batch_x_ptr_t<__half>(maxd);
  }
}

const void* combine_ptr(int maxd) {
  switch (maxd) {
    case 4: return reinterpret_cast<const void*>(&batch_combine_kernel<4>);
    case 8: return reinterpret_cast<const void*>(&batch_combine_kernel<8>);
    case 12: return reinterpret_cast<const void*>(&batch_combine_kernel<12>);
    case 16: return reinterpret_cast<const void*>(&batch_combine_kernel<16>);
    default: return reinterpret_cast<const void*>(&batch_combine_kernel<24>);
  }
}

void free_plan(triot_plan_impl* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_pairs) cudaFree(p->d_pairs);
  if (p->d_tile_pair) cudaFree(p->d_tile_pair);
  if (p->d_xtile_pair) cudaFree(p->d_xtile_pair);
  if (p->d_fill_pair) cudaFree(p->d_fill_pair);
  if (p->d_slots) cudaFree(p->d_slots);
  if (p->d_ws) cudaFree(p->d_ws);
  delete p;
}

int enqueue(triot_plan_impl* p, cudaStream_t s) {
  cudaError_t e;
  // 1. zero fill of every y (the pad)
  int es = dtype_size(p->dtype);
  void* fargs[] = {(void*)&p->d_pairs, (void*)&p->d_fill_pair, (void*)&p->nfill, (void*)&p->npairs, (void*)&es};
  e = cudaLaunchKernel(reinterpret_cast<const void*>(&batch_fill_kernel), dim3(p->fgrid), dim3(256), fargs, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch fill launch");
  // 2. x-driven passes: fused (x*x and the moment) or embed then product
  const void* fx = batch_x_ptr(p->dtype, p->maxd);
  const int xmodes_fused[] = {BM_FUSED};
  const int xmodes_phased[] = {BM_EMBED, BM_PRODUCT};
  const int* xm = p->mode == TRIOT_BATCH_FUSED ? xmodes_fused : xmodes_phased;
  const int nxm = p->mode == TRIOT_BATCH_FUSED ? 1 : 2;
  for (int k = 0; k < nxm; ++k) {
    int mode = xm[k];
    void* args[] = {(void*)&p->d_pairs, (void*)&p->d_xtile_pair, (void*)&p->nxtiles, (void*)&p->npairs,
                    (void*)&mode, (void*)&p->d_slots};
    e = cudaLaunchKernel(fx, dim3(p->xgrid), dim3(kBatchThreads), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch x kernel launch");
  }
  // 3. phased: the moment of y over y's rows
  int xtiles = 1;
  if (p->mode != TRIOT_BATCH_FUSED) {
    int mode = BM_MOMENT;
    void* args[] = {(void*)&p->d_pairs, (void*)&p->d_tile_pair, (void*)&p->ntiles, (void*)&p->npairs,
                    (void*)&mode, (void*)&p->d_slots};
    e = cudaLaunchKernel(batch_ptr(p->dtype, p->maxd), dim3(p->grid), dim3(kBatchThreads), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch moment launch");
    xtiles = 0;
  }
  void* cargs[] = {(void*)&p->d_pairs, (void*)&p->d_slots, (void*)&xtiles};
  e = cudaLaunchKernel(combine_ptr(p->maxd), dim3(p->npairs), dim3(256), cargs, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch combine launch");
  return TRIOT_OK;
}

}  // namespace

void st_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_triot_device_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_triot_device_flag, &zero, sizeof(int));
  *flag = v;
}

}  // namespace triot

using namespace triot;

struct triot_plan : triot_plan_impl {};

extern "C" {

int triot_batch_plan_create(const triot_batch_desc* descs, int n, int dtype, int mode,
                            const triot_tune* tune, triot_plan** out) {
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  *out = nullptr;
  if (!descs || n <= 0) return fail(TRIOT_ERR_ARG, "need at least one descriptor");
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (mode != TRIOT_BATCH_FUSED && mode != TRIOT_BATCH_PHASED) return fail(TRIOT_ERR_ARG, "unknown batch mode");
  if (tune && (tune->tile_elems < 0 || tune->tile_elems > (1 << 20) || tune->ctas_per_sm < 0 ||
               tune->ctas_per_sm > 32))
    return fail(TRIOT_ERR_ARG, "tile_elems or ctas_per_sm out of range");
  const int es = dtype_size(dtype);
  // every descriptor is checked before anything touches the GPU
  for (int i = 0; i < n; ++i) {
    const triot_batch_desc& d = descs[i];
    char buf[160];
    if (d.rank < 1 || d.rank > kMaxRank) {
      snprintf(buf, sizeof buf, "descriptor %d: rank %d outside [1, %d]", i, d.rank, kMaxRank);
      return fail(TRIOT_ERR_RANK, buf);
    }
    long long ny = 1, nx = 1;
    for (int a = 0; a < d.rank; ++a) {
      if (d.xshape[a] < 1 || d.yshape[a] < 1 || d.xshape[a] > d.yshape[a] || d.yshape[a] >= (1ll << 31)) {
        snprintf(buf, sizeof buf, "descriptor %d: axis %d needs 1 <= x extent <= y extent < 2^31", i, a);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      if (ny > (1ll << 40) / d.yshape[a]) {
        snprintf(buf, sizeof buf, "descriptor %d: more than 2^40 elements", i);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      ny *= d.yshape[a];
      nx *= d.xshape[a];
    }
    if (!d.x || !d.y || !d.moment_out) {
      snprintf(buf, sizeof buf, "descriptor %d: NULL pointer", i);
      return fail(TRIOT_ERR_NULL, buf);
    }
    if (overlaps_bytes(d.x, size_t(nx) * es, d.y, size_t(ny) * es)) {
      snprintf(buf, sizeof buf, "descriptor %d: x and y overlap", i);
      return fail(TRIOT_ERR_ALIAS, buf);
    }
  }
  DeviceInfo dev;
  int st = device_info(dev);
  if (st) return st;
  // geometry: the caller's values, else the tuned ones for this batch's key, else defaults
  TuneCfg tuned;
  {
    long long ny_total = 0;
    for (int i = 0; i < n; ++i) {
      long long ny = 1;
      for (int a = 0; a < descs[i].rank; ++a) ny *= descs[i].yshape[a];
      ny_total += ny;
    }
    tuned = tune_lookup_key(batch_key(dtype, mode, n, ny_total));
  }
  const long long target = (tune && tune->tile_elems > 0) ? tune->tile_elems
                           : tuned.tile_elems > 0           ? tuned.tile_elems
                                                            : 1024;
  std::vector<PairDev> host(n);
  std::vector<int> tile_pair, xtile_pair, fill_pair;
  int maxrank = 1;
  long long ntiles = 0, nxtiles = 0, nfill = 0;
  size_t max_ws = 16;
  for (int i = 0; i < n; ++i) {
    const triot_batch_desc& d = descs[i];
    long long ny = 1, nx = 1;
    for (int a = 0; a < d.rank; ++a) {
      ny *= d.yshape[a];
      nx *= d.xshape[a];
    }
    const long long rows = ny / d.yshape[d.rank - 1];
    if (rows > 0xFFFFFFFFll) return fail(TRIOT_ERR_SHAPE, "a pair has more than 2^32 rows");
    PairDev& p = host[i];
    memset(&p, 0, sizeof p);
    p.D = d.rank;
    p.rows = rows;
    p.inner = d.yshape[d.rank - 1];
    p.xinner = d.xshape[d.rank - 1];
    p.x = d.x;
    p.y = d.y;
    p.out = d.moment_out;
    long long xs = p.xinner;
    for (int k = 0; k < d.rank - 1; ++k) {
      const int a = d.rank - 2 - k;
      p.div[k] = make_fastdiv((uint32_t)d.yshape[a]);
      p.xstride[k] = xs;
      p.xext[k] = (unsigned)d.xshape[a];
      xs *= d.xshape[a];
    }
    p.inner_div = make_fastdiv((uint32_t)p.inner);
    {
      int bit = 0;
      for (int k = 0; k < d.rank - 1; ++k) {
        const long long ext = d.yshape[d.rank - 2 - k];
        int b = 1;
        while (b < 32 && (1ll << b) < ext) ++b;
        p.dshift[k] = (unsigned char)(bit < 64 ? bit : 0);
        p.dbits[k] = (unsigned char)b;
        bit += b;
      }
      p.packed = bit <= 64 ? 1 : 0;
    }
    if (p.inner <= target) {
      long long R = std::max(1ll, std::min<long long>(kWarpRows, target / p.inner));
      R = std::min(R, rows);
      p.rows_per_tile = (int)R;
      p.segs = 1;
      p.seg_len = p.inner;
      p.ntiles = (rows + R - 1) / R;
    } else {
      p.rows_per_tile = 1;
      p.segs = (p.inner + target - 1) / target;
      p.seg_len = ((p.inner + p.segs - 1) / p.segs + 31) / 32 * 32;
      p.segs = (p.inner + p.seg_len - 1) / p.seg_len;
      p.ntiles = rows * p.segs;
    }
    p.tile_begin = ntiles;
    ntiles += p.ntiles;
    for (long long t = 0; t < p.ntiles; ++t) tile_pair.push_back(i);
    // zero-fill tiles of y
    p.ny = ny;
    p.fill_begin = nfill;
    p.fill_ntiles = (ny * es + kFillTileBytes - 1) / kFillTileBytes;
    nfill += p.fill_ntiles;
    for (long long t = 0; t < p.fill_ntiles; ++t) fill_pair.push_back(i);
    // x-row tiles
    p.xrows = nx / p.xinner;
    {
      long long ys = p.inner;
      for (int k = 0; k < d.rank - 1; ++k) {
        const int a = d.rank - 2 - k;
        p.xdiv[k] = make_fastdiv((uint32_t)d.xshape[a]);
        p.ystride[k] = ys;
        ys *= d.yshape[a];
      }
    }
    const long long xtarget = target;
    if (p.xinner <= xtarget) {
      long long R = std::max(1ll, std::min(256ll, xtarget / p.xinner));
      R = std::min(R, p.xrows);
      p.xrows_per_tile = (int)R;
      p.xsegs = 1;
      p.xseg_len = p.xinner;
      p.xntiles = (p.xrows + R - 1) / R;
    } else {
      p.xrows_per_tile = 1;
      p.xsegs = (p.xinner + xtarget - 1) / xtarget;
      p.xseg_len = ((p.xinner + p.xsegs - 1) / p.xsegs + 31) / 32 * 32;
      p.xsegs = (p.xinner + p.xseg_len - 1) / p.xseg_len;
      p.xntiles = p.xrows * p.xsegs;
    }
    p.xtile_begin = nxtiles;
    nxtiles += p.xntiles;
    for (long long t = 0; t < p.xntiles; ++t) xtile_pair.push_back(i);
    if (ntiles >= (1ll << 31) || nxtiles >= (1ll << 31) || nfill >= (1ll << 31))
      return fail(TRIOT_ERR_ARG, "batch has more than 2^31 tiles");
    maxrank = std::max(maxrank, d.rank);
    // workspace of the plain per-pair moment launches
    MomentLaunch L;
    st = plan_moment_call(d.rank, d.yshape, dtype, d.y, nullptr, L);
    if (st) return st;
    max_ws = std::max(max_ws, moment_ws_bytes(L));
  }
  const int maxd = maxrank <= 4 ? 4 : maxrank <= 8 ? 8 : maxrank <= 12 ? 12 : maxrank <= 16 ? 16 : 24;
  triot_plan* p = new triot_plan();
  p->dtype = dtype;
  p->mode = mode;
  p->maxd = maxd;
  p->npairs = n;
  p->ntiles = ntiles;
  p->descs.assign(descs, descs + n);
  const int cps = (tune && tune->ctas_per_sm > 0) ? tune->ctas_per_sm
                  : tuned.ctas_per_sm > 0           ? tuned.ctas_per_sm
                                                    : 4;
  p->tile_elems = (int)target;
  p->ctas_per_sm = cps;
  p->nxtiles = nxtiles;
  p->nfill = nfill;
  p->grid = (int)std::max(1ll, std::min<long long>((ntiles + kBatchWarps - 1) / kBatchWarps, (long long)dev.sms * cps));
  p->xgrid = (int)std::max(1ll, std::min<long long>((nxtiles + kBatchWarps - 1) / kBatchWarps, (long long)dev.sms * cps));
  p->fgrid = (int)std::max(1ll, std::min<long long>(nfill, (long long)dev.sms * 8));
  const size_t b_pairs = sizeof(PairDev) * n, b_map = sizeof(int) * ntiles, b_xmap = sizeof(int) * nxtiles,
               b_fmap = sizeof(int) * nfill,
               b_slots = sizeof(double) * (maxd + 1) * std::max(ntiles, nxtiles);
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_pairs, b_pairs)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_tile_pair, b_map)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_xtile_pair, b_xmap)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_fill_pair, b_fmap)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_slots, b_slots)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ws, max_ws)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_pairs, host.data(), b_pairs, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_tile_pair, tile_pair.data(), b_map, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_xtile_pair, xtile_pair.data(), b_xmap, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_fill_pair, fill_pair.data(), b_fmap, cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "batch plan allocation");
  }
  p->ws_bytes = max_ws;
  p->dev_bytes = b_pairs + b_map + b_xmap + b_fmap + b_slots + max_ws;
  *out = p;
  return ok();
}

int triot_batch_run(triot_plan* p, void* stream) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!p->exec) {
    // capture on a private stream (the caller's may be the legacy default stream)
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    int st = enqueue(p, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if ((e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    p->graph = g;
  }
  if ((e = cudaGraphLaunch(p->exec, s)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return ok();
}

int triot_batch_run_plain(triot_plan* p, void* stream) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  for (const triot_batch_desc& d : p->descs) {
    int st = launch_rows(ROW_EMBED, d.rank, d.xshape, d.x, d.yshape, d.y, p->dtype, 0, s, nullptr);
    if (!st) st = launch_rows(ROW_PRODUCT, d.rank, d.xshape, d.x, d.yshape, d.y, p->dtype, 0, s, nullptr);
    if (!st) st = moment_call(d.rank, d.yshape, d.y, p->dtype, d.moment_out, p->d_ws, p->ws_bytes, s, nullptr);
    if (st) return st;
  }
  return ok();
}

int triot_batch_plan_info(const triot_plan* p, size_t* device_bytes, int64_t* tiles) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  if (device_bytes) *device_bytes = p->dev_bytes;
  if (tiles) *tiles = p->ntiles;
  return ok();
}

int triot_batch_plan_geometry(const triot_plan* p, triot_tune* out) {
  if (!p || !out) return fail(TRIOT_ERR_NULL, "plan or out is NULL");
  out->threads = kBatchThreads;
  out->tile_elems = p->tile_elems;
  out->ctas_per_sm = p->ctas_per_sm;
  out->unroll = 0;
  return ok();
}

int triot_batch_plan_destroy(triot_plan* p) {
  free_plan(p);
  return ok();
}

int triot_batch_autotune(const triot_batch_desc* descs, int n, int dtype, int mode, void* stream,
                         triot_tune* best) {
  if (!descs || n <= 0) return fail(TRIOT_ERR_ARG, "need at least one descriptor");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(e, "cudaEventCreate");
  }
  float best_ms = 1e30f;
  triot_tune best_t{0, 0, 0, 0};
  int rc = TRIOT_OK;
  for (int tile : {256, 512, 1024, 2048, 4096}) {
    for (int cps : {2, 4, 8}) {
      triot_tune t{0, tile, cps, 0};
      triot_plan* p = nullptr;
      if ((rc = triot_batch_plan_create(descs, n, dtype, mode, &t, &p))) break;
      // the first run captures the graph; it and one more are warm-up
      for (int w = 0; w < 2 && rc == TRIOT_OK; ++w) rc = triot_batch_run(p, stream);
      std::vector<float> ms;
      for (int r = 0; r < 3 && rc == TRIOT_OK; ++r) {
        cudaEventRecord(a, s);
        rc = triot_batch_run(p, stream);
        cudaEventRecord(b, s);
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) { rc = cuda_fail(e, "batch autotune"); break; }
        float v = 0.f;
        cudaEventElapsedTime(&v, a, b);
        ms.push_back(v);
      }
      triot_batch_plan_destroy(p);
      if (rc) break;
      std::sort(ms.begin(), ms.end());
      if (ms[ms.size() / 2] < best_ms) {
        best_ms = ms[ms.size() / 2];
        best_t = t;
      }
    }
    if (rc) break;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  long long ny_total = 0;
  for (int i = 0; i < n; ++i) {
    long long ny = 1;
    for (int ax = 0; ax < descs[i].rank; ++ax) ny *= descs[i].yshape[ax];
    ny_total += ny;
  }
  TuneCfg tc;
  tc.tile_elems = best_t.tile_elems;
  tc.ctas_per_sm = best_t.ctas_per_sm;
  tune_store_key(batch_key(dtype, mode, n, ny_total), tc);
  if (best) *best = best_t;
  return ok();
}

}  // extern "C"
