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
// innermost) in a strided order; a row's tuple is decoded once (Algorithm 4 with
// magic-number division) into each tensor's row offset, and the lanes test the row's
// elements (coalesced along the innermost axis), each lane keeping the least and greatest
// inner digit and a count.  A row with a counted element (a warp vote) updates the outer
// axes' least and greatest digits with the row's digits.  Shorter rows are streamed in CTA
// tiles of whole rows (bbox_rows_kernel).  Per CTA the warps' boxes are merged (min / max / sum, exact and independent of
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
  long long tile_rows;                    // short rows: rows of a CTA tile (a multiple of rp)
  int rp;                                 // short rows: rows per pass of the CTA's threads
  int slo;                                // short rows: the split decode's first low axis (0: none)
  long long P;                            // product of the extents of axes slo .. D-2
  FastDiv Pdiv;
  FastDiv ldiv;                           // short rows: divisor L
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

// Short rows (fewer than 32 elements): CTA tiles of consecutive rows.  Thread t always takes
// column t mod L of rows t div L, t div L + RP, .. (RP = floor(threads / L) rows per pass),
// so a warp's loads read contiguous stretches of every tensor and no element index is ever
// divided.  Per tile: (1) every row's offsets are decoded once (Algorithm 4 with magic-number
// division) into shared memory; (2) the tile's elements are tested, kBoxU per thread in
// flight, each counted element flagging its row; (3) the flagged rows' digits are decoded
// and the outer axes' least and greatest digits merged with one warp min / max per axis
// (lane a of every warp keeps axis a's running values).  Two buffers of row offsets and
// flags: while a tile streams (2), step (3) of the CTA's previous tile and step (1) of its
// next run between the tile's first loads and their use, so a tile costs one barrier.
constexpr int kBoxU = 4;
constexpr int kBoxTileElems = 4096;  // elements of a short-row tile (at most kBoxTileRows rows)
constexpr int kBoxTileRows = 512;
constexpr int kBoxTableEntries = 1024;  // P * N offsets of the split decode

// resident CTAs per SM the register budget is sized for (the kernel is latency-bound: more
// warps, more loads in flight)
__host__ __device__ constexpr int box_rows_ctas(int n) { return n <= 2 ? 8 : (n == 3 ? 6 : 5); }

template <typename B, int N>
__global__ void __launch_bounds__(kBoxWarps * 32, box_rows_ctas(N))
    bbox_rows_kernel(const __grid_constant__ BoxGeom g, long long* __restrict__ slots) {
  __shared__ unsigned s_lo[kBoxWarps][kMaxRank], s_hi[kBoxWarps][kMaxRank];
  __shared__ unsigned long long s_cnt[kBoxWarps];
  __shared__ long long s_off[2][N][kBoxTileRows];  // two tiles: one streams, the next is decoded
  __shared__ unsigned char s_flag[2][kBoxTileRows];
  __shared__ long long s_tlo[kBoxTableEntries];  // offsets of the innermost outer axes' values
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int D = g.D;     // >= 2 here (a short innermost axis and at least one outer axis)
  const int IN = D - 2;  // the innermost outer axis
  const long long R = g.tile_rows;  // a multiple of RP
  const int RP = g.rp;
  uint32_t col;
  const uint32_t rl = fdivmod((uint32_t)tid, g.ldiv, col);  // first row of this thread in a tile
  const bool lact = (int)rl < RP;                             // threads past RP * L idle
  const B* X[N];
#pragma unroll
  for (int k = 0; k < N; ++k) X[k] = static_cast<const B*>(g.x[k]) + (long long)col * g.stride[k][D - 1];
  unsigned mylo = 0xFFFFFFFFu, myhi = 0u;  // lane a: axis a's least / greatest digit
  unsigned jlo = 0xFFFFFFFFu, jhi = 0u;    // the inner axis
  unsigned long long cnt = 0;
  const long long ntiles = (g.rows + R - 1) / R;
  // offsets over the outer axes a0 .. a1 (a0 <= a1) of the mixed-radix number r
  auto decode = [&](uint32_t r, int a0, int a1, long long (&off)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) off[k] = 0;
    for (int a = a1; a >= a0; --a) {
      uint32_t d = r;
      if (a > a0) {
        const uint32_t q1 = fdiv(r, g.div[a]);
        d = r - q1 * g.div[a].d;
        r = q1;
      }
#pragma unroll
      for (int k = 0; k < N; ++k) off[k] += (long long)d * g.stride[k][a];
    }
  };
  // Row r = h P + p splits into its digits on the outer axes below g.slo (h) and from g.slo
  // (p < P, the innermost outer axes).  With P >= 32 (g.slo > 0) the offsets of every p are a
  // table built once per CTA, and the 32 consecutive rows of a warp span at most two values
  // of h, decoded by lanes 0 and 1 and shared by shuffles; otherwise every row is decoded.
  const bool split = g.slo > 0;
  if (split)
    for (int p = tid; p < (int)g.P; p += nth) {
      long long off[N];
      decode((uint32_t)p, g.slo, IN, off);
#pragma unroll
      for (int k = 0; k < N; ++k) s_tlo[p * N + k] = off[k];
    }
  // step (3) for tile `prev` (flags in buffer b, read and cleared by row q = q0 + tid), then
  // step (1) for tile `next` into buffer b; called by every thread together
  auto merge_and_decode = [&](long long prev, long long next, int b) {
    if (prev >= 0) {
      for (long long q0 = 0; q0 < R; q0 += nth) {  // uniform trip count: the warp votes below
        const long long q = q0 + tid;
        const long long r = prev * R + q;
        const bool f = q < R && r < g.rows && s_flag[b][q];
        if (q < R) s_flag[b][q] = 0;
        if (__any_sync(0xffffffffu, f)) {
          uint32_t rr = f ? (uint32_t)r : 0u;
          for (int a = IN; a >= 0; --a) {
            uint32_t d = rr;
            if (a > 0) {
              const uint32_t q1 = fdiv(rr, g.div[a]);
              d = rr - q1 * g.div[a].d;
              rr = q1;
            }
            const unsigned mn = __reduce_min_sync(0xffffffffu, f ? d : 0xFFFFFFFFu);
            const unsigned mx = __reduce_max_sync(0xffffffffu, f ? d : 0u);
            if (lane == a) {
              mylo = min(mylo, mn);
              myhi = max(myhi, mx);
            }
          }
        }
      }
    }
    if (next >= 0) {
      for (long long q0 = 0; q0 < R; q0 += nth) {  // uniform trip count: the shuffles below
        const long long q = q0 + tid;
        const long long r = next * R + q;
        const bool ok = q < R && r < g.rows;
        long long off[N];
        if (split) {
          // the warp's rows start at rw (lane 0); p of this lane, and whether it is in h0 + 1
          const uint32_t rw = (uint32_t)(next * R + q0 + (tid & ~31));
          uint32_t p0;
          const uint32_t h0 = fdivmod(rw, g.Pdiv, p0);
          uint32_t pl = p0 + (uint32_t)lane;
          const bool second = pl >= (uint32_t)g.P;
          if (second) pl -= (uint32_t)g.P;
          long long ho[N];
#pragma unroll
          for (int k = 0; k < N; ++k) ho[k] = 0;
          if (lane < 2) decode(h0 + (uint32_t)lane, 0, g.slo - 1, ho);
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const long long hA = __shfl_sync(0xffffffffu, ho[k], 0);
            const long long hB = __shfl_sync(0xffffffffu, ho[k], 1);
            off[k] = (second ? hB : hA) + (ok ? s_tlo[pl * N + k] : 0ll);
          }
        } else if (ok) {
          decode((uint32_t)r, 0, IN, off);
        }
        if (ok) {
#pragma unroll
          for (int k = 0; k < N; ++k) s_off[b][k][q] = off[k];
        }
      }
    }
  };
  // tile k streams from buffer k mod 2 while the flags of tile k-1 are merged and tile k+1
  // is decoded into the other buffer, between the first loads of tile k and their use
  long long prev = -1;
  int cb = 0;
  for (int q = tid; q < 2 * kBoxTileRows; q += nth) (&s_flag[0][0])[q] = 0;
  __syncthreads();  // the table of the split decode is complete
  if (blockIdx.x < ntiles) merge_and_decode(-1, blockIdx.x, 0);
  __syncthreads();
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long next = tile + gridDim.x < ntiles ? tile + gridDim.x : -1;
    const int nrows = (int)(g.rows - tile * R < R ? g.rows - tile * R : R);
    for (int q0 = 0; q0 < nrows; q0 += RP * kBoxU) {  // the same trip count in every thread
      B v[kBoxU][N];
#pragma unroll
      for (int u = 0; u < kBoxU; ++u) {
        const int q = q0 + (int)rl + u * RP;
#pragma unroll
        for (int k = 0; k < N; ++k) v[u][k] = (lact && q < nrows) ? __ldg(X[k] + s_off[cb][k][q]) : (B)0;
      }
      if (q0 == 0) merge_and_decode(prev, next, cb ^ 1);
#pragma unroll
      for (int u = 0; u < kBoxU; ++u) {
        const int q = q0 + (int)rl + u * RP;
        bool c = lact && q < nrows;
#pragma unroll
        for (int k = 0; k < N; ++k) c = c & nz_bits(v[u][k]);
        if (c) {
          ++cnt;
          s_flag[cb][q] = 1;
        }
      }
    }
    __syncthreads();
    prev = tile;
    cb ^= 1;
  }
  merge_and_decode(prev, -1, cb ^ 1);
  if (cnt) {  // this thread's column was counted
    jlo = col;
    jhi = col;
  }
  jlo = __reduce_min_sync(0xffffffffu, jlo);
  jhi = __reduce_max_sync(0xffffffffu, jhi);
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane <= IN) {
    s_lo[warp][lane] = mylo;
    s_hi[warp][lane] = myhi;
  }
  if (lane == 0) {
    s_lo[warp][D - 1] = jlo;
    s_hi[warp][D - 1] = jhi;
    s_cnt[warp] = cnt;
  }
  __syncthreads();
  // a warp's axis values may come from rows counted by other warps (the flags are per CTA),
  // so the CTA merges every warp's values whether or not the warp itself counted
  long long* slot = slots + (long long)blockIdx.x * (2 * D + 1);
  unsigned long long ctot = 0;
  for (int w = 0; w < kBoxWarps; ++w) ctot += s_cnt[w];
  if (tid < D) {
    const int a = tid;
    unsigned l = 0xFFFFFFFFu, h = 0u;
    for (int w = 0; w < kBoxWarps; ++w) {
      l = min(l, s_lo[w][a]);
      h = max(h, s_hi[w][a]);
    }
    slot[2 * a] = ctot ? (long long)l : LLONG_MAX;
    slot[2 * a + 1] = ctot ? (long long)h : -1;
  }
  if (tid == 0) slot[2 * D] = (long long)ctot;
}

// merge the CTAs' slots; write [lo_0, hi_0, .., count] in the caller's axis order (axes of
// extent 1 in I: 0 .. 0 when anything counted); nothing counted: lo 0, hi -1 everywhere
constexpr int kBoxCombineWarps = 32;

__global__ void __launch_bounds__(kBoxCombineWarps * 32) bbox_combine_kernel(const __grid_constant__ BoxGeom g, int nslots,
                                                           const long long* __restrict__ slots,
                                                           long long* __restrict__ out) {
  // warp w reads slots w, w + NW, ..; lane c keeps component c (and c + 32) of a slot, whose
  // 2D + 1 values are contiguous: [lo_0, hi_0, .., lo_{D-1}, hi_{D-1}, count]
  constexpr int NW = kBoxCombineWarps;
  __shared__ long long s_part[NW][2 * kMaxRank + 1];
  __shared__ long long s_lo[kMaxRank], s_hi[kMaxRank];
  __shared__ unsigned long long s_cnt;
  const int D = g.D, C = 2 * D + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto init = [&](int c) -> long long { return c == 2 * D ? 0ll : ((c & 1) ? -1ll : LLONG_MAX); };
  auto fold = [&](int c, long long acc, long long v) -> long long {
    return c == 2 * D ? acc + v : ((c & 1) ? max(acc, v) : min(acc, v));
  };
  constexpr int U = 8;  // slots a warp has in flight
  long long a0 = init(lane), a1 = init(lane + 32);
  for (int k0 = warp; k0 < nslots; k0 += NW * U) {
    long long v0[U], v1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + u * NW;
      const long long* sl = slots + (long long)k * C;
      v0[u] = (k < nslots && lane < C) ? sl[lane] : init(lane);
      v1[u] = (k < nslots && lane + 32 < C) ? sl[lane + 32] : init(lane + 32);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      a0 = fold(lane, a0, v0[u]);
      a1 = fold(lane + 32, a1, v1[u]);
    }
  }
  if (lane < C) s_part[warp][lane] = a0;
  if (lane + 32 < C) s_part[warp][lane + 32] = a1;
  __syncthreads();
  if (threadIdx.x < C) {
    const int c = threadIdx.x;
    long long acc = init(c);
    for (int w = 0; w < NW; ++w) acc = fold(c, acc, s_part[w][c]);
    if (c == 2 * D) s_cnt = (unsigned long long)acc;
    else if (c & 1) s_hi[c >> 1] = acc;
    else s_lo[c >> 1] = acc;
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
  L.short_rows = g.D >= 2 && g.L < 32 && g.rows < (1ll << 31);
  g.rp = (int)std::max(1ll, (long long)(kBoxWarps * 32) / std::max(1ll, g.L));
  g.tile_rows = (long long)g.rp * std::max(1, std::min(kBoxTileElems / (g.rp * (int)std::max(1ll, g.L)),
                                                       kBoxTileRows / g.rp));
  g.ldiv = make_fastdiv((uint32_t)std::max(1ll, std::min<long long>(g.L, 1ll << 30)));
  // the split decode: the most innermost outer axes whose P offsets per tensor fit the table
  g.slo = 0;
  g.P = 1;
  if (L.short_rows) {
    long long P = 1;
    int a = g.D - 2;
    while (a >= 0 && P * g.ext[a] * n <= kBoxTableEntries) P *= g.ext[a--];
    if (P >= 32 && a >= 0) {  // at least one axis left above the split
      g.slo = a + 1;
      g.P = P;
    }
  }
  g.Pdiv = make_fastdiv((uint32_t)g.P);
  // short rows: CTA tiles of rows, a few CTAs per SM; long rows: a warp per row
  const long long want = L.short_rows ? (g.rows + g.tile_rows - 1) / g.tile_rows
                                      : (g.rows + kBoxWarps - 1) / kBoxWarps;
  L.grid = L.empty ? 1 : (int)std::max(1ll, std::min(want, (long long)dev.sms * (L.short_rows ? box_rows_ctas(n) : 8)));
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
  e = cudaLaunchKernel(reinterpret_cast<const void*>(&bbox_combine_kernel), dim3(1), dim3(kBoxCombineWarps * 32),
                       cargs, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "bounding box combine launch");
  return ok();
}

}  // extern "C"
