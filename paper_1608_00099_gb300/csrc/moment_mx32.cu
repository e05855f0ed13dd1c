// f32 / bf16 / f16 moment by marginals (Algorithms 10 and 11), accumulated in f32.
//
// The same split as the f64 kernel (moment_mx.cu): row axes 0 .. s-1 and column axes
// s .. D-1 view the tensor as R rows of C contiguous elements; the row axes' moments come
// from the rows' masses and the column axes' moments from the columns' masses.  A warp
// owns one tile of columns and a contiguous range of rows.  When every row starts on a
// 16-byte boundary, lane l reads kMx32J / V vectors of V = 16 / (element size) elements
// per row (vector k covers columns (l + 32k) V .. (l + 32k) V + V - 1 of the tile), else it
// reads kMx32J single elements (columns l + 32j); loads run two rows ahead.  Per element the
// work is one f32 add into its column's sum and one into the row's mass (a tree over the
// lane's elements).  The row's digits are warp-uniform and advance like Algorithm 3: the
// four innermost row axes are credited every row from the row's mass (so that carries past
// them, and the lazy hand-over of pending masses to the axes above, come at most every 16
// rows for any shape), the other row axes at their carries.
//
// Accuracy: every plain f32 sum has at most kMx32Window + J terms (a window of rows, or a
// row's J elements); window results are added into compensated f32 pairs (two-sum), the
// lanes' pairs are added across the warp the same way, and only then does f64 come in (one
// conversion per warp and component, a fixed-order sum per CTA).  So the error stays below
// about (kMx32Window + J + 2) * 2^-24 of sum |p[t]| t_i, the narrow FP64 pipe is barely used,
// and results are identical from run to run.  Non-finite values propagate as in a plain sum;
// finite data whose partial sums exceed the f32 range give inf (an f32-accumulation limit).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "float_moment.cuh"
#include "kernels.h"
#include "mx.cuh"

namespace triot {
namespace {

constexpr int kEager = 4;  // innermost row axes credited every row

// compensated f32 pair h + l
struct CF {
  float h, l;
};
__device__ __forceinline__ void cf_add(CF& a, float v) {  // a += v (Knuth two-sum)
  const float s = a.h + v, bp = s - a.h;
  a.l += (a.h - (s - bp)) + (v - bp);
  a.h = s;
}
__device__ __forceinline__ void cf_add(CF& a, const CF& b) {
  cf_add(a, b.h);
  a.l += b.l;
}
__device__ __forceinline__ void cf_mac(CF& a, const CF& b, uint32_t t) {  // a += b * t
  const float tf = (float)t, p = b.h * tf;
  cf_add(a, p);
  a.l += fmaf(b.h, tf, -p) + b.l * tf;
}

// the lane's cold state (local memory): the row levels above the eager axes, and totals
struct Mx32Cold {
  CF Aa[kMaxRank];         // row axes 0 .. s-1-kEager: sums of mass * digit
  CF Qa[kMaxRank];         // their pending masses (level i: not yet credited to axes <= i)
  uint32_t td[kMaxRank];   // digits of row axes 0 .. s-1-kEager (warp-uniform)
  CF Tot[kMaxRank + 1];    // the lane's totals per component (moments, then the mass)
  CF colsum[kMx32J];       // column sums over the warp's rows
  CF Sc[kEager];           // the eager axes' sums over the warp's rows
};

// Pending mass `pend` of the level below the eager axes (axis L = s-1-kEager): credited to
// every axis the carry changes (with its old digit) and handed to the axis above; with
// carry = false (a window end) it is only credited and handed up, digits unchanged.
__device__ __noinline__ void mx32_cold_step(const MxGeom& g, Mx32Cold& st, CF pend, bool carry) {
  int i = g.s - 1 - kEager;
  bool moving = carry;
  while (i >= 0) {
    CF tot = pend;
    cf_add(tot, st.Qa[i]);
    st.Qa[i] = CF{0.f, 0.f};
    cf_mac(st.Aa[i], tot, st.td[i]);
    pend = tot;
    if (moving) {
      const uint32_t nt = st.td[i] + 1;
      if (i > 0 && nt == (uint32_t)g.ext[i]) {
        st.td[i] = 0;  // wraps: the carry goes on
      } else {
        st.td[i] = nt;
        moving = false;
        // mass still pending for the axes above i
        if (i > 0) {
          cf_add(st.Qa[i - 1], tot);
          return;
        }
      }
    }
    --i;
  }
  cf_add(st.Tot[g.D], pend);  // past axis 0: the mass
}

template <typename T> struct Unpack {
  __device__ static float at(const uint4& v, int i) { return FPiece<T>::get(v, i); }
};

__device__ __forceinline__ uint4 ld_stream16(const void* q) {
  uint4 v;
  asm volatile("ld.global.cs.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(q));
  return v;
}

// column of element j of this lane's row slice
template <int V>
__device__ __forceinline__ long long mx32_col(long long c0, int lane, int j) {
  return V > 1 ? c0 + (long long)(lane + 32 * (j / V)) * V + (j % V) : c0 + lane + 32 * j;
}

// V > 1: vector loads of V elements (kMx32J / V per lane and row); V == 1: single elements
template <typename T, int V>
__global__ void __launch_bounds__(kMx32Warps * 32, kMx32MinCtas) moment_mx32_kernel(
    const __grid_constant__ MxGeom g, const T* __restrict__ p, double* __restrict__ partial) {
  constexpr int J = kMx32J;        // elements per lane and row
  constexpr int NV = J / V;        // loads per lane and row
  constexpr int NW = kMx32Warps;
  constexpr int TW = 32 * J;       // columns of the tile
  __shared__ CF s_col[NW][TW];     // the warps' column sums, exchanged at the end
  __shared__ double wsum[NW][kMaxRank + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, s = g.s;
  // the CTA: one tile, a contiguous range of rows; its warps split the range
  const long long tile = blockIdx.x % g.tiles, pc = blockIdx.x / g.tiles;
  const long long cr0 = g.R * pc / g.parts, cr1 = g.R * (pc + 1) / g.parts;
  const long long r0 = cr0 + (cr1 - cr0) * warp / NW, r1 = cr0 + (cr1 - cr0) * (warp + 1) / NW;
  const long long c0 = tile * TW;  // first column of the tile
  uint32_t okmask = 0;             // bit k: load k of this lane lies inside the tensor
#pragma unroll
  for (int k = 0; k < NV; ++k) okmask |= (mx32_col<V>(c0, lane, k * V) < g.C ? 1u : 0u) << k;
  const bool full = okmask == ((1u << NV) - 1u);

  Mx32Cold st;
  for (int i = 0; i <= D; ++i) st.Tot[i] = CF{0.f, 0.f};
  for (int i = 0; i < s; ++i) {
    st.Aa[i] = CF{0.f, 0.f};
    st.Qa[i] = CF{0.f, 0.f};
  }
#pragma unroll
  for (int j = 0; j < J; ++j) st.colsum[j] = CF{0.f, 0.f};
  // ---- hot state: window column sums (plain f32) and the eager row axes.  The row's mass
  // is added across the warp every row, so every lane carries the same row-side state.
  float cs[J];
#pragma unroll
  for (int j = 0; j < J; ++j) cs[j] = 0.f;
  float S[kEager], Qh = 0.f;  // eager axes s-1-k: sum of row mass * digit; pending mass above
  uint32_t t[kEager], E[kEager];
#pragma unroll
  for (int k = 0; k < kEager; ++k) {
    S[k] = 0.f;
    st.Sc[k] = CF{0.f, 0.f};
    t[k] = 0;
    E[k] = s - 1 - k >= 0 ? (uint32_t)g.ext[s - 1 - k] : 0xFFFFFFFFu;  // absent: never wraps
  }
  if (r1 > r0) {
    uint32_t q = (uint32_t)r0;  // R < 2^31
    for (int a = s - 1; a >= 0; --a) {
      uint32_t d = q;
      if (a > 0) {
        const uint32_t q1 = fdiv(q, g.div[a]);
        d = q - q1 * g.div[a].d;
        q = q1;
      }
      const int k = s - 1 - a;
#pragma unroll
      for (int e = 0; e < kEager; ++e)
        if (e == k) t[e] = d;
      if (k >= kEager) st.td[a] = d;
    }
  }

  const T* lanep = p + (r0 * g.C + mx32_col<V>(c0, lane, 0));
  using Raw = typename std::conditional<(V > 1), uint4, float>::type;
  auto load = [&](Raw (&v)[NV], long long r) {
    const T* q = lanep + (r - r0) * g.C;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      if constexpr (V > 1) {
        v[k] = (full || (okmask >> k & 1u)) ? ld_stream16(q + 32 * k * V) : make_uint4(0, 0, 0, 0);
      } else {
        v[k] = (full || (okmask >> k & 1u)) ? FPiece<T>::ld(q, 32 * k) : 0.f;
      }
    }
  };
  int wrow = 0;
  // window end: plain f32 window sums into the compensated sums; the pending mass of the
  // cold levels is credited with the current digits
  auto end_window = [&]() {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      cf_add(st.colsum[j], cs[j]);
      cs[j] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < kEager; ++k) {
      cf_add(st.Sc[k], S[k]);
      S[k] = 0.f;
    }
    mx32_cold_step(g, st, CF{Qh, 0.f}, false);
    Qh = 0.f;
  };
  auto row = [&](const Raw (&v)[NV]) {
    float x[J];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
      for (int i = 0; i < V; ++i) {
        if constexpr (V > 1) x[k * V + i] = Unpack<T>::at(v[k], i);
        else x[k] = v[k];
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) cs[j] += x[j];
#pragma unroll
    for (int w = 1; w < J; w *= 2)
#pragma unroll
      for (int j = 0; j + w < J; j += 2 * w) x[j] += x[j + w];
    float m = x[0];
    // the row's mass over the warp (xor butterfly: the same value in every lane)
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) m += __shfl_xor_sync(0xffffffffu, m, off);
#pragma unroll
    for (int k = 0; k < kEager; ++k) S[k] = fmaf(m, (float)t[k], S[k]);
    Qh += m;
    // the next row's digits: carries through the eager axes, then the cold levels
    if (++t[0] == E[0]) {
      t[0] = 0;
      if (++t[1] == E[1]) {
        t[1] = 0;
        if (++t[2] == E[2]) {
          t[2] = 0;
          if (++t[3] == E[3]) {
            t[3] = 0;
            mx32_cold_step(g, st, CF{Qh, 0.f}, true);
            Qh = 0.f;
          }
        }
      }
    }
    if (++wrow == g.win) {
      end_window();
      wrow = 0;
    }
  };
  if (r1 > r0) {
    Raw va[NV], vb[NV], vc[NV];
    load(va, r0);
    if (r0 + 1 < r1) load(vb, r0 + 1);
    for (long long r = r0; r < r1; r += 3) {
      if (r + 2 < r1) load(vc, r + 2);
      row(va);
      if (r + 1 >= r1) break;
      if (r + 3 < r1) load(va, r + 3);
      row(vb);
      if (r + 2 >= r1) break;
      if (r + 4 < r1) load(vb, r + 4);
      row(vc);
    }
    end_window();
  }
  // row-side components of this warp (every lane holds the same values): lane 0's
#pragma unroll
  for (int k = 0; k < kEager; ++k)
    if (s - 1 - k >= 0) cf_add(st.Tot[s - 1 - k], st.Sc[k]);
  for (int i = 0; i + kEager < s; ++i) cf_add(st.Tot[i], st.Aa[i]);
  if (lane == 0) {
    for (int i = 0; i < s; ++i) wsum[warp][i] = (double)st.Tot[i].h + (double)st.Tot[i].l;
    wsum[warp][D] = (double)st.Tot[D].h + (double)st.Tot[D].l;
  }
  // column sums to shared memory (tile-relative columns), then per thread two columns of
  // the tile summed over the warps in a fixed order and weighted by their digits
#pragma unroll
  for (int j = 0; j < J; ++j) s_col[warp][mx32_col<V>(0, lane, j)] = st.colsum[j];
  __syncthreads();
  float M[kMaxRank];  // column axis s + k
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) M[k] = 0.f;
#pragma unroll
  for (int h = 0; h < TW / (NW * 32); ++h) {
    const int c = threadIdx.x + h * NW * 32;
    if (c0 + c >= g.C) continue;
    CF w{0.f, 0.f};
#pragma unroll
    for (int u = 0; u < NW; ++u) cf_add(w, s_col[u][c]);
    const float wf = w.h + w.l;
    uint32_t col = (uint32_t)(c0 + c);
#pragma unroll
    for (int k = 0; k < kMaxRank; ++k) {
      const int b = D - 1 - k;  // column axes from the innermost
      if (b < s) break;
      uint32_t d = col;
      if (b > s) {
        const uint32_t q = fdiv(col, g.div[b]);
        d = col - q * g.div[b].d;
        col = q;
      }
      M[k] = fmaf(wf, (float)d, M[k]);
    }
  }
  __syncthreads();
  // the column moments over the CTA: warp trees, then the warps in a fixed order
#pragma unroll
  for (int k = 0; k < kMaxRank; ++k) {
    if (k >= D - s) break;
    float v = M[k];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) wsum[warp][D - 1 - k] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

}  // namespace

const void* moment_mx32_kernel_ptr(int dtype, int V) {
  switch (dtype) {
    case DT_F32: return V > 1 ? reinterpret_cast<const void*>(&moment_mx32_kernel<float, 4>)
                              : reinterpret_cast<const void*>(&moment_mx32_kernel<float, 1>);
    case DT_BF16: return V > 1 ? reinterpret_cast<const void*>(&moment_mx32_kernel<__nv_bfloat16, 8>)
                               : reinterpret_cast<const void*>(&moment_mx32_kernel<__nv_bfloat16, 1>);
    case DT_F16: return V > 1 ? reinterpret_cast<const void*>(&moment_mx32_kernel<__half, 8>)
                              : reinterpret_cast<const void*>(&moment_mx32_kernel<__half, 1>);
  }
  return nullptr;
}

}  // namespace triot
