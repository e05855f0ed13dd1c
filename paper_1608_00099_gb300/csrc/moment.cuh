// Tuple-weighted moment  m_i = sum_t p[t] * t_i  (Algorithms 10 and 11) and its mass.
//
// Work split: the flat index range is cut into lane segments of S elements; 32 lane
// segments form a warp segment and persistent warps loop over warp segments.  Each lane
// walks its segment in order, carrying its tuple like the paper's advance_tuple
// (Algorithm 3).  Instead of d multiply-adds per element, a lane accumulates the mass and
// the inner-index-weighted mass of the current row, and pushes the row's mass up the
// axes only when a carry happens ("carry-propagated" sums): at a carry into axis i the
// pending mass of the block that just ended is weighted by t_i.  The per-element cost is
// two accumulations; axis i is touched once per prod_{j>i} s_j elements, the same
// geometric-series amortisation Section 1 gives for advance_tuple.
//
// Staging: each lane needs its own contiguous run, so the warp copies 32 pieces of 128
// bytes (one per lane) into a warp-private shared-memory stage with 16-byte cp.async
// (coalesced in global memory; rows padded to 144 bytes so the lanes' reads are
// bank-conflict free), double-buffered.
//
// Arithmetic: f32/bf16/f16 input accumulates in f32 with compensated (two-sum) adds at
// row and carry level.  f64 input accumulates in exact two's-complement fixed point: GB300
// runs f64 at ~1/70 of its f32 rate, which cannot keep up with HBM; integer adds can.
// Per-block partials (f64) are combined by combine_kernel in exact fixed point, so the
// result does not depend on the order of the partials.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "fixed.cuh"

namespace triot {

constexpr int kStageRowBytes = 144;      // 128 data bytes + 16 pad per lane row
constexpr int kStageBytes = 32 * kStageRowBytes;
constexpr int kFixGuard = 16;            // fraction bits below a chunk's exponent (f64 path)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Stage chunk `chunk` of warp segment `ws` (32 pieces of 128 bytes) into `buf`.
template <int ES>
__device__ __forceinline__ void stage_chunk(const MomentGeom& g, const unsigned char* p,
                                            unsigned char* buf, long long ws, int chunk,
                                            int lane) {
  constexpr int C = 128 / ES;
  const long long nbytes = g.n * ES;
  if (g.aligned) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int piece = q * 4 + (lane >> 3), part = lane & 7;
      const long long byte =
          ((ws * 32 + piece) * g.seg + (long long)chunk * C) * ES + part * 16;
      long long rem = nbytes - byte;
      const int nb = rem >= 16 ? 16 : (rem > 0 ? int(rem) : 0);
      cp_async16(buf + piece * kStageRowBytes + part * 16, nb ? (const void*)(p + byte) : (const void*)p, nb);
    }
  } else {
    // unaligned base: plain element loads (coalesced across lanes), then shared stores
    for (int i = lane; i < 32 * C; i += 32) {
      const int piece = i / C, off = i - piece * C;
      const long long idx = (ws * 32 + piece) * g.seg + (long long)chunk * C + off;
      unsigned char* d = buf + piece * kStageRowBytes + off * ES;
      if (ES == 8) {
        *reinterpret_cast<unsigned long long*>(d) =
            idx < g.n ? reinterpret_cast<const unsigned long long*>(p)[idx] : 0ull;
      } else if (ES == 4) {
        *reinterpret_cast<unsigned*>(d) = idx < g.n ? reinterpret_cast<const unsigned*>(p)[idx] : 0u;
      } else {
        *reinterpret_cast<unsigned short*>(d) =
            idx < g.n ? reinterpret_cast<const unsigned short*>(p)[idx] : (unsigned short)0;
      }
    }
  }
}

// tuple of flat index k over the effective shape (digits peeled innermost first, Alg 4)
template <int D>
__device__ __forceinline__ void decode_tuple(const MomentGeom& g, long long k, uint32_t (&t)[D]) {
  if (g.n32) {
    uint32_t rem = (uint32_t)k;
#pragma unroll
    for (int i = D - 1; i >= 1; --i) {
      const uint32_t q = fdiv(rem, g.div[i]);
      t[i] = rem - q * g.div[i].d;
      rem = q;
    }
    t[0] = rem;
  } else {
    long long rem = k;
#pragma unroll
    for (int i = D - 1; i >= 1; --i) {
      const long long q = rem / g.ext[i];
      t[i] = (uint32_t)(rem - q * g.ext[i]);
      rem = q;
    }
    t[0] = (uint32_t)rem;
  }
}

// ====================================================================== f32 accumulation

struct Comp32 {  // s + e, updated with Knuth's branch-free two-sum
  float s, e;
  __device__ __forceinline__ void zero() { s = 0.f; e = 0.f; }
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + e; }
};

template <typename T>
__device__ __forceinline__ float elem_f32(const unsigned char* row, int j) {
  if constexpr (sizeof(T) == 4) {
    return reinterpret_cast<const float*>(row)[j];
  } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
    return __uint_as_float(((unsigned)reinterpret_cast<const unsigned short*>(row)[j]) << 16);
  } else {
    return __half2float(reinterpret_cast<const __half*>(row)[j]);
  }
}

template <typename T, int D>
__global__ void __launch_bounds__(kMomentWarps * 32) moment_f32_kernel(
    const __grid_constant__ MomentGeom g, const T* __restrict__ p, double* __restrict__ partial) {
  constexpr int ES = sizeof(T);
  constexpr int C = 128 / ES;
  __shared__ __align__(16) unsigned char stage[kMomentWarps][2][kStageBytes];
  __shared__ double wsum[kMomentWarps][kMaxRank + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kMomentWarps + warp;
  const long long tw = (long long)gridDim.x * kMomentWarps;
  const long long nseg = gw < g.nwarpseg ? (g.nwarpseg - gw + tw - 1) / tw : 0;
  const long long nsteps = nseg * g.nchunks;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
  const uint32_t L = (uint32_t)g.ext[D - 1];

  Comp32 A[D], P[D];  // P[0]: mass; P[k], k >= 1: pending mass of the block of axis k-1
#pragma unroll
  for (int i = 0; i < D; ++i) { A[i].zero(); P[i].zero(); }
  uint32_t t[D];
#pragma unroll
  for (int i = 0; i < D; ++i) t[i] = 0;
  float mp = 0.f, wp = 0.f, jl = 0.f;  // segment mass, local-index-weighted mass, local index
  uint32_t t0 = 0;                      // inner index at the start of the current run
  bool active = false;                  // the current lane segment starts inside the tensor

  // end of a run of one row: push the run into the row accumulators
  auto flush_run = [&]() {
    A[D - 1].add(wp);
    A[D - 1].add((float)t0 * mp);
    P[D - 1].add(mp);
    mp = 0.f; wp = 0.f; jl = 0.f;
  };
  // carry out of the inner axis (row end): pending masses move up while axes wrap
  auto carry = [&]() {
#pragma unroll
    for (int i = D - 2; i >= 0; --i) {
      const float pm = P[i + 1].value();
      A[i].add((float)t[i] * pm);
      P[i].add(pm);
      P[i + 1].zero();
      if (i > 0) {
        if (++t[i] < (uint32_t)g.ext[i]) break;
        t[i] = 0;
      } else {
        ++t[0];
      }
    }
  };
  // end of a lane segment: flush every pending level (the tuple is that of the last
  // element processed, so each pending mass is weighted by its own digit)
  auto flush_all = [&]() {
    flush_run();
#pragma unroll
    for (int i = D - 2; i >= 0; --i) {
      const float pm = P[i + 1].value();
      A[i].add((float)t[i] * pm);
      P[i].add(pm);
      P[i + 1].zero();
    }
  };

  if (nsteps > 0) {
    stage_chunk<ES>(g, pb, stage[warp][0], gw, 0, lane);
    cp_async_commit();
  }
  for (long long s = 0; s < nsteps; ++s) {
    const long long ws = gw + (s / g.nchunks) * tw;
    const int chunk = (int)(s % g.nchunks);
    if (s + 1 < nsteps) {
      const long long ws1 = gw + ((s + 1) / g.nchunks) * tw;
      stage_chunk<ES>(g, pb, stage[warp][(s + 1) & 1], ws1, (int)((s + 1) % g.nchunks), lane);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    if (chunk == 0) {
      // a lane segment that starts at or past the end holds only zero fill: skip it
      const long long k0 = (ws * 32 + lane) * g.seg;
      active = k0 < g.n;
      if (active) {
        decode_tuple<D>(g, k0, t);
        t0 = t[D - 1];
      }
    }
    if (active) {
      const unsigned char* row = stage[warp][s & 1] + lane * kStageRowBytes;
#pragma unroll 4
      for (int j = 0; j < C; ++j) {
        const float x = elem_f32<T>(row, j);
        mp += x;
        wp = fmaf(jl, x, wp);
        jl += 1.0f;
        if (++t[D - 1] == L) {
          flush_run();
          t[D - 1] = 0;
          t0 = 0;
          carry();
        }
      }
      flush_run();
      t0 = t[D - 1];
      if (chunk == g.nchunks - 1) flush_all();
    }
    __syncwarp();
  }

  // warp reduction of the compensated pairs (xor butterfly: fixed order)
  double* ws_out = wsum[warp];
#pragma unroll
  for (int i = 0; i <= D; ++i) {
    Comp32 v = (i < D) ? A[i] : P[0];
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, v.s, off);
      const float oe = __shfl_xor_sync(0xffffffffu, v.e, off);
      v.add(os);
      v.e += oe;
    }
    if (lane == 0) ws_out[i] = (double)v.s + (double)v.e;
  }
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kMomentWarps; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

// ====================================================================== f64 fixed point
//
// Each lane reads its 16-element chunk from shared memory twice.  First pass: the chunk's
// largest exponent field E_c (zeros and subnormals count as exponent 1) and whether a
// non-finite value is present.  Second pass, one run at a time (a run = the part of the
// chunk inside one row): an f64 with biased exponent e and significand m (53 bits,
// implicit bit included) is m * 2^(e-1075); relative to E_c it is c = m >> (E_c - e)
// units of 2^(E_c-1075), exact for the chunk maximum and truncated below its last bit
// for smaller elements.  A run keeps P = sum c and Q = sum of the running P, so that the
// run's inner-index-weighted sum sum_k k c_k = n P - Q needs no multiply per element.
// Runs move into the lane's 128-bit accumulators, whose unit is 2^(E_L-1075-16) for the
// largest exponent E_L the lane has seen (accumulators shift right when E_L grows).
// Non-finite elements are summed separately in f64 so that they propagate.

template <int D>
__global__ void __launch_bounds__(kMomentWarps * 32, (D <= 12 ? 4 : 2)) moment_f64_kernel(
    const __grid_constant__ MomentGeom g, const double* __restrict__ p,
    double* __restrict__ partial) {
  constexpr int ES = 8;
  constexpr int C = 16;
  __shared__ __align__(16) unsigned char stage[kMomentWarps][2][kStageBytes];
  __shared__ double wsum[kMomentWarps][kMaxRank + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kMomentWarps + warp;
  const long long tw = (long long)gridDim.x * kMomentWarps;
  const long long nseg = gw < g.nwarpseg ? (g.nwarpseg - gw + tw - 1) / tw : 0;
  const long long nsteps = nseg * g.nchunks;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
  const uint32_t L = (uint32_t)g.ext[D - 1];

  __int128 A[D], P[D];  // P[0]: mass; P[k], k >= 1: pending mass of the block of axis k-1
#pragma unroll
  for (int i = 0; i < D; ++i) { A[i] = 0; P[i] = 0; }
  int EL = 0;                         // lane reference exponent (0: nothing seen yet)
  bool special = false;               // a non-finite element was seen
  double Asp[D], Psp = 0.0;           // f64 sums of non-finite elements
#pragma unroll
  for (int i = 0; i < D; ++i) Asp[i] = 0.0;
  uint32_t t[D];
#pragma unroll
  for (int i = 0; i < D; ++i) t[i] = 0;
  uint32_t ti = 0;                    // inner index (digit of axis D-1)
  bool active = false;                // the current lane segment starts inside the tensor

  // a run (P: sum of c, W: sum of local index * c, t0: inner index of its first element)
  auto add_run = [&](long long Pr, long long Wr, uint32_t t0, int Ec) {
    if (Pr == 0 && Wr == 0) return;
    if (Ec > EL) {
      if (EL != 0) {
#pragma unroll
        for (int i = 0; i < D; ++i) { A[i] = shr_arith(A[i], Ec - EL); P[i] = shr_arith(P[i], Ec - EL); }
      }
      EL = Ec;
    }
    const __int128 M = (__int128)Pr;
    const __int128 W = (__int128)Wr + (__int128)Pr * (__int128)(unsigned long long)t0;
    if (EL == Ec) {
      P[D - 1] += M << kFixGuard;
      A[D - 1] += W << kFixGuard;
    } else {
      const int sc = kFixGuard - (EL - Ec);
      P[D - 1] += scale_shift(M, sc);
      A[D - 1] += scale_shift(W, sc);
    }
  };
  // row end: the row's pending mass moves up while axes wrap (carry of Algorithm 3)
  auto carry = [&]() {
#pragma unroll
    for (int i = D - 2; i >= 0; --i) {
      const __int128 pm = P[i + 1];
      A[i] += pm * (__int128)(unsigned long long)t[i];
      P[i] += pm;
      P[i + 1] = 0;
      if (i > 0) {
        if (++t[i] < (uint32_t)g.ext[i]) break;
        t[i] = 0;
      } else {
        ++t[0];
      }
    }
  };
  auto flush_levels = [&]() {
#pragma unroll
    for (int i = D - 2; i >= 0; --i) {
      const __int128 pm = P[i + 1];
      A[i] += pm * (__int128)(unsigned long long)t[i];
      P[i] += pm;
      P[i + 1] = 0;
    }
  };
  // one chunk, runs split at row ends; SPECIAL chunks route non-finite values to f64
  auto do_chunk = [&](const unsigned long long* row, int Ec, auto special_tag) {
    constexpr bool SPECIAL = decltype(special_tag)::value;
    int j = 0;
    while (j < C) {
      // active lanes keep ti < L, so every run has at least one element
      const int left = ti < L ? (int)(L - ti) : C;
      const int n = left < C - j ? left : C - j;
      long long Pr = 0, Q = 0;
      for (int k = 0; k < n; ++k) {
        const unsigned long long b = row[j + k];
        const uint32_t hi = (uint32_t)(b >> 32);
        const uint32_t ef = hi & 0x7FF00000u;
        if (SPECIAL && ef == 0x7FF00000u) {
          const double v = __longlong_as_double((long long)b);
#pragma unroll
          for (int i = 0; i < D - 1; ++i) Asp[i] += v * (double)t[i];
          Asp[D - 1] += v * (double)(ti + (uint32_t)k);
          Psp += v;
          Q += Pr;
          continue;
        }
        const uint32_t e = (ef > 0x00100000u ? ef : 0x00100000u) >> 20;
        const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
        const uint32_t sh = (uint32_t)Ec - e;
        long long c = (long long)(m >> (sh < 63u ? sh : 63u));
        c = ((int)hi < 0) ? -c : c;
        Pr += c;
        Q += Pr;
      }
      add_run(Pr, (long long)n * Pr - Q, ti, Ec);
      j += n;
      ti += (uint32_t)n;
      if (ti == L) {
        ti = 0;
        carry();
      }
    }
  };

  // Fast chunk: every element finite, non-negative and normal, exponents within 32 binades
  // of the chunk maximum.  Then m >> sh needs two 32-bit funnel shifts and no sign or
  // subnormal handling: about nine integer instructions per element.
  auto do_chunk_fast = [&](const uint2* row2, uint32_t ec) {
    int j = 0;
    while (j < C) {
      const int left = ti < L ? (int)(L - ti) : C;
      const int n = left < C - j ? left : C - j;
      unsigned long long Pr = 0, Q = 0;
#pragma unroll 2
      for (int k = 0; k < n; ++k) {
        const uint2 b = row2[j + k];
        const uint32_t sh = ec - (b.y >> 20);
        const uint32_t mh = (b.y & 0x000FFFFFu) | 0x00100000u;
        const uint32_t cl = __funnelshift_r(b.x, mh, sh);
        const uint32_t ch = mh >> sh;
        Pr += ((unsigned long long)ch << 32) | cl;
        Q += Pr;
      }
      add_run((long long)Pr, (long long)((unsigned long long)n * Pr - Q), ti, (int)ec);
      j += n;
      ti += (uint32_t)n;
      if (ti == L) {
        ti = 0;
        carry();
      }
    }
  };

  if (nsteps > 0) {
    stage_chunk<ES>(g, pb, stage[warp][0], gw, 0, lane);
    cp_async_commit();
  }
  for (long long s = 0; s < nsteps; ++s) {
    const long long ws = gw + (s / g.nchunks) * tw;
    const int chunk = (int)(s % g.nchunks);
    if (s + 1 < nsteps) {
      const long long ws1 = gw + ((s + 1) / g.nchunks) * tw;
      stage_chunk<ES>(g, pb, stage[warp][(s + 1) & 1], ws1, (int)((s + 1) % g.nchunks), lane);
    }
    cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    if (chunk == 0) {
      // a lane segment that starts at or past the end holds only zero fill: skip it (for
      // D = 1 its decoded inner index would not be below L)
      const long long k0 = (ws * 32 + lane) * g.seg;
      active = k0 < g.n;
      if (active) {
        decode_tuple<D>(g, k0, t);
        ti = t[D - 1];
      }
    }
    if (active) {
    const unsigned long long* row =
        reinterpret_cast<const unsigned long long*>(stage[warp][s & 1] + lane * kStageRowBytes);
    // unsigned max / min of the high words: for non-negative values they order by exponent;
    // a negative value (sign bit) or a non-finite one pushes the max to 0x7FF00000 or above,
    // a zero or subnormal pulls the min below 0x00100000
    uint32_t hmax = 0u, hmin = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < C; j += 2) {
      const uint4 v = *reinterpret_cast<const uint4*>(row + j);
      hmax = max(hmax, max(v.y, v.w));
      hmin = min(hmin, min(v.y, v.w));
    }
    if (hmax < 0x7FF00000u && hmin >= 0x00100000u && (hmax >> 20) - (hmin >> 20) < 32u) {
      do_chunk_fast(reinterpret_cast<const uint2*>(row), hmax >> 20);
    } else {
      // general chunk: largest finite exponent field (zeros and subnormals count as 1)
      uint32_t emaxf = 0x00100000u, efin = 0x00100000u;
#pragma unroll
      for (int j = 0; j < C; j += 2) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + j);
        const uint32_t f0 = v.y & 0x7FF00000u, f1 = v.w & 0x7FF00000u;
        emaxf = max(emaxf, max(f0, f1));
        efin = max(efin, max(f0 == 0x7FF00000u ? 0u : f0, f1 == 0x7FF00000u ? 0u : f1));
      }
      if (emaxf != 0x7FF00000u) {
        do_chunk(row, (int)(emaxf >> 20), std::false_type());
      } else {
        special = true;
        do_chunk(row, (int)(efin >> 20), std::true_type());
      }
    }
    if (chunk == g.nchunks - 1) flush_levels();
    }
    __syncwarp();
  }

  // warp reduction: align lanes to the warp's largest exponent, then exact integer sums
  const int EW = (int)__reduce_max_sync(0xffffffffu, (unsigned)EL);
  const bool any_special = __any_sync(0xffffffffu, special);
  double* ws_out = wsum[warp];
#pragma unroll
  for (int i = 0; i <= D; ++i) {
    __int128 v = (i < D) ? A[i] : P[0];
    v = (EL == 0) ? (__int128)0 : shr_arith(v, EW - EL);
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)((unsigned __int128)v >> 64);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
      const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
      const unsigned __int128 sum = (((unsigned __int128)hi << 64) | lo) + (((unsigned __int128)ohi << 64) | olo);
      lo = (unsigned long long)sum;
      hi = (unsigned long long)(sum >> 64);
    }
    double dv = 0.0;
    if (EW != 0) {
      const __int128 tot = (__int128)(((unsigned __int128)hi << 64) | lo);
      dv = ldexp(i128_to_double(tot), EW - 1075 - kFixGuard);
    }
    if (any_special) {
      double sp = (i < D) ? Asp[i] : Psp;
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, off);
      dv += sp;
    }
    if (lane == 0) ws_out[i] = dv;
  }
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kMomentWarps; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

}  // namespace triot
