// f64 moment by marginals (Algorithms 10 and 11), in exact fixed point.
//
// The canonical axes are split in two: row axes 0 .. s-1 and column axes s .. D-1, so the
// tensor is an R x C matrix (R rows of C contiguous elements).  A moment splits the same
// way: for a row axis i,  m_i = sum over rows r of  t_i(r) * (mass of row r),  and for a
// column axis a,  m_a = sum over columns c of  t_a(c) * (mass of column c).  Each warp owns
// one tile of 32*J columns (lane l holds columns l, l + 32, ..., l + 32(J-1) of the tile)
// and a contiguous range of rows.  Rows are read straight from HBM with coalesced loads
// (the warp reads 32 x J x 8 contiguous bytes of a row), three rows ahead of the one being
// summed; every element costs one load, its conversion to fixed point and two integer
// adds: one into its column's sum, one into the lane's part of the row's mass.  The row's
// digits are the same for the whole warp and advance like Algorithm 3 (one increment per
// row, carries at wraps), so the tuple arithmetic is per row, not per element:
//   * the innermost row axis is credited every row:  S1 += (row mass) * t_{s-1};
//   * the mass of the other row axes waits in pending sums, credited to axis i (times its
//     digit) only when t_i changes, and then handed to the axis above.
// Column sums are turned into the column axes' moments once per window, from the digits
// of the lane's columns.
//
// Fixed point: inside a window (at most kMxWindow rows of the warp) every element is the
// integer c = m >> (E_W - e) in units of 2^(E_W - 1075): m its 53-bit significand, e its
// biased exponent, E_W the largest exponent the lane has seen in the window (all sums shift
// right when it grows).  Sums are exact; truncation bounds the error of every output by
// 2^-52 * (largest |p| of the lane's window) per element.  At the window end the sums are
// rounded once to f64.  Non-finite elements are summed separately in f64, so that they
// propagate as they would in a plain sum.
//
// Layout of the code: the per-row loop keeps all of its state in registers and stays
// small; everything that runs at most once per row wrap, window or warp (carries past the
// innermost row axis, window ends, rebasing, non-finite values) is out of line and works on
// the lane's cold state in local memory.
#include <utility>

#include "mx.cuh"
#include "fixed.cuh"
#include "kernels.h"

namespace triot {
namespace {

// c = m >> sh for sh in [0, 2^32): the PTX shift clamps amounts above 64 (result 0)
__device__ __forceinline__ unsigned long long shr_clamp(unsigned long long m, uint32_t sh) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(m), "r"(sh));
  return r;
}

// streaming 8-byte load (read once: evict first)
__device__ __forceinline__ unsigned long long ld_stream(const unsigned long long* q) {
  unsigned long long v;
  asm volatile("ld.global.cs.L2::256B.u64 %0, [%1];" : "=l"(v) : "l"(q));
  return v;
}

// digit of column `col` on column axis a (s <= a < D)
__device__ __forceinline__ uint32_t mx_col_digit(const MxGeom& g, uint32_t col, int a) {
  for (int b = g.D - 1; b > a; --b) col = fdiv(col, g.div[b]);
  return a == g.s ? col : col - fdiv(col, g.div[a]) * g.div[a].d;
}

// The lane's cold state (local memory): touched at carries, window ends and rare rows.
template <int J>
struct MxCold {
  long long cs[J];                  // column sums, handed over at a window end or rebase
  __int128 Aa[kMaxRank];            // row axes 0 .. s-2: sums of mass * digit
  __int128 Qa[kMaxRank];            // row levels 0 .. s-3: pending masses
  __int128 Mtot;                    // mass credited to every row axis
  uint32_t td[kMaxRank];            // digits of row axes 0 .. s-2 (warp-uniform)
  double Ad[kMaxRank + 1];          // the lane's f64 totals per component
  double sp[kMaxRank + 1];          // non-finite elements (plain f64 sums)
  int special;                      // sp holds something
};

// A carry out of the innermost row axis: the pending mass `pend` of level s-2 is credited
// to each changing axis with its old digit and handed to the axis above (Algorithm 3's
// carry, lazily).
template <int J>
__device__ __noinline__ void mx_carry(const MxGeom& g, MxCold<J>& st, __int128 pend) {
  const int s = g.s;
  int i = s - 2;
  while (true) {
    __int128 tot = pend;
    if (i < s - 2) {
      tot += st.Qa[i];
      st.Qa[i] = 0;
    }
    mac128x32(st.Aa[i], tot, st.td[i]);
    const uint32_t nt = st.td[i] + 1;
    if (i > 0 && nt == (uint32_t)g.ext[i]) {
      st.td[i] = 0;
      pend = tot;
      --i;
      continue;
    }
    st.td[i] = nt;
    if (i > 0) st.Qa[i - 1] += tot;  // still pending for the axes above i
    else st.Mtot += tot;
    return;
  }
}

// Window end: credit every pending mass (Qh: level s-2), round the window's sums (column
// sums in st.cs, S1 for the innermost row axis) to f64 once.
template <int J>
__device__ __noinline__ void mx_end_window(const MxGeom& g, MxCold<J>& st, __int128 Qh, __int128 S1,
                                           int EW, long long cbase, uint32_t colok) {
  const int s = g.s, D = g.D;
  __int128 pend = Qh;
  for (int i = s - 2; i >= 0; --i) {
    if (i < s - 2) {
      pend += st.Qa[i];
      st.Qa[i] = 0;
    }
    mac128x32(st.Aa[i], pend, st.td[i]);
  }
  st.Mtot += pend;
  if (EW != 0) {
    const int sc = EW - 1075;
    for (int i = 0; i + 1 < s; ++i) {
      st.Ad[i] += fixed_to_double(st.Aa[i], sc);
      st.Aa[i] = 0;
    }
    st.Ad[s - 1] += fixed_to_double(S1, sc);
    st.Ad[D] += fixed_to_double(st.Mtot, sc);
    // column axes: each of the lane's columns decoded once into all its digits
    __int128 acc[kMaxRank];
    for (int a = s; a < D; ++a) acc[a] = 0;
    for (int j = 0; j < J; ++j) {
      if (!(colok >> j & 1u)) continue;
      uint32_t c = (uint32_t)(cbase + 32 * j);
      for (int a = D - 1; a >= s; --a) {
        uint32_t d = c;
        if (a > s) {
          const uint32_t q = fdiv(c, g.div[a]);
          d = c - q * g.div[a].d;
          c = q;
        }
        mac64x32(acc[a], st.cs[j], d);
      }
    }
    for (int a = s; a < D; ++a) st.Ad[a] += fixed_to_double(acc[a], sc);
  }
  st.Mtot = 0;
}

// every fixed-point sum of the cold state shifts right by d (a larger window exponent)
template <int J>
__device__ __noinline__ void mx_rebase_cold(const MxGeom& g, MxCold<J>& st, int d) {
  for (int j = 0; j < J; ++j) st.cs[j] = shr64(st.cs[j], d);
  for (int i = 0; i + 1 < g.s; ++i) st.Aa[i] = shr_arith(st.Aa[i], d);
  for (int i = 0; i + 2 < g.s; ++i) st.Qa[i] = shr_arith(st.Qa[i], d);
  st.Mtot = shr_arith(st.Mtot, d);
}

// non-finite element v at column col of the current row: plain f64 sums
template <int J>
__device__ __noinline__ void mx_special(const MxGeom& g, MxCold<J>& st, double v, uint32_t t1,
                                        uint32_t col) {
  if (!st.special) {
    for (int i = 0; i <= g.D; ++i) st.sp[i] = 0.0;
    st.special = 1;
  }
  for (int i = 0; i + 1 < g.s; ++i) st.sp[i] += v * (double)st.td[i];
  st.sp[g.s - 1] += v * (double)t1;
  for (int a = g.s; a < g.D; ++a) st.sp[a] += v * (double)mx_col_digit(g, col, a);
  st.sp[g.D] += v;
}

// General conversion of the lane's J elements of one row (from the warp's shared-memory
// slot, J doubles per lane, lane-major): the window exponent is raised to the row's largest
// finite exponent first (the cold sums shift right; the hot ones are returned shifted in
// the returned shift), then every element converts exactly -- signed, zero, subnormal, tiny --
// and a non-finite one goes to the plain f64 sums.  The element integers are written back
// over the slot (as long long).  Out of line: rows of positive normal values, or of signed
// values within the window, never come here.
struct MxExp {
  int ew;     // the window exponent after the row
  int shift;  // how far the hot sums must shift right (0: the exponent did not grow)
};
template <int J>
__device__ __noinline__ MxExp mx_row_general(const MxGeom& g, MxCold<J>& st, unsigned long long* slot,
                                             int EW, uint32_t t1, long long cbase) {
  int emax = 0;
  for (int j = 0; j < J; ++j) {
    const uint32_t ef = (uint32_t)(slot[j * 32] >> 32) & 0x7FF00000u;
    if (ef != 0x7FF00000u) emax = max(emax, (int)((ef > 0x00100000u ? ef : 0x00100000u) >> 20));
  }
  MxExp r{EW, 0};
  if (emax > EW) {
    if (EW != 0) {
      r.shift = emax - EW;
      mx_rebase_cold<J>(g, st, emax - EW);
    }
    r.ew = emax;
  }
  for (int j = 0; j < J; ++j) {
    const unsigned long long b = slot[j * 32];
    const uint32_t ef = (uint32_t)(b >> 32) & 0x7FF00000u;
    long long c = 0;
    if (ef == 0x7FF00000u) {
      mx_special<J>(g, st, __longlong_as_double((long long)b), t1, (uint32_t)(cbase + 32 * j));
    } else {
      const int e = (int)((ef > 0x00100000u ? ef : 0x00100000u) >> 20);
      const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (ef ? 0x0010000000000000ull : 0ull);
      const long long x = (long long)shr_clamp(m, (uint32_t)(r.ew - e));
      c = (b >> 63) ? -x : x;
    }
    slot[j * 32] = (unsigned long long)c;
  }
  return r;
}

template <int J>
__global__ void __launch_bounds__(kMxWarps * 32, kMxMinCtas) moment_mx64_kernel(
    const __grid_constant__ MxGeom g, const double* __restrict__ p, double* __restrict__ partial) {
  __shared__ double wsum[kMxWarps][kMaxRank + 1];
  __shared__ unsigned long long s_slot[kMxWarps][J * 32];  // the general path's row, per warp
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, s = g.s;
  const long long gw = (long long)blockIdx.x * kMxWarps + warp;
  const long long tile = gw % g.tiles, part = gw / g.tiles;
  const bool active = part < g.parts;
  const long long r0 = active ? g.R * part / g.parts : 0;
  const long long r1 = active ? g.R * (part + 1) / g.parts : 0;
  const long long c0 = tile * 32 * J;            // first column of the tile
  const long long cbase = c0 + lane;             // column of slot j: cbase + 32 j
  const long long ncols = g.C - c0 < 32 * J ? g.C - c0 : 32 * J;
  const bool full_tile = ncols == 32 * J;
  uint32_t colok = 0;                            // bit j: column slot j lies inside the tensor
#pragma unroll
  for (int j = 0; j < J; ++j) colok |= (cbase + 32 * j < g.C ? 1u : 0u) << j;

  MxCold<J> st;
  for (int i = 0; i <= D; ++i) st.Ad[i] = 0.0;
  for (int i = 0; i + 1 < s; ++i) {
    st.Aa[i] = 0;
    st.Qa[i] = 0;
  }
  st.Mtot = 0;
  st.special = 0;

  // ---- hot state (registers)
  long long cs[J];                      // column sums (fixed point, the window)
  __int128 S1 = 0;                      // innermost row axis: sum of row mass * t1
  __int128 Qh = 0;                      // mass pending at row level s-2 (s = 1: the mass)
  int EW = 0;                           // window exponent (0: nothing seen)
  uint32_t t1 = 0;                      // digit of the innermost row axis
  const uint32_t E1 = s >= 2 ? (uint32_t)g.ext[s - 1] : 0xFFFFFFFFu;  // axis 0 never wraps
#pragma unroll
  for (int j = 0; j < J; ++j) cs[j] = 0;
  if (r1 > r0) {
    // digits of the first row (magic-number division, Algorithm 4)
    if (g.r32) {
      uint32_t q = (uint32_t)r0;
      for (int a = s - 1; a >= 1; --a) {
        const uint32_t q1 = fdiv(q, g.div[a]);
        const uint32_t d = q - q1 * g.div[a].d;
        if (a == s - 1) t1 = d;
        else st.td[a] = d;
        q = q1;
      }
      if (s == 1) t1 = q;
      else st.td[0] = q;
    } else {
      long long q = r0;
      for (int a = s - 1; a >= 1; --a) {
        const long long q1 = q / g.ext[a];
        const uint32_t d = (uint32_t)(q - q1 * g.ext[a]);
        if (a == s - 1) t1 = d;
        else st.td[a] = d;
        q = q1;
      }
      if (s == 1) t1 = (uint32_t)q;
      else st.td[0] = (uint32_t)q;
    }
  }
  auto end_window = [&]() {
#pragma unroll
    for (int j = 0; j < J; ++j) st.cs[j] = cs[j];
    mx_end_window<J>(g, st, Qh, S1, EW, cbase, colok);
#pragma unroll
    for (int j = 0; j < J; ++j) cs[j] = 0;
    Qh = 0;
    S1 = 0;
    EW = 0;
  };

  // ---- rows: loads straight from HBM into a ring of four row buffers, so that while one
  // row is summed the next three are in flight (3 x 32 x J x 8 bytes per warp)
  const unsigned long long* prow =
      reinterpret_cast<const unsigned long long*>(p) + (r0 * g.C + cbase);  // slot 0, row r0
  auto load = [&](unsigned long long (&v)[J], long long r) {
    const unsigned long long* q = prow + (r - r0) * g.C;
    if (full_tile) {
#pragma unroll
      for (int j = 0; j < J; ++j) v[j] = ld_stream(q + 32 * j);
    } else {
#pragma unroll
      for (int j = 0; j < J; ++j) v[j] = (colok >> j & 1u) ? ld_stream(q + 32 * j) : 0ull;
    }
  };
  int wrow = 0;
  auto row = [&](const unsigned long long (&v)[J]) {
    uint32_t hmax = 0, hmin = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const uint32_t hi = (uint32_t)(v[j] >> 32);
      hmax = max(hmax, hi);
      hmin = min(hmin, hi);
    }
    // no new exponent and positive, finite values everywhere in the warp's row
    const bool steady = hmax < 0x7FF00000u && (int)(hmax >> 20) <= EW;
    long long rp = 0;
    if (__all_sync(0xffffffffu, steady && hmin >= 0x00100000u && EW - (int)(hmin >> 20) < 32)) {
      // normal values within 32 binades of the window exponent: 32-bit funnel shifts
      const uint32_t ec = (uint32_t)EW;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const uint32_t hi = (uint32_t)(v[j] >> 32), lo = (uint32_t)v[j];
        const uint32_t sh = ec - (hi >> 20);
        const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
        const long long c =
            (long long)(((unsigned long long)(mh >> sh) << 32) | __funnelshift_r(lo, mh, sh));
        cs[j] += c;
        rp += c;
      }
    } else if (__all_sync(0xffffffffu, steady && EW >= 54)) {
      // zeros, subnormals and tiny values too (a window exponent of 54 or more sends them
      // to their exact fixed-point value, 0 when they are below the window): a clamped
      // 64-bit shift
      const uint32_t ec = (uint32_t)EW;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const uint32_t hi = (uint32_t)(v[j] >> 32);
        const unsigned long long m = (v[j] & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
        const long long c = (long long)shr_clamp(m, ec - (hi >> 20));
        cs[j] += c;
        rp += c;
      }
    } else {
      // everything else (signs, a new exponent, a small window exponent, non-finite
      // values), out of line through the warp's shared-memory slot
      unsigned long long* slot = &s_slot[warp][lane];
#pragma unroll
      for (int j = 0; j < J; ++j) slot[j * 32] = v[j];
      const MxExp ex = mx_row_general<J>(g, st, slot, EW, t1, cbase);
      EW = ex.ew;
      if (ex.shift) {
        const int hs = ex.shift;
#pragma unroll
        for (int j = 0; j < J; ++j) cs[j] = shr64(cs[j], hs);
        S1 = shr_arith(S1, hs);
        Qh = shr_arith(Qh, hs);
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const long long c = (long long)slot[j * 32];
        cs[j] += c;
        rp += c;
      }
    }
    mac64x32(S1, rp, t1);
    Qh += rp;
    if (++t1 == E1) {
      t1 = 0;
      mx_carry<J>(g, st, Qh);
      Qh = 0;
    }
    if (++wrow == g.win) {
      end_window();
      wrow = 0;
    }
  };
  if (r1 > r0) {
    unsigned long long va[J], vb[J], vc[J], vd[J];
    load(va, r0);
    if (r0 + 1 < r1) load(vb, r0 + 1);
    if (r0 + 2 < r1) load(vc, r0 + 2);
    for (long long r = r0; r < r1; r += 4) {
      if (r + 3 < r1) load(vd, r + 3);
      row(va);
      if (r + 1 >= r1) break;
      if (r + 4 < r1) load(va, r + 4);
      row(vb);
      if (r + 2 >= r1) break;
      if (r + 5 < r1) load(vb, r + 5);
      row(vc);
      if (r + 3 >= r1) break;
      if (r + 6 < r1) load(vc, r + 6);
      row(vd);
    }
    end_window();
  }

  // warp sum of the lane totals: exact in 128-bit fixed point relative to the warp's largest
  // exponent (integer shuffles), or an f64 xor-order sum when a lane holds a non-finite value
#pragma unroll 1
  for (int i = 0; i <= D; ++i) {
    double v = st.special ? st.Ad[i] + st.sp[i] : st.Ad[i];
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FFull);
    if (__any_sync(0xffffffffu, e == 0x7FF)) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) wsum[warp][i] = v;
      continue;
    }
    unsigned long long mant = bits & 0x000FFFFFFFFFFFFFull;
    if (e) mant |= 1ull << 52;
    else e = 1;
    const int ew = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    const int d = ew - e;  // v = mant * 2^(e - 1075) = (mant << (64 - d)) * 2^(ew - 1139)
    __int128 x = 0;
    if (d <= 64) x = (__int128)((unsigned __int128)mant << (64 - d));
    else if (d < 64 + 53) x = (__int128)(mant >> (d - 64));
    if (bits >> 63) x = -x;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const unsigned __int128 u = (unsigned __int128)x;
      const unsigned w0 = __shfl_xor_sync(0xffffffffu, (unsigned)u, off);
      const unsigned w1 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 32), off);
      const unsigned w2 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 64), off);
      const unsigned w3 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 96), off);
      x += (__int128)(((unsigned __int128)w3 << 96) | ((unsigned __int128)w2 << 64) |
                      ((unsigned __int128)w1 << 32) | (unsigned __int128)w0);
    }
    if (lane == 0) wsum[warp][i] = fixed_to_double(x, ew - 1139);
  }
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kMxWarps; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

}  // namespace

const void* moment_mx64_kernel_ptr() { return reinterpret_cast<const void*>(&moment_mx64_kernel<kMxJ>); }

}  // namespace triot
