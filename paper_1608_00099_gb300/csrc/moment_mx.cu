// f64 moment by marginals (Algorithms 10 and 11), in exact fixed point.
//
// The canonical axes are split in two: row axes 0 .. s-1 and column axes s .. D-1, so the
// tensor is an R x C matrix (R rows of C contiguous elements).  A moment splits the same
// way: for a row axis i,  m_i = sum over rows r of  t_i(r) * (mass of row r),  and for a
// column axis a,  m_a = sum over columns c of  t_a(c) * (mass of column c).  Each warp owns
// one tile of 32*J columns (lane l holds columns l, l + 32, ..., l + 32(J-1) of the tile)
// and a contiguous range of rows.  Each row's segment of the tile (up to 2 KB, contiguous)
// is staged into shared memory by one bulk copy issued by lane 0, kMxStages rows ahead, so
// the loads in flight cost no registers; every element then costs one shared-memory read,
// its conversion to fixed point and two integer adds: one into its column's sum, one into
// the lane's part of the row's mass.
// The row's digits are the same for the whole warp and advance like Algorithm 3 (one
// increment per row, carries at wraps), so the tuple arithmetic is per row, not per
// element:
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
#include <utility>

#include "mx.cuh"
#include "fixed.cuh"
#include "kernels.h"
#include "sync.cuh"

namespace triot {
namespace {

// set when a bounded wait for a staged row gives up (read by triot_device_status)
__device__ int g_mx_flag = 0;

// c = m >> sh for sh in [0, 2^32): the PTX shift clamps amounts above 64 (result 0)
__device__ __forceinline__ unsigned long long shr_clamp(unsigned long long m, uint32_t sh) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(m), "r"(sh));
  return r;
}

// Digits of row r on the row axes 0 .. s-1 (axis s-1 is the innermost row axis).
__device__ void mx_row_digits(const MxGeom& g, long long r, uint32_t* td) {
  if (g.r32) {
    uint32_t q = (uint32_t)r;
    for (int a = g.s - 1; a >= 1; --a) {
      const uint32_t q1 = fdiv(q, g.div[a]);
      td[a] = q - q1 * g.div[a].d;
      q = q1;
    }
    td[0] = q;
  } else {
    long long q = r;
    for (int a = g.s - 1; a >= 1; --a) {
      const long long q1 = q / g.ext[a];
      td[a] = (uint32_t)(q - q1 * g.ext[a]);
      q = q1;
    }
    td[0] = (uint32_t)q;
  }
}

// digit of column `col` on column axis a (s <= a < D)
__device__ __forceinline__ uint32_t mx_col_digit(const MxGeom& g, uint32_t col, int a) {
  for (int b = g.D - 1; b > a; --b) col = fdiv(col, g.div[b]);
  return a == g.s ? col : col - fdiv(col, g.div[a]) * g.div[a].d;
}

// non-finite element v at row digits td (innermost t1) and column col: plain f64 sums
__device__ __noinline__ void mx_special(const MxGeom& g, double v, const uint32_t* td, uint32_t t1,
                                        uint32_t col, double* sp) {
  for (int i = 0; i + 1 < g.s; ++i) sp[i] += v * (double)td[i];
  sp[g.s - 1] += v * (double)t1;
  for (int a = g.s; a < g.D; ++a) sp[a] += v * (double)mx_col_digit(g, col, a);
  sp[g.D] += v;
}

// General conversion of a lane's J elements of one row at window exponent EW (at least the
// exponent of every finite element): signed, zero, subnormal and tiny values exactly; a
// non-finite element gives 0 and sets its bit in the returned mask.  Out of line, so that
// the hot loop stays small: rows of positive normal values never come here.
template <int J>
__device__ __noinline__ unsigned mx_convert_general(const unsigned long long* v, int EW, long long* c) {
  unsigned spec = 0;
  for (int j = 0; j < J; ++j) {
    const unsigned long long b = v[j];
    const uint32_t ef = (uint32_t)(b >> 32) & 0x7FF00000u;
    if (ef == 0x7FF00000u) {
      spec |= 1u << j;
      c[j] = 0;
      continue;
    }
    const int e = (int)((ef > 0x00100000u ? ef : 0x00100000u) >> 20);
    const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (ef ? 0x0010000000000000ull : 0ull);
    const long long x = (long long)shr_clamp(m, (uint32_t)(EW - e));
    c[j] = (b >> 63) ? -x : x;
  }
  return spec;
}

// the largest biased exponent of the finite elements among v[0 .. J-1] (subnormals and zeros
// count as 1), 0 when all are non-finite
template <int J>
__device__ __noinline__ int mx_row_emax(const unsigned long long* v) {
  int emax = 0;
  for (int j = 0; j < J; ++j) {
    const uint32_t ef = (uint32_t)(v[j] >> 32) & 0x7FF00000u;
    if (ef != 0x7FF00000u) emax = max(emax, (int)((ef > 0x00100000u ? ef : 0x00100000u) >> 20));
  }
  return emax;
}

template <int J>
__global__ void __launch_bounds__(kMxWarps * 32, kMxMinCtas) moment_mx64_kernel(
    const __grid_constant__ MxGeom g, const double* __restrict__ p, double* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double wsum[kMxWarps][kMaxRank + 1];
  __shared__ __align__(8) unsigned long long s_bar[kMxWarps][kMxStages];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    for (int q = 0; q < kMxStages; ++q) {
      const unsigned a = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const int D = g.D, s = g.s;
  const long long gw = (long long)blockIdx.x * kMxWarps + warp;
  const long long tile = gw % g.tiles, part = gw / g.tiles;
  const bool active = part < g.parts;
  const long long r0 = active ? g.R * part / g.parts : 0;
  const long long r1 = active ? g.R * (part + 1) / g.parts : 0;
  const long long cbase = tile * 32 * J + lane;  // column of slot j: cbase + 32 j

  // ---- lane state
  long long cs[J];                      // column sums (fixed point, the window)
  __int128 S1 = 0;                      // innermost row axis: sum of row mass * t1
  __int128 Qh = 0;                      // mass pending at row level s-2 (s = 1: the mass)
  __int128 Mtot = 0;                    // mass credited to every row axis
  int EW = 0;                           // window exponent (0: nothing seen)
  __int128 Aa[kMaxRank];                // row axes 0 .. s-2: sums of mass * digit
  __int128 Qa[kMaxRank];                // row levels 0 .. s-3: pending masses
  uint32_t td[kMaxRank];                // digits of row axes 0 .. s-2 (warp-uniform)
  double Ad[kMaxRank + 1];              // the lane's f64 totals per component
  double sp[kMaxRank + 1];              // non-finite elements (plain f64 sums)
  bool special = false;
#pragma unroll
  for (int j = 0; j < J; ++j) cs[j] = 0;
  for (int i = 0; i <= D; ++i) Ad[i] = 0.0;
  for (int i = 0; i + 1 < s; ++i) { Aa[i] = 0; Qa[i] = 0; }
  uint32_t t1 = 0;
  const uint32_t E1 = s >= 2 ? (uint32_t)g.ext[s - 1] : 0xFFFFFFFFu;  // axis 0 never wraps
  if (r1 > r0) {
    uint32_t dg[kMaxRank];
    mx_row_digits(g, r0, dg);
    for (int i = 0; i + 1 < s; ++i) td[i] = dg[i];
    t1 = dg[s - 1];
  }
  uint32_t colok = 0;  // bit j: column slot j lies inside the tensor
#pragma unroll
  for (int j = 0; j < J; ++j) colok |= (cbase + 32 * j < g.C ? 1u : 0u) << j;

  auto rebase = [&](int e_new) {
    if (EW != 0) {
      const int d = e_new - EW;
#pragma unroll
      for (int j = 0; j < J; ++j) cs[j] = shr64(cs[j], d);
      S1 = shr_arith(S1, d);
      Qh = shr_arith(Qh, d);
      Mtot = shr_arith(Mtot, d);
      for (int i = 0; i + 1 < s; ++i) Aa[i] = shr_arith(Aa[i], d);
      for (int i = 0; i + 2 < s; ++i) Qa[i] = shr_arith(Qa[i], d);
    }
    EW = e_new;
  };
  // a carry out of the innermost row axis: credit the pending mass of each changing axis
  // with its old digit and hand it to the axis above (Algorithm 3's carry, lazily)
  auto carry = [&]() {
    __int128 pend = Qh;
    Qh = 0;
    int i = s - 2;
    while (true) {
      __int128 tot = pend;
      if (i < s - 2) { tot += Qa[i]; Qa[i] = 0; }
      mac128x32(Aa[i], tot, td[i]);
      const uint32_t nt = td[i] + 1;
      if (i > 0 && nt == (uint32_t)g.ext[i]) {
        td[i] = 0;
        pend = tot;
        --i;
        continue;
      }
      td[i] = nt;
      if (i > 0) Qa[i - 1] += tot;  // still pending for the axes above i
      else Mtot += tot;
      break;
    }
  };
  // window end: credit every pending mass, round the window's sums to f64 once, reset
  auto end_window = [&]() {
    __int128 pend = Qh;
    Qh = 0;
    for (int i = s - 2; i >= 0; --i) {
      if (i < s - 2) { pend += Qa[i]; Qa[i] = 0; }
      mac128x32(Aa[i], pend, td[i]);
    }
    Mtot += pend;
    if (EW != 0) {
      const int sc = EW - 1075;
      for (int i = 0; i + 1 < s; ++i) { Ad[i] += fixed_to_double(Aa[i], sc); Aa[i] = 0; }
      Ad[s - 1] += fixed_to_double(S1, sc);
      Ad[D] += fixed_to_double(Mtot, sc);
      for (int a = s; a < D; ++a) {
        __int128 acc = 0;
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (colok >> j & 1u) mac64x32(acc, cs[j], mx_col_digit(g, (uint32_t)(cbase + 32 * j), a));
        Ad[a] += fixed_to_double(acc, sc);
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j) cs[j] = 0;
    S1 = 0;
    Mtot = 0;
    EW = 0;
  };
  // one row: v[j] holds the bits of column slot j (0 where the column is outside C)
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
        const long long c = (long long)(((unsigned long long)(mh >> sh) << 32) | __funnelshift_r(lo, mh, sh));
        cs[j] += c;
        rp += c;
      }
    } else if (__all_sync(0xffffffffu, steady && EW >= 54)) {
      // zeros, subnormals and tiny values too (a window exponent of 54 or more sends them to
      // 0 or their exact fixed-point value): one clamped 64-bit shift
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
      // anything else: the row's largest finite exponent first, so that the whole row
      // converts at one scale, then the general conversion out of line
      const int emax = mx_row_emax<J>(v);
      if (emax > EW) rebase(emax);
      long long c[J];
      const unsigned spec = mx_convert_general<J>(v, EW, c);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        cs[j] += c[j];
        rp += c[j];
      }
      if (spec) {
        if (!special) {
          for (int i = 0; i <= D; ++i) sp[i] = 0.0;
          special = true;
        }
        for (int j = 0; j < J; ++j)
          if (spec >> j & 1u)
            mx_special(g, __longlong_as_double((long long)v[j]), td, t1, (uint32_t)(cbase + 32 * j), sp);
      }
    }
    mac64x32(S1, rp, t1);
    Qh += rp;
    if (++t1 == E1) {
      t1 = 0;
      carry();
    }
    if (++wrow == g.win) {
      end_window();
      wrow = 0;
    }
  };
  // ---- staged rows: lane 0 copies each row's tile segment into one of the warp's NS stages
  // with a bulk copy (widened to 16-byte bounds; completion on the stage's mbarrier), so
  // NS - 1 rows are in flight while one is summed
  unsigned char* stages = dsm + (size_t)warp * kMxStages * kMxStageBytes;
  const long long c0 = tile * 32 * J;                     // first column of the tile
  const long long ncols = g.C - c0 < 32 * J ? g.C - c0 : 32 * J;
  const bool full_tile = ncols == 32 * J;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
  auto seg_start = [&](long long r) { return pb + (r * g.C + c0) * 8; };
  auto issue = [&](long long r, int q) {
    const unsigned long long a = reinterpret_cast<unsigned long long>(seg_start(r));
    const unsigned long long a16 = a & ~15ull, e16 = (a + 8 * ncols + 15) & ~15ull;
    const unsigned nb = (unsigned)(e16 - a16);
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
    // this lane's earlier reads of the stage (generic proxy) come before the async write
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(nb) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            (unsigned)__cvta_generic_to_shared(stages + q * kMxStageBytes)),
        "l"(a16), "r"(nb), "r"(bar)
        : "memory");
  };
  unsigned phase = 0;          // parity of the current use of each stage
  long long issued = r0;       // next row to stage
  bool timed_out = false;
  if (r1 > r0) {
    if (lane == 0)
      for (int q = 0; q < kMxStages && issued < r1; ++q) issue(issued++, q);
    else
      issued = r0 + (r1 - r0 < kMxStages ? r1 - r0 : kMxStages);
    int q = 0;
    long long r = r0;
    for (; r < r1; ++r) {
      const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bar, (phase >> q) & 1u, kWaitLimit));
      if (!ok) {  // the copy did not land: record it and stop (results are not to be used)
        if (lane == 0) atomicExch(&g_mx_flag, 1);
        timed_out = true;
        break;
      }
      phase ^= 1u << q;
      const unsigned char* buf = stages + q * kMxStageBytes +
                                 (reinterpret_cast<unsigned long long>(seg_start(r)) & 15ull);
      unsigned long long v[J];
      if (full_tile) {
#pragma unroll
        for (int j = 0; j < J; ++j) v[j] = *reinterpret_cast<const unsigned long long*>(buf + 8 * (lane + 32 * j));
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j)
          v[j] = (colok >> j & 1u) ? *reinterpret_cast<const unsigned long long*>(buf + 8 * (lane + 32 * j)) : 0ull;
      }
      __syncwarp();
      if (issued < r1) {
        if (lane == 0) issue(issued, q);
        ++issued;
      }
      row(v);
      if (++q == kMxStages) q = 0;
    }
    if (timed_out) {
      // rows r .. issued-1 may still be in flight into this warp's stages (each stage holds
      // at most one of them): wait for them, bounded, before the CTA's shared memory goes
      for (long long x = r; x < issued; ++x) {
        const int k = (int)((x - r0) % kMxStages);
        const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][k]);
        mbar_wait_bounded(bar, (phase >> k) & 1u, kWaitLimit);
      }
    }
    end_window();
  }

  // warp sum of the lane totals: exact in 128-bit fixed point relative to the warp's largest
  // exponent (integer shuffles), or an f64 xor-order sum when a lane holds a non-finite value
  auto reduce_out = [&](double v, int slot) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FFull);
    if (__any_sync(0xffffffffu, e == 0x7FF)) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) wsum[warp][slot] = v;
      return;
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
    if (lane == 0) wsum[warp][slot] = fixed_to_double(x, ew - 1139);
  };
#pragma unroll 1
  for (int i = 0; i <= D; ++i) reduce_out(special ? Ad[i] + sp[i] : Ad[i], i);
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

void mx_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_mx_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_mx_flag, &zero, sizeof(int));
  *flag = v;
}

}  // namespace triot
