// f64 moment for tensors whose trailing axes form short blocks (Algorithms 10 and 11),
// in exact fixed point.
//
// The last m axes (B <= 16 elements together) form a block; the axes in front of them are
// the outer axes 0 .. DO-1.  The tensor is cut into rounds of 32 chunks, a chunk being K
// whole blocks (CB = K*B elements, 16..30).  Each warp owns a contiguous range of rounds;
// per round it stages the round's 32*CB contiguous elements into shared memory with one bulk
// TMA copy (cp.async.bulk, completion on an mbarrier; rows padded for conflict-free reads
// take 16-byte cp.async instead) and lane l sums chunk l.  So a lane visits blocks b, b+1, .., b+K-1,
// then jumps by 32K-K+1 blocks to its chunk of the next round: its tuple advances by one
// (advance_tuple, Algorithm 3) or by a constant whose mixed-radix digits are precomputed.
//
// Fixed point: within a window (at most kB64Window elements of a lane) every element is the
// integer c = m >> (E_W - e) in units of 2^(E_W - 1075), e its biased exponent, m its 53-bit
// significand and E_W the largest exponent the window has seen (the sums shift right when
// E_W grows).  Per lane and window:
//   * column sums cs[j] (64-bit, one register pair per column; B is a template parameter),
//     which give the block axes' moments sum_j cs[j] * digit_a(j) at the window end;
//   * the three innermost outer axes summed eagerly once per chunk from its block masses:
//     the chunk's K blocks cross at most one wrap of axis DO-1 (when K <= its extent), so
//     they split into two runs with fixed digits, and A1 += t1 * M + sum_k k bm_k - E1 * Mb,
//     A2 += t2 * Ma + t2' * Mb, A3 likewise (M = Ma + Mb the masses before and after the
//     wrap); lanes with different digits run the same instructions;
//   * the remaining outer axes summed lazily: a chunk's mass waits in the pending mass of
//     axis DO-4 and is credited (A_i += pending * t_i) only when t_i changes, then moves up.
// At the window end the sums are rounded once to f64 and added to the lane's f64 totals.
// Truncation below the window maximum's last bit bounds the error of every output by
// 2^-52 * max|p| (over the window) per element; relative to sum |p| t_i that is at most
// kB64Window * 2^-52 (2.3e-13), and for data of similar magnitudes near 2^-52.  Non-finite
// elements are summed separately in f64 so that they propagate as they would in a plain sum.
#include <utility>

#include "kernels.h"
#include "moment.cuh"
#include "sync.cuh"

namespace triot {
namespace {

// set when a bounded wait for a bulk copy gives up (read by triot_device_status)
__device__ int g_b64_flag = 0;

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// non-finite element: plain f64 sums of v * t_i (rare; kept out of line)
__device__ __noinline__ void add_special(double v, uint32_t t1, uint32_t t2, uint32_t t3,
                                         LaneCol<uint32_t, kB64Warps * 32> tc, int DO, int m,
                                         const unsigned char* dig_j, double* Asp, double* Isp,
                                         double* Psp) {
  if (DO >= 1) Asp[DO - 1] += v * (double)t1;
  if (DO >= 2) Asp[DO - 2] += v * (double)t2;
  if (DO >= 3) Asp[DO - 3] += v * (double)t3;
  for (int i = 0; i + 3 < DO; ++i) Asp[i] += v * (double)tc[i];
  for (int a = 0; a < m; ++a) Isp[a] += v * (double)dig_j[a * 16];
  *Psp += v;
}

template <int B>
__global__ void __launch_bounds__(kB64Warps * 32, 6) moment_b64_kernel(
    const __grid_constant__ MomentGeom g, const double* __restrict__ p,
    double* __restrict__ partial) {
  constexpr int K = b64_blocks_per_chunk(B);
  constexpr int CB = K * B;                          // elements per chunk (one lane, one round)
  constexpr int H = CB / 2;                          // 16-byte pieces per chunk
  constexpr int ROW = b64_row_bytes(B);              // staged bytes per chunk
  constexpr int PAD = ROW - CB * 8;                  // 0 or 16
  constexpr int NW = kB64Warps;
  constexpr int NS = kB64Stages;
  constexpr int T = NW * 32;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double wsum[NW][kMaxRank + 1];
  __shared__ unsigned char s_dig[4][16];             // digits of block column j on block axis a
  __shared__ uint32_t s_jd[kMaxRank];                // digits of the round jump per outer axis
  __shared__ __align__(8) unsigned long long s_bar[NW][NS];  // one mbarrier per stage

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, m = g.m, DO = D - m;
  if (threadIdx.x < 16) {
    uint32_t u = threadIdx.x;
    for (int a = 0; a < 4; ++a) s_dig[a][threadIdx.x] = 0;
    for (int a = D - 1; a >= DO; --a) {
      const uint32_t e = (uint32_t)g.ext[a];
      s_dig[a - DO][threadIdx.x] = (unsigned char)(u % e);
      u /= e;
    }
  }
  if (threadIdx.x == 32) {
    // a lane's next block after its chunk is 32K - K + 1 blocks on; the outermost axis keeps
    // the remainder (it never wraps inside the tensor)
    uint32_t J = 32u * K - (K - 1);  // below 2^32: magic-number division (Alg 4)
    for (int a = DO - 1; a >= 1; --a) {
      const uint32_t q = fdiv(J, g.div[a]);
      s_jd[a] = J - q * g.div[a].d;
      J = q;
    }
    if (DO >= 1) s_jd[0] = J;
  }
  if ((threadIdx.x & 31) == 0) {
    for (int q = 0; q < NS; ++q) {
      const unsigned a = (unsigned)__cvta_generic_to_shared(&s_bar[threadIdx.x >> 5][q]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long W = (long long)gridDim.x * NW;
  const long long gw = (long long)blockIdx.x * NW + warp;
  const long long r0 = g.nround * gw / W, r1 = g.nround * (gw + 1) / W;  // this warp's rounds
  const long long nbytes = g.n * 8;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
  // extents of axes DO-1, DO-2, DO-3 (the outermost axis never wraps inside the tensor)
  const uint32_t E1 = DO >= 2 ? (uint32_t)g.ext[DO - 1] : 0xFFFFFFFFu;
  const uint32_t E2 = DO >= 3 ? (uint32_t)g.ext[DO - 2] : 0xFFFFFFFFu;
  const uint32_t E3 = DO >= 4 ? (uint32_t)g.ext[DO - 3] : 0xFFFFFFFFu;
  const uint32_t j1 = DO >= 1 ? s_jd[DO - 1] : 0u;
  const uint32_t j2 = DO >= 2 ? s_jd[DO - 2] : 0u;
  const uint32_t j3 = DO >= 3 ? s_jd[DO - 3] : 0u;
  bool jcold = false;  // the jump changes a digit above axis DO-3 by itself
  for (int i = 0; i + 3 < DO; ++i) jcold = jcold || s_jd[i] != 0u;
  const bool per_round = (uint32_t)K <= E1;  // a chunk crosses at most one wrap of axis DO-1

  // round r (32 chunks, contiguous) into stage q.  Dense rows (PAD == 0) of an aligned,
  // complete round: one bulk copy issued by lane 0, completing on the stage's mbarrier.
  // Otherwise the lanes copy 16-byte pieces (cp.async, tracked by the same mbarrier) or
  // elements (unaligned input), and lane 0 adds the one expected arrival after them.
  auto stage_round = [&](long long r, int q) {
    unsigned char* buf = dsm + ((size_t)warp * NS + q) * 32 * ROW;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
    const long long base = r * (32ll * CB * 8);
    constexpr unsigned kBytes = 32u * CB * 8u;
    const bool full = base + (long long)kBytes <= nbytes;
    if (g.aligned && full && PAD == 0) {
      if (lane == 0) {
        // the lanes' reads of this stage (previous use) precede the async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(kBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                (unsigned)__cvta_generic_to_shared(buf)),
            "l"(pb + base), "r"(kBytes), "r"(bar)
            : "memory");
      }
      return;
    }
    if (g.aligned) {
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const int pc = h * 32 + lane;
        unsigned char* dst = buf + pc * 16 + (pc / H) * PAD;
        const long long off = base + (long long)pc * 16;
        if (full) {
          cp_async16(dst, pb + off, 16);
        } else {
          const long long rem = nbytes - off;
          const int nb = rem >= 16 ? 16 : (rem > 0 ? (int)rem : 0);
          cp_async16(dst, nb ? (const void*)(pb + off) : (const void*)pb, nb);
        }
      }
      // the stage's mbarrier also waits for this lane's copies (pending count +1 now, the
      // arrival when they land)
      asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    } else {
      for (int i = lane; i < 32 * CB; i += 32) {
        const int row = i / CB, off = i - row * CB;
        const long long idx = r * (32ll * CB) + i;
        *reinterpret_cast<unsigned long long*>(buf + row * ROW + off * 8) =
            idx < g.n ? reinterpret_cast<const unsigned long long*>(p)[idx] : 0ull;
      }
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  };
  // bounded wait for stage q's copy (parity of its current use); on time-out the sticky
  // device flag is set and the (incomplete) stage is used anyway, so the kernel ends
  unsigned phase = 0;
  auto wait_stage = [&](int q) {
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
    const unsigned par = (phase >> q) & 1u;
    if (!mbar_wait_bounded(bar, par, kWaitLimit) && lane == 0) atomicExch(&g_b64_flag, 1);
    phase ^= 1u << q;
  };

  // ---- lane state (window sums in fixed point)
  long long cs[B];                      // column sums
  __int128 A1 = 0, A2 = 0, A3 = 0;      // axes DO-1, DO-2, DO-3: sum of mass * digit
  __int128 Q4 = 0;                      // mass not yet credited to axis DO-4 (or the mass)
  __int128 Mtot = 0;                    // mass that left the outermost level
  uint32_t t1 = 0, t2 = 0, t3 = 0;      // digits of axes DO-1, DO-2, DO-3
  int es = 0;                           // window exponent (0: nothing seen)
#pragma unroll
  for (int j = 0; j < B; ++j) cs[j] = 0;
  // axes 0 .. DO-4 and the lane's f64 totals: lane-major dynamic shared memory after the
  // stages (touched at carries and window ends; run-time axis index)
  unsigned char* st_base = dsm + (size_t)b64_stage_bytes(B);
  const LaneCol<__int128, T> Ac{reinterpret_cast<__int128*>(st_base) + threadIdx.x};
  st_base += (size_t)b64_levels(DO) * T * 16;
  const LaneCol<__int128, T> Qc{reinterpret_cast<__int128*>(st_base) + threadIdx.x};
  st_base += (size_t)b64_qlevels(DO) * T * 16;
  const LaneCol<double, T> Ads{reinterpret_cast<double*>(st_base) + threadIdx.x};
  st_base += (size_t)DO * T * 8;
  const LaneCol<uint32_t, T> tc{reinterpret_cast<uint32_t*>(st_base) + threadIdx.x};
  for (int i = 0; i < b64_levels(DO); ++i) { Ac[i] = 0; tc[i] = 0; }
  for (int i = 0; i < b64_qlevels(DO); ++i) Qc[i] = 0;
  for (int i = 0; i < DO; ++i) Ads[i] = 0.0;
  double Asp[kMaxRank];  // non-finite elements (local memory; written only when one occurs)
  double Ind[4] = {0.0, 0.0, 0.0, 0.0}, Isp[4] = {0.0, 0.0, 0.0, 0.0};
  double Md = 0.0, Psp = 0.0;
  bool special = false;

  auto rebase = [&](int e_new) {
    if (es != 0) {
      const int d = e_new - es;
#pragma unroll
      for (int j = 0; j < B; ++j) cs[j] = shr64(cs[j], d);
      A1 = shr_arith(A1, d);
      A2 = shr_arith(A2, d);
      A3 = shr_arith(A3, d);
      Q4 = shr_arith(Q4, d);
      Mtot = shr_arith(Mtot, d);
      for (int i = 0; i < b64_levels(DO); ++i) Ac[i] = shr_arith(Ac[i], d);
      for (int i = 0; i < b64_qlevels(DO); ++i) Qc[i] = shr_arith(Qc[i], d);
    }
    es = e_new;
  };
  // digits of axes DO-4 .. 0 advance by inc_i = (jump digit if `jump`) + carry.  Every axis
  // up to the outermost one that changes first hands its pending mass to the axis above
  // (crediting it with its current digit), so no mass is ever credited with a wrong digit.
  auto cold_step = [&](uint32_t carry_in, bool jump) {
    int h = -1;  // outermost changing axis
    {
      uint32_t carry = carry_in;
      for (int i = DO - 4; i >= 0; --i) {
        const uint32_t inc = (jump ? s_jd[i] : 0u) + carry;
        if (inc) h = i;
        carry = (i > 0 && tc[i] + inc >= (uint32_t)g.ext[i]) ? 1u : 0u;
        if (!jump && !carry) break;
      }
    }
    if (h < 0) return;
    uint32_t carry = carry_in;
    __int128 pend = Q4;
    Q4 = 0;
    for (int i = DO - 4; i >= h; --i) {
      const uint32_t t = tc[i];
      mac128x32(Ac[i], pend, t);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0;
      } else {
        Mtot += pend;
      }
      const uint32_t inc = (jump ? s_jd[i] : 0u) + carry;
      uint32_t nt = t + inc;
      carry = 0;
      if (i > 0 && nt >= (uint32_t)g.ext[i]) {
        nt -= (uint32_t)g.ext[i];
        carry = 1;
      }
      tc[i] = nt;
    }
    if (h > 0) Qc[h - 1] += pend;
  };
  // from a chunk's last block to the lane's first block of its next round
  auto jump = [&]() {
    t1 += j1;
    const uint32_t c1 = t1 >= E1 ? 1u : 0u;
    t1 -= c1 ? E1 : 0u;
    t2 += j2 + c1;
    const uint32_t c2 = t2 >= E2 ? 1u : 0u;
    t2 -= c2 ? E2 : 0u;
    t3 += j3 + c2;
    const uint32_t c3 = t3 >= E3 ? 1u : 0u;
    t3 -= c3 ? E3 : 0u;
    if (c3 || jcold) cold_step(c3, jcold);
  };
  // one block at a time (chunks with non-finite or unusual elements, or K > E1)
  auto block_end = [&](long long bm, bool last_in_chunk) {
    mac64x32(A1, bm, t1);
    if (DO >= 2) mac64x32(A2, bm, t2);
    if (DO >= 3) mac64x32(A3, bm, t3);
    Q4 += bm;
    if (!last_in_chunk) {
      const uint32_t w1 = (++t1 == E1) ? 1u : 0u;
      t1 = w1 ? 0u : t1;
      t2 += w1;
      const uint32_t w2 = (t2 == E2) ? 1u : 0u;
      t2 = w2 ? 0u : t2;
      t3 += w2;
      const uint32_t w3 = (t3 == E3) ? 1u : 0u;
      t3 = w3 ? 0u : t3;
      if (w3) cold_step(1u, false);
    } else {
      jump();
    }
  };
  // a whole chunk from its K block masses (K <= E1: at most one wrap of axis DO-1, after
  // block kw = E1 - t1); then the jump to the next round
  auto chunk_end = [&](const long long (&bmv)[K]) {
    long long M = 0, Wk = 0, Mb = 0;
    const uint32_t kw = E1 - t1;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      M += bmv[k];
      Wk += (long long)k * bmv[k];
      Mb += ((uint32_t)k >= kw) ? bmv[k] : 0ll;
    }
    const long long Ma = M - Mb;
    const bool wrap1 = kw < (uint32_t)K;
    uint32_t t2b = t2, t3b = t3;
    bool c3 = false;
    if (wrap1) {
      t2b = t2 + 1;
      if (t2b == E2) {
        t2b = 0;
        t3b = t3 + 1;
        if (t3b == E3) {
          t3b = 0;
          c3 = true;
        }
      }
    }
    mac64x32(A1, M, t1);
    A1 += Wk;
    mac64x32(A1, -Mb, E1);
    if (DO >= 2) {
      mac64x32(A2, Ma, t2);
      mac64x32(A2, Mb, t2b);
    }
    if (DO >= 3) {
      mac64x32(A3, Ma, t3);
      mac64x32(A3, Mb, t3b);
    }
    if (!c3) {
      Q4 += M;
    } else {
      Q4 += Ma;
      cold_step(1u, false);
      Q4 += Mb;
    }
    t1 = t1 + (uint32_t)(K - 1) - (wrap1 ? E1 : 0u);
    t2 = t2b;
    t3 = t3b;
    jump();
  };
  // window end: credit every pending mass, round the window's sums to f64 once
  auto end_window = [&]() {
    __int128 pend = Q4;
    Q4 = 0;
    for (int i = DO - 4; i >= 0; --i) {
      mac128x32(Ac[i], pend, tc[i]);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0;
      }
    }
    Mtot += pend;
    if (es != 0) {
      const int sc = es - 1075;
      if (DO >= 1) Ads[DO - 1] += fixed_to_double(A1, sc);
      if (DO >= 2) Ads[DO - 2] += fixed_to_double(A2, sc);
      if (DO >= 3) Ads[DO - 3] += fixed_to_double(A3, sc);
      for (int i = 0; i + 3 < DO; ++i) Ads[i] += fixed_to_double(Ac[i], sc);
      Md += fixed_to_double(Mtot, sc);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        if (a >= m) break;
        __int128 s = 0;
#pragma unroll
        for (int j = 0; j < B; ++j) mac128(s, cs[j], (long long)s_dig[a][j]);
        Ind[a] += fixed_to_double(s, sc);
      }
    }
#pragma unroll
    for (int j = 0; j < B; ++j) cs[j] = 0;
    A1 = 0;
    A2 = 0;
    A3 = 0;
    Mtot = 0;
    for (int i = 0; i < b64_levels(DO); ++i) Ac[i] = 0;
    es = 0;
  };

  const long long nsteps = r1 - r0;
  if (nsteps > 0) {
    // tuple of this lane's first block (the outermost axis takes the remainder)
    const long long blk = (r0 * 32 + lane) * K;
    auto set_digit = [&](int a, uint32_t v) {
      if (a == DO - 1) t1 = v;
      else if (a == DO - 2) t2 = v;
      else if (a == DO - 3) t3 = v;
      else tc[a] = v;
    };
    if (g.n32) {
      uint32_t r32 = (uint32_t)blk;
      for (int a = DO - 1; a >= 1; --a) {
        const uint32_t q = fdiv(r32, g.div[a]);
        set_digit(a, r32 - q * g.div[a].d);
        r32 = q;
      }
      if (DO >= 1) set_digit(0, r32);
    } else {
      long long q = blk;
      for (int a = DO - 1; a >= 1; --a) {
        const long long q1 = q / g.ext[a];
        set_digit(a, (uint32_t)(q - q1 * g.ext[a]));
        q = q1;
      }
      if (DO >= 1) set_digit(0, (uint32_t)q);
    }
  }

  long long ri = r0;                    // next round to stage
#pragma unroll
  for (int q = 0; q < NS - 1; ++q)
    if (ri < r1) stage_round(ri++, q);
  // window phases staggered across warps, so that the window ends (a burst of work with no
  // copy in flight) of the warps sharing an SM do not coincide
  int buf = 0, wpos = (int)(gw % g.win);
  for (long long s = 0; s < nsteps; ++s) {
    wait_stage(buf);
    __syncwarp();
    if (ri < r1) stage_round(ri++, buf == 0 ? NS - 1 : buf - 1);
    const unsigned char* row = dsm + ((size_t)warp * NS + buf) * 32 * ROW + lane * ROW;
    // unsigned max / min of the high words, as trees (short dependency chains)
    uint32_t mx[H], mn[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
      const uint4 v = *reinterpret_cast<const uint4*>(row + 16 * h);
      mx[h] = max(v.y, v.w);
      mn[h] = min(v.y, v.w);
    }
#pragma unroll
    for (int w = 1; w < H; w *= 2)
#pragma unroll
      for (int h = 0; h + w < H; h += 2 * w) {
        mx[h] = max(mx[h], mx[h + w]);
        mn[h] = min(mn[h], mn[h + w]);
      }
    const uint32_t hmax = mx[0], hmin = mn[0];
    // positive, normal and finite: the lean conversion
    const bool clean = hmax < 0x7FF00000u && hmin >= 0x00100000u;
    if (clean) {
      if ((int)(hmax >> 20) > es) rebase((int)(hmax >> 20));
    } else {
      uint32_t efin = 0x00100000u;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + 16 * h);
        const uint32_t f0 = v.y & 0x7FF00000u, f1 = v.w & 0x7FF00000u;
        if (f0 != 0x7FF00000u) efin = max(efin, f0);
        if (f1 != 0x7FF00000u) efin = max(efin, f1);
      }
      if ((int)(efin >> 20) > es) rebase((int)(efin >> 20));
    }
    const uint32_t ec = (uint32_t)es;
    if (clean && ec - (hmin >> 20) < 32u) {
      long long cb[B];   // the block's elements; its mass is their sum taken as a tree
      long long bmv[K];  // the chunk's block masses
#pragma unroll
      for (int idx = 0; idx < CB; idx += 2) {
        const uint4 v = *reinterpret_cast<const uint4*>(row + 8 * idx);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t lo = h ? v.z : v.x, hi = h ? v.w : v.y;
          const uint32_t sh = ec - (hi >> 20);
          const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
          const long long c =
              (long long)(((unsigned long long)(mh >> sh) << 32) | __funnelshift_r(lo, mh, sh));
          const int j = (idx + h) % B;
          cs[j] += c;
          cb[j] = c;
          if (j == B - 1) {
#pragma unroll
            for (int w = 1; w < B; w *= 2)
#pragma unroll
              for (int q = 0; q + w < B; q += 2 * w) cb[q] += cb[q + w];
            bmv[(idx + h) / B] = cb[0];
          }
        }
      }
      if (per_round) {
        chunk_end(bmv);
      } else {
#pragma unroll
        for (int k = 0; k < K; ++k) block_end(bmv[k], k == K - 1);
      }
    } else {
      long long bm = 0;
#pragma unroll
      for (int idx = 0; idx < CB; ++idx) {
        const int j = idx % B;
        const unsigned long long b = *reinterpret_cast<const unsigned long long*>(row + 8 * idx);
        const uint32_t hi = (uint32_t)(b >> 32);
        const uint32_t ef = hi & 0x7FF00000u;
        long long c = 0;
        if (ef == 0x7FF00000u) {
          if (!special) {
            for (int i = 0; i < DO; ++i) Asp[i] = 0.0;
            special = true;
          }
          add_special(__longlong_as_double((long long)b), t1, t2, t3, tc, DO, m, &s_dig[0][j], Asp,
                      Isp, &Psp);
        } else {
          const uint32_t e = (ef > 0x00100000u ? ef : 0x00100000u) >> 20;
          const unsigned long long mm = (b & 0x000FFFFFFFFFFFFFull) | (ef ? (1ull << 52) : 0ull);
          const uint32_t sh = ec - e;
          c = (long long)(mm >> (sh < 63u ? sh : 63u));
          if ((int)hi < 0) c = -c;
        }
        cs[j] += c;
        bm += c;
        if (j == B - 1) {
          block_end(bm, idx == CB - 1);
          bm = 0;
        }
      }
    }
    if (++wpos == g.win || s + 1 == nsteps) {
      end_window();
      wpos = 0;
    }
    if (++buf == NS) buf = 0;
    __syncwarp();
  }

  // warp sum of the lane totals: exact in 128-bit fixed point relative to the warp's largest
  // exponent (integer shuffles; the narrow FP64 pipe is left alone), or an f64 xor-order sum
  // when a lane holds a non-finite value
  double* ws_out = wsum[warp];
  auto reduce_out = [&](double v, double sp, int slot) {
    if (special) v += sp;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FFull);
    if (__any_sync(0xffffffffu, e == 0x7FF)) {
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) ws_out[slot] = v;
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
    if (lane == 0) ws_out[slot] = fixed_to_double(x, ew - 1139);
  };
  for (int i = 0; i < DO; ++i) reduce_out(Ads[i], special ? Asp[i] : 0.0, i);
#pragma unroll
  for (int a = 0; a < 4; ++a)
    if (a < m) reduce_out(Ind[a], Isp[a], DO + a);
  reduce_out(Md, Psp, D);
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

template <int... N>
const void* pick(int b, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_b64_kernel<N + 1>)...};
  return table[b - 1];
}

}  // namespace

void b64_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_b64_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_b64_flag, &zero, sizeof(int));
  *flag = v;
}

const void* moment_blk64_kernel_ptr(int B, int DO) {
  if (B < 1 || B > 16 || DO < 0 || DO >= kMaxRank) return nullptr;
  return pick(B, std::make_integer_sequence<int, 16>{});
}

}  // namespace triot
