// f32 / bf16 / f16 moment for tensors whose trailing axes form short blocks (Algorithms 10
// and 11), accumulated in f32.
//
// The last m axes (B <= 16 elements together) form a block; the axes in front of them are
// the outer axes 0 .. DO-1.  The tensor is cut into rounds of 32 chunks, a chunk being K
// whole blocks (a whole number of 16-byte pieces, at least 128 bytes).  Each warp owns a
// contiguous range of rounds and stages one round at a time into shared memory (one bulk
// TMA copy, cp.async.bulk completing on an mbarrier, when the lane rows need no padding;
// 16-byte cp.async tracked by the same mbarrier otherwise); lane l sums chunk l.  A lane
// visits blocks b, b+1, .., b+K-1 and then jumps 32K-K+1 blocks to its chunk of the next
// round: its tuple advances by one (advance_tuple, Algorithm 3) or by a constant whose
// mixed-radix digits are precomputed.
//
// Per element the work is two f32 adds: the element's column sum cs[j] (registers; B is a
// template parameter), which gives the block axes' moments sum_j cs[j] * digit_a(j), and
// its share of the block's mass (a tree over the block).  Per block the mass is credited to
// the three innermost outer axes (A += mass * digit) and added to the pending mass of the
// axes above, which is credited to an axis (A_i += pending * t_i) only when its digit
// changes.
//
// Accuracy: every plain f32 sum of a lane runs over at most kB32Terms terms (a window is at
// most kB32Terms blocks of a lane); at the window end each sum is added across the warp in
// f32 (a fixed xor tree) into the warp's compensated f32 totals (two-sum pairs), which are
// added in f64 at the end.  Block masses are trees of at most 16 elements and the block
// axes' moments sums of at most 16 products, so every output is within about (kB32Terms +
// 30) * 2^-24 (5.6e-6) of sum |p| t_i.  Non-finite elements propagate as in a plain sum (an
// infinite mass times a zero digit gives NaN, as in the definition); finite data whose
// partial sums exceed the f32 range overflow to inf.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

#include "blk32.cuh"
#include "common.cuh"
#include "fixed.cuh"
#include "float_moment.cuh"
#include "kernels.h"

namespace triot {
namespace {

// set when a bounded wait for a staged round gives up (read by triot_device_status)
__device__ int g_b32_flag = 0;

template <typename T, int B>
__global__ void __launch_bounds__(kB32Warps * 32) moment_b32_kernel(
    const __grid_constant__ MomentGeom g, const T* __restrict__ p, double* __restrict__ partial) {
  constexpr int ES = sizeof(T);
  constexpr int K = b32_blocks_per_chunk(B, ES);
  constexpr int CB = K * B;                      // elements per chunk (one lane, one round)
  constexpr int EPP = 16 / ES;                   // elements per 16-byte piece
  constexpr int H = CB / EPP;                    // pieces per chunk
  constexpr int ROW = b32_row_bytes(B, ES);      // staged bytes per chunk
  constexpr int PAD = ROW - CB * ES;             // 0 or 16
  constexpr int NW = kB32Warps;
  constexpr int NS = kB32Stages;
  constexpr int TH = NW * 32;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float wtot[NW][2][kMaxRank + 1];    // the warps' totals: compensated f32 pairs
  __shared__ float s_dig[4][16];                 // digit of block column j on block axis a
  __shared__ uint32_t s_jd[kMaxRank];            // digits of the round jump per outer axis
  __shared__ __align__(8) unsigned long long s_bar[NW][NS];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, m = g.m, DO = D - m;
  if (threadIdx.x < 16) {
    uint32_t u = threadIdx.x;
    for (int a = 0; a < 4; ++a) s_dig[a][threadIdx.x] = 0.f;
    for (int a = D - 1; a >= DO; --a) {
      const uint32_t e = (uint32_t)g.ext[a];
      s_dig[a - DO][threadIdx.x] = (float)(u % e);
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
  if (lane == 0) {
    for (int q = 0; q < NS; ++q) {
      const unsigned a = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i <= kMaxRank; ++i) wtot[warp][0][i] = wtot[warp][1][i] = 0.f;
  }
  __syncthreads();

  const long long W = (long long)gridDim.x * NW;
  const long long gw = (long long)blockIdx.x * NW + warp;
  const long long r0 = g.nround * gw / W, r1 = g.nround * (gw + 1) / W;  // this warp's rounds
  const long long nbytes = g.n * ES;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);
  // extents of axes DO-1, DO-2, DO-3 (the outermost axis never wraps inside the tensor)
  const uint32_t E1 = DO >= 2 ? (uint32_t)g.ext[DO - 1] : 0xFFFFFFFFu;
  const uint32_t E2 = DO >= 3 ? (uint32_t)g.ext[DO - 2] : 0xFFFFFFFFu;
  const uint32_t E3 = DO >= 4 ? (uint32_t)g.ext[DO - 3] : 0xFFFFFFFFu;
  const uint32_t j1 = DO >= 1 ? s_jd[DO - 1] : 0u;
  const uint32_t j2 = DO >= 2 ? s_jd[DO - 2] : 0u;
  const uint32_t j3 = DO >= 3 ? s_jd[DO - 3] : 0u;
  int jtop = DO;  // outermost axis above DO-3 that the jump changes by itself (DO: none)
  for (int i = DO - 4; i >= 0; --i)
    if (s_jd[i] != 0u) jtop = i;
  const bool jcold = jtop < DO;

  // round r (32 chunks, contiguous) into stage q
  auto stage_round = [&](long long r, int q) {
    unsigned char* buf = dsm + ((size_t)warp * NS + q) * 32 * ROW;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
    const long long base = r * (32ll * CB * ES);
    constexpr unsigned kBytes = 32u * CB * ES;
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
          fm_cp16(dst, pb + off, 16);
        } else {
          const long long rem = nbytes - off;
          const int nb = rem >= 16 ? 16 : (rem > 0 ? (int)rem : 0);
          fm_cp16(dst, nb ? (const void*)(pb + off) : (const void*)pb, nb);
        }
      }
      // the stage's mbarrier also waits for this lane's copies
      asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    } else {
      for (int i = lane; i < 32 * CB; i += 32) {
        const int row = i / CB, off = i - row * CB;
        const long long idx = r * (32ll * CB) + i;
        unsigned char* d = buf + row * ROW + off * ES;
        if (ES == 4) {
          *reinterpret_cast<unsigned*>(d) = idx < g.n ? reinterpret_cast<const unsigned*>(p)[idx] : 0u;
        } else {
          *reinterpret_cast<unsigned short*>(d) =
              idx < g.n ? reinterpret_cast<const unsigned short*>(p)[idx] : (unsigned short)0;
        }
      }
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  };
  // bounded wait for stage q's copy; on time-out the sticky device flag is set and the
  // (incomplete) stage is used anyway, so the kernel ends
  unsigned phase = 0;
  auto wait_stage = [&](int q) {
    fm_wait((unsigned)__cvta_generic_to_shared(&s_bar[warp][q]), (phase >> q) & 1u, lane, &g_b32_flag);
    phase ^= 1u << q;
  };

  // ---- lane state
  float cs[B];                            // column sums of the window
  float A1 = 0.f, A2 = 0.f, A3 = 0.f;     // axes DO-1, DO-2, DO-3: sum of mass * digit
  float Q4 = 0.f;                         // mass not yet credited to axis DO-4 (or the mass)
  float Mtot = 0.f;                       // mass that left the outermost level
  uint32_t t1 = 0, t2 = 0, t3 = 0;        // digits of axes DO-1, DO-2, DO-3
#pragma unroll
  for (int j = 0; j < B; ++j) cs[j] = 0.f;
  // the sums, digits and pending masses of axes 0 .. DO-4: lane-major dynamic shared memory
  // after the stages (touched at carries and window ends; run-time axis index)
  unsigned char* st_base = dsm + (size_t)b32_stage_bytes(B, ES);
  const LaneCol<float, TH> Ac{reinterpret_cast<float*>(st_base) + threadIdx.x};
  st_base += (size_t)b32_levels(DO) * TH * 4;
  const LaneCol<uint32_t, TH> tc{reinterpret_cast<uint32_t*>(st_base) + threadIdx.x};
  st_base += (size_t)b32_levels(DO) * TH * 4;
  const LaneCol<float, TH> Qc{reinterpret_cast<float*>(st_base) + threadIdx.x};
  for (int i = 0; i < b32_levels(DO); ++i) { Ac[i] = 0.f; tc[i] = 0; }
  for (int i = 0; i < b32_qlevels(DO); ++i) Qc[i] = 0.f;

  // digits of axes DO-4 .. 0 advance by inc_i = (jump digit if `jump`) + carry.  First the
  // outermost axis that changes (h); then every axis from DO-4 up to h hands its pending
  // mass to the axis above, crediting it with its current digit first, so no mass is
  // credited with a wrong digit.
  auto cold_step = [&](uint32_t carry_in, bool jump) {
    int h = -1;
    {
      uint32_t carry = carry_in;
      for (int i = DO - 4; i >= 0; --i) {
        const uint32_t inc = (jump ? s_jd[i] : 0u) + carry;
        if (inc) h = i;
        carry = (i > 0 && tc[i] + inc >= (uint32_t)g.ext[i]) ? 1u : 0u;
        if (!carry && (!jump || i <= jtop)) break;
      }
    }
    if (h < 0) return;
    uint32_t carry = carry_in;
    float pend = Q4;
    Q4 = 0.f;
    for (int i = DO - 4; i >= h; --i) {
      const uint32_t t = tc[i];
      Ac[i] = fmaf(pend, (float)t, Ac[i]);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0.f;
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
  // a block's mass: credited to the eager axes, pending for the others; then the next block
  auto block_end = [&](float bm, bool last_in_chunk) {
    A1 = fmaf(bm, (float)t1, A1);
    if (DO >= 2) A2 = fmaf(bm, (float)t2, A2);
    if (DO >= 3) A3 = fmaf(bm, (float)t3, A3);
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
  // one window sum of every lane into the warp's compensated total
  auto warp_add = [&](float v, int slot) { fm_warp_add(v, &wtot[warp][0][slot], &wtot[warp][1][slot], lane); };
  // window end: credit every pending mass, move the window's sums into the warp's totals
  auto end_window = [&]() {
    float pend = Q4;
    Q4 = 0.f;
    for (int i = DO - 4; i >= 0; --i) {
      Ac[i] = fmaf(pend, (float)tc[i], Ac[i]);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0.f;
      }
    }
    Mtot += pend;
    if (DO >= 1) warp_add(A1, DO - 1);
    if (DO >= 2) warp_add(A2, DO - 2);
    if (DO >= 3) warp_add(A3, DO - 3);
    for (int i = 0; i + 3 < DO; ++i) {
      warp_add(Ac[i], i);
      Ac[i] = 0.f;
    }
    warp_add(Mtot, D);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (a >= m) break;
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < B; ++j) s = fmaf(cs[j], s_dig[a][j], s);
      warp_add(s, DO + a);
    }
#pragma unroll
    for (int j = 0; j < B; ++j) cs[j] = 0.f;
    A1 = 0.f;
    A2 = 0.f;
    A3 = 0.f;
    Mtot = 0.f;
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

  long long ri = r0;  // next round to stage
#pragma unroll
  for (int q = 0; q < NS - 1; ++q)
    if (ri < r1) stage_round(ri++, q);
  // window phases staggered across warps (the window ends of warps sharing an SM spread out)
  int buf = 0, wpos = (int)(gw % g.win);
  for (long long s = 0; s < nsteps; ++s) {
    wait_stage(buf);
    __syncwarp();
    if (ri < r1) stage_round(ri++, buf == 0 ? NS - 1 : buf - 1);
    const unsigned char* row = dsm + ((size_t)warp * NS + buf) * 32 * ROW + lane * ROW;
    uint4 v[H];
#pragma unroll
    for (int h = 0; h < H; ++h) v[h] = *reinterpret_cast<const uint4*>(row + 16 * h);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float cb[B];
#pragma unroll
      for (int j = 0; j < B; ++j) {
        const int idx = k * B + j;
        const float x = FPiece<T>::get(v[idx / EPP], idx % EPP);
        cs[j] += x;
        cb[j] = x;
      }
#pragma unroll
      for (int w = 1; w < B; w *= 2)
#pragma unroll
        for (int q = 0; q + w < B; q += 2 * w) cb[q] += cb[q + w];
      block_end(cb[0], k == K - 1);
    }
    if (++wpos == g.win || s + 1 == nsteps) {
      end_window();
      wpos = 0;
    }
    if (++buf == NS) buf = 0;
    __syncwarp();
  }

  __syncthreads();
  if (threadIdx.x <= D) partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = fm_cta_total<NW>(wtot, threadIdx.x);
}

template <typename T, int... N>
const void* pick(int b, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_b32_kernel<T, N + 1>)...};
  return table[b - 1];
}

}  // namespace

void b32_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_b32_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_b32_flag, &zero, sizeof(int));
  *flag = v;
}

// block sizes 1 .. 16 (1: a single element, every extent 1)
const void* moment_blk32_kernel_ptr(int dtype, int B) {
  if (B < 1 || B > 16) return nullptr;
  auto seq = std::make_integer_sequence<int, 16>{};
  switch (dtype) {
    case DT_F32: return pick<float>(B, seq);
    case DT_BF16: return pick<__nv_bfloat16>(B, seq);
    case DT_F16: return pick<__half>(B, seq);
  }
  return nullptr;
}

}  // namespace triot
