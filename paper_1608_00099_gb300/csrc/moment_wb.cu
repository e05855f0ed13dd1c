// f32 / bf16 / f16 moment for tensors whose trailing axes form blocks of 32 .. 256 elements
// (Algorithms 10 and 11), accumulated in f32: one block at a time per warp.
//
// The last m axes form a block of B elements (32 <= B <= 256); the axes in front of them
// are the outer axes 0 .. DO-1.  Each warp owns a contiguous range of blocks.  When a block
// is a whole number of 512-byte rows, lane l reads 16-byte vectors of it directly (columns
// 16/es * (l + 32 v) ..; several blocks' loads in flight); otherwise the warp walks its
// range in steps of U whole blocks (at most kWBStepBytes), each staged into shared memory
// by one bulk TMA copy (cp.async.bulk over the step widened to 16-byte bounds, completing
// on an mbarrier; 16-byte cp.async with zero fill for the tensor's last bytes), and lane l
// reads columns l, l + 32, .. (C = ceil(B / 32)).  Each element is added to the lane's
// column sum; the lane's share of the block's mass goes to the outer axes.  All lanes of a
// warp are in the same block, so the outer digits are the same in every lane: advancing the
// tuple by one block (advance_tuple, Algorithm 3) is a uniform branch.  The two innermost
// outer axes take mass * digit per block; the axes above keep a pending mass that is
// credited (A_i += pending * t_i) only when their digit changes.  The block axes' moments
// are sum_j digit_a(j) * colsum_j.
//
// Accuracy: every plain f32 sum of a lane runs over at most kWBTerms terms (a window is at
// most kWBTerms blocks); at the window end each sum is added across the warp in f32 (a
// fixed xor tree) into the warp's compensated f32 totals (two-sum pairs), added in f64 at
// the end. Every output is then within about (kWBTerms + 20) * 2^-24 (5.0e-6) of sum |p|
// t_i. Non-finite elements propagate as in a plain sum; finite data whose partial sums
// exceed the f32 range overflow to inf.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "blk32.cuh"
#include "common.cuh"
#include "fixed.cuh"
#include "float_moment.cuh"
#include "kernels.h"

namespace triot {
namespace {

// set when a bounded wait for a staged step gives up (read by triot_device_status)
__device__ int g_wb_flag = 0;

// a staged element as f32 (exact for every type)
__device__ __forceinline__ float wb_elem(const unsigned char* s, float*) {
  return *reinterpret_cast<const float*>(s);
}
__device__ __forceinline__ float wb_elem(const unsigned char* s, __nv_bfloat16*) {
  return __uint_as_float((unsigned)*reinterpret_cast<const unsigned short*>(s) << 16);
}
__device__ __forceinline__ float wb_elem(const unsigned char* s, __half*) {
  return __half2float(__ushort_as_half(*reinterpret_cast<const unsigned short*>(s)));
}

template <typename T, int C, bool VEC>
__global__ void __launch_bounds__(kWBWarps * 32, 4) moment_wb_kernel(
    const __grid_constant__ MomentGeom g, const T* __restrict__ p, double* __restrict__ partial) {
  constexpr int ES = sizeof(T);
  constexpr int NW = kWBWarps;
  constexpr int NS = kWBStages;
  constexpr int TH = NW * 32;
  constexpr int EPV = 16 / ES;                  // elements per 16-byte vector
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float s_cdig[8][kWBMaxC * 32];     // digit of block column j on block axis a
  __shared__ float wtot[NW][2][kMaxRank + 1];   // the warps' totals: compensated f32 pairs
  __shared__ __align__(8) unsigned long long s_bar[NW][NS];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, m = g.m, DO = D - m, B = g.B;
  for (int j = threadIdx.x; j < kWBMaxC * 32; j += TH) {
    uint32_t u = (uint32_t)j;
    for (int a = 0; a < 8; ++a) s_cdig[a][j] = 0.f;
    if (j < B) {
      for (int a = D - 1; a >= DO; --a) {
        const uint32_t e = (uint32_t)g.ext[a];
        s_cdig[a - DO][j] = (float)(u % e);
        u /= e;
      }
    }
  }
  if (lane == 0) {
    for (int i = 0; i <= kMaxRank; ++i) wtot[warp][0][i] = wtot[warp][1][i] = 0.f;
    for (int q = 0; q < NS; ++q) {
      const unsigned a = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long nb = g.nround;  // blocks
  const long long W = (long long)gridDim.x * NW;
  const long long gw = (long long)blockIdx.x * NW + warp;
  const long long q0 = nb * gw / W, q1 = nb * (gw + 1) / W;  // this warp's blocks
  // extents of axes DO-1 and DO-2 (the outermost axis never wraps inside the tensor)
  const uint32_t E1 = DO >= 2 ? (uint32_t)g.ext[DO - 1] : 0xFFFFFFFFu;
  const uint32_t E2 = DO >= 3 ? (uint32_t)g.ext[DO - 2] : 0xFFFFFFFFu;
  const int U = g.nchunks;                           // blocks per step
  const long long nsteps = (q1 - q0 + U - 1) / U;
  const long long nbytes = g.n * ES;
  const unsigned char* pb = reinterpret_cast<const unsigned char*>(p);

  // step st (blocks q0 + st * U ..) into stage q, widened to 16-byte bounds
  auto stage_step = [&](long long st, int q) {
    const long long qb = q0 + st * U;
    const long long ub = (q1 - qb) < U ? (q1 - qb) : U;
    unsigned char* buf = dsm + ((size_t)warp * NS + q) * kWBStageBytes;
    const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[warp][q]);
    const long long sb = qb * B * ES, eb = (qb + ub) * B * ES;
    const long long a0 = sb & ~15ll, a1 = (eb + 15) & ~15ll;
    if (g.aligned && a1 <= nbytes) {
      if (lane == 0) {
        // the lanes' reads of this stage (previous use) precede the async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((unsigned)(a1 - a0))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                (unsigned)__cvta_generic_to_shared(buf)),
            "l"(pb + a0), "r"((unsigned)(a1 - a0)), "r"(bar)
            : "memory");
      }
      return;
    }
    if (g.aligned) {
      // the tensor's last bytes: 16-byte pieces, zero-filled past its end
      for (long long off = a0 + 16 * lane; off < a1; off += 512) {
        const long long rem = nbytes - off;
        const int nbt = rem >= 16 ? 16 : (rem > 0 ? (int)rem : 0);
        fm_cp16(buf + (off - a0), nbt ? (const void*)(pb + off) : (const void*)pb, nbt);
      }
      asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
    } else {
      // unaligned base: element copies to the same offsets
      for (long long i = lane; i < ub * B; i += 32) {
        unsigned char* d = buf + (sb - a0) + i * ES;
        const long long idx = qb * B + i;
        if (ES == 4) *reinterpret_cast<unsigned*>(d) = reinterpret_cast<const unsigned*>(p)[idx];
        else *reinterpret_cast<unsigned short*>(d) = reinterpret_cast<const unsigned short*>(p)[idx];
      }
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
  };
  // bounded wait for stage q's copy; on time-out the sticky device flag is set and the
  // (incomplete) stage is used anyway, so the kernel ends
  unsigned phase = 0;
  auto wait_stage = [&](int q) {
    fm_wait((unsigned)__cvta_generic_to_shared(&s_bar[warp][q]), (phase >> q) & 1u, lane, &g_wb_flag);
    phase ^= 1u << q;
  };

  // ---- lane state
  float cs[C];                   // column sums of the window
  float A1 = 0.f, A2 = 0.f;      // axes DO-1, DO-2: sum of mass * digit
  float Q3 = 0.f;                // mass not yet credited to axis DO-3 (or the mass)
  float Mtot = 0.f;              // mass that left the outermost level
#pragma unroll
  for (int r = 0; r < C; ++r) cs[r] = 0.f;
  uint32_t t1 = 0, t2 = 0;        // digits of axes DO-1, DO-2 (the same in every lane)
  // axes 0 .. DO-3: sums, digits and pending masses, lane-major in dynamic shared memory
  unsigned char* st_base = dsm + (size_t)wb_stage_smem(VEC);
  const LaneCol<float, TH> Ac{reinterpret_cast<float*>(st_base) + threadIdx.x};
  st_base += (size_t)wb_levels(DO) * TH * 4;
  const LaneCol<uint32_t, TH> tc{reinterpret_cast<uint32_t*>(st_base) + threadIdx.x};
  st_base += (size_t)wb_levels(DO) * TH * 4;
  const LaneCol<float, TH> Qc{reinterpret_cast<float*>(st_base) + threadIdx.x};
  for (int i = 0; i < wb_levels(DO); ++i) { Ac[i] = 0.f; tc[i] = 0; }
  for (int i = 0; i < wb_qlevels(DO); ++i) Qc[i] = 0.f;

  // a carry into axis DO-3: first the outermost axis whose digit changes (h); then every
  // axis from DO-3 up to h hands its pending mass to the axis above, crediting it with its
  // current digit first, so no mass is credited with a wrong digit
  auto cold_carry = [&]() {
    int h = DO - 3;
    while (h > 0 && tc[h] + 1 == (uint32_t)g.ext[h]) --h;
    float pend = Q3;
    Q3 = 0.f;
    for (int i = DO - 3; i >= h; --i) {
      const uint32_t t = tc[i];
      Ac[i] = fmaf(pend, (float)t, Ac[i]);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0.f;
      } else {
        Mtot += pend;
      }
      tc[i] = i > h ? 0u : t + 1;
    }
    if (h > 0) Qc[h - 1] += pend;
  };
  // block column of this lane's column slot r
  auto col = [&](int r) { return VEC ? (lane + 32 * (r / EPV)) * EPV + r % EPV : lane + 32 * r; };
  // one window sum of every lane into the warp's compensated total
  auto warp_add = [&](float v, int slot) { fm_warp_add(v, &wtot[warp][0][slot], &wtot[warp][1][slot], lane); };
  // window end: credit every pending mass, move the window's sums into the warp's totals
  auto end_window = [&]() {
    float pend = Q3;
    Q3 = 0.f;
    for (int i = DO - 3; i >= 0; --i) {
      Ac[i] = fmaf(pend, (float)tc[i], Ac[i]);
      if (i > 0) {
        pend += Qc[i - 1];
        Qc[i - 1] = 0.f;
      }
    }
    Mtot += pend;
    if (DO >= 1) warp_add(A1, DO - 1);
    if (DO >= 2) warp_add(A2, DO - 2);
    for (int i = 0; i + 2 < DO; ++i) {
      warp_add(Ac[i], i);
      Ac[i] = 0.f;
    }
    warp_add(Mtot, D);
    for (int a = 0; a < m; ++a) {
      float s = 0.f;
#pragma unroll
      for (int r = 0; r < C; ++r) s = fmaf(cs[r], s_cdig[a][col(r)], s);
      warp_add(s, DO + a);
    }
#pragma unroll
    for (int r = 0; r < C; ++r) cs[r] = 0.f;
    A1 = 0.f;
    A2 = 0.f;
    Mtot = 0.f;
  };

  if (q1 > q0) {
    // tuple of the warp's first block (the outermost axis takes the remainder)
    auto set_digit = [&](int a, uint32_t v) {
      if (a == DO - 1) t1 = v;
      else if (a == DO - 2) t2 = v;
      else tc[a] = v;
    };
    if (g.n32) {
      uint32_t r32 = (uint32_t)q0;
      for (int a = DO - 1; a >= 1; --a) {
        const uint32_t q = fdiv(r32, g.div[a]);
        set_digit(a, r32 - q * g.div[a].d);
        r32 = q;
      }
      if (DO >= 1) set_digit(0, r32);
    } else {
      long long q = q0;
      for (int a = DO - 1; a >= 1; --a) {
        const long long qq = q / g.ext[a];
        set_digit(a, (uint32_t)(q - qq * g.ext[a]));
        q = qq;
      }
      if (DO >= 1) set_digit(0, (uint32_t)q);
    }
  }

  // one block: the lane's C column values (in slot order); `win` = check for the window end
  // here (the vector path checks once per group of blocks, so the window end has a single
  // call site in its loop)
  int wpos = 0;
  auto do_block = [&](const float (&x)[C], auto win) {
    float part = 0.f;
#pragma unroll
    for (int r = 0; r < C; ++r) {
      cs[r] += x[r];
      part += x[r];
    }
    A1 = fmaf(part, (float)t1, A1);
    A2 = fmaf(part, (float)t2, A2);
    Q3 += part;
    // the next block (the same step in every lane)
    if (++t1 == E1) {
      t1 = 0;
      if (++t2 == E2) {
        t2 = 0;
        cold_carry();
      }
    }
    if (decltype(win)::value && ++wpos == kWBTerms) {
      end_window();
      wpos = 0;
    }
  };

  if (VEC && g.aligned) {
    // direct 16-byte loads: lane l holds vectors l, l + 32, .. of each block; groups of UV
    // blocks, the next group's loads issued before the current group is summed
    constexpr int CV = VEC ? C / EPV : 1;
    constexpr int UV = 8 / CV;
    static_assert(kWBTerms % UV == 0, "a window is a whole number of vector steps");
    const uint4* pv = reinterpret_cast<const uint4*>(p);
    const long long bv = B / EPV;  // vectors per block
    // group of UV blocks from block q into registers (blocks past q1 read as zeros)
    auto load = [&](uint4 (&xv)[UV][CV], long long q) {
#pragma unroll
      for (int u = 0; u < UV; ++u)
#pragma unroll
        for (int v = 0; v < CV; ++v)
          xv[u][v] = (q + u < q1) ? __ldcs(pv + (q + u) * bv + lane + 32 * v) : make_uint4(0u, 0u, 0u, 0u);
    };
    auto process = [&](const uint4 (&xv)[UV][CV], long long q) {
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        if (q + u >= q1) break;
        float x[C];
#pragma unroll
        for (int r = 0; r < C; ++r) x[r] = FPiece<T>::get(xv[u][r / EPV], r % EPV);
        do_block(x, std::false_type{});
      }
      // UV divides kWBTerms, so a window holds exactly kWBTerms blocks
      wpos += UV;
      if (wpos == kWBTerms) {
        end_window();
        wpos = 0;
      }
    };
    // two register buffers: the next group's loads are in flight while a group is summed
    uint4 xa[UV][CV], xb[UV][CV];
    if (q0 < q1) load(xa, q0);
    for (long long q = q0; q < q1; q += 2 * UV) {
      if (q + UV < q1) load(xb, q + UV);
      process(xa, q);
      if (q + UV >= q1) break;
      if (q + 2 * UV < q1) load(xa, q + 2 * UV);
      process(xb, q + UV);
    }
  } else if (VEC) {
    // unaligned base: element loads at the same columns
    for (long long q = q0; q < q1; ++q) {
      float x[C];
#pragma unroll
      for (int r = 0; r < C; ++r) x[r] = FPiece<T>::ld(p, q * B + col(r));
      do_block(x, std::true_type{});
    }
  } else {
    long long si = 0;  // next step to stage
#pragma unroll
    for (int q = 0; q < NS - 1; ++q)
      if (si < nsteps) stage_step(si++, q);
    int buf = 0;
    for (long long st = 0; st < nsteps; ++st) {
      wait_stage(buf);
      __syncwarp();
      if (si < nsteps) stage_step(si++, buf == 0 ? NS - 1 : buf - 1);
      const long long qb = q0 + st * U;
      const int ub = (int)((q1 - qb) < U ? (q1 - qb) : U);
      const unsigned char* sbuf =
          dsm + ((size_t)warp * NS + buf) * kWBStageBytes + ((qb * B * ES) & 15) + lane * ES;
      for (int u = 0; u < ub; ++u) {
        const unsigned char* bl = sbuf + (size_t)u * B * ES;
        float x[C];
#pragma unroll
        for (int r = 0; r < C; ++r)
          x[r] = (r < C - 1 || lane + 32 * r < B) ? wb_elem(bl + 32 * r * ES, (T*)nullptr) : 0.f;
        do_block(x, std::true_type{});
      }
      if (++buf == NS) buf = 0;
      __syncwarp();
    }
  }
  if (wpos > 0) end_window();

  __syncthreads();
  if (threadIdx.x <= D) partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = fm_cta_total<NW>(wtot, threadIdx.x);
}

template <typename T, int... N>
const void* pick(int c, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_wb_kernel<T, N + 1, false>)...};
  return table[c - 1];
}

}  // namespace

void wb_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_wb_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_wb_flag, &zero, sizeof(int));
  *flag = v;
}

// blocks of 32 .. 256 elements
const void* moment_wb_kernel_ptr(int dtype, int B) {
  if (B < 32 || B > kWBMaxC * 32) return nullptr;
  const int c = (B + 31) / 32;
  const int es = dtype == DT_F32 ? 4 : 2;
  if (wb_vec(B, es)) {  // f32: B = 128 or 256; 16-bit: B = 256
    if (dtype == DT_F32) return c == 4 ? (const void*)&moment_wb_kernel<float, 4, true>
                                       : (const void*)&moment_wb_kernel<float, 8, true>;
    if (dtype == DT_BF16) return (const void*)&moment_wb_kernel<__nv_bfloat16, 8, true>;
    if (dtype == DT_F16) return (const void*)&moment_wb_kernel<__half, 8, true>;
    return nullptr;
  }
  auto seq = std::make_integer_sequence<int, kWBMaxC>{};
  switch (dtype) {
    case DT_F32: return pick<float>(c, seq);
    case DT_BF16: return pick<__nv_bfloat16>(c, seq);
    case DT_F16: return pick<__half>(c, seq);
  }
  return nullptr;
}

}  // namespace triot
