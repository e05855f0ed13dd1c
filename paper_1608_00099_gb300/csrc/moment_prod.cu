// Moment of a product of tensors over the intersection I of their shapes: Algorithm 11's
// tuple-weighted sum with the weight w[t] = x_0[t] * x_1[t] * ... formed on the fly (with
// two tensors the mass is benchmark 2's inner product over the tuples both shapes share,
// Section 3), so the product is never written to memory.
//
// Work split: rows of I (its last axis) in rounds of 32; each warp owns a contiguous range
// of rounds and lane l takes row l of each round, loading that row from every tensor with
// the tensor's own strides (Algorithm 2 per tensor).  A lane's row tuple advances by 32 rows
// per round: a constant whose mixed-radix digits are precomputed, carried like
// advance_tuple (Algorithm 3).
//
// Arithmetic: w is formed left to right in double for f64 tensors and in float for f32,
// bf16 and f16 tensors (each multiply rounded to nearest even).  Each w becomes the integer
// c = m >> (E_W - e) of the lane's current fixed-point window (at most kMProdWindow
// elements; E_W the largest exponent seen in the window; float weights keep 24 extra
// fraction bits).  Per row: the mass P = sum c and the inner-axis sum sum_j j c; the three
// innermost outer axes are credited eagerly per row (A += P * t), the remaining axes lazily
// when their digit changes.  At a window end the sums are rounded once to f64 and added to
// the lane's totals; lane totals are summed per warp exactly in 128-bit fixed point.
// Non-finite weights are summed separately in f64 so that they propagate.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>
#include <utility>

#include "common.cuh"
#include "fixed.cuh"
#include "kernels.h"

namespace triot {
namespace {

// element loads in the product's compute type (bf16 and f16 convert to float exactly)
__device__ __forceinline__ double ld_w(const double* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_w(const float* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float ld_w(const __nv_bfloat16* p, long long i) {
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
  return __uint_as_float((unsigned)b << 16);
}
__device__ __forceinline__ float ld_w(const __half* p, long long i) {
  const unsigned short b = __ldg(reinterpret_cast<const unsigned short*>(p) + i);
  return __half2float(__ushort_as_half(b));
}
__device__ __forceinline__ double mul_w(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_w(float a, float b) { return __fmul_rn(a, b); }

// the compute type's binary layout: w = m * 2^(e - kBias) (e >= 1 after clamping
// subnormals); fixed-point units are 2^(E_W - kBias - kGuard)
template <typename CT> struct WBits;
template <> struct WBits<double> {
  static constexpr int kBias = 1075, kGuard = 0, kEmax = 0x7FF;
  __device__ static int exp_of(double w) {
    return (int)(((unsigned long long)__double_as_longlong(w) >> 52) & 0x7FF);
  }
  __device__ static void split(double w, int& e, unsigned long long& m, bool& neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(w);
    e = (int)((b >> 52) & 0x7FF);
    m = (b & 0x000FFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
    neg = (b >> 63) != 0;
  }
};
template <> struct WBits<float> {
  static constexpr int kBias = 150, kGuard = 24, kEmax = 0xFF;
  __device__ static int exp_of(float w) { return (int)((__float_as_uint(w) >> 23) & 0xFF); }
  __device__ static void split(float w, int& e, unsigned long long& m, bool& neg) {
    const unsigned b = __float_as_uint(w);
    e = (int)((b >> 23) & 0xFF);
    m = ((unsigned long long)((b & 0x7FFFFFu) | (e ? 0x800000u : 0u))) << 24;
    neg = (b >> 31) != 0;
  }
};

template <typename T> struct ComputeOf { using type = float; };
template <> struct ComputeOf<double> { using type = double; };

// non-finite weight: plain f64 sums of v * t_i (rare; kept out of line)
__device__ __noinline__ void mprod_special(double v, uint32_t t1, uint32_t t2, uint32_t t3,
                                           LaneCol<uint32_t, kMProdWarps * 32> tc, int DO,
                                           long long j, double* Asp, double* Isp, double* Psp) {
  if (DO >= 1) Asp[DO - 1] += v * (double)t1;
  if (DO >= 2) Asp[DO - 2] += v * (double)t2;
  if (DO >= 3) Asp[DO - 3] += v * (double)t3;
  for (int i = 0; i + 3 < DO; ++i) Asp[i] += v * (double)tc[i];
  *Isp += v * (double)j;
  *Psp += v;
}

template <typename T, int NT>
__global__ void __launch_bounds__(kMProdWarps * 32) moment_prod_kernel(
    const __grid_constant__ MProdGeom g, double* __restrict__ partial) {
  using CT = typename ComputeOf<T>::type;
  using Bits = WBits<CT>;
  constexpr int NW = kMProdWarps;
  constexpr int TH = NW * 32;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double wsum[NW][kMaxRank + 1];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int D = g.D, DO = D - 1;
  const long long L = g.L;
  const long long W = (long long)gridDim.x * NW;
  const long long gw = (long long)blockIdx.x * NW + warp;
  const long long r0 = g.nround * gw / W, r1 = g.nround * (gw + 1) / W;

  const uint32_t E1 = DO >= 2 ? (uint32_t)g.ext[DO - 1] : 0xFFFFFFFFu;
  const uint32_t E2 = DO >= 3 ? (uint32_t)g.ext[DO - 2] : 0xFFFFFFFFu;
  const uint32_t E3 = DO >= 4 ? (uint32_t)g.ext[DO - 3] : 0xFFFFFFFFu;
  const uint32_t j1 = DO >= 1 ? g.jd[DO - 1] : 0u;
  const uint32_t j2 = DO >= 2 ? g.jd[DO - 2] : 0u;
  const uint32_t j3 = DO >= 3 ? g.jd[DO - 3] : 0u;
  bool jcold = false;
  for (int i = 0; i + 3 < DO; ++i) jcold = jcold || g.jd[i] != 0u;

  // axes 0 .. DO-4 and the lane's f64 totals of the outer axes: lane-major dynamic shared
  // memory (touched at carries and window ends; run-time axis index)
  unsigned char* st_base = dsm;
  const LaneCol<__int128, TH> Ac{reinterpret_cast<__int128*>(st_base) + threadIdx.x};
  st_base += (size_t)mprod_levels(DO) * TH * 16;
  const LaneCol<__int128, TH> Qc{reinterpret_cast<__int128*>(st_base) + threadIdx.x};
  st_base += (size_t)mprod_qlevels(DO) * TH * 16;
  const LaneCol<double, TH> Ads{reinterpret_cast<double*>(st_base) + threadIdx.x};
  st_base += (size_t)DO * TH * 8;
  const LaneCol<uint32_t, TH> tc{reinterpret_cast<uint32_t*>(st_base) + threadIdx.x};
  for (int i = 0; i < mprod_levels(DO); ++i) { Ac[i] = 0; tc[i] = 0; }
  for (int i = 0; i < mprod_qlevels(DO); ++i) Qc[i] = 0;
  for (int i = 0; i < DO; ++i) Ads[i] = 0.0;

  __int128 A1 = 0, A2 = 0, A3 = 0;      // axes DO-1, DO-2, DO-3: sum of row mass * digit
  __int128 AI = 0;                      // the row axis: sum of j * c
  __int128 Q4 = 0;                      // mass not yet credited to axis DO-4 (or the mass)
  __int128 Mtot = 0;                    // mass that left the outermost level
  long long P = 0;                      // mass of the current row (window units)
  __int128 Wr = 0;                      // sum of j * c over the current row
  uint32_t t1 = 0, t2 = 0, t3 = 0;      // digits of axes DO-1, DO-2, DO-3
  int es = 0;                           // window exponent (0: nothing seen)
  int welem = 0;                        // elements in the window
  double Asp[kMaxRank];                 // non-finite weights (written only when one occurs)
  double Dinner = 0.0, Md = 0.0, Isp = 0.0, Psp = 0.0;
  bool special = false;

  auto rebase = [&](int e_new) {
    if (es != 0) {
      const int d = e_new - es;
      P = shr64(P, d);
      Wr = shr_arith(Wr, d);
      A1 = shr_arith(A1, d);
      A2 = shr_arith(A2, d);
      A3 = shr_arith(A3, d);
      AI = shr_arith(AI, d);
      Q4 = shr_arith(Q4, d);
      Mtot = shr_arith(Mtot, d);
      for (int i = 0; i < mprod_levels(DO); ++i) Ac[i] = shr_arith(Ac[i], d);
      for (int i = 0; i < mprod_qlevels(DO); ++i) Qc[i] = shr_arith(Qc[i], d);
    }
    es = e_new;
  };
  // digits of axes DO-4 .. 0 advance by (jump digit if `jump`) + carry; every axis up to
  // the outermost one that changes first hands its pending mass up (credited with its
  // current digit)
  auto cold_step = [&](uint32_t carry_in, bool jump) {
    int h = -1;
    {
      uint32_t carry = carry_in;
      for (int i = DO - 4; i >= 0; --i) {
        const uint32_t inc = (jump ? g.jd[i] : 0u) + carry;
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
      const uint32_t inc = (jump ? g.jd[i] : 0u) + carry;
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
  // the row's (or part row's) mass and inner sum, credited with the row's digits
  auto credit_row = [&]() {
    if (DO >= 1) mac64x32(A1, P, t1);
    if (DO >= 2) mac64x32(A2, P, t2);
    if (DO >= 3) mac64x32(A3, P, t3);
    Q4 += P;
    AI += Wr;
    P = 0;
    Wr = 0;
  };
  // to the lane's row of the next round: 32 rows on
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
      const int sc = es - Bits::kBias - Bits::kGuard;
      if (DO >= 1) Ads[DO - 1] += fixed_to_double(A1, sc);
      if (DO >= 2) Ads[DO - 2] += fixed_to_double(A2, sc);
      if (DO >= 3) Ads[DO - 3] += fixed_to_double(A3, sc);
      for (int i = 0; i + 3 < DO; ++i) Ads[i] += fixed_to_double(Ac[i], sc);
      Dinner += fixed_to_double(AI, sc);
      Md += fixed_to_double(Mtot, sc);
    }
    A1 = 0;
    A2 = 0;
    A3 = 0;
    AI = 0;
    Mtot = 0;
    for (int i = 0; i < mprod_levels(DO); ++i) Ac[i] = 0;
    es = 0;
    welem = 0;
  };

  if (r1 > r0) {
    // tuple of this lane's first row (the outermost axis takes the remainder)
    const long long row0 = r0 * 32 + lane;
    auto set_digit = [&](int a, uint32_t v) {
      if (a == DO - 1) t1 = v;
      else if (a == DO - 2) t2 = v;
      else if (a == DO - 3) t3 = v;
      else tc[a] = v;
    };
    if (g.n32) {
      uint32_t r32 = (uint32_t)row0;
      for (int a = DO - 1; a >= 1; --a) {
        const uint32_t q = fdiv(r32, g.div[a]);
        set_digit(a, r32 - q * g.div[a].d);
        r32 = q;
      }
      if (DO >= 1) set_digit(0, r32);
    } else {
      long long q = row0;
      for (int a = DO - 1; a >= 1; --a) {
        const long long q1 = q / g.ext[a];
        set_digit(a, (uint32_t)(q - q1 * g.ext[a]));
        q = q1;
      }
      if (DO >= 1) set_digit(0, (uint32_t)q);
    }
  }

  const T* xs[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) xs[k] = static_cast<const T*>(g.x[k]);
  long long sj[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) sj[k] = g.unit_inner ? 1 : g.stride[k][D - 1];

  // offsets of row `rw` in every tensor, decoded from scratch (Algorithm 4, then Horner)
  auto decode_offsets = [&](long long rw, long long (&o)[NT]) {
#pragma unroll
    for (int k = 0; k < NT; ++k) o[k] = 0;
    long long q = rw;
    for (int a = DO - 1; a >= 0; --a) {
      long long dgt;
      if (a == 0) {
        dgt = q;
      } else if (g.n32) {
        const uint32_t qq = fdiv((uint32_t)q, g.div[a]);
        dgt = (long long)((uint32_t)q - qq * g.div[a].d);
        q = qq;
      } else {
        const long long qq = q / g.ext[a];
        dgt = q - qq * g.ext[a];
        q = qq;
      }
#pragma unroll
      for (int k = 0; k < NT; ++k) o[k] += dgt * g.stride[k][a];
    }
  };
  // offsets of the lane's row in the next round, from the current digits: the same carries
  // as jump() makes, applied to the offsets (a fresh decode when an axis above DO-3 moves)
  auto next_offsets = [&](const long long (&o)[NT], long long rw, long long (&on)[NT]) {
    const uint32_t a1 = t1 + j1;
    const uint32_t c1 = a1 >= E1 ? 1u : 0u;
    const uint32_t a2 = t2 + j2 + c1;
    const uint32_t c2 = a2 >= E2 ? 1u : 0u;
    const uint32_t a3 = t3 + j3 + c2;
    const uint32_t c3 = a3 >= E3 ? 1u : 0u;
    if (c3 || jcold) {
      decode_offsets(rw + 32, on);
      return;
    }
    const long long d1 = (long long)j1 - (c1 ? (long long)E1 : 0ll);
    const long long d2 = (long long)(j2 + c1) - (c2 ? (long long)E2 : 0ll);
    const long long d3 = (long long)(j3 + c2);
#pragma unroll
    for (int k = 0; k < NT; ++k) {
      long long v = o[k];
      if (DO >= 1) v += d1 * g.stride[k][DO - 1];
      if (DO >= 2) v += d2 * g.stride[k][DO - 2];
      if (DO >= 3) v += d3 * g.stride[k][DO - 3];
      on[k] = v;
    }
  };
  // one element's weight into the window's fixed point (or the f64 special sums)
  auto add_elem = [&](CT w, long long j) {
    int e;
    unsigned long long mm;
    bool neg;
    Bits::split(w, e, mm, neg);
    if (e == Bits::kEmax) {
      if (!special) {
        for (int i = 0; i < DO; ++i) Asp[i] = 0.0;
        special = true;
      }
      mprod_special((double)w, t1, t2, t3, tc, DO, j, Asp, &Isp, &Psp);
      return;
    }
    const int e1 = e > 1 ? e : 1;
    if (e1 > es) rebase(e1);
    const int sh = es - e1;
    long long c = sh < 64 ? (long long)(mm >> sh) : 0ll;
    if (neg) c = -c;
    P += c;
    mac64x32(Wr, c, (uint32_t)j);
  };

  long long off[NT];
#pragma unroll
  for (int k = 0; k < NT; ++k) off[k] = 0;
  if (r1 > r0) decode_offsets(r0 * 32 + lane, off);
  for (long long r = r0; r < r1; ++r) {
    const long long row = r * 32 + lane;
    if (row >= g.nrows) break;
    if (L <= kMProdWindow) {
      if (welem + L > kMProdWindow) end_window();
      // the row in batches of kMProdLC: all loads of a batch first, one exponent check, the
      // batch's sums sum c and sum u c in 64 bits (u < kMProdLC), one 128-bit update each
      auto row_batches = [&](auto unit) {
        constexpr bool kUnit = decltype(unit)::value;
        const T* pk[NT];
#pragma unroll
        for (int k = 0; k < NT; ++k) pk[k] = xs[k] + off[k];
        for (long long j0 = 0; j0 < L; j0 += kMProdLC) {
          const int cnt = (L - j0) < kMProdLC ? (int)(L - j0) : kMProdLC;
          CT w[kMProdLC];
#pragma unroll
          for (int u = 0; u < kMProdLC; ++u) {
            if (u < cnt) {
              const long long j = j0 + u;
              CT v = ld_w(pk[0], kUnit ? j : j * sj[0]);
#pragma unroll
              for (int k = 1; k < NT; ++k) v = mul_w(v, ld_w(pk[k], kUnit ? j : j * sj[k]));
              w[u] = v;
            } else {
              w[u] = CT(0);
            }
          }
          int emax = 0;
          bool odd = false;  // a non-finite weight in the batch
#pragma unroll
          for (int u = 0; u < kMProdLC; ++u) {
            const int e = Bits::exp_of(w[u]);
            odd = odd || e == Bits::kEmax;
            emax = e > emax ? e : emax;
          }
          if (odd) {
            for (int u = 0; u < cnt; ++u) add_elem(w[u], j0 + u);
            continue;
          }
          if ((emax > 1 ? emax : 1) > es) rebase(emax > 1 ? emax : 1);
          long long pb = 0, ub = 0;
#pragma unroll
          for (int u = 0; u < kMProdLC; ++u) {
            int e;
            unsigned long long mm;
            bool neg;
            Bits::split(w[u], e, mm, neg);
            const int sh = es - (e > 1 ? e : 1);
            long long c = sh < 64 ? (long long)(mm >> sh) : 0ll;
            if (neg) c = -c;
            pb += c;
            ub += (long long)u * c;
          }
          P += pb;
          mac64x32(Wr, pb, (uint32_t)j0);
          Wr += ub;
        }
      };
      if (g.unit_inner) row_batches(std::true_type{});
      else row_batches(std::false_type{});
      welem += (int)L;
    } else {
      // a row longer than the window: element by element, closing windows mid-row
      if (welem > 0) end_window();
      for (long long j = 0; j < L; ++j) {
        if (welem == kMProdWindow) {
          credit_row();
          end_window();
        }
        CT v = ld_w(xs[0], off[0] + j * sj[0]);
#pragma unroll
        for (int k = 1; k < NT; ++k) v = mul_w(v, ld_w(xs[k], off[k] + j * sj[k]));
        add_elem(v, j);
        ++welem;
      }
    }
    long long offn[NT];
    next_offsets(off, row, offn);
    credit_row();
    jump();
#pragma unroll
    for (int k = 0; k < NT; ++k) off[k] = offn[k];
  }
  end_window();

  // warp sum of the lane totals: exact in 128-bit fixed point relative to the warp's largest
  // exponent, or an f64 xor-order sum when a lane holds a non-finite value
  double* ws_out = wsum[warp];
  auto reduce_out = [&](double v, double sp, int slot) {
    if (special) v += sp;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    int e = (int)((bits >> 52) & 0x7FFull);
    if (__any_sync(0xffffffffu, e == 0x7FF)) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) ws_out[slot] = v;
      return;
    }
    unsigned long long mant = bits & 0x000FFFFFFFFFFFFFull;
    if (e) mant |= 1ull << 52;
    else e = 1;
    const int ew = (int)__reduce_max_sync(0xffffffffu, (unsigned)e);
    const int d = ew - e;
    __int128 x = 0;
    if (d <= 64) x = (__int128)((unsigned __int128)mant << (64 - d));
    else if (d < 64 + 53) x = (__int128)(mant >> (d - 64));
    if (bits >> 63) x = -x;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const unsigned __int128 u = (unsigned __int128)x;
      const unsigned w0 = __shfl_xor_sync(0xffffffffu, (unsigned)u, o);
      const unsigned w1 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 32), o);
      const unsigned w2 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 64), o);
      const unsigned w3 = __shfl_xor_sync(0xffffffffu, (unsigned)(u >> 96), o);
      x += (__int128)(((unsigned __int128)w3 << 96) | ((unsigned __int128)w2 << 64) |
                      ((unsigned __int128)w1 << 32) | (unsigned __int128)w0);
    }
    if (lane == 0) ws_out[slot] = fixed_to_double(x, ew - 1139);
  };
  for (int i = 0; i < DO; ++i) reduce_out(Ads[i], special ? Asp[i] : 0.0, i);
  reduce_out(Dinner, Isp, DO);
  reduce_out(Md, Psp, D);
  __syncthreads();
  if (threadIdx.x <= D) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < NW; ++w) acc += wsum[w][threadIdx.x];
    partial[(long long)blockIdx.x * (D + 1) + threadIdx.x] = acc;
  }
}

template <typename T, int... N>
const void* pick_n(int n, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_prod_kernel<T, N + 1>)...};
  return table[n - 1];
}

}  // namespace

const void* moment_prod_kernel_ptr(int dtype, int ntensors) {
  if (ntensors < 1 || ntensors > kMProdMaxTensors) return nullptr;
  auto seq = std::make_integer_sequence<int, kMProdMaxTensors>{};
  switch (dtype) {
    case DT_F64: return pick_n<double>(ntensors, seq);
    case DT_F32: return pick_n<float>(ntensors, seq);
    case DT_BF16: return pick_n<__nv_bfloat16>(ntensors, seq);
    case DT_F16: return pick_n<__half>(ntensors, seq);
  }
  return nullptr;
}

}  // namespace triot
