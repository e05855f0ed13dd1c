// Moment of a product of tensors on short rows (rows of I shorter than 8 elements), the
// same reduction as moment_prod.cu (Algorithm 11 with the weight w[t] = x_0[t] * x_1[t] * ..
// formed left to right, in double for f64 tensors and in float otherwise) for shapes whose
// rows are too short for a lane per row to amortise its per-row bookkeeping.
//
// CTA tiles of consecutive rows of I.  Thread t always takes column t mod L of rows
// t div L, t div L + RP, .. of a tile (RP = floor(threads / L) rows per pass), so each load
// instruction of a warp reads contiguous stretches of every tensor.  Per tile:
//   (1) every row's offset in every tensor is decoded once (Algorithm 4 with magic-number
//       division) into shared memory;
//   (2) every element's weight is formed and kept in shared memory (as a double, exact),
//       and the CTA takes the largest exponent E among the tile's weights;
//   (3) a thread per row converts the row's weights to the tile's fixed point (the integer
//       c = m >> (E - e), m the 53-bit significand, e the exponent: exact sums, at most
//       2^-52 of the tile's largest |w| dropped per element), forms the row mass P and the
//       inner-axis sum sum_j j c, decodes the row's digits and adds t_i P for every outer
//       axis i across the warp (exact 128-bit sums, lane i keeping axis i; an axis whose
//       digit is the same in all the warp's rows takes digit times the warp's mass).  The
//       tile's sums are rounded once to f64.  A tile holding a non-finite weight is summed
//       in plain f64 instead, so that infinities and NaN propagate as in a plain sum.
// The CTA's per-lane totals are added per component in a fixed order into its partial
// vector; the combine kernel adds the partial vectors exactly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

#include "common.cuh"
#include "fixed.cuh"
#include "kernels.h"
#include "mprod_rows.h"

namespace triot {
namespace {

constexpr int kMPRThreads = kMPRowsWarps * 32;
constexpr int kMPRU = 4;  // passes whose loads a thread has in flight
constexpr int kMPRowsEager = 3;  // innermost outer axes summed per thread

// an element in the product's compute type (bf16 and f16 convert to float exactly)
__device__ __forceinline__ double mpr_load(const double* p) { return __ldg(p); }
__device__ __forceinline__ float mpr_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float mpr_load(const __nv_bfloat16* p) {
  return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short*>(p)) << 16);
}
__device__ __forceinline__ float mpr_load(const __half* p) {
  return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
}
__device__ __forceinline__ double mpr_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mpr_mul(float a, float b) { return __fmul_rn(a, b); }

template <typename T> struct MPRCompute { using type = float; };
template <> struct MPRCompute<double> { using type = double; };

// biased exponent of a double (0 for zero and subnormals, 0x7FF for inf and NaN)
__device__ __forceinline__ int mpr_exp(double w) {
  return (int)(((unsigned long long)__double_as_longlong(w) >> 52) & 0x7FF);
}

// w as an integer in units of 2^(E - 1075): exact when w's exponent is E, truncated toward
// zero by E - e bits otherwise (E >= the exponent of every finite w of the tile)
__device__ __forceinline__ long long mpr_fix(double w, int E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int sh = E - (e ? e : 1);
  const long long c = sh >= 64 ? 0ll : (long long)(m >> sh);
  return (b >> 63) ? -c : c;
}

// exact warp sum of a 128-bit integer (xor butterfly on 32-bit words)
__device__ __forceinline__ __int128 mpr_warp_sum(__int128 x) {
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
  return x;
}

__device__ __forceinline__ double mpr_warp_sum(double v) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T, int N>
__global__ void __launch_bounds__(kMPRThreads) mprod_rows_kernel(const __grid_constant__ MProdGeom g,
                                                                 const __grid_constant__ MPRowsGeom rg,
                                                                 double* __restrict__ partial) {
  using CT = typename MPRCompute<T>::type;
  __shared__ long long s_off[N][kMPRowsTileRows];
  __shared__ double s_w[kMPRowsTileElems];
  __shared__ int s_emax[kMPRowsWarps];
  __shared__ int s_special;
  __shared__ double s_tot[kMPRowsWarps][kMaxRank + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int D = g.D;        // >= 2 here
  const int IN = D - 2;     // the innermost outer axis
  const int L = (int)g.L;   // 1 < L < 8
  const int R = rg.tile_rows;
  const int RP = rg.rp;
  uint32_t col;
  const uint32_t rl = fdivmod((uint32_t)tid, rg.ldiv, col);
  const bool lact = (int)rl < RP;  // threads past RP * L idle in the streaming step
  const T* X[N];
#pragma unroll
  for (int k = 0; k < N; ++k) X[k] = static_cast<const T*>(g.x[k]) + (long long)col * g.stride[k][D - 1];
  double tot = 0.0;  // lane a: this warp's f64 total of component a from tiles summed in f64
  // fixed-point sums in units of 2^(EW - 1075), EW the largest exponent the CTA has seen:
  // this thread's rows on the kMPRowsEager innermost outer axes (Ae[k]: axis IN - k), their
  // mass and inner-axis sum; lane a: the warp's sum of outer axis a above those
  __int128 Ae[kMPRowsEager], Am = 0, Ai = 0, Ah = 0;
#pragma unroll
  for (int k = 0; k < kMPRowsEager; ++k) Ae[k] = 0;
  int EW = 0;
  const long long ntiles = (g.nrows + R - 1) / R;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long row0 = tile * R;
    const int nrows = (int)(g.nrows - row0 < R ? g.nrows - row0 : R);
    // (1) row offsets
    for (int q = tid; q < nrows; q += kMPRThreads) {
      uint32_t r = (uint32_t)(row0 + q);
      long long off[N];
#pragma unroll
      for (int k = 0; k < N; ++k) off[k] = 0;
      for (int a = IN; a >= 0; --a) {
        uint32_t d = r;
        if (a > 0) {
          const uint32_t q1 = fdiv(r, g.div[a]);
          d = r - q1 * g.div[a].d;
          r = q1;
        }
#pragma unroll
        for (int k = 0; k < N; ++k) off[k] += (long long)d * g.stride[k][a];
      }
#pragma unroll
      for (int k = 0; k < N; ++k) s_off[k][q] = off[k];
    }
    if (tid == 0) s_special = 0;
    __syncthreads();
    // (2) weights
    int emax = 0;
    bool spec = false;
    for (int q0 = 0; q0 < nrows; q0 += RP * kMPRU) {
      CT v[kMPRU][N];
#pragma unroll
      for (int u = 0; u < kMPRU; ++u) {
        const int q = q0 + (int)rl + u * RP;
        const bool ok = lact && q < nrows;
#pragma unroll
        for (int k = 0; k < N; ++k) v[u][k] = ok ? mpr_load(X[k] + s_off[k][q]) : CT(0);
      }
#pragma unroll
      for (int u = 0; u < kMPRU; ++u) {
        const int q = q0 + (int)rl + u * RP;
        if (lact && q < nrows) {
          CT w = v[u][0];
#pragma unroll
          for (int k = 1; k < N; ++k) w = mpr_mul(w, v[u][k]);
          const double wd = (double)w;
          s_w[q * L + (int)col] = wd;
          const int e = mpr_exp(wd);
          if (e == 0x7FF) spec = true;
          else emax = max(emax, e ? e : 1);
        }
      }
    }
    emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)emax);
    spec = __any_sync(0xffffffffu, spec);
    if (lane == 0) {
      s_emax[warp] = emax;
      if (spec) s_special = 1;
    }
    __syncthreads();
    int E = 0;
#pragma unroll
    for (int w = 0; w < kMPRowsWarps; ++w) E = max(E, s_emax[w]);
    const bool special = s_special != 0;
    if (!special && E > EW) {  // the CTA's exponent grows: every fixed-point sum shifts right
      if (EW > 0) {
        const int sh = E - EW;
#pragma unroll
        for (int k = 0; k < kMPRowsEager; ++k) Ae[k] = shr_arith(Ae[k], sh);
        Am = shr_arith(Am, sh);
        Ai = shr_arith(Ai, sh);
        Ah = shr_arith(Ah, sh);
      }
      EW = E;
    }
    // (3) rows: a thread per row (the trip count is the same in every thread of the CTA)
    for (int q0 = 0; q0 < nrows; q0 += kMPRThreads) {
      const int q = q0 + tid;
      const bool ok = q < nrows;
      if (!special) {
        long long P = 0, Pi = 0;
        if (ok)
          for (int j = 0; j < L; ++j) {
            const long long c = mpr_fix(s_w[q * L + j], EW);
            P += c;
            Pi += c * j;
          }
        Am += P;
        Ai += Pi;
        // the row's digits: the innermost outer axes into this thread's sums; above them the
        // warp's rows are consecutive, so on most axes every row of the warp has the same
        // digit d and the axis takes d times the warp's mass, and only an axis whose digit
        // varies across the warp takes a sum of its own (rows past the tile have P = 0 and
        // take the digits of the warp's first row)
        const uint32_t r0w = (uint32_t)(row0 + q0 + (tid & ~31));
        uint32_t r = ok ? (uint32_t)(row0 + q) : r0w;
#pragma unroll
        for (int k = 0; k < kMPRowsEager; ++k) {
          const int a = IN - k;
          if (a < 0) break;
          uint32_t d = r;
          if (a > 0) {
            const uint32_t q1 = fdiv(r, g.div[a]);
            d = r - q1 * g.div[a].d;
            r = q1;
          }
          mac64x32(Ae[k], P, d);
        }
        long long xm = 0;
        bool have_xm = false;
        for (int a = IN - kMPRowsEager; a >= 0; --a) {
          uint32_t d = r;
          if (a > 0) {
            const uint32_t q1 = fdiv(r, g.div[a]);
            d = r - q1 * g.div[a].d;
            r = q1;
          }
          const uint32_t d0 = __shfl_sync(0xffffffffu, d, 0);
          if (__all_sync(0xffffffffu, d == d0)) {
            if (!have_xm) {  // the warp's mass (|P| < 2^56: the sum of 32 fits 64 bits)
              xm = P;
#pragma unroll
              for (int off = 16; off >= 1; off >>= 1) xm += __shfl_xor_sync(0xffffffffu, xm, off);
              have_xm = true;
            }
            if (lane == a) mac64x32(Ah, xm, d0);
          } else {
            __int128 x = 0;
            mac64x32(x, P, d);
            x = mpr_warp_sum(x);
            if (lane == a) Ah += x;
          }
        }
      } else {
        double P = 0.0, Pi = 0.0;
        if (ok)
          for (int j = 0; j < L; ++j) {
            const double w = s_w[q * L + j];
            P += w;
            Pi += w * (double)j;
          }
        uint32_t r = ok ? (uint32_t)(row0 + q) : 0u;
        for (int a = IN; a >= 0; --a) {
          uint32_t d = r;
          if (a > 0) {
            const uint32_t q1 = fdiv(r, g.div[a]);
            d = r - q1 * g.div[a].d;
            r = q1;
          }
          const double x = mpr_warp_sum(ok ? P * (double)d : 0.0);
          if (lane == a) tot += x;
        }
        const double xi = mpr_warp_sum(Pi), xm = mpr_warp_sum(P);
        if (lane == D - 1) tot += xi;
        if (lane == D) tot += xm;
      }
    }
    __syncthreads();  // s_off, s_w and s_emax are rewritten by the next tile
  }
  // the warp's fixed-point sums (exact), rounded once to f64, plus its f64 totals
  {
    const __int128 wm = mpr_warp_sum(Am), wi = mpr_warp_sum(Ai);
    __int128 own = (lane < D - 1 && IN - lane >= kMPRowsEager) ? Ah : (__int128)0;
#pragma unroll
    for (int k = 0; k < kMPRowsEager; ++k) {
      const __int128 we = mpr_warp_sum(Ae[k]);
      if (lane == IN - k) own = we;
    }
    if (lane == D - 1) own = wi;
    if (lane == D) own = wm;
    if (lane <= D) s_tot[warp][lane] = tot + (EW > 0 ? fixed_to_double(own, EW - 1075) : 0.0);
  }
  __syncthreads();
  if (tid <= D) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kMPRowsWarps; ++w) s += s_tot[w][tid];
    partial[(long long)blockIdx.x * (D + 1) + tid] = s;
  }
}

template <typename T, int... I>
const void* mpr_pick(int n, std::integer_sequence<int, I...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&mprod_rows_kernel<T, I + 1>)...};
  return table[n - 1];
}

}  // namespace

const void* moment_prod_rows_kernel_ptr(int dtype, int ntensors) {
  if (ntensors < 1 || ntensors > kMProdMaxTensors) return nullptr;
  auto seq = std::make_integer_sequence<int, kMProdMaxTensors>{};
  switch (dtype) {
    case DT_F64: return mpr_pick<double>(ntensors, seq);
    case DT_F32: return mpr_pick<float>(ntensors, seq);
    case DT_BF16: return mpr_pick<__nv_bfloat16>(ntensors, seq);
    case DT_F16: return mpr_pick<__half>(ntensors, seq);
  }
  return nullptr;
}

}  // namespace triot
