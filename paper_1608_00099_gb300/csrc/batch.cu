// Batched pipeline: thousands of independent (x, y) pairs of uneven rank and shape, each
// embedded (x into a zero-padded y), multiplied (y[t] *= x[t] over x's shape) and reduced
// to its tuple-weighted moment, in one persistent launch driven by a device work list
// and replayed from a CUDA graph.  Section 4 suggests partitioning independent work
// across processors with per-processor pre-results combined afterwards; here a tile of a
// pair is the unit of work and each tile writes its moment pre-result to a fixed slot.
//
// Fused mode: a tile reads x once and writes y once.  The value written is
// x[t] * x[t] inside x's shape and +0 outside, which is exactly embed followed by the
// in-place product (the product of a tile reads only what that tile wrote), and the
// tile's moment pre-result is accumulated from the same registers.
// Phased mode: the same kernel runs three times (embed, product, moment) for comparison.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/triot.h"
#include "internal.h"
#include "fixed.cuh"
#include "rows.cuh"

namespace triot {

constexpr int kBatchRows = 128;       // rows decoded per tile (shared-memory table)
constexpr int kBatchThreads = 256;

enum { BM_FUSED = 0, BM_EMBED = 1, BM_PRODUCT = 2, BM_MOMENT = 3 };

struct PairDev {
  int D;                        // rank
  int rows_per_tile;
  long long rows;               // rows of y (product of its outer extents)
  long long inner;              // y's inner extent
  long long xinner;             // x's inner extent
  long long segs;               // segments per row (>= 1)
  long long seg_len;
  long long tile_begin;         // first global tile of the pair
  long long ntiles;
  const void* x;
  void* y;
  double* out;
  FastDiv div[kMaxRank];        // y's outer extents, innermost first
  FastDiv inner_div;
  long long xstride[kMaxRank];  // x's strides for the outer axes, innermost first
  unsigned xext[kMaxRank];      // x's outer extents, innermost first
};

__device__ int g_triot_device_flag = 0;

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

template <typename T>
__device__ __forceinline__ typename AccOf<T>::type to_acc(T v) { return (typename AccOf<T>::type)v; }
template <>
__device__ __forceinline__ float to_acc<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_acc<__half>(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T zero_of() { return T(0); }
template <> __device__ __forceinline__ __nv_bfloat16 zero_of<__nv_bfloat16>() { return __ushort_as_bfloat16(0); }
template <> __device__ __forceinline__ __half zero_of<__half>() { return __ushort_as_half(0); }

template <typename T, int MAXD>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(
    const PairDev* __restrict__ pairs, const int* __restrict__ tile_pair, long long ntiles,
    int npairs, int mode, double* __restrict__ slots) {
  using Acc = typename AccOf<T>::type;
  constexpr int NV = MAXD + 1;  // moment slots: MAXD axes + mass
  __shared__ PairDev pd;
  __shared__ long long s_xoff[kBatchRows];
  __shared__ unsigned s_dig[kBatchRows][MAXD];
  __shared__ Acc s_red[kBatchThreads / 32][NV];
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pi = tile_pair[tile];
    if (pi < 0 || pi >= npairs) {  // corrupted work list: flag it and skip the tile
      if (tid == 0) atomicExch(&g_triot_device_flag, 1);
      continue;
    }
    {
      const int* src = reinterpret_cast<const int*>(pairs + pi);
      int* dst = reinterpret_cast<int*>(&pd);
      for (int w = tid; w < int(sizeof(PairDev) / sizeof(int)); w += nth) dst[w] = src[w];
    }
    __syncthreads();
    const int D = pd.D;
    const int nout = D - 1;
    const long long lt = tile - pd.tile_begin;
    long long row0, nrows, col0, E;
    if (pd.segs == 1) {
      row0 = lt * pd.rows_per_tile;
      nrows = pd.rows - row0 < pd.rows_per_tile ? pd.rows - row0 : pd.rows_per_tile;
      col0 = 0;
      E = nrows * pd.inner;
    } else {
      row0 = lt / pd.segs;
      col0 = (lt - row0 * pd.segs) * pd.seg_len;
      nrows = 1;
      E = pd.inner - col0 < pd.seg_len ? pd.inner - col0 : pd.seg_len;
    }
    // phase 1: tuple digits and x offset of every row of the tile
    for (int q = tid; q < nrows; q += nth) {
      uint32_t rem = (uint32_t)(row0 + q);
      long long xo = 0;
      bool inside = true;
#pragma unroll
      for (int k = 0; k < MAXD; ++k) {
        if (k < nout) {
          uint32_t t;
          if (k + 1 < nout) {
            const uint32_t qq = fdiv(rem, pd.div[k]);
            t = rem - qq * pd.div[k].d;
            rem = qq;
          } else {
            t = rem;
          }
          s_dig[q][k] = t;
          xo += (long long)t * pd.xstride[k];
          inside = inside && (t < pd.xext[k]);
        }
      }
      s_xoff[q] = inside ? xo : -1;
    }
    __syncthreads();
    // phase 2: elements
    Acc acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = Acc(0);
    const T* __restrict__ X = static_cast<const T*>(pd.x);
    T* __restrict__ Y = static_cast<T*>(pd.y);
    for (long long e = tid; e < E; e += nth) {
      long long q, c;
      if (pd.segs == 1) {
        uint32_t cc;
        q = fdivmod((uint32_t)e, pd.inner_div, cc);
        c = cc;
      } else {
        q = 0;
        c = col0 + e;
      }
      const long long yi = (row0 + q) * pd.inner + c;
      const long long xo = s_xoff[q];
      const bool inside = xo >= 0 && c < pd.xinner;
      Acc v = Acc(0);
      if (mode == BM_FUSED) {
        T o = zero_of<T>();
        if (inside) {
          const T xv = X[xo + c];
          o = mul_rn(xv, xv);
        }
        Y[yi] = o;
        v = to_acc<T>(o);
      } else if (mode == BM_EMBED) {
        Y[yi] = inside ? X[xo + c] : zero_of<T>();
      } else if (mode == BM_PRODUCT) {
        if (inside) Y[yi] = mul_rn(Y[yi], X[xo + c]);
      } else {
        v = to_acc<T>(Y[yi]);
      }
      if ((mode == BM_FUSED || mode == BM_MOMENT) && v != Acc(0)) {
#pragma unroll
        for (int k = 0; k < MAXD; ++k)
          if (k < nout) acc[k] += (Acc)s_dig[q][k] * v;  // axis D-2-k
        acc[MAXD - 1] += (Acc)c * v;                      // inner axis
        acc[MAXD] += v;                                   // mass
      }
    }
    if (mode == BM_FUSED || mode == BM_MOMENT) {
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        Acc v = acc[i];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) s_red[warp][i] = v;
      }
      __syncthreads();
      // slot layout per tile: axis 0 .. D-1 (outermost first), then the mass
      for (int i = tid; i < NV; i += nth) {
        double s = 0.0;
        for (int w = 0; w < nth / 32; ++w) s += (double)s_red[w][i];
        int axis;
        if (i == MAXD) axis = D;                        // mass
        else if (i == MAXD - 1) axis = D - 1;           // inner axis
        else axis = (i < nout) ? D - 2 - i : -1;        // outer digit k -> axis D-2-k
        if (axis >= 0) slots[tile * NV + axis] = s;
      }
    }
    __syncthreads();
  }
}

// Exact per-pair combine of the tiles' moment pre-results (as combine_kernel, per pair).
template <int MAXD>
__global__ void __launch_bounds__(256) batch_combine_kernel(const PairDev* __restrict__ pairs,
                                                            const double* __restrict__ slots) {
  constexpr int NV = MAXD + 1;
  const PairDev& pd = pairs[blockIdx.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int comp = warp; comp <= pd.D; comp += blockDim.x / 32) {
    unsigned emax = 0;
    int bad = 0;
    for (long long k = lane; k < pd.ntiles; k += 32) {
      const unsigned long long b =
          (unsigned long long)__double_as_longlong(slots[(pd.tile_begin + k) * NV + comp]);
      const unsigned e = (unsigned)((b >> 52) & 0x7FF);
      if (e == 0x7FF) bad = 1;
      else emax = e > emax ? e : emax;
    }
    emax = __reduce_max_sync(0xffffffffu, emax);
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    double result;
    if (bad) {
      double acc = 0.0;
      if (lane == 0)
        for (long long k = 0; k < pd.ntiles; ++k) acc += slots[(pd.tile_begin + k) * NV + comp];
      result = acc;
    } else {
      const int E = emax ? (int)emax : 1;
      __int128 acc = 0;
      for (long long k = lane; k < pd.ntiles; k += 32) {
        const unsigned long long b =
            (unsigned long long)__double_as_longlong(slots[(pd.tile_begin + k) * NV + comp]);
        const int e = (int)((b >> 52) & 0x7FF);
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
        const __int128 v = scale_shift((__int128)m, 56 - (E - (e ? e : 1)));
        acc += (b >> 63) ? -v : v;
      }
      unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)((unsigned __int128)acc >> 64);
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) {
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
        const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
        const unsigned __int128 sum = (((unsigned __int128)hi << 64) | lo) + (((unsigned __int128)ohi << 64) | olo);
        lo = (unsigned long long)sum;
        hi = (unsigned long long)(sum >> 64);
      }
      const __int128 tot = (__int128)(((unsigned __int128)hi << 64) | lo);
      result = (emax == 0 && tot == 0) ? 0.0 : ldexp(i128_to_double(tot), E - 1075 - 56);
    }
    if (lane == 0) pd.out[comp] = result;
  }
}

// ====================================================================== host side

struct triot_plan_impl {
  int dtype = 0, mode = 0, maxd = 0, npairs = 0;
  long long ntiles = 0;
  int grid = 0;
  std::vector<triot_batch_desc> descs;     // host copy for the plain per-pair launches
  PairDev* d_pairs = nullptr;
  int* d_tile_pair = nullptr;
  double* d_slots = nullptr;
  void* d_ws = nullptr;                    // moment workspace of the plain launches
  size_t ws_bytes = 0;
  size_t dev_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
};

namespace {

template <typename T, int... M>
const void* batch_ptr_t(int maxd) {
  switch (maxd) {
    case 4: return reinterpret_cast<const void*>(&batch_kernel<T, 4>);
    case 8: return reinterpret_cast<const void*>(&batch_kernel<T, 8>);
    case 12: return reinterpret_cast<const void*>(&batch_kernel<T, 12>);
    case 16: return reinterpret_cast<const void*>(&batch_kernel<T, 16>);
    default: return reinterpret_cast<const void*>(&batch_kernel<T, 24>);
  }
}

const void* batch_ptr(int dtype, int maxd) {
  switch (dtype) {
    case DT_F64: return batch_ptr_t<double>(maxd);
    case DT_F32: return batch_ptr_t<float>(maxd);
    case DT_BF16: return batch_ptr_t<__nv_bfloat16>(maxd);
    default: return batch_ptr_t<__half>(maxd);
  }
}

const void* combine_ptr(int maxd) {
  switch (maxd) {
    case 4: return reinterpret_cast<const void*>(&batch_combine_kernel<4>);
    case 8: return reinterpret_cast<const void*>(&batch_combine_kernel<8>);
    case 12: return reinterpret_cast<const void*>(&batch_combine_kernel<12>);
    case 16: return reinterpret_cast<const void*>(&batch_combine_kernel<16>);
    default: return reinterpret_cast<const void*>(&batch_combine_kernel<24>);
  }
}

void free_plan(triot_plan_impl* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_pairs) cudaFree(p->d_pairs);
  if (p->d_tile_pair) cudaFree(p->d_tile_pair);
  if (p->d_slots) cudaFree(p->d_slots);
  if (p->d_ws) cudaFree(p->d_ws);
  delete p;
}

int enqueue(triot_plan_impl* p, cudaStream_t s) {
  const void* fn = batch_ptr(p->dtype, p->maxd);
  const int modes_fused[] = {BM_FUSED};
  const int modes_phased[] = {BM_EMBED, BM_PRODUCT, BM_MOMENT};
  const int* modes = p->mode == TRIOT_BATCH_FUSED ? modes_fused : modes_phased;
  const int nm = p->mode == TRIOT_BATCH_FUSED ? 1 : 3;
  for (int m = 0; m < nm; ++m) {
    int mode = modes[m];
    void* args[] = {(void*)&p->d_pairs, (void*)&p->d_tile_pair, (void*)&p->ntiles, (void*)&p->npairs,
                    (void*)&mode, (void*)&p->d_slots};
    cudaError_t e = cudaLaunchKernel(fn, dim3(p->grid), dim3(kBatchThreads), args, 0, s);
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
  }
  void* cargs[] = {(void*)&p->d_pairs, (void*)&p->d_slots};
  cudaError_t e = cudaLaunchKernel(combine_ptr(p->maxd), dim3(p->npairs), dim3(256), cargs, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch combine launch");
  return TRIOT_OK;
}

}  // namespace

void st_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_triot_device_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_triot_device_flag, &zero, sizeof(int));
  *flag = v;
}

}  // namespace triot

using namespace triot;

struct triot_plan : triot_plan_impl {};

extern "C" {

int triot_batch_plan_create(const triot_batch_desc* descs, int n, int dtype, int mode,
                            const triot_tune* tune, triot_plan** out) {
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  *out = nullptr;
  if (!descs || n <= 0) return fail(TRIOT_ERR_ARG, "need at least one descriptor");
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (mode != TRIOT_BATCH_FUSED && mode != TRIOT_BATCH_PHASED) return fail(TRIOT_ERR_ARG, "unknown batch mode");
  const int es = dtype_size(dtype);
  DeviceInfo dev;
  int st = device_info(dev);
  if (st) return st;
  const long long target = (tune && tune->tile_elems > 0) ? tune->tile_elems : 4096;
  if (target < 1) return fail(TRIOT_ERR_ARG, "tile_elems out of range");
  std::vector<PairDev> host(n);
  std::vector<int> tile_pair;
  int maxrank = 1;
  long long ntiles = 0;
  size_t max_ws = 16;
  for (int i = 0; i < n; ++i) {
    const triot_batch_desc& d = descs[i];
    char buf[160];
    if (d.rank < 1 || d.rank > kMaxRank) {
      snprintf(buf, sizeof buf, "descriptor %d: rank %d outside [1, %d]", i, d.rank, kMaxRank);
      return fail(TRIOT_ERR_RANK, buf);
    }
    long long ny = 1, nx = 1;
    for (int a = 0; a < d.rank; ++a) {
      if (d.xshape[a] < 1 || d.yshape[a] < 1 || d.xshape[a] > d.yshape[a] || d.yshape[a] >= (1ll << 31)) {
        snprintf(buf, sizeof buf, "descriptor %d: axis %d needs 1 <= x extent <= y extent < 2^31", i, a);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      ny *= d.yshape[a];
      nx *= d.xshape[a];
    }
    if (!d.x || !d.y || !d.moment_out) {
      snprintf(buf, sizeof buf, "descriptor %d: NULL pointer", i);
      return fail(TRIOT_ERR_NULL, buf);
    }
    if (overlaps_bytes(d.x, size_t(nx) * es, d.y, size_t(ny) * es)) {
      snprintf(buf, sizeof buf, "descriptor %d: x and y overlap", i);
      return fail(TRIOT_ERR_ALIAS, buf);
    }
    const long long rows = ny / d.yshape[d.rank - 1];
    if (rows > 0xFFFFFFFFll) return fail(TRIOT_ERR_SHAPE, "a pair has more than 2^32 rows");
    PairDev& p = host[i];
    memset(&p, 0, sizeof p);
    p.D = d.rank;
    p.rows = rows;
    p.inner = d.yshape[d.rank - 1];
    p.xinner = d.xshape[d.rank - 1];
    p.x = d.x;
    p.y = d.y;
    p.out = d.moment_out;
    long long xs = p.xinner;
    for (int k = 0; k < d.rank - 1; ++k) {
      const int a = d.rank - 2 - k;
      p.div[k] = make_fastdiv((uint32_t)d.yshape[a]);
      p.xstride[k] = xs;
      p.xext[k] = (unsigned)d.xshape[a];
      xs *= d.xshape[a];
    }
    p.inner_div = make_fastdiv((uint32_t)p.inner);
    if (p.inner <= target) {
      long long R = std::max(1ll, std::min<long long>(kBatchRows, target / p.inner));
      R = std::min(R, rows);
      p.rows_per_tile = (int)R;
      p.segs = 1;
      p.seg_len = p.inner;
      p.ntiles = (rows + R - 1) / R;
    } else {
      p.rows_per_tile = 1;
      p.segs = (p.inner + target - 1) / target;
      p.seg_len = (p.inner + p.segs - 1) / p.segs;
      p.segs = (p.inner + p.seg_len - 1) / p.seg_len;
      p.ntiles = rows * p.segs;
    }
    p.tile_begin = ntiles;
    ntiles += p.ntiles;
    if (ntiles >= (1ll << 31)) return fail(TRIOT_ERR_ARG, "batch has more than 2^31 tiles");
    for (long long t = 0; t < p.ntiles; ++t) tile_pair.push_back(i);
    maxrank = std::max(maxrank, d.rank);
    // workspace of the plain per-pair moment launches
    MomentLaunch L;
    st = plan_moment_call(d.rank, d.yshape, dtype, d.y, nullptr, L);
    if (st) return st;
    max_ws = std::max(max_ws, moment_ws_bytes(L));
  }
  const int maxd = maxrank <= 4 ? 4 : maxrank <= 8 ? 8 : maxrank <= 12 ? 12 : maxrank <= 16 ? 16 : 24;
  triot_plan* p = new triot_plan();
  p->dtype = dtype;
  p->mode = mode;
  p->maxd = maxd;
  p->npairs = n;
  p->ntiles = ntiles;
  p->descs.assign(descs, descs + n);
  const int cps = (tune && tune->ctas_per_sm > 0) ? tune->ctas_per_sm : 4;
  p->grid = (int)std::max(1ll, std::min<long long>(ntiles, (long long)dev.sms * cps));
  const size_t b_pairs = sizeof(PairDev) * n, b_map = sizeof(int) * ntiles,
               b_slots = sizeof(double) * (maxd + 1) * ntiles;
  cudaError_t e;
  if ((e = cudaMalloc(&p->d_pairs, b_pairs)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_tile_pair, b_map)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_slots, b_slots)) != cudaSuccess ||
      (e = cudaMalloc(&p->d_ws, max_ws)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_pairs, host.data(), b_pairs, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMemcpy(p->d_tile_pair, tile_pair.data(), b_map, cudaMemcpyHostToDevice)) != cudaSuccess) {
    free_plan(p);
    return cuda_fail(e, "batch plan allocation");
  }
  p->ws_bytes = max_ws;
  p->dev_bytes = b_pairs + b_map + b_slots + max_ws;
  *out = p;
  return ok();
}

int triot_batch_run(triot_plan* p, void* stream) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (!p->exec) {
    // capture on a private stream (the caller's may be the legacy default stream)
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(e, "cudaStreamBeginCapture");
    }
    int st = enqueue(p, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    if ((e = cudaGraphInstantiate(&p->exec, g, 0)) != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    p->graph = g;
  }
  if ((e = cudaGraphLaunch(p->exec, s)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  return ok();
}

int triot_batch_run_plain(triot_plan* p, void* stream) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  for (const triot_batch_desc& d : p->descs) {
    int st = launch_rows(ROW_EMBED, d.rank, d.xshape, d.x, d.yshape, d.y, p->dtype, 0, s, nullptr);
    if (!st) st = launch_rows(ROW_PRODUCT, d.rank, d.xshape, d.x, d.yshape, d.y, p->dtype, 0, s, nullptr);
    if (!st) st = moment_call(d.rank, d.yshape, d.y, p->dtype, d.moment_out, p->d_ws, p->ws_bytes, s, nullptr);
    if (st) return st;
  }
  return ok();
}

int triot_batch_plan_info(const triot_plan* p, size_t* device_bytes, int64_t* tiles) {
  if (!p) return fail(TRIOT_ERR_NULL, "plan is NULL");
  if (device_bytes) *device_bytes = p->dev_bytes;
  if (tiles) *tiles = p->ntiles;
  return ok();
}

int triot_batch_plan_destroy(triot_plan* p) {
  free_plan(p);
  return ok();
}

}  // extern "C"
