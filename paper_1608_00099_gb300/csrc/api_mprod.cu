// C ABI of the moment of a product of tensors (Algorithm 11 with several weight tensors;
// for two tensors the mass is benchmark 2's inner product over the shared tuples):
// validation, canonicalisation of the intersection, launch of the kernel and the combine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/triot.h"
#include "internal.h"
#include "kernels.h"
#include "mprod_rows.h"

namespace triot {
namespace {

struct MProdLaunch {
  MProdGeom g;
  MPRowsGeom rg;  // the short-row kernel's tiles
  CombineGeom cg;
  int grid = 0;
  size_t smem = 0;
  bool empty = false;
  bool rows = false;  // the short-row kernel (moment_prod_rows.cu)
};

bool mul_overflows(int64_t a, int64_t b) { return a != 0 && b > INT64_MAX / a; }

int mprod_occupancy(const void* fn, size_t dyn, int& occ) {
  struct Entry { const void* fn; size_t dyn; int dev; int occ; };
  static std::mutex mu;
  static std::vector<Entry> table;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& x : table)
    if (x.fn == fn && x.dyn == dyn && x.dev == dev) { occ = x.occ; return TRIOT_OK; }
  // the attribute is per kernel: cover the largest rank once
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, mprod_dyn_smem(kMaxRank - 1));
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic shared memory)");
  int o = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, kMProdWarps * 32, dyn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  occ = o > 0 ? o : 1;
  table.push_back({fn, dyn, dev, occ});
  return TRIOT_OK;
}

int plan_mprod(int rank, int n, const int64_t* const* shapes, int dtype, const void* const* ptrs,
               MProdLaunch& L) {
  char buf[256];
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    return fail(TRIOT_ERR_RANK, buf);
  }
  if (n < 1 || n > kMProdMaxTensors) {
    snprintf(buf, sizeof buf, "ntensors %d outside [1, %d]", n, kMProdMaxTensors);
    return fail(TRIOT_ERR_ARG, buf);
  }
  if (!shapes) return fail(TRIOT_ERR_NULL, "shapes is NULL");
  int64_t I[kMaxRank];
  for (int k = 0; k < n; ++k) {
    if (!shapes[k]) return fail(TRIOT_ERR_NULL, "a shape pointer is NULL");
    for (int i = 0; i < rank; ++i) {
      const int64_t e = shapes[k][i];
      if (e < 0) {
        snprintf(buf, sizeof buf, "negative extent on axis %d of tensor %d", i, k);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      if (e >= (int64_t(1) << 31)) {
        snprintf(buf, sizeof buf, "extent %lld on axis %d of tensor %d must be < 2^31", (long long)e, i, k);
        return fail(TRIOT_ERR_SHAPE, buf);
      }
      I[i] = k == 0 ? e : std::min(I[i], e);
    }
  }
  // element strides of every tensor (row-major in its own shape)
  int64_t st[kMProdMaxTensors][kMaxRank];
  for (int k = 0; k < n; ++k) {
    int64_t s = 1;
    for (int i = rank - 1; i >= 0; --i) {
      st[k][i] = s;
      const int64_t e = shapes[k][i] > 0 ? shapes[k][i] : 1;
      if (mul_overflows(s, e)) return fail(TRIOT_ERR_SHAPE, "element count overflows int64");
      s *= e;
    }
  }
  int64_t total = 1;
  for (int i = 0; i < rank; ++i) {
    if (mul_overflows(total, I[i])) return fail(TRIOT_ERR_SHAPE, "element count overflows int64");
    total *= I[i];
  }
  L = MProdLaunch();
  MProdGeom& g = L.g;
  CombineGeom& cg = L.cg;
  cg.rank = rank;
  // drop I's unit axes (their digit is always 0)
  int D = 0;
  for (int i = 0; i < rank; ++i) {
    if (I[i] == 1) continue;
    g.ext[D] = I[i];
    for (int k = 0; k < n; ++k) g.stride[k][D] = st[k][i];
    cg.orig[D] = i;
    ++D;
  }
  if (D == 0) {  // a single element
    g.ext[0] = 1;
    for (int k = 0; k < n; ++k) g.stride[k][0] = 0;
    cg.orig[0] = rank - 1;
    D = 1;
  }
  g.D = D;
  cg.D = D;
  for (int k = 0; k < n; ++k) g.x[k] = ptrs ? ptrs[k] : nullptr;
  g.unit_inner = 1;
  for (int k = 0; k < n; ++k) g.unit_inner = g.unit_inner && g.stride[k][D - 1] == 1;
  for (int a = 0; a < D; ++a) g.div[a] = make_fastdiv((uint32_t)std::max<int64_t>(1, g.ext[a]));
  L.empty = total == 0;
  g.L = g.ext[D - 1];
  g.nrows = L.empty ? 0 : total / g.L;
  g.nround = (g.nrows + 31) / 32;
  g.n32 = g.nrows < (int64_t(1) << 32);
  // digits of a 32-row step over the outer axes; the outermost axis takes the remainder
  {
    unsigned long long J = 32;
    for (int a = D - 2; a >= 1; --a) {
      g.jd[a] = (uint32_t)(J % (unsigned long long)g.ext[a]);
      J /= (unsigned long long)g.ext[a];
    }
    if (D >= 2) g.jd[0] = (uint32_t)J;
  }
  if (L.empty) {
    cg.nparts = 0;
    return TRIOT_OK;
  }
  DeviceInfo dev;
  int s = device_info(dev);
  if (s) return s;
  // rows shorter than kMPRowsMaxL: CTA tiles of rows, streamed with a fixed column per thread
  if (D >= 2 && g.L < kMPRowsMaxL && g.nrows < (int64_t(1) << 31)) {
    const void* fr = moment_prod_rows_kernel_ptr(dtype, n);
    if (!fr) return fail(TRIOT_ERR_ARG, "no kernel for this dtype and tensor count");
    L.rows = true;
    MPRowsGeom& rg = L.rg;
    rg.rp = (kMPRowsWarps * 32) / (int)g.L;
    rg.tile_rows = rg.rp * std::max(1, std::min(kMPRowsTileElems / (rg.rp * (int)g.L), kMPRowsTileRows / rg.rp));
    rg.ldiv = make_fastdiv((uint32_t)g.L);
    int occ = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fr, kMPRowsWarps * 32, 0);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    const long long ntiles = (g.nrows + rg.tile_rows - 1) / rg.tile_rows;
    L.grid = (int)std::max(1ll, std::min(ntiles, (long long)dev.sms * std::max(1, occ)));
    L.smem = 0;
    cg.nparts = L.grid;
    if (L.grid > kMaxMomentParts) return fail(TRIOT_ERR_ARG, "grid exceeds the partial limit");
    return TRIOT_OK;
  }
  const void* fn = moment_prod_kernel_ptr(dtype, n);
  if (!fn) return fail(TRIOT_ERR_ARG, "no kernel for this dtype and tensor count");
  L.smem = (size_t)mprod_dyn_smem(D - 1);
  int occ = 1;
  if ((s = mprod_occupancy(fn, L.smem, occ))) return s;
  const long long need = (g.nround + kMProdWarps - 1) / kMProdWarps;
  const long long cap = (long long)dev.sms * occ;
  L.grid = (int)std::max(1ll, std::min(need, cap));
  cg.nparts = L.grid;
  if (L.grid > kMaxMomentParts) return fail(TRIOT_ERR_ARG, "grid exceeds the partial limit");
  return TRIOT_OK;
}

size_t mprod_ws_bytes(const MProdLaunch& L) {
  const size_t b = size_t(L.grid) * size_t(L.g.D + 1) * sizeof(double);
  return b < 16 ? 16 : b;
}

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" {

int triot_moment_product_workspace_size(int rank, int ntensors, const int64_t* const* shapes, int dtype,
                                        size_t* bytes) {
  if (!bytes) return fail(TRIOT_ERR_NULL, "bytes is NULL");
  MProdLaunch L;
  int st = plan_mprod(rank, ntensors, shapes, dtype, nullptr, L);
  if (st) return st;
  *bytes = mprod_ws_bytes(L);
  return ok();
}

int triot_moment_product(int rank, int ntensors, const int64_t* const* shapes, const void* const* tensors,
                         int dtype, double* out, void* workspace, size_t workspace_bytes, void* stream) {
  MProdLaunch L;
  int st = plan_mprod(rank, ntensors, shapes, dtype, tensors, L);
  if (st) return st;
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if (!L.empty) {
    if (!tensors) return fail(TRIOT_ERR_NULL, "tensors is NULL");
    for (int k = 0; k < ntensors; ++k)
      if (!tensors[k]) return fail(TRIOT_ERR_NULL, "a tensor pointer is NULL");
  }
  if (!workspace) return fail(TRIOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % 16) return fail(TRIOT_ERR_WORKSPACE, "workspace is not 16-byte aligned");
  if (workspace_bytes < mprod_ws_bytes(L)) {
    char buf[128];
    snprintf(buf, sizeof buf, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes,
             mprod_ws_bytes(L));
    return fail(TRIOT_ERR_WORKSPACE, buf);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  double* part = static_cast<double*>(workspace);
  if (!L.empty) {
    if (L.rows) {
      void* args[] = {(void*)&L.g, (void*)&L.rg, (void*)&part};
      e = cudaLaunchKernel(moment_prod_rows_kernel_ptr(dtype, ntensors), dim3(L.grid), dim3(kMPRowsWarps * 32), args,
                           0, s);
    } else {
      void* args[] = {(void*)&L.g, (void*)&part};
      e = cudaLaunchKernel(moment_prod_kernel_ptr(dtype, ntensors), dim3(L.grid), dim3(kMProdWarps * 32), args,
                           L.smem, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "moment-product kernel launch");
  }
  // the combine is a programmatic dependent of the kernel: its launch overlaps the kernel's
  // tail and its first instruction waits for the kernel's completion
  const double* partc = part;
  void* cargs[] = {(void*)&L.cg, (void*)&partc, (void*)&out};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.g.D + 1);
  cfg.blockDim = dim3(kCombineThreadsHost);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = L.empty ? 0 : 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, combine_kernel_ptr(), cargs);
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel launch");
  return ok();
}

}  // extern "C"
