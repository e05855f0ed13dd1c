// C ABI of the TRIOT hot path: validation, canonicalisation, per-rank dispatch, launch.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/triot.h"
#include "blk32.cuh"
#include "internal.h"
#include "kernels.h"
#include "plan.h"

namespace triot {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int ok() { return TRIOT_OK; }

int cuda_fail(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  return fail(TRIOT_ERR_CUDA, buf);
}

// ------------------------------------------------------------------ devices
int device_info(DeviceInfo& out) {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& d : cache)
    if (d.device == dev) { out = d; return TRIOT_OK; }
  DeviceInfo d;
  d.device = dev;
  e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  snprintf(d.name, sizeof d.name, "%.*s", (int)sizeof d.name - 1, prop.name);
  cache.push_back(d);
  out = d;
  return TRIOT_OK;
}

bool valid_dtype(int dt) { return dt >= TRIOT_F64 && dt <= TRIOT_F16; }

bool overlaps_bytes(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + nb && y < x + na;
}

static int64_t count(int rank, const int64_t* s) {
  int64_t n = 1;
  for (int i = 0; i < rank; ++i) n *= s[i];
  return n;
}

// ------------------------------------------------------------------ row ops
int launch_rows(int op, int rank, const int64_t* xshape, const void* x, const int64_t* yshape,
                const void* y, int dtype, unsigned flags, cudaStream_t stream,
                const TuneCfg* force, const int64_t* xdata, const int64_t* ydata) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (op == ROW_EMBED && (flags & ~TRIOT_EMBED_NOPAD)) return fail(TRIOT_ERR_ARG, "unknown embed flag");
  Canon c;
  bool x_empty = false;
  std::string err;
  int st = canon_rows(op, rank, xshape, yshape, c, x_empty, err, xdata, ydata);
  if (st) return fail(st, err);
  const int es = dtype_size(dtype);
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape);
  // embed writes all of y even when x is empty
  const bool work = (op == ROW_EMBED) ? (ny > 0) : !c.empty;
  if (!work) return ok();
  if ((op != ROW_EMBED || nx > 0) && !x) return fail(TRIOT_ERR_NULL, "x is NULL");
  if (!y) return fail(TRIOT_ERR_NULL, "y is NULL");
  // (views: the caller checks the whole containers)
  if (!xdata && !ydata && x && nx > 0 && overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es))
    return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  DeviceInfo dev;
  if ((st = device_info(dev))) return st;
  TuneCfg t = force ? *force : tune_lookup(op == ROW_EMBED ? TRIOT_OP_EMBED : op == ROW_CROP ? TRIOT_OP_CROP : TRIOT_OP_PRODUCT,
                                           dtype, c);
  // A = written tensor, B = read tensor
  const void* A = (op == ROW_CROP) ? x : y;
  const void* B = (op == ROW_CROP) ? y : x;
  RowLaunch L;
  plan_rows(op, c, x_empty, es, A, B, flags, t, dev, L);
  if (op == ROW_CROP && !L.g.a_dense) return fail(TRIOT_ERR_ARG, "internal: crop into a strided tensor");
  const void* fn = (op == ROW_EMBED) ? (L.g.a_dense ? embed_kernel_ptr(es, L.g.nouter)
                                                    : embed_view_kernel_ptr(es, L.g.nouter))
                   : (op == ROW_CROP) ? crop_kernel_ptr(es, L.g.nouter)
                                      : product_kernel_ptr(dtype, L.g.nouter);
  if (!fn) return fail(TRIOT_ERR_RANK, "no kernel for this effective rank");
  if (L.block < 32 || L.block > 1024 || L.block % 32) return fail(TRIOT_ERR_ARG, "threads must be a multiple of 32 in [32, 1024]");
  // an empty x leaves B unused; give the kernel a valid (never dereferenced) pointer
  const void* Bk = B ? B : A;
  void* args[] = {(void*)&L.g, (void*)&A, (void*)&Bk};
  cudaError_t e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.block), args, L.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "row kernel launch");
  return ok();
}

// ------------------------------------------------------------------ moment
static int moment_occupancy(const void* fn, int threads, size_t dyn, size_t dyn_max, int& occ) {
  struct Entry { const void* fn; size_t dyn; int dev; int occ; };
  static std::mutex mu;
  static std::vector<Entry> table;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& x : table)
    if (x.fn == fn && x.dyn == dyn && x.dev == dev) { occ = x.occ; return TRIOT_OK; }
  if (dyn > 0) {
    // opt in to the largest dynamic shared memory any launch of this kernel can need (the
    // attribute is per kernel, so it must cover every rank, not just this call's)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(max dynamic shared memory)");
  }
  int o = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, threads, dyn);
  if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
  occ = o > 0 ? o : 1;
  table.push_back({fn, dyn, dev, occ});
  return TRIOT_OK;
}

int plan_moment_call(int rank, const int64_t* shape, int dtype, const void* p, const TuneCfg* force,
                     MomentLaunch& L) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  Canon c;
  std::string err;
  int st = canon_moment(rank, shape, c, err);
  if (st) return fail(st, err);
  DeviceInfo dev;
  if ((st = device_info(dev))) return st;
  TuneCfg t = force ? *force : tune_lookup(TRIOT_OP_MOMENT, dtype, c);
  {
    // the marginal split (rows x columns) when the axes give good rows and columns
    const bool f64 = dtype == DT_F64;
    const void* fmx = f64 ? moment_mx64_kernel_ptr() : moment_mx32_kernel_ptr(dtype, 2);
    const int nw = f64 ? kMxWarps : kMx32Warps;
    int occ = 1;
    if ((st = moment_occupancy(fmx, nw * 32, 0, 0, occ))) return st;
    const int cps = t.ctas_per_sm > 0 ? t.ctas_per_sm : occ;
    // only large tensors (float storage also needs rows that can be read 16 bytes at a
    // time; f64 a few rows per warp): the column pass and the row-side set-up at a warp's
    // start and end need enough rows to pay off, and smaller tensors, which are
    // latency-bound, are served better by the row and block kernels below
    const bool eligible = c.total >= (f64 ? kMx64MinElems : kMx32MinElems);
    if (eligible && plan_moment_mx(c, rank, dtype_size(dtype), p, (long long)dev.sms * cps * nw, L) &&
        (f64 || (L.mx.C * dtype_size(dtype)) % 16 == 0) &&
        (!f64 || L.mx.R >= kMxMinRowsPerWarp * L.mx.parts))
      return TRIOT_OK;
    L = MomentLaunch();
  }
  const int m = moment_block_axes(c, dtype);
  int B = 1;
  for (int a = c.D - m; a < c.D; ++a) B *= (int)c.ext[a];
  const void* fn = moment_kernel_ptr(dtype, c.D, m, B);
  if (!fn) return fail(TRIOT_ERR_RANK, "no moment kernel for this effective rank");
  int occ = 1;
  const int es = dtype_size(dtype), Bk = B < 1 ? 1 : B;
  const bool b64 = m > 0 && dtype == DT_F64;
  const bool wb = m > 0 && dtype != DT_F64 && Bk >= 32;
  const bool b32 = m > 0 && dtype != DT_F64 && Bk < 32;
  const size_t dyn = b64 ? (size_t)b64_dyn_smem(Bk, c.D - m)
                     : b32 ? (size_t)b32_dyn_smem(Bk, es, c.D - m)
                     : wb ? (size_t)wb_dyn_smem(c.D - m, wb_vec(Bk, es)) : 0;
  const size_t dyn_max = b64 ? (size_t)b64_dyn_smem(Bk, kMaxRank - 1)
                         : b32 ? (size_t)b32_dyn_smem(Bk, es, kMaxRank - 1)
                         : wb ? (size_t)wb_dyn_smem(kMaxRank - 1, wb_vec(Bk, es)) : 0;
  const int threads = (b64 ? kB64Warps : b32 ? kB32Warps : wb ? kWBWarps : kMomentWarps) * 32;
  if ((st = moment_occupancy(fn, threads, dyn, dyn_max, occ))) return st;
  L.kind = MOMENT_KIND_ROWS_BLOCKS;
  plan_moment(c, rank, dtype_size(dtype), m, p, t, dev, occ, L);
  L.smem = dyn;
  if (L.grid > kMaxMomentParts) return fail(TRIOT_ERR_ARG, "moment grid exceeds the partial limit");
  return TRIOT_OK;
}

size_t moment_ws_bytes(const MomentLaunch& L) {
  const size_t b = size_t(L.grid) * size_t(L.g.D + 1) * sizeof(double);
  return b < 16 ? 16 : b;
}

int launch_moment(const MomentLaunch& L, int dtype, const void* p, double* out, void* ws,
                  cudaStream_t stream) {
  cudaError_t e;
  if (L.kind == MOMENT_KIND_MX) {
    double* part = static_cast<double*>(ws);
    void* args[] = {(void*)&L.mx, (void*)&p, (void*)&part};
    const void* fn = dtype == DT_F64 ? moment_mx64_kernel_ptr() : moment_mx32_kernel_ptr(dtype, L.mx.V);
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.warps * 32), args, 0, stream);
    if (e != cudaSuccess) return cuda_fail(e, "moment kernel launch");
  } else if (!L.empty) {
    const void* fn = moment_kernel_ptr(dtype, L.g.D, L.g.m, L.g.B);
    if (!fn) return fail(TRIOT_ERR_RANK, "no moment kernel for this effective rank");
    double* part = static_cast<double*>(ws);
    void* args[] = {(void*)&L.g, (void*)&p, (void*)&part};
    e = cudaLaunchKernel(fn, dim3(L.grid), dim3(L.warps * 32), args, L.smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "moment kernel launch");
  }
  const double* partc = static_cast<const double*>(ws);
  void* cargs[] = {(void*)&L.cg, (void*)&partc, (void*)&out};
  // the combine as a programmatic dependent launch (it waits for the moment kernel itself)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.g.D + 1);
  cfg.blockDim = dim3(kCombineThreadsHost);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = L.empty ? 0 : 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelExC(&cfg, combine_kernel_ptr(), cargs);
  if (e != cudaSuccess) return cuda_fail(e, "combine kernel launch");
  return ok();
}

int moment_call(int rank, const int64_t* shape, const void* p, int dtype, double* out, void* ws,
                size_t ws_bytes, cudaStream_t stream, const TuneCfg* force) {
  MomentLaunch L;
  int st = plan_moment_call(rank, shape, dtype, p, force, L);
  if (st) return st;
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if (!L.empty && !p) return fail(TRIOT_ERR_NULL, "p is NULL");
  if (!ws) return fail(TRIOT_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 16) return fail(TRIOT_ERR_WORKSPACE, "workspace is not 16-byte aligned");
  if (ws_bytes < moment_ws_bytes(L)) {
    char buf[128];
    snprintf(buf, sizeof buf, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, moment_ws_bytes(L));
    return fail(TRIOT_ERR_WORKSPACE, buf);
  }
  return launch_moment(L, dtype, p, out, ws, stream);
}

}  // namespace triot

using namespace triot;

// ====================================================================== C ABI

extern "C" {

const char* triot_last_error(void) { return g_err.c_str(); }

const char* triot_version(void) { return "triot-gb300 1.0 sm_103a"; }

int triot_embed(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                int dtype, unsigned flags, void* stream) {
  return launch_rows(ROW_EMBED, rank, xshape, x, yshape, y, dtype, flags, (cudaStream_t)stream, nullptr);
}

int triot_crop(int rank, const int64_t* xshape, void* x, const int64_t* yshape, const void* y,
               int dtype, void* stream) {
  // crop writes x: pass x as the written tensor through the same launcher
  return launch_rows(ROW_CROP, rank, xshape, x, yshape, y, dtype, 0, (cudaStream_t)stream, nullptr);
}

int triot_product(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                  int dtype, void* stream) {
  return launch_rows(ROW_PRODUCT, rank, xshape, x, yshape, y, dtype, 0, (cudaStream_t)stream, nullptr);
}

int triot_moment_workspace_size(int rank, const int64_t* shape, int dtype, size_t* bytes) {
  if (!bytes) return fail(TRIOT_ERR_NULL, "bytes is NULL");
  MomentLaunch L;
  int st = plan_moment_call(rank, shape, dtype, nullptr, nullptr, L);
  if (st) return st;
  *bytes = moment_ws_bytes(L);
  return ok();
}

int triot_moment_plan(int rank, const int64_t* shape, int dtype, int* kernel, int* grid, int64_t* rows,
                      int64_t* cols) {
  MomentLaunch L;
  int st = plan_moment_call(rank, shape, dtype, nullptr, nullptr, L);
  if (st) return st;
  int k = TRIOT_MK_ROWS;
  if (L.kind == MOMENT_KIND_MX) k = TRIOT_MK_MARGINALS;
  else if (L.g.m > 0 && dtype == DT_F64) k = TRIOT_MK_BLOCKS64;
  else if (L.g.m > 0 && L.g.B >= 32) k = TRIOT_MK_WARPBLOCKS;
  else if (L.g.m > 0) k = TRIOT_MK_BLOCKS32;
  if (kernel) *kernel = k;
  if (grid) *grid = L.empty ? 0 : L.grid;
  if (rows) *rows = L.kind == MOMENT_KIND_MX ? L.mx.R : 0;
  if (cols) *cols = L.kind == MOMENT_KIND_MX ? L.mx.C : 0;
  return ok();
}

int triot_moment(int rank, const int64_t* shape, const void* p, int dtype, double* out,
                 void* workspace, size_t workspace_bytes, void* stream) {
  return moment_call(rank, shape, p, dtype, out, workspace, workspace_bytes, (cudaStream_t)stream, nullptr);
}

int triot_canonicalize(int op, int rank, const int64_t* xshape, const int64_t* yshape, int* eff_rank,
                       int64_t* ext, int64_t* xstride, int64_t* ystride, int64_t* xbound, int* orig) {
  if (!eff_rank || !ext) return fail(TRIOT_ERR_NULL, "output pointer is NULL");
  Canon c;
  std::string err;
  int st;
  if (op == TRIOT_OP_MOMENT) {
    st = canon_moment(rank, xshape, c, err);
    if (st) return fail(st, err);
    *eff_rank = c.D;
    for (int i = 0; i < c.D; ++i) {
      ext[i] = c.ext[i];
      if (xstride) xstride[i] = 0;
      if (ystride) ystride[i] = 0;
      if (xbound) xbound[i] = c.ext[i];
      if (orig) orig[i] = c.orig[i];
    }
    return ok();
  }
  const int rop = op == TRIOT_OP_EMBED ? ROW_EMBED : op == TRIOT_OP_CROP ? ROW_CROP : op == TRIOT_OP_PRODUCT ? ROW_PRODUCT : -1;
  if (rop < 0) return fail(TRIOT_ERR_ARG, "unknown op");
  bool x_empty = false;
  st = canon_rows(rop, rank, xshape, yshape, c, x_empty, err);
  if (st) return fail(st, err);
  *eff_rank = c.D;
  // A is the written tensor (y for embed/product, x for crop), B the read one
  for (int i = 0; i < c.D; ++i) {
    ext[i] = c.ext[i];
    if (xstride) xstride[i] = (rop == ROW_CROP) ? c.sa[i] : c.sb[i];
    if (ystride) ystride[i] = (rop == ROW_CROP) ? c.sb[i] : c.sa[i];
    if (xbound) xbound[i] = c.bound[i];
    if (orig) orig[i] = c.orig[i];
  }
  return ok();
}

int triot_fastdiv_check(uint32_t d, const uint32_t* n, size_t count, uint32_t* q, uint32_t* r) {
  if (d == 0) return fail(TRIOT_ERR_ARG, "divisor is zero");
  if (count && (!n || !q || !r)) return fail(TRIOT_ERR_NULL, "array pointer is NULL");
  const FastDiv f = make_fastdiv(d);
  for (size_t k = 0; k < count; ++k) {
    uint32_t rr;
    q[k] = fdivmod(n[k], f, rr);
    r[k] = rr;
  }
  return ok();
}

int triot_device_status(void) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
  int flag = 0, flag2 = 0, flag3 = 0, flag4 = 0, flag5 = 0;
  st_read_device_flag(&flag);
  b64_read_device_flag(&flag2);
  b32_read_device_flag(&flag3);
  wb_read_device_flag(&flag4);
  selftest_read_device_flag(&flag5);
  return (flag || flag2 || flag3 || flag4 || flag5) ? fail(TRIOT_ERR_DEVICE, "a device-side guard tripped")
                                                    : ok();
}

}  // extern "C"
