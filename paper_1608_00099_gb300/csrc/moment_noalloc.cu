// triot_moment_noalloc: the moment for callers that cannot allocate device memory.
//
// triot_moment needs a caller-provided workspace for its per-block partial sums.  Some
// callers have no way to get one: they cannot call cudaMalloc (for example a plugin or
// callback that runs where device allocation is forbidden or would synchronise the
// device, or an application whose device memory is handed out entirely by its own pool).
// This entry point keeps the partial sums in a fixed file-scope device array instead, so
// the call itself allocates nothing.  The array is part of the library image: every GPU
// that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {

// The partials scratch: TRIOT_MOMENT_NOALLOC_MAX_DOUBLES doubles (512 KiB).
static __device__ __align__(256) double g_moment_scratch[TRIOT_MOMENT_NOALLOC_MAX_DOUBLES];

namespace {

// Device address of g_moment_scratch, looked up once per device with that device current.
// In host code the array's name is only a host-side stand-in; kernels must be given the
// address cudaGetSymbolAddress returns.
int scratch_address(double** out) {
  static std::mutex mu;
  static double* addr[64] = {};
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(TRIOT_ERR_ARG, "device ordinal out of range for the scratch table");
  std::lock_guard<std::mutex> lk(mu);
  if (!done[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_moment_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(moment scratch)");
    addr[dev] = static_cast<double*>(p);
    done[dev] = true;
  }
  *out = addr[dev];
  return TRIOT_OK;
}

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" int triot_moment_noalloc(int rank, const int64_t* shape, const void* p, int dtype,
                                    double* out, void* stream) {
  MomentLaunch L;
  int st = plan_moment_call(rank, shape, dtype, p, nullptr, L);
  if (st) return st;
  if (!out) return fail(TRIOT_ERR_NULL, "out is NULL");
  if (!L.empty && !p) return fail(TRIOT_ERR_NULL, "p is NULL");
  const size_t need = size_t(L.grid) * size_t(L.g.D + 1);
  if (need > size_t(TRIOT_MOMENT_NOALLOC_MAX_DOUBLES)) {
    char buf[192];
    snprintf(buf, sizeof buf,
             "moment needs %zu partial doubles but the no-allocation scratch holds %d; use triot_moment "
             "with a caller workspace",
             need, TRIOT_MOMENT_NOALLOC_MAX_DOUBLES);
    return fail(TRIOT_ERR_WORKSPACE, buf);
  }
  double* scratch = nullptr;
  if ((st = scratch_address(&scratch))) return st;
  // Every partial the combine reads is written by the moment kernel of this call first,
  // so nothing in the scratch needs clearing.
  return launch_moment(L, dtype, p, out, scratch, (cudaStream_t)stream);
}
