// Self-test of the failure path of the bounded waits: a wait that gives up must leave a
// status the host can read, and the context must stay usable.  The kernel waits on an
// mbarrier that expects one arrival no thread makes and that no copy targets, so nothing
// is in flight while it waits, and the wait ends after `limit` polls.
#include <cuda_runtime.h>

#include "../../include/triot.h"
#include "internal.h"
#include "sync.cuh"

namespace triot {
namespace {

__device__ int g_selftest_flag = 0;

__global__ void __launch_bounds__(32) wait_timeout_kernel(int limit) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned a = (unsigned)__cvta_generic_to_shared(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // phase 0 never completes: every lane's wait runs out
  if (!mbar_wait_bounded(a, 0u, limit) && threadIdx.x == 0) atomicExch(&g_selftest_flag, 1);
  __syncwarp();
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(a) : "memory");
}

}  // namespace

void selftest_read_device_flag(int* flag) {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_selftest_flag, sizeof(int));
  const int zero = 0;
  cudaMemcpyToSymbol(g_selftest_flag, &zero, sizeof(int));
  *flag = v;
}

}  // namespace triot

using namespace triot;

extern "C" int triot_selftest_wait_timeout(int limit, void* stream) {
  if (limit < 1 || limit > 4096) return fail(TRIOT_ERR_ARG, "limit outside [1, 4096]");
  void* args[] = {(void*)&limit};
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(&wait_timeout_kernel), dim3(1), dim3(32),
                                   args, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "self-test kernel launch");
  return ok();
}
