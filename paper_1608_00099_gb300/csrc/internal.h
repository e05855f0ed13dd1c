// Internal host-side interfaces shared by the C ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "plan.h"

namespace triot {

constexpr int kMaxMomentParts = 16384;   // partial vectors a moment launch may produce
constexpr int kCombineThreadsHost = 256;  // threads of the combine kernel

int fail(int code, const std::string& msg);
int ok();
int cuda_fail(cudaError_t e, const char* what);
int device_info(DeviceInfo& out);
bool valid_dtype(int dt);
bool overlaps_bytes(const void* a, size_t na, const void* b, size_t nb);

// row ops with an explicit geometry (force != nullptr) or the cached one
// xdata / ydata: container shapes when x / y are views (their pointers already carry the
// view's bias); nullptr for whole tensors
int launch_rows(int op, int rank, const int64_t* xshape, const void* x, const int64_t* yshape,
                const void* y, int dtype, unsigned flags, cudaStream_t stream, const TuneCfg* force,
                const int64_t* xdata = nullptr, const int64_t* ydata = nullptr);

// moment: plan, workspace bytes, launch
int plan_moment_call(int rank, const int64_t* shape, int dtype, const void* p, const TuneCfg* force,
                     MomentLaunch& L);
size_t moment_ws_bytes(const MomentLaunch& L);
int launch_moment(const MomentLaunch& L, int dtype, const void* p, double* out, void* ws,
                  cudaStream_t stream);
int moment_call(int rank, const int64_t* shape, const void* p, int dtype, double* out, void* ws,
                size_t ws_bytes, cudaStream_t stream, const TuneCfg* force);

// tuning cache (tune.cpp)
TuneCfg tune_lookup(int op, int dtype, const Canon& c);
void tune_store(int op, int dtype, const Canon& c, const TuneCfg& t);
// batches (TRIOT_OP_BATCH): keyed by dtype, mode and size class
std::string batch_key(int dtype, int mode, long long npairs, long long ny_total);
TuneCfg tune_lookup_key(const std::string& k);
void tune_store_key(const std::string& k, const TuneCfg& t);

// device-side guard flag (batch.cu)
void st_read_device_flag(int* flag);
// the bounded-wait self-test's flag (selftest.cu)
void selftest_read_device_flag(int* flag);

}  // namespace triot
