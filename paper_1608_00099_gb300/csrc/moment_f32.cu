// Instantiations of the f32-accumulating moment kernel (f32, bf16, f16 storage) for every
// rank, and the dtype/rank dispatch of the moment.
#include <utility>

#include "kernels.h"
#include "moment.cuh"

namespace triot {
const void* moment_f64_ptr(int D);
namespace {
template <typename T, int... N>
const void* pick(int d, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_f32_kernel<T, N + 1>)...};
  return table[d - 1];
}
}  // namespace

const void* moment_kernel_ptr(int dtype, int D, int m, int B) {
  if (D < 1 || D > kMaxRank) return nullptr;
  if (m > 0) {
    if (m > D) return nullptr;
    if (B < 1) B = 1;  // an empty tensor: no launch, any instantiation serves the planner
    if (dtype == DT_F64) return moment_blk64_kernel_ptr(B, D - m);
    return B >= 32 ? moment_wb_kernel_ptr(dtype, B) : moment_blk32_kernel_ptr(dtype, B);
  }
  auto seq = std::make_integer_sequence<int, kMaxRank>{};
  switch (dtype) {
    case DT_F64: return moment_f64_ptr(D);
    case DT_F32: return pick<float>(D, seq);
    case DT_BF16: return pick<__nv_bfloat16>(D, seq);
    case DT_F16: return pick<__half>(D, seq);
  }
  return nullptr;
}
}  // namespace triot
