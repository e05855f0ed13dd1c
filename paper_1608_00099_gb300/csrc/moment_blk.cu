// Instantiations of the block-column moment kernel (f32, bf16, f16 storage) for every
// number of outer axes.
#include <utility>

#include "kernels.h"
#include "moment.cuh"

namespace triot {
namespace {
template <typename T, int... N>
const void* pick(int d, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_blk_kernel<T, N>)...};
  return table[d];
}
}  // namespace

const void* moment_blk_kernel_ptr(int dtype, int DO) {
  if (DO < 0 || DO >= kMaxRank) return nullptr;
  auto seq = std::make_integer_sequence<int, kMaxRank>{};
  switch (dtype) {
    case DT_F32: return pick<float>(DO, seq);
    case DT_BF16: return pick<__nv_bfloat16>(DO, seq);
    case DT_F16: return pick<__half>(DO, seq);
  }
  return nullptr;
}
}  // namespace triot
