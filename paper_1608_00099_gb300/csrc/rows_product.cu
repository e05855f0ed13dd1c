// Instantiations of the product row kernel by dtype for every rank.
#include <utility>

#include "kernels.h"
#include "rows.cuh"

namespace triot {
namespace {
template <typename T, int... N>
const void* pick(int n, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&rows_kernel<ROW_PRODUCT, T, N>)...};
  return table[n];
}
}  // namespace

const void* product_kernel_ptr(int dtype, int nouter) {
  if (nouter < 0 || nouter >= kMaxRank) return nullptr;
  auto seq = std::make_integer_sequence<int, kMaxRank>{};
  switch (dtype) {
    case DT_F64: return pick<double>(nouter, seq);
    case DT_F32: return pick<float>(nouter, seq);
    case DT_BF16: return pick<__nv_bfloat16>(nouter, seq);
    case DT_F16: return pick<__half>(nouter, seq);
  }
  return nullptr;
}
}  // namespace triot
