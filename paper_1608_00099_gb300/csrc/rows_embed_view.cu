// Instantiations of the embed row kernel for a view of a larger tensor (the written rows
// addressed through the view's strides, Section 4's biased slice), by element size and rank.
#include <utility>

#include "kernels.h"
#include "rows.cuh"

namespace triot {
namespace {
template <typename T, int... N>
const void* pick(int n, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&rows_kernel<ROW_EMBED_S, T, N>)...};
  return table[n];
}
}  // namespace

const void* embed_view_kernel_ptr(int es, int nouter) {
  if (nouter < 0 || nouter >= kMaxRank) return nullptr;
  auto seq = std::make_integer_sequence<int, kMaxRank>{};
  if (es == 8) return pick<unsigned long long>(nouter, seq);
  if (es == 4) return pick<unsigned int>(nouter, seq);
  if (es == 2) return pick<unsigned short>(nouter, seq);
  return nullptr;
}
}  // namespace triot
