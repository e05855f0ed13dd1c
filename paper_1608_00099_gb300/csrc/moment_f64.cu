// Instantiations of the f64 (fixed-point) moment kernel for every rank.
#include <utility>

#include "kernels.h"
#include "moment.cuh"

namespace triot {
namespace {
template <int... N>
const void* pick(int d, std::integer_sequence<int, N...>) {
  static const void* const table[] = {reinterpret_cast<const void*>(&moment_f64_kernel<N + 1>)...};
  return table[d - 1];
}
}  // namespace

const void* moment_f64_ptr(int D) { return pick(D, std::make_integer_sequence<int, kMaxRank>{}); }
}  // namespace triot
