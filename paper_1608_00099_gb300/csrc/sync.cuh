// Bounded waits on shared-memory mbarriers (completion of staged bulk copies).
#pragma once

namespace triot {

// try_wait polls of a wait for a staged copy before it gives up
constexpr int kWaitLimit = 1 << 22;

// Poll the phase of parity `par` of the mbarrier at shared address `bar` at most `limit`
// times; true once the phase has completed.  A caller that gets false records it in its
// sticky device flag (read by triot_device_status) and goes on, so the kernel always ends.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned par, int limit) {
  unsigned done = 0;
  for (int it = 0; it < limit && !done; ++it)
    asm volatile(
        "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2; selp.u32 %0, 1, 0, P; }"
        : "=r"(done)
        : "r"(bar), "r"(par)
        : "memory");
  return done != 0;
}

}  // namespace triot
