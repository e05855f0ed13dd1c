// Launch geometry of the block-column moment for f32, bf16 and f16 storage (float sums),
// shared by the host planner and the kernel.
#pragma once

namespace triot {

constexpr int kB32Warps = 4;    // warps per CTA
constexpr int kB32Stages = 2;   // staged rounds per warp
constexpr int kB32Terms = 64;   // blocks (and column terms) a lane sums in one float window

// blocks per chunk: a chunk is a whole number of 16-byte pieces and at least 128 bytes
__host__ __device__ constexpr int b32_blocks_per_chunk(int b, int es) {
  int k = 1;
  while ((k * b * es) % 16 != 0 || k * b * es < 128) ++k;
  return k;
}
// bytes of one lane row of a stage: the chunk, plus 16 bytes when its piece count is even,
// so that the lanes' 16-byte reads at equal offsets fall in distinct banks
__host__ __device__ constexpr int b32_row_bytes(int b, int es) {
  return b32_blocks_per_chunk(b, es) * b * es +
         (((b32_blocks_per_chunk(b, es) * b * es / 16) & 1) ? 0 : 16);
}
__host__ __device__ constexpr int b32_stage_bytes(int b, int es) {
  return kB32Warps * kB32Stages * 32 * b32_row_bytes(b, es);
}
// outer axes 0 .. DO-4 keep a lane's sums and digits in shared memory, axes 0 .. DO-5 a
// pending mass (lane-major, after the stages)
__host__ __device__ constexpr int b32_levels(int DO) { return DO >= 4 ? DO - 3 : 0; }
__host__ __device__ constexpr int b32_qlevels(int DO) { return DO >= 5 ? DO - 4 : 0; }
__host__ __device__ constexpr int b32_dyn_smem(int b, int es, int DO) {
  return b32_stage_bytes(b, es) + kB32Warps * 32 * (b32_levels(DO) * 8 + b32_qlevels(DO) * 4);
}

// Warp-block moment (f32, bf16, f16): blocks of B = 32..256 elements (the trailing axes),
// one block at a time per warp, lane l holding columns l, l + 32, .. (C = ceil(B / 32)).
// A step is U whole blocks (U * B * es <= kWBStepBytes), staged by one bulk copy.
constexpr int kWBWarps = 4;          // warps per CTA
constexpr int kWBStages = 3;         // staged steps per warp
constexpr int kWBMaxC = 8;           // columns per lane (B <= 256)
constexpr int kWBStepBytes = 4096;   // bytes of one step (whole blocks)
constexpr int kWBStageBytes = kWBStepBytes + 32;  // a stage: the step widened to 16-byte bounds
constexpr int kWBTerms = 64;         // blocks a lane sums in one float window
// blocks of a whole number of 512-byte rows (32 lanes x 16 bytes) are read with direct
// 16-byte loads instead of staged copies
__host__ __device__ constexpr bool wb_vec(int b, int es) { return (b * es) % 512 == 0; }
// dynamic shared memory: the stages (staged reads only), then (lane-major) the sums and
// digits of outer axes 0 .. DO-3 and the pending masses of axes 0 .. DO-4
__host__ __device__ constexpr int wb_levels(int DO) { return DO >= 3 ? DO - 2 : 0; }
__host__ __device__ constexpr int wb_qlevels(int DO) { return DO >= 4 ? DO - 3 : 0; }
__host__ __device__ constexpr int wb_stage_smem(bool vec) {
  return vec ? 0 : kWBWarps * kWBStages * kWBStageBytes;
}
__host__ __device__ constexpr int wb_dyn_smem(int DO, bool vec) {
  return wb_stage_smem(vec) + kWBWarps * 32 * (wb_levels(DO) * 8 + wb_qlevels(DO) * 4);
}

}  // namespace triot
