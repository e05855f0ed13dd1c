// Internal definitions shared by the host planner and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fastdiv.cuh"

namespace triot {

constexpr int kMaxRank = 24;
constexpr int kMomentWarps = 4;     // warps per CTA of the row-mode moment kernels

// f64 block-column moment: blocks of B elements per staged chunk (the smallest count that
// covers 16 elements with an even number of elements, so chunks are whole 16-byte pieces)
__host__ __device__ constexpr int b64_blocks_per_chunk(int b) {
  return (((16 + b - 1) / b) * b) % 2 ? (16 + b - 1) / b + 1 : (16 + b - 1) / b;
}

// f64 block kernel: warps per CTA, staged rounds per warp, bytes of one lane row of a stage
// (an odd number of 16-byte units: conflict-free 16-byte reads across lanes), and its dynamic
// shared memory: the stages, then lane-major per-axis state (128-bit axis sums and 32-bit
// digits of axes 0..DO-4, 128-bit pending masses of axes 0..DO-5, and the lane's f64 totals
// of axes 0..DO-1)
constexpr int kB64Warps = 2;
constexpr int kB64Stages = 2;
constexpr int kB64Window = 1024;  // elements a lane sums in one fixed-point window
__host__ __device__ constexpr int b64_row_bytes(int b) {
  return b64_blocks_per_chunk(b) * b * 8 + (((b64_blocks_per_chunk(b) * b / 2) & 1) ? 0 : 16);
}
__host__ __device__ constexpr int b64_stage_bytes(int b) { return kB64Warps * kB64Stages * 32 * b64_row_bytes(b); }
__host__ __device__ constexpr int b64_levels(int DO) { return DO >= 4 ? DO - 3 : 0; }
__host__ __device__ constexpr int b64_qlevels(int DO) { return DO >= 5 ? DO - 4 : 0; }
__host__ __device__ constexpr int b64_dyn_smem(int b, int DO) {
  return b64_stage_bytes(b) +
         kB64Warps * 32 * (b64_levels(DO) * 20 + b64_qlevels(DO) * 16 + DO * 8);
}

// ROW_EMBED_S: embed into a view of a larger tensor (A's row offsets from its strides); a
// separate instantiation so that the dense embed's row decode carries no extra branch
enum RowOp { ROW_EMBED = 0, ROW_CROP = 1, ROW_PRODUCT = 2, ROW_EMBED_S = 3 };

// Element types of the kernels.
enum Dtype { DT_F64 = 0, DT_F32 = 1, DT_BF16 = 2, DT_F16 = 3 };

inline int dtype_size(int dt) { return dt == DT_F64 ? 8 : dt == DT_F32 ? 4 : 2; }

// ------------------------------------------------------------------ canonical form
//
// A call's shapes reduced for launch (Section 4: trivial axes are ignored; adjacent axes
// that are contiguous in every tensor behave as one axis).  Axes are listed outermost
// first.  Strides are in elements.  For embed the iteration space is y and `bound` holds
// x's extent per axis; for crop it is x; for product it is the intersection I; for the
// moment it is p (no merging: every axis has its own output).
struct Canon {
  int D = 0;                       // effective rank, >= 1
  int64_t ext[kMaxRank];           // iteration extents
  int64_t sa[kMaxRank];            // strides of tensor A (the written tensor)
  int64_t sb[kMaxRank];            // strides of tensor B (the read tensor)
  int64_t bound[kMaxRank];         // embed: x's extent per axis
  int orig[kMaxRank];              // moment: original axis of each effective axis
  int64_t total = 0;               // number of iterated elements
  bool empty = false;              // some iteration extent is zero
};

// ------------------------------------------------------------------ row kernels
//
// The iteration space is viewed as `rows` rows of `inner` contiguous elements; a row is a
// tuple of the outer axes.  Outer-axis data is stored innermost first: entry k describes
// canonical axis D-2-k.  A tile is either a run of whole rows or one segment of a row.
struct RowInfo {
  long long a;   // offset of the row in A
  long long b;   // offset of the row in B, or -1 (embed: row outside x)
};

struct RowGeom {
  int nouter;                      // outer axes (D - 1)
  int path;                        // PATH_* below, uniform for the launch
  FastDiv div[kMaxRank];           // outer extents (innermost first) for the decode
  long long ext[kMaxRank];         // outer extents (innermost first)
  long long sa[kMaxRank];          // A strides per outer axis
  long long sb[kMaxRank];          // B strides per outer axis
  long long bound[kMaxRank];       // embed: x extent per outer axis
  long long rows;                  // number of rows
  long long inner;                 // row length (iteration)
  long long b_inner;               // embed: x's extent of the inner axis
  long long rows_per_tile;         // multi-row tiles
  long long segs_per_row;          // > 1: a tile is one segment of a row
  long long seg_len;               // segment length (multiple of the vector width)
  long long ntiles;
  FastDiv inner_div;               // divisor = inner (only when inner < 2^31)
  FastDiv seg_div;                 // divisor = segs_per_row
  int rows32;                      // rows fit the 32-bit decode
  int nopad;                       // embed: skip writing the pad
  int a_dense;                     // A's rows lie back to back (offset = row * inner); 0 for
                                   // a view of a larger tensor (host: selects ROW_EMBED_S)
};

enum {
  PATH_VEC = 0,   // vector slots inside one row; B loaded as a vector
  PATH_ROW = 1,   // vector slots inside one row; B loaded per element
  PATH_GEN = 2    // one element at a time (any row length, any alignment)
};

// ------------------------------------------------------------------ moment
struct MomentGeom {
  int D;                           // effective rank
  int m;                           // block mode: the last m axes form blocks of B elements
  int B;                           // (m = 0: row mode, the inner axis alone)
  int nchunks;                     // chunks per lane segment (the last may be partial); warp
                                   // blocks: blocks per staged step
  long long n;                     // elements
  long long seg;                   // lane segment length S (multiple of the chunk)
  long long nwarpseg;              // warp segments (32 lane segments each)
  int n32;                         // n < 2^32: 32-bit decode
  int aligned;                     // p is 16-byte aligned: cp.async staging
  long long nround;                // block kernels: rounds of 32 chunks (warp blocks: blocks)
  int win;                         // block kernels: rounds (warp blocks: blocks) per window
  FastDiv div[kMaxRank];           // extents (axis order, outermost first)
  long long ext[kMaxRank];         // extents (axis order, outermost first)
};

// Moment of a product of tensors over the intersection I of their shapes.  I's unit axes
// are dropped (their digit is always 0); axis D-1 is the row (inner) axis.
constexpr int kMProdMaxTensors = 4;
constexpr int kMProdWarps = 4;           // warps per CTA
constexpr int kMProdWindow = 1024;       // elements a lane sums in one fixed-point window
constexpr int kMProdLC = 8;              // row elements a lane loads before using any
struct MProdGeom {
  int D;                                 // rank of the canonical I (>= 1)
  int unit_inner;                        // every tensor has stride 1 on the row axis
  long long L;                           // row length (extent of axis D-1)
  long long nrows;                       // rows: product of the extents of axes 0..D-2
  long long nround;                      // rounds of 32 rows
  long long ext[kMaxRank];               // extents of I
  FastDiv div[kMaxRank];                 // the same, for the 32-bit decode
  int n32;                               // nrows < 2^32
  uint32_t jd[kMaxRank];                 // digits of a 32-row step, axes 0..D-2 (axis 0 takes
                                         // the remainder)
  const void* x[kMProdMaxTensors];       // the tensors
  long long stride[kMProdMaxTensors][kMaxRank];  // their element strides on I's axes
};
__host__ __device__ constexpr int mprod_levels(int DO) { return DO >= 4 ? DO - 3 : 0; }
__host__ __device__ constexpr int mprod_qlevels(int DO) { return DO >= 5 ? DO - 4 : 0; }
__host__ __device__ constexpr int mprod_dyn_smem(int DO) {
  return kMProdWarps * 32 * (mprod_levels(DO) * 20 + mprod_qlevels(DO) * 16 + DO * 8);
}

struct CombineGeom {
  int D;                           // effective rank
  int rank;                        // caller's rank (output length rank + 1)
  int nparts;                      // partial vectors in the workspace
  int orig[kMaxRank];              // output index of each effective axis
};

}  // namespace triot
