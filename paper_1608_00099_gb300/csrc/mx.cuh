// Geometry of the moment by marginals (moment_mx.cu): the canonical tensor viewed as an
// R x C matrix of rows (axes 0 .. s-1) and columns (axes s .. D-1).
#pragma once
#include "common.cuh"

namespace triot {

constexpr int kMxWarps = 12;     // warps per CTA
constexpr int kMxMinCtas = 1;    // resident CTAs per SM the register budget is sized for
constexpr int kMxJ = 8;          // columns per lane: a warp tile is 32 * kMxJ columns
constexpr int kMxWindow = 1023;  // rows a lane sums in one fixed-point window (|c| < 2^53)
constexpr int kMxMaxGrid = 16384;  // CTAs (partial vectors) of one launch at most
constexpr long long kMx64MinElems = 1ll << 21;  // f64 tensors this large or larger
constexpr int kMxMinRowsPerWarp = 4;            // and at least this many rows per warp

struct MxGeom {
  int D;                         // effective rank
  int V;                         // float kernel: elements per vector load (1: scalar loads)
  int W;                         // columns of a warp tile
  int s;                         // row axes 0 .. s-1, column axes s .. D-1 (1 <= s < D)
  long long R;                   // rows (< 2^31)
  long long C;                   // columns (< 2^31)
  long long tiles;               // column tiles of W columns
  long long parts;               // row ranges per tile (one warp each)
  int win;                       // rows per fixed-point window
  int r32;                       // R < 2^32: 32-bit row decode
  long long ext[kMaxRank];       // extents (axis order, outermost first)
  FastDiv div[kMaxRank];
};

// float storage (f32, bf16, f16), accumulated in f32: a lane holds kMx32J elements per
// row, as vectors of V = 16 bytes / element size when rows are 16-byte aligned (else V = 1);
// a warp tile is 32 * kMx32J columns; plain f32 sums of at most kMx32Window rows
constexpr int kMx32Warps = 8;
constexpr int kMx32MinCtas = 2;
constexpr int kMx32J = 16;       // elements per lane and row
constexpr int kMx32Window = 64;  // rows per f32 window
constexpr long long kMx32MinElems = 1ll << 25;  // float tensors this large or larger

}  // namespace triot
