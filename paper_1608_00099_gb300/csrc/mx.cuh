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

struct MxGeom {
  int D;                         // effective rank
  int s;                         // row axes 0 .. s-1, column axes s .. D-1 (1 <= s < D)
  long long R;                   // rows (< 2^31)
  long long C;                   // columns (< 2^31)
  long long tiles;               // column tiles of 32 * kMxJ columns
  long long parts;               // row ranges per tile (one warp each)
  int win;                       // rows per fixed-point window
  int r32;                       // R < 2^32: 32-bit row decode
  long long ext[kMaxRank];       // extents (axis order, outermost first)
  FastDiv div[kMaxRank];
};

}  // namespace triot
