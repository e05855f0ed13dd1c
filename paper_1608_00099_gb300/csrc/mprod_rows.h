// Launch geometry of the short-row kernel of the moment of a product (moment_prod_rows.cu):
// rows of I shorter than kMPRowsMaxL elements, streamed in CTA tiles of whole rows.
#pragma once
#include "common.cuh"

namespace triot {

constexpr int kMPRowsWarps = 8;
constexpr int kMPRowsMaxL = 8;
constexpr int kMPRowsTileRows = 512;    // rows of a tile at most
constexpr int kMPRowsTileElems = 2048;  // elements of a tile at most

struct MPRowsGeom {
  int tile_rows;  // rows of a CTA tile (a multiple of rp)
  int rp;         // rows per pass of the CTA's threads: floor(threads / L)
  FastDiv ldiv;   // divisor L
};

}  // namespace triot
