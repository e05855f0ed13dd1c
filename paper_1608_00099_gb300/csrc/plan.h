// Host planning: argument validation, shape canonicalisation and launch geometry.
#pragma once
#include <stdint.h>

#include <string>

#include "common.cuh"
#include "mx.cuh"

namespace triot {

// Launch knobs of one kernel family; 0 = default.
struct TuneCfg {
  int threads = 0;
  int tile_elems = 0;
  int ctas_per_sm = 0;
  int unroll = 0;
};

struct DeviceInfo {
  int device = 0;
  int sms = 152;
  char name[128] = {0};
};

// Validate and canonicalise a row operation (ROW_EMBED / ROW_CROP / ROW_PRODUCT).
// Returns a triot_status code; on error `err` says why.
// xdata / ydata: shapes of the containers the operands are views of (strides come from
// them; nullptr: the operand is its own container).
int canon_rows(int op, int rank, const int64_t* xshape, const int64_t* yshape, Canon& c,
               bool& x_empty, std::string& err, const int64_t* xdata = nullptr,
               const int64_t* ydata = nullptr);
// Validate and canonicalise a moment (drop extent-1 axes, keep the axis map).
int canon_moment(int rank, const int64_t* shape, Canon& c, std::string& err);

// Launch geometry of a row kernel.  `es` is the element size in bytes.
struct RowLaunch {
  RowGeom g;
  int grid = 0, block = 0;
  size_t smem = 0;
};
void plan_rows(int op, const Canon& c, bool x_empty, int es, const void* A, const void* B,
               unsigned flags, const TuneCfg& t, const DeviceInfo& dev, RowLaunch& L);

struct MomentLaunch {
  MomentGeom g;
  CombineGeom cg;
  int kind = 0;        // MOMENT_KIND_* below
  MxGeom mx;           // MOMENT_KIND_MX: the marginal split
  int grid = 0;        // CTAs of the moment kernel (= number of partial vectors)
  int warps = 4;       // warps per CTA
  size_t smem = 0;     // dynamic shared memory per CTA (block kernels: stages, outer-axis state)
  bool empty = false;  // nothing to sum: only the combine runs (it writes zeros)
};
enum { MOMENT_KIND_ROWS_BLOCKS = 0, MOMENT_KIND_MX = 1 };
// The marginal split of a f64 moment (moment_mx.cu): false when no split of the canonical
// axes gives rows and columns the kernel can use well.  `target_warps` = warps of a full GPU.
// (es: element size; p: the data, whose alignment decides vector loads for float storage)
bool plan_moment_mx(const Canon& c, int rank, int es, const void* p, long long target_warps,
                    MomentLaunch& L);
// `occ` = resident CTAs per SM of the chosen kernel (from the occupancy calculator).
void plan_moment(const Canon& c, int rank, int es, int m, const void* p, const TuneCfg& t,
                 const DeviceInfo& dev, int occ, MomentLaunch& L);
// block-column mode: number of trailing axes forming a block of at most 16 elements
// (0 = row mode, for inner extents above 16)
int moment_block_axes(const Canon& c, int dtype);

// lane segment length chosen for the moment (exposed for the workspace bound)
long long moment_segment(const Canon& c, int es, long long target_lanes);

}  // namespace triot
