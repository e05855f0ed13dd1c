// Host planning of the moment (Algorithms 10 and 11): validation, canonicalisation (Section
// 4: trivial axes are ignored) and the lane-segment / block-column work split.
#include "plan.h"

#include <algorithm>
#include <cstdio>

#include "../../include/triot.h"
#include "blk32.cuh"

namespace triot {

namespace {

bool mul_overflows(int64_t a, int64_t b) {
  return a != 0 && b > INT64_MAX / a;
}

long long gcd_ll(long long a, long long b) {
  while (b) { long long t = a % b; a = b; b = t; }
  return a;
}

}  // namespace

int canon_moment(int rank, const int64_t* shape, Canon& c, std::string& err) {
  char buf[256];
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    err = buf;
    return TRIOT_ERR_RANK;
  }
  if (!shape) { err = "shape pointer is NULL"; return TRIOT_ERR_NULL; }
  c = Canon();
  c.total = 1;
  for (int i = 0; i < rank; ++i) {
    if (shape[i] < 0) {
      snprintf(buf, sizeof buf, "negative extent on axis %d", i);
      err = buf;
      return TRIOT_ERR_SHAPE;
    }
    if (shape[i] >= (int64_t(1) << 31)) {
      snprintf(buf, sizeof buf, "moment axis %d extent %lld must be < 2^31", i, (long long)shape[i]);
      err = buf;
      return TRIOT_ERR_SHAPE;
    }
    if (mul_overflows(c.total, shape[i])) { err = "element count overflows int64"; return TRIOT_ERR_SHAPE; }
    c.total *= shape[i];
  }
  c.empty = (c.total == 0);
  int D = 0;
  for (int i = 0; i < rank; ++i) {
    if (shape[i] == 1) continue;
    c.ext[D] = shape[i];
    c.orig[D] = i;
    c.sa[D] = c.sb[D] = 0;
    c.bound[D] = shape[i];
    ++D;
  }
  if (D == 0) {  // a single element: its tuple is all zeros
    c.ext[0] = 1;
    c.orig[0] = 0;
    D = 1;
  }
  c.D = D;
  return TRIOT_OK;
}
long long moment_segment(const Canon& c, int es, long long target_lanes) {
  // A lane segment is a whole number of 128-byte chunks.  When it is also a multiple of
  // the inner extent L (and of L * s_{D-2}), every lane of a warp reaches its row ends
  // (and the next carries) at the same step, so the carry code runs without divergence.
  // Each segment costs a tuple decode and a flush of D levels (~24 D instructions), so
  // segments are preferably at least 24 D elements long -- unless the tensor is too small
  // to give every lane of a full GPU some work, in which case parallelism wins.
  const long long C = 128 / es;
  const long long L = c.ext[c.D - 1];
  auto lcm = [](long long a, long long b) { return a / gcd_ll(a, b) * b; };
  const long long base0 = (L > 0 && lcm(C, L) <= 4096) ? lcm(C, L) : C;
  long long base1 = base0;
  if (c.D >= 2 && L > 0) {
    const long long blk = L * c.ext[c.D - 2];
    if (blk > 0 && blk <= 4096 && lcm(C, blk) <= 4096) base1 = lcm(C, blk);
  }
  const long long smin = std::max(C, 24ll * c.D);
  auto up = [&](long long b, long long lo) { return (lo + b - 1) / b * b; };
  const long long cands[4] = {up(base1, smin), up(base0, smin), base0, C};
  for (long long s : cands)
    if (c.total >= s * target_lanes) return s;
  // too small for every lane: the largest chunk multiple that still fills the lanes
  long long s = (c.total / std::max(1ll, target_lanes)) / C * C;
  return std::max(C, s);
}

int moment_block_axes(const Canon& c, int dtype) {
  // the trailing axes whose product stays within `cap` elements
  auto axes = [&](long long cap, long long& b) {
    b = 1;
    int m = 0;
    for (int a = c.D - 1; a >= 0; --a) {
      if (b * c.ext[a] > cap) break;
      b *= c.ext[a];
      ++m;
    }
    return m;
  };
  long long b = 1;
  if (dtype != DT_F64) {
    // float storage: warp blocks of up to 256 elements when the trailing axes reach 128
    // elements or form whole 512-byte rows (shorter warp blocks leave lanes idle and lose
    // to the chunked kernel's blocks of at most 16)
    const int m = axes((long long)kWBMaxC * 32, b);
    if (b >= 128 || (b >= 32 && wb_vec((int)b, dtype_size(dtype)))) return m;
  }
  return axes(16, b);
}

bool plan_moment_mx(const Canon& c, int rank, int es, const void* p, long long target_warps,
                    MomentLaunch& L) {
  if (c.empty || c.D < 2) return false;
  // columns of a warp tile: f64 32 * kMxJ; float storage 32 * kMx32J (vector loads of V
  // elements when every row starts on a 16-byte boundary, else V = 1)
  auto tile_width = [&](long long C, int& V) -> long long {
    if (es == 8) {
      V = 1;
      return 32ll * kMxJ;
    }
    const bool vec = (reinterpret_cast<uintptr_t>(p) % 16) == 0 && (C * es) % 16 == 0;
    V = vec ? 16 / es : 1;
    return 32ll * kMx32J;
  };
  // split after axis s-1: the best use of the tiles' columns, then columns near 2^12
  int best_s = 0;
  double best_score = -1.0;
  for (int s = 1; s < c.D; ++s) {
    long long C = 1, R = 1;
    for (int a = s; a < c.D; ++a) C *= c.ext[a];
    for (int a = 0; a < s; ++a) R *= c.ext[a];
    int V = 1;
    const long long W = tile_width(C, V);
    if (C >= (1ll << 31) || R >= (1ll << 31) || C < W / 2) continue;
    const long long tiles = (C + W - 1) / W;
    const double eff = double(C) / double(tiles * W);
    if (eff < 0.8) continue;
    double lc = 0.0;
    for (long long v = C; v > 1; v >>= 1) lc += 1.0;
    const double score = eff - 0.01 * (lc > 12.0 ? lc - 12.0 : 12.0 - lc);
    if (score > best_score) {
      best_score = score;
      best_s = s;
    }
  }
  if (best_s == 0) return false;
  MxGeom& g = L.mx;
  g = MxGeom();
  g.D = c.D;
  g.s = best_s;
  g.C = 1;
  g.R = 1;
  for (int a = best_s; a < c.D; ++a) g.C *= c.ext[a];
  for (int a = 0; a < best_s; ++a) g.R *= c.ext[a];
  for (int i = 0; i < c.D; ++i) {
    g.ext[i] = c.ext[i];
    g.div[i] = make_fastdiv((uint32_t)c.ext[i]);
  }
  g.r32 = g.R < (1ll << 32);
  g.W = (int)tile_width(g.C, g.V);
  g.tiles = (g.C + g.W - 1) / g.W;
  const int nw = es == 8 ? kMxWarps : kMx32Warps;
  long long grid;
  if (es == 8) {
    // one warp per (tile, row range): enough ranges to fill the GPU, whole warps per CTA
    const long long parts = std::max(1ll, std::min(g.R, target_warps / g.tiles));
    g.parts = parts;
    const long long rows_per_warp = (g.R + parts - 1) / parts;
    g.win = (int)std::min<long long>(kMxWindow, std::max(1ll, rows_per_warp));
    grid = (g.tiles * parts + nw - 1) / nw;
  } else {
    // one CTA per (tile, row range), its warps splitting the range: the CTA's warps share
    // their tile's columns, so the column axes' moments are formed once per CTA
    const long long parts = std::max(1ll, std::min((g.R + nw - 1) / nw, target_warps / nw / g.tiles));
    g.parts = parts;
    g.win = kMx32Window;
    grid = g.tiles * parts;
  }
  if (grid > kMxMaxGrid) return false;
  L.kind = MOMENT_KIND_MX;
  L.grid = (int)grid;
  L.warps = nw;
  L.smem = 0;
  L.empty = false;
  // the row/block geometry is unused, but the effective rank must be right for the
  // workspace size and the combine
  L.g = MomentGeom();
  L.g.D = c.D;
  CombineGeom& cg = L.cg;
  cg = CombineGeom();
  cg.D = c.D;
  cg.rank = rank;
  cg.nparts = L.grid;
  for (int i = 0; i < c.D; ++i) cg.orig[i] = c.orig[i];
  return true;
}

void plan_moment(const Canon& c, int rank, int es, int m, const void* p, const TuneCfg& t,
                 const DeviceInfo& dev, int occ, MomentLaunch& L) {
  MomentGeom& g = L.g;
  g = MomentGeom();
  const int D = c.D;
  g.D = D;
  g.n = c.total;
  for (int i = 0; i < D; ++i) {
    g.ext[i] = c.ext[i];
    g.div[i] = make_fastdiv((uint32_t)c.ext[i]);
  }
  g.n32 = c.total < (int64_t(1) << 32);
  g.aligned = (reinterpret_cast<uintptr_t>(p) % 16) == 0;
  const int cps = t.ctas_per_sm > 0 ? t.ctas_per_sm : occ;
  const long long max_ctas = (long long)dev.sms * std::max(1, cps);
  long long Bm = 1;  // block size (block modes)
  for (int a = D - m; a < D; ++a) Bm *= c.ext[a];
  const bool wb = m > 0 && es != 8 && Bm >= 32;
  const int warps = (m > 0 && es == 8) ? kB64Warps : wb ? kWBWarps : m > 0 ? kB32Warps : kMomentWarps;
  L.warps = warps;
  const long long target_lanes = max_ctas * warps * 32;
  const long long C = 128 / es;
  g.m = m;
  if (wb) {
    // warp blocks: each warp a contiguous range of whole blocks (g.nround counts blocks),
    // steps of U = g.nchunks blocks (at most kWBStepBytes), windows of kWBTerms blocks
    g.B = (int)Bm;
    g.nround = c.total / Bm;
    g.win = kWBTerms;
    g.seg = Bm;
    g.nchunks = (int)std::max(1ll, (long long)kWBStepBytes / (Bm * es));
    const long long units = (g.nround + g.nchunks - 1) / g.nchunks;
    g.nwarpseg = c.empty ? 0 : units;
    const long long need = (units + warps - 1) / warps;
    L.empty = c.empty;
    L.grid = c.empty ? 0 : (int)std::max(1ll, std::min(need, max_ctas));
    CombineGeom& cg = L.cg;
    cg = CombineGeom();
    cg.D = D;
    cg.rank = rank;
    cg.nparts = L.grid;
    for (int i = 0; i < D; ++i) cg.orig[i] = c.orig[i];
    return;
  }
  if (m > 0) {
    long long B = 1;
    for (int a = D - m; a < D; ++a) B *= c.ext[a];
    if (B < 1) B = 1;
    g.B = (int)B;
    const long long K = es == 8 ? b64_blocks_per_chunk((int)B) : b32_blocks_per_chunk((int)B, es);
    const long long CB = K * B;
    // rounds of 32 chunks of K whole blocks each; every warp takes a contiguous share of the
    // rounds (the kernel splits them evenly), one chunk per lane and round
    g.seg = CB;
    g.nchunks = 1;
    g.nround = (c.total + 32 * CB - 1) / (32 * CB);
    if (es == 8) {
      // a fixed-point window: at most kB64Window elements per lane and 512 per block column
      // (a column sum of 512 elements below 2^53 stays below 2^62)
      g.win = (int)std::max(1ll, std::min((long long)kB64Window, 512 * B) / CB);
    } else {
      // a float window: at most kB32Terms blocks per lane
      g.win = (int)std::max(1ll, (long long)kB32Terms / K);
    }
  } else {
    g.B = 0;
    g.seg = moment_segment(c, es, target_lanes);
    g.nchunks = (int)(g.seg / C);
  }
  g.nwarpseg = c.empty ? 0 : (c.total + 32 * g.seg - 1) / (32 * g.seg);
  long long need = (g.nwarpseg + warps - 1) / warps;
  long long grid = std::min(need, max_ctas);
  L.empty = c.empty;
  L.grid = c.empty ? 0 : (int)std::max(1ll, grid);
  CombineGeom& cg = L.cg;
  cg = CombineGeom();
  cg.D = D;
  cg.rank = rank;
  cg.nparts = L.grid;
  for (int i = 0; i < D; ++i) cg.orig[i] = c.orig[i];
}

}  // namespace triot
