// Host planning of the row operations (embed, crop, product): validation
// (check_tensor_pack_bounds, Algorithm 8), canonicalisation (Section 4: trivial axes are
// ignored; contiguous neighbours merge) and tiling.
#include "plan.h"

#include <algorithm>
#include <cstdio>

#include "../../include/triot.h"

namespace triot {

namespace {

void strides_of(int rank, const int64_t* shape, int64_t* st) {
  int64_t s = 1;
  for (int i = rank - 1; i >= 0; --i) {
    st[i] = s;
    s *= (shape[i] > 0 ? shape[i] : 1);
  }
}

bool mul_overflows(int64_t a, int64_t b) {
  return a != 0 && b > INT64_MAX / a;
}

}  // namespace

int canon_rows(int op, int rank, const int64_t* xshape, const int64_t* yshape, Canon& c,
               bool& x_empty, std::string& err, const int64_t* xdata, const int64_t* ydata) {
  char buf[256];
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    err = buf;
    return TRIOT_ERR_RANK;
  }
  if (!xshape || !yshape) { err = "shape pointer is NULL"; return TRIOT_ERR_NULL; }
  int64_t nx = 1, ny = 1;
  for (int i = 0; i < rank; ++i) {
    if (xshape[i] < 0 || yshape[i] < 0) {
      snprintf(buf, sizeof buf, "negative extent on axis %d", i);
      err = buf;
      return TRIOT_ERR_SHAPE;
    }
    if ((op == ROW_EMBED || op == ROW_CROP) && xshape[i] > yshape[i]) {
      snprintf(buf, sizeof buf, "x extent %lld exceeds y extent %lld on axis %d",
               (long long)xshape[i], (long long)yshape[i], i);
      err = buf;
      return TRIOT_ERR_SHAPE;
    }
    if (mul_overflows(nx, xshape[i]) || mul_overflows(ny, yshape[i])) {
      err = "element count overflows int64";
      return TRIOT_ERR_SHAPE;
    }
    nx *= xshape[i];
    ny *= yshape[i];
  }
  int64_t ext[kMaxRank], sx[kMaxRank], sy[kMaxRank], sa[kMaxRank], sb[kMaxRank], bound[kMaxRank];
  // strides from the containers' shapes (a view addresses its container, Section 4)
  strides_of(rank, xdata ? xdata : xshape, sx);
  strides_of(rank, ydata ? ydata : yshape, sy);
  x_empty = (nx == 0);
  for (int i = 0; i < rank; ++i) {
    if (op == ROW_EMBED) { ext[i] = yshape[i]; sa[i] = sy[i]; sb[i] = sx[i]; bound[i] = xshape[i]; }
    else if (op == ROW_CROP) { ext[i] = xshape[i]; sa[i] = sx[i]; sb[i] = sy[i]; bound[i] = xshape[i]; }
    else {
      ext[i] = std::min(xshape[i], yshape[i]);
      sa[i] = sy[i];
      sb[i] = sx[i];
      bound[i] = ext[i];
    }
  }
  c = Canon();
  c.total = 1;
  for (int i = 0; i < rank; ++i) c.total *= ext[i];
  c.empty = (c.total == 0);
  // drop unit axes, then merge neighbours that are contiguous in both tensors (and, for
  // embed, full in x on the inner side)
  int D = 0;
  for (int i = 0; i < rank; ++i) {
    if (ext[i] == 1) continue;
    if (D > 0) {
      const int j = D - 1;  // previous kept (outer) axis; axis i is the inner candidate
      const bool contiguous = (c.sa[j] == sa[i] * ext[i]) && (c.sb[j] == sb[i] * ext[i]);
      const bool full = (op != ROW_EMBED) || (bound[i] == ext[i]);
      if (contiguous && full && !mul_overflows(c.ext[j], ext[i])) {
        c.ext[j] *= ext[i];
        c.bound[j] = c.bound[j] * ext[i];
        c.sa[j] = sa[i];
        c.sb[j] = sb[i];
        continue;
      }
    }
    c.ext[D] = ext[i];
    c.sa[D] = sa[i];
    c.sb[D] = sb[i];
    c.bound[D] = bound[i];
    c.orig[D] = i;
    ++D;
  }
  // rows must run over unit stride in both tensors: otherwise add a unit inner axis
  if (D == 0 || c.sa[D - 1] != 1 || c.sb[D - 1] != 1) {
    if (D == kMaxRank) {
      // every axis kept and the innermost is strided: impossible (the last original axis
      // always has unit stride in every tensor unless it was dropped)
      err = "internal: no room for a unit inner axis";
      return TRIOT_ERR_SHAPE;
    }
    c.ext[D] = 1;
    c.sa[D] = 1;
    c.sb[D] = 1;
    c.bound[D] = x_empty ? 0 : 1;
    c.orig[D] = rank - 1;
    ++D;
  }
  c.D = D;
  return TRIOT_OK;
}
void plan_rows(int op, const Canon& c, bool x_empty, int es, const void* A, const void* B,
               unsigned flags, const TuneCfg& t, const DeviceInfo& dev, RowLaunch& L) {
  RowGeom& g = L.g;
  g = RowGeom();
  const int D = c.D;
  const int vec = 16 / es;
  g.nouter = D - 1;
  long long rows = 1;
  for (int k = 0; k < g.nouter; ++k) {
    const int a = D - 2 - k;
    g.ext[k] = c.ext[a];
    g.sa[k] = c.sa[a];
    g.sb[k] = c.sb[a];
    g.bound[k] = c.bound[a];
    rows *= c.ext[a];
  }
  g.rows = rows;
  g.inner = c.ext[D - 1];
  g.b_inner = c.bound[D - 1];
  if (op == ROW_EMBED && x_empty) {
    // nothing of x is visible: every row lies outside
    if (g.nouter > 0) g.bound[g.nouter - 1] = 0;
    else g.b_inner = 0;
  }
  g.rows32 = rows <= 0xFFFFFFFFll;
  for (int k = 0; k < g.nouter; ++k)
    g.div[k] = make_fastdiv(g.ext[k] < 0xFFFFFFFFll ? (uint32_t)g.ext[k] : 1u);
  g.nopad = (op == ROW_EMBED && (flags & TRIOT_EMBED_NOPAD)) ? 1 : 0;
  {
    long long expect = g.inner;
    g.a_dense = 1;
    for (int k = 0; k < g.nouter; ++k) {
      if (g.sa[k] != expect) g.a_dense = 0;
      expect *= g.ext[k];
    }
  }

  const bool a_al = (reinterpret_cast<uintptr_t>(A) % 16) == 0;
  const bool b_al = (reinterpret_cast<uintptr_t>(B) % 16) == 0;
  // vector accesses to A need every row of A 16-byte aligned: A's start and all its row
  // strides (automatic for a dense A whose rows are whole vectors; a view's rows may not be)
  bool row_ok = (g.inner % vec == 0) && a_al;
  for (int k = 0; k < g.nouter; ++k) row_ok = row_ok && (g.sa[k] % vec == 0);
  bool vec_ok = row_ok && b_al;
  for (int k = 0; k < g.nouter; ++k) vec_ok = vec_ok && (g.sb[k] % vec == 0);
  if (op == ROW_EMBED) vec_ok = vec_ok && (g.b_inner % vec == 0);
  g.path = vec_ok ? PATH_VEC : (row_ok ? PATH_ROW : PATH_GEN);

  long long target = t.tile_elems > 0 ? t.tile_elems : (32768 / es);
  // small problems: shrink tiles so that every SM gets several (down to 64 vectors)
  if (t.tile_elems <= 0) {
    const long long spread = (c.total + 4ll * dev.sms - 1) / (4ll * dev.sms);
    target = std::min(target, std::max(64ll * vec, spread));
  }
  if (target < vec) target = vec;
  if (g.inner <= target) {
    long long R = std::max(1ll, target / g.inner);
    R = std::min(R, 1024ll);
    R = std::min(R, std::max(1ll, rows));
    g.rows_per_tile = R;
    g.segs_per_row = 1;
    g.seg_len = g.inner;
    g.ntiles = (rows + R - 1) / R;
  } else {
    long long segs = (g.inner + target - 1) / target;
    long long len = (g.inner + segs - 1) / segs;
    len = (len + vec - 1) / vec * vec;
    segs = (g.inner + len - 1) / len;
    g.rows_per_tile = 1;
    g.segs_per_row = segs;
    g.seg_len = len;
    g.ntiles = rows * segs;
  }
  g.inner_div = make_fastdiv(g.inner < 0xFFFFFFFFll ? (uint32_t)g.inner : 1u);
  g.seg_div = make_fastdiv(g.segs_per_row < 0xFFFFFFFFll ? (uint32_t)g.segs_per_row : 1u);

  const int threads = t.threads > 0 ? t.threads : 256;
  const int cps = t.ctas_per_sm > 0 ? t.ctas_per_sm : 4;
  long long grid = std::min<long long>(g.ntiles, (long long)dev.sms * cps);
  L.grid = (int)std::max(1ll, grid);
  L.block = threads;
  L.smem = (size_t)g.rows_per_tile * sizeof(RowInfo);
}

}  // namespace triot
