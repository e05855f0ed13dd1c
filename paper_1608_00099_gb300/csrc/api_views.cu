// C ABI of the view operations: embed, crop and product on a window of y that starts at a
// tuple `ystart` (Section 4: a slice references its tensor and adds a bias, the flat index of
// its start tuple, to every flat index computed with the tensor's own shape).  The row
// kernels run unchanged on the view: strides from y's shape, y's pointer advanced by the bias.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/triot.h"
#include "internal.h"

namespace triot {
namespace {

// validates the window and returns the bias (elements) of ystart in y
int window_bias(int rank, const int64_t* xshape, const int64_t* yshape, const int64_t* ystart,
                bool x_must_fit, int64_t& bias) {
  char buf[256];
  if (rank < 1 || rank > kMaxRank) {
    snprintf(buf, sizeof buf, "rank %d outside [1, %d]", rank, kMaxRank);
    return fail(TRIOT_ERR_RANK, buf);
  }
  if (!xshape || !yshape || !ystart) return fail(TRIOT_ERR_NULL, "a shape or start pointer is NULL");
  bias = 0;
  for (int i = 0; i < rank; ++i) {
    if (xshape[i] < 0 || yshape[i] < 0 || ystart[i] < 0) {
      snprintf(buf, sizeof buf, "negative extent or start on axis %d", i);
      return fail(TRIOT_ERR_SHAPE, buf);
    }
    if (ystart[i] > yshape[i] || (x_must_fit && ystart[i] + xshape[i] > yshape[i])) {
      snprintf(buf, sizeof buf, "window start %lld + extent %lld exceeds y extent %lld on axis %d",
               (long long)ystart[i], (long long)(x_must_fit ? xshape[i] : 0), (long long)yshape[i], i);
      return fail(TRIOT_ERR_SHAPE, buf);
    }
  }
  // Horner (Algorithm 2) on y's shape
  for (int i = 0; i < rank; ++i) bias = bias * (yshape[i] > 0 ? yshape[i] : 1) + ystart[i];
  return TRIOT_OK;
}

int64_t count(int rank, const int64_t* s) {
  int64_t n = 1;
  for (int i = 0; i < rank; ++i) n *= s[i];
  return n;
}

const void* advance(const void* p, int64_t elems, int dtype) {
  return p ? static_cast<const char*>(p) + elems * dtype_size(dtype) : p;
}

}  // namespace
}  // namespace triot

using namespace triot;

extern "C" {

int triot_crop_at(int rank, const int64_t* xshape, void* x, const int64_t* yshape, const void* y,
                  const int64_t* ystart, int dtype, void* stream) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  int64_t bias;
  int st = window_bias(rank, xshape, yshape, ystart, true, bias);
  if (st) return st;
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape);
  const int es = dtype_size(dtype);
  if (nx > 0 && x && y && overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es))
    return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  // x[t] = y[ystart + t]: the read view of y has x's extent
  return launch_rows(ROW_CROP, rank, xshape, x, xshape, advance(y, bias, dtype), dtype, 0,
                     (cudaStream_t)stream, nullptr, nullptr, yshape);
}

int triot_product_at(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                     const int64_t* ystart, int dtype, void* stream) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  int64_t bias;
  int st = window_bias(rank, xshape, yshape, ystart, false, bias);
  if (st) return st;
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape);
  const int es = dtype_size(dtype);
  if (nx > 0 && x && y && overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es))
    return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  // y[ystart + t] *= x[t] over the tuples of x that fit: the view of y is y's remainder
  int64_t yview[kMaxRank];
  for (int i = 0; i < rank; ++i) yview[i] = yshape[i] - ystart[i];
  return launch_rows(ROW_PRODUCT, rank, xshape, x, yview, advance(y, bias, dtype), dtype, 0,
                     (cudaStream_t)stream, nullptr, nullptr, yshape);
}

int triot_embed_at(int rank, const int64_t* xshape, const void* x, const int64_t* yshape, void* y,
                   const int64_t* ystart, int dtype, unsigned flags, void* stream) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  if (flags & ~TRIOT_EMBED_NOPAD) return fail(TRIOT_ERR_ARG, "unknown embed flag");
  int64_t bias;
  int st = window_bias(rank, xshape, yshape, ystart, true, bias);
  if (st) return st;
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape);
  const int es = dtype_size(dtype);
  if (nx > 0 && x && y && overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es))
    return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  cudaStream_t s = (cudaStream_t)stream;
  if (!(flags & TRIOT_EMBED_NOPAD) && ny > 0) {
    // the pad: an embed of an empty tensor writes +0 over all of y
    int64_t zero[kMaxRank];
    for (int i = 0; i < rank; ++i) zero[i] = 0;
    if ((st = launch_rows(ROW_EMBED, rank, zero, nullptr, yshape, y, dtype, 0, s, nullptr))) return st;
  }
  if (nx == 0) return ok();
  // y[ystart + t] = x[t]: the written view of y has x's extent (every tuple inside)
  return launch_rows(ROW_EMBED, rank, xshape, x, xshape, advance(y, bias, dtype), dtype,
                     TRIOT_EMBED_NOPAD, s, nullptr, nullptr, yshape);
}

// ---- windows on both sides (Section 4: views over the intersecting support of two tensors)

namespace {
int views_check(int rank, const int64_t* ext, const int64_t* xshape, const int64_t* xstart,
                const int64_t* yshape, const int64_t* ystart, int64_t& xbias, int64_t& ybias) {
  int st = window_bias(rank, ext, xshape, xstart, true, xbias);
  if (st) return st;
  return window_bias(rank, ext, yshape, ystart, true, ybias);
}
}  // namespace

int triot_copy_views(int rank, const int64_t* ext, const int64_t* xshape, const void* x,
                     const int64_t* xstart, const int64_t* yshape, void* y, const int64_t* ystart,
                     int dtype, void* stream) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  int64_t xb, yb;
  int st = views_check(rank, ext, xshape, xstart, yshape, ystart, xb, yb);
  if (st) return st;
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape), ne = count(rank, ext);
  const int es = dtype_size(dtype);
  if (ne == 0) return ok();
  if (!x || !y) return fail(TRIOT_ERR_NULL, "x or y is NULL");
  if (overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es)) return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  // an embed of x's window into y's window with nothing to pad: every tuple is written
  return launch_rows(ROW_EMBED, rank, ext, advance(x, xb, dtype), ext, advance(y, yb, dtype), dtype,
                     TRIOT_EMBED_NOPAD, (cudaStream_t)stream, nullptr, xshape, yshape);
}

int triot_product_views(int rank, const int64_t* ext, const int64_t* xshape, const void* x,
                        const int64_t* xstart, const int64_t* yshape, void* y, const int64_t* ystart,
                        int dtype, void* stream) {
  if (!valid_dtype(dtype)) return fail(TRIOT_ERR_DTYPE, "unknown dtype code");
  int64_t xb, yb;
  int st = views_check(rank, ext, xshape, xstart, yshape, ystart, xb, yb);
  if (st) return st;
  const int64_t nx = count(rank, xshape), ny = count(rank, yshape), ne = count(rank, ext);
  const int es = dtype_size(dtype);
  if (ne == 0) return ok();
  if (!x || !y) return fail(TRIOT_ERR_NULL, "x or y is NULL");
  if (overlaps_bytes(x, size_t(nx) * es, y, size_t(ny) * es)) return fail(TRIOT_ERR_ALIAS, "x and y overlap");
  return launch_rows(ROW_PRODUCT, rank, ext, advance(x, xb, dtype), ext, advance(y, yb, dtype), dtype, 0,
                     (cudaStream_t)stream, nullptr, xshape, yshape);
}

int triot_product_support(int rank, const int64_t* xshape, const void* x, const int64_t* xorigin,
                          const int64_t* yshape, void* y, const int64_t* yorigin, int dtype, void* stream) {
  if (rank < 1 || rank > kMaxRank) return fail(TRIOT_ERR_RANK, "rank outside [1, 24]");
  if (!xshape || !yshape || !xorigin || !yorigin) return fail(TRIOT_ERR_NULL, "a shape or origin pointer is NULL");
  int64_t ext[kMaxRank], xs[kMaxRank], ys[kMaxRank];
  for (int i = 0; i < rank; ++i) {
    if (xshape[i] < 0 || yshape[i] < 0) return fail(TRIOT_ERR_SHAPE, "negative extent");
    const int64_t lim = int64_t(1) << 62;
    if (xorigin[i] <= -lim || xorigin[i] >= lim || yorigin[i] <= -lim || yorigin[i] >= lim)
      return fail(TRIOT_ERR_SHAPE, "origin outside (-2^62, 2^62)");
    // the supports [origin, origin + shape) intersect in [lo, hi)
    const int64_t lo = std::max(xorigin[i], yorigin[i]);
    const int64_t hi = std::min(xorigin[i] + xshape[i], yorigin[i] + yshape[i]);
    ext[i] = hi > lo ? hi - lo : 0;
    xs[i] = hi > lo ? lo - xorigin[i] : 0;
    ys[i] = hi > lo ? lo - yorigin[i] : 0;
  }
  return triot_product_views(rank, ext, xshape, x, xs, yshape, y, ys, dtype, stream);
}

}  // extern "C"
