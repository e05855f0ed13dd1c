// TRIOT CPU oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-purpose restatement of what the GPU path computes, written
// from Heyl & Serang, "TRIOT: Faster tensor manipulation in C++11" (arXiv 1608.00099).
// Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load this
// library.  The product path (the CUDA library) never calls, links or includes it, and
// this file includes nothing from the CUDA path.
//
// Conventions
//  * Tensors are dense and row-major (Section 1: "assuming row-major order of the flat
//    vector").  A shape is `dim` extents; tuples and flat indices are 64-bit unsigned.
//  * Iteration follows the paper's tuple iteration: a tuple starts at all zeros and is
//    advanced lexicographically with carries (Algorithm 3); flat indices are computed
//    with Horner's rule (Section 1, Algorithm 2).
//  * Floating point: products are one IEEE multiply in the storage type for f64/f32.
//    For bf16/f16 the exact product of the stored inputs is formed in f64 (exact: at most
//    22 significant bits, exponent well inside f64's range) and rounded once, to nearest
//    with ties to even, by round_to_format() below.  Moments are Neumaier-compensated f64
//    sums (Neumaier 1974), so the oracle's own error is far below the 1e-12 tolerance.
//  * Element type codes: 0 = f64, 1 = f32, 2 = bf16, 3 = f16.
//
// Parity pins (tests/test_oracle_pins.py) check every exported function against values
// the paper prints, closed forms, numpy/torch library routines and brute force.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

typedef uint64_t u64;

namespace {

enum { T_F64 = 0, T_F32 = 1, T_BF16 = 2, T_F16 = 3 };

// ------------------------------------------------------------------ index arithmetic

// The flat index of a tuple (Section 1): sum over axes of t_i times the number of
// elements in one step of axis i, i.e. the product of the extents right of i.  Evaluated
// as a left fold that scales the index so far by the next axis' extent and adds that
// axis' digit -- the nested (Horner) form of the same sum that Algorithm 2 uses.
u64 tuple_to_index(const u64* tup, const u64* shape, unsigned dim) {
  u64 flat = 0;
  for (unsigned axis = 0; axis < dim; ++axis) flat = flat * shape[axis] + tup[axis];
  return flat;
}

// Lexicographic successor of a tuple (the increment Algorithm 3 defines): the rightmost
// axis that has not reached its last value goes up by one and every axis right of it
// restarts at zero.  When all axes after the first are at their last value the first
// axis is the one raised, so the step after the final tuple gives (shape[0], 0, ..., 0).
void advance_tuple(u64* tup, const u64* shape, unsigned dim) {
  unsigned grow = dim - 1;
  while (grow > 0 && tup[grow] + 1 == shape[grow]) --grow;
  tup[grow] += 1;
  for (unsigned axis = grow + 1; axis < dim; ++axis) tup[axis] = 0;
}

// The digits of a flat index with respect to `shape` (the inverse of tuple_to_index):
// the last axis' digit is the remainder by its extent, the quotient carries the rest.
void index_to_tuple(u64 index, const u64* shape, unsigned dim, u64* tup) {
  for (unsigned n = dim; n-- > 0;) {
    tup[n] = index % shape[n];
    index /= shape[n];
  }
}

// What Algorithm 4 computes: the flat index, in `new_shape`, of the tuple whose flat index
// in `shape` is `index` -- the tuple recovered digit by digit, then flattened again.
u64 reindex(u64 index, const u64* shape, const u64* new_shape, unsigned dim) {
  std::vector<u64> tup(dim);
  index_to_tuple(index, shape, dim, tup.data());
  return tuple_to_index(tup.data(), new_shape, dim);
}

// The same map when every extent is a power of two (Algorithm 12): an axis' digit is a
// bit field of the index, so the digits come out with masks and shifts and the new flat
// index is assembled by shifting each digit into a field of the new axis' width.
u64 reindex_pow2(u64 index, const unsigned* log_shape, const unsigned* new_log_shape,
                 unsigned dim) {
  std::vector<u64> digit(dim);
  for (unsigned n = dim; n-- > 0;) {
    digit[n] = index & ((u64(1) << log_shape[n]) - 1);
    index >>= log_shape[n];
  }
  u64 flat = 0;
  for (unsigned axis = 0; axis < dim; ++axis) flat = (flat << new_log_shape[axis]) + digit[axis];
  return flat;
}

u64 count_of(const u64* shape, unsigned dim) {
  u64 n = 1;
  for (unsigned i = 0; i < dim; ++i) n *= shape[i];
  return n;
}

size_t elem_size(int t) { return t == T_F64 ? 8 : t == T_F32 ? 4 : 2; }

// ------------------------------------------------------------------ number formats

// Round a double to the nearest value of a binary floating-point format with `p` bits
// of precision (implicit bit included), minimum normal exponent `emin`, maximum exponent
// `emax` and `ebits` exponent bits; ties go to the even significand (IEEE 754-2008,
// roundTiesToEven).  Returns the encoded bit pattern (sign | exponent | fraction).
// Written from the format definition: the representable values near |v| are integer
// multiples of the quantum 2^q, q = max(floor(log2|v|), emin) - (p - 1).
uint32_t round_to_format(double v, int p, int emin, int emax, int ebits) {
  const int fbits = p - 1;
  const uint32_t sign = std::signbit(v) ? (uint32_t(1) << (ebits + fbits)) : 0u;
  const uint32_t exp_all_ones = (uint32_t(1) << ebits) - 1;
  if (std::isnan(v)) return sign | (exp_all_ones << fbits) | (uint32_t(1) << (fbits - 1));
  const double a = std::fabs(v);
  if (std::isinf(a)) return sign | (exp_all_ones << fbits);
  if (a == 0.0) return sign;
  int e2;
  (void)std::frexp(a, &e2);       // a = f * 2^e2 with f in [0.5, 1)
  int e = e2 - 1;                 // floor(log2 a)
  int q = (e > emin ? e : emin) - fbits;
  double n = std::ldexp(a, -q);   // exact: a power-of-two scaling inside double range
  double fl = std::floor(n);
  double frac = n - fl;           // exact (n < 2^53)
  double r = fl;
  if (frac > 0.5 || (frac == 0.5 && std::fmod(fl, 2.0) != 0.0)) r = fl + 1.0;
  const double two_p = std::ldexp(1.0, p);
  if (r == two_p) {               // rounded up into the next binade
    r = two_p / 2.0;
    q += 1;
  }
  const int unbiased = q + fbits; // exponent of the leading bit when normal
  if (unbiased > emax) return sign | (exp_all_ones << fbits);  // overflow -> infinity
  const uint32_t ri = uint32_t(r);
  if (ri < (uint32_t(1) << fbits)) return sign | ri;           // subnormal (q == emin - fbits)
  const int bias = (1 << (ebits - 1)) - 1;
  const uint32_t ebiased = uint32_t(unbiased + bias);
  return sign | (ebiased << fbits) | (ri - (uint32_t(1) << fbits));
}

double bits_to_double(uint32_t bits, int p, int ebits) {
  const int fbits = p - 1;
  const uint32_t emask = (uint32_t(1) << ebits) - 1;
  const bool neg = (bits >> (ebits + fbits)) & 1u;
  const uint32_t eb = (bits >> fbits) & emask;
  const uint32_t f = bits & ((uint32_t(1) << fbits) - 1);
  const int bias = (1 << (ebits - 1)) - 1;
  double mag;
  if (eb == emask) mag = f ? NAN : INFINITY;
  else if (eb == 0) mag = std::ldexp(double(f), 1 - bias - fbits);
  else mag = std::ldexp(double(f + (uint32_t(1) << fbits)), int(eb) - bias - fbits);
  return neg ? -mag : mag;
}

double load_as_double(const void* base, u64 i, int t) {
  switch (t) {
    case T_F64: return static_cast<const double*>(base)[i];
    case T_F32: return double(static_cast<const float*>(base)[i]);
    case T_BF16: return bits_to_double(static_cast<const uint16_t*>(base)[i], 8, 8);
    default: return bits_to_double(static_cast<const uint16_t*>(base)[i], 11, 5);
  }
}

// y[iy] = y[iy] * x[ix] in the storage type (single rounding).
void multiply_into(void* y, u64 iy, const void* x, u64 ix, int t) {
  switch (t) {
    case T_F64: {
      double* yy = static_cast<double*>(y);
      yy[iy] = yy[iy] * static_cast<const double*>(x)[ix];
      break;
    }
    case T_F32: {
      float* yy = static_cast<float*>(y);
      yy[iy] = yy[iy] * static_cast<const float*>(x)[ix];
      break;
    }
    case T_BF16: {
      uint16_t* yy = static_cast<uint16_t*>(y);
      const double exact = bits_to_double(yy[iy], 8, 8) *
                           bits_to_double(static_cast<const uint16_t*>(x)[ix], 8, 8);
      yy[iy] = uint16_t(round_to_format(exact, 8, -126, 127, 8));
      break;
    }
    default: {
      uint16_t* yy = static_cast<uint16_t*>(y);
      const double exact = bits_to_double(yy[iy], 11, 5) *
                           bits_to_double(static_cast<const uint16_t*>(x)[ix], 11, 5);
      yy[iy] = uint16_t(round_to_format(exact, 11, -14, 15, 5));
      break;
    }
  }
}

// Neumaier's improved Kahan-Babuska summation.
struct NeumaierSum {
  double s = 0.0, c = 0.0;
  void add(double v) {
    const double t = s + v;
    if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
  }
  // Once the running sum is non-finite, the plain sum of Algorithms 10/11 is that value
  // (inf, or NaN after inf - inf); the correction term (inf - inf there) carries nothing.
  double value() const { return std::isfinite(s) ? s + c : s; }
};

// split [0, n) into `parts` contiguous ranges (the outer-axis partition of Section 4)
void split_range(u64 n, unsigned parts, unsigned j, u64* lo, u64* hi) {
  *lo = n * j / parts;
  *hi = n * (j + 1) / parts;
}

unsigned clamp_threads(int nthreads, u64 outer) {
  unsigned n = nthreads < 1 ? 1u : unsigned(nthreads);
  if (outer < n) n = outer ? unsigned(outer) : 1u;
  return n;
}

}  // namespace

extern "C" {

int oracle_version(void) { return 1; }

u64 oracle_tuple_to_index(const u64* tup, const u64* shape, unsigned dim) {
  return tuple_to_index(tup, shape, dim);
}
void oracle_advance_tuple(u64* tup, const u64* shape, unsigned dim) {
  advance_tuple(tup, shape, dim);
}
u64 oracle_reindex(u64 index, const u64* shape, const u64* new_shape, unsigned dim) {
  return reindex(index, shape, new_shape, dim);
}
u64 oracle_reindex_pow2(u64 index, const unsigned* log_shape, const unsigned* new_log_shape,
                        unsigned dim) {
  return reindex_pow2(index, log_shape, new_log_shape, dim);
}

// Visit `count` tuples of `shape` from zero with Algorithm 3 and write each visited
// tuple's Horner index (Algorithm 2) to out[k].  Used to pin k-th tuple == k.
void oracle_enumerate(const u64* shape, unsigned dim, u64 count, u64* out_index,
                      u64* out_carries) {
  std::vector<u64> t(dim, 0), prev(dim, 0);
  for (u64 k = 0; k < count; ++k) {
    out_index[k] = tuple_to_index(t.data(), shape, dim);
    prev = t;
    advance_tuple(t.data(), shape, dim);
    u64 changed = 0;  // axes touched by this advance = carries + 1
    for (unsigned i = 0; i < dim; ++i) changed += (t[i] != prev[i]);
    if (out_carries) out_carries[k] = changed;
  }
}

uint32_t oracle_round_to_format(double v, int p, int emin, int emax, int ebits) {
  return round_to_format(v, p, emin, emax, ebits);
}
double oracle_format_to_double(uint32_t bits, int p, int ebits) {
  return bits_to_double(bits, p, ebits);
}
// element-wise widening of a stored tensor to f64 (bit-exact)
void oracle_to_f64(int dtype, const void* src, u64 n, double* dst) {
  for (u64 i = 0; i < n; ++i) dst[i] = load_as_double(src, i, dtype);
}
// element-wise rounding of f64 values to a storage type, RN-even, single rounding
void oracle_from_f64(int dtype, const double* src, u64 n, void* dst) {
  for (u64 i = 0; i < n; ++i) {
    switch (dtype) {
      case T_F64: static_cast<double*>(dst)[i] = src[i]; break;
      case T_F32: {
        const uint32_t b = round_to_format(src[i], 24, -126, 127, 8);
        std::memcpy(static_cast<float*>(dst) + i, &b, 4);
        break;
      }
      case T_BF16: static_cast<uint16_t*>(dst)[i] = uint16_t(round_to_format(src[i], 8, -126, 127, 8)); break;
      default: static_cast<uint16_t*>(dst)[i] = uint16_t(round_to_format(src[i], 11, -14, 15, 5)); break;
    }
  }
}

// ------------------------------------------------------------------ embed / crop

// Embed: y <- 0 everywhere, then y[t] = x[t] for every tuple t of x's shape.
// This is the copy of benchmark 1 (Section 3, Algorithm 13's tuple iteration) run in the
// other direction: the loop walks x's tuples with Algorithm 3 and addresses y with
// Algorithm 2.  Requires xshape[i] <= yshape[i].  `nthreads` > 1 splits the outermost
// axis of x into contiguous ranges, one per std::thread (the outer-loop partition the
// paper suggests in Section 4); the result does not depend on it.
void oracle_embed(int dtype, unsigned dim, const u64* xshape, const void* x,
                  const u64* yshape, void* y, int nthreads) {
  const size_t es = elem_size(dtype);
  const u64 ny = count_of(yshape, dim);
  std::memset(y, 0, size_t(ny) * es);
  const u64 nx = count_of(xshape, dim);
  if (nx == 0) return;
  const u64 inner = nx / xshape[0];  // elements per outermost slab of x
  const unsigned nt = clamp_threads(nthreads, xshape[0]);
  auto work = [&](unsigned j) {
    u64 lo, hi;
    split_range(xshape[0], nt, j, &lo, &hi);
    std::vector<u64> t(dim, 0);
    t[0] = lo;
    const char* xs = static_cast<const char*>(x);
    char* ys = static_cast<char*>(y);
    for (u64 k = lo * inner; k < hi * inner; ++k) {
      const u64 iy = tuple_to_index(t.data(), yshape, dim);
      std::memcpy(ys + iy * es, xs + k * es, es);
      advance_tuple(t.data(), xshape, dim);
    }
  };
  if (nt == 1) { work(0); return; }
  std::vector<std::thread> th;
  for (unsigned j = 0; j < nt; ++j) th.emplace_back(work, j);
  for (auto& h : th) h.join();
}

// Crop: x[k] = y[t] for the k-th tuple t of x's shape (Algorithm 13, tuple iteration).
void oracle_crop(int dtype, unsigned dim, const u64* xshape, void* x, const u64* yshape,
                 const void* y, int nthreads) {
  const size_t es = elem_size(dtype);
  const u64 nx = count_of(xshape, dim);
  if (nx == 0) return;
  const u64 inner = nx / xshape[0];
  const unsigned nt = clamp_threads(nthreads, xshape[0]);
  auto work = [&](unsigned j) {
    u64 lo, hi;
    split_range(xshape[0], nt, j, &lo, &hi);
    std::vector<u64> t(dim, 0);
    t[0] = lo;
    char* xs = static_cast<char*>(x);
    const char* ys = static_cast<const char*>(y);
    for (u64 k = lo * inner; k < hi * inner; ++k) {
      const u64 iy = tuple_to_index(t.data(), yshape, dim);
      std::memcpy(xs + k * es, ys + iy * es, es);
      advance_tuple(t.data(), xshape, dim);
    }
  };
  if (nt == 1) { work(0); return; }
  std::vector<std::thread> th;
  for (unsigned j = 0; j < nt; ++j) th.emplace_back(work, j);
  for (auto& h : th) h.join();
}

// Expected values of the embedded y on the flat window [begin, begin + count) of y, one
// element at a time: decode `begin` to a tuple of y's shape (the digit peeling of
// Algorithm 4), then walk y's tuples with Algorithm 3; an element is x[t] when t lies in
// x's shape and +0 otherwise.  Lets tests check windows of a y too large to rebuild.
void oracle_embed_window(int dtype, unsigned dim, const u64* xshape, const void* x,
                         const u64* yshape, u64 begin, u64 count, void* out) {
  const size_t es = elem_size(dtype);
  std::vector<u64> t(dim);
  index_to_tuple(begin, yshape, dim, t.data());
  const char* xs = static_cast<const char*>(x);
  char* os = static_cast<char*>(out);
  for (u64 k = 0; k < count; ++k) {
    bool inside = true;
    for (unsigned i = 0; i < dim; ++i) inside = inside && (t[i] < xshape[i]);
    if (inside) std::memcpy(os + k * es, xs + tuple_to_index(t.data(), xshape, dim) * es, es);
    else std::memset(os + k * es, 0, es);
    advance_tuple(t.data(), yshape, dim);
  }
}

// ------------------------------------------------------------------ product

// y[t] <- y[t] * x[t] for every tuple t of the intersection I = elementwise min of the two
// shapes ("visiting only tuple indices shared by both", Section 3, benchmark 2); y outside
// I is untouched.  Walks I's tuples with Algorithm 3 and addresses both tensors with
// Algorithm 2 -- apply_tensors with y as the destination (Algorithm 9).
void oracle_product(int dtype, unsigned dim, const u64* xshape, const void* x,
                    const u64* yshape, void* y, int nthreads) {
  std::vector<u64> I(dim);
  for (unsigned i = 0; i < dim; ++i) I[i] = xshape[i] < yshape[i] ? xshape[i] : yshape[i];
  const u64 n = count_of(I.data(), dim);
  if (n == 0) return;
  const u64 inner = n / I[0];
  const unsigned nt = clamp_threads(nthreads, I[0]);
  auto work = [&](unsigned j) {
    u64 lo, hi;
    split_range(I[0], nt, j, &lo, &hi);
    std::vector<u64> t(dim, 0);
    t[0] = lo;
    for (u64 k = lo * inner; k < hi * inner; ++k) {
      multiply_into(y, tuple_to_index(t.data(), yshape, dim), x,
                    tuple_to_index(t.data(), xshape, dim), dtype);
      advance_tuple(t.data(), I.data(), dim);
    }
  };
  if (nt == 1) { work(0); return; }
  std::vector<std::thread> th;
  for (unsigned j = 0; j < nt; ++j) th.emplace_back(work, j);
  for (auto& h : th) h.join();
}

// The product applied to a flat window [begin, begin + count) of y only: `ywin` holds
// y[begin .. begin+count) on entry and the multiplied values on exit.  Elements whose
// tuple (decoded as in oracle_embed_window) lies in I are multiplied by x[t].
void oracle_product_window(int dtype, unsigned dim, const u64* xshape, const void* x,
                           const u64* yshape, u64 begin, u64 count, void* ywin) {
  std::vector<u64> t(dim);
  index_to_tuple(begin, yshape, dim, t.data());
  for (u64 k = 0; k < count; ++k) {
    bool inside = true;
    for (unsigned i = 0; i < dim; ++i) inside = inside && (t[i] < xshape[i]) && (t[i] < yshape[i]);
    if (inside) multiply_into(ywin, k, x, tuple_to_index(t.data(), xshape, dim), dtype);
    advance_tuple(t.data(), yshape, dim);
  }
}

// ------------------------------------------------------------------ moment

// out[i] = sum over tuples t of p's shape of p[t] * t_i, i = 0..dim-1, tuples zero-based
// (the counter starts at 0, Algorithm 10); out[dim] = sum of p[t] (the mass).  This is
// Algorithm 11's tuple-weighted sum with a single weight tensor: the loop walks p's
// tuples with Algorithm 3 and the counter is visible to the summand.  Sums are
// Neumaier-compensated in f64; `nthreads` > 1 splits the outermost axis into contiguous
// ranges whose pre-results are combined afterwards in thread order (Section 4's
// reduce-like scheme).
void oracle_moment(int dtype, unsigned dim, const u64* shape, const void* p, double* out,
                   int nthreads) {
  for (unsigned i = 0; i <= dim; ++i) out[i] = 0.0;
  const u64 n = count_of(shape, dim);
  if (n == 0) return;
  const u64 inner = n / shape[0];
  const unsigned nt = clamp_threads(nthreads, shape[0]);
  std::vector<NeumaierSum> partial(size_t(nt) * (dim + 1));
  auto work = [&](unsigned j) {
    u64 lo, hi;
    split_range(shape[0], nt, j, &lo, &hi);
    std::vector<u64> t(dim, 0);
    t[0] = lo;
    NeumaierSum* acc = &partial[size_t(j) * (dim + 1)];
    for (u64 k = lo * inner; k < hi * inner; ++k) {
      const double v = load_as_double(p, k, dtype);
      for (unsigned i = 0; i < dim; ++i) acc[i].add(v * double(t[i]));
      acc[dim].add(v);
      advance_tuple(t.data(), shape, dim);
    }
  };
  if (nt == 1) work(0);
  else {
    std::vector<std::thread> th;
    for (unsigned j = 0; j < nt; ++j) th.emplace_back(work, j);
    for (auto& h : th) h.join();
  }
  for (unsigned i = 0; i <= dim; ++i) {
    NeumaierSum total;
    for (unsigned j = 0; j < nt; ++j) total.add(partial[size_t(j) * (dim + 1) + i].value());
    out[i] = total.value();
  }
}

// ------------------------------------------------------------------ convolution

// Section 3, benchmark 3: x[t] <- x[t] + y[t] * x[t] - z[t] for every tuple t of x's shape,
// each tensor addressed with its own shape (Algorithm 2; y and z contain x's shape).  The
// expression is evaluated left to right, ((y*x) then x + that, then minus z), each
// operation rounded to nearest even: in double for f64, in float for f32, and in float for
// bf16 / f16 with one final rounding to the storage format.
void oracle_apply_xpyxmz(int dtype, unsigned dim, const u64* xshape, void* x, const u64* yshape,
                         const void* y, const u64* zshape, const void* z) {
  const u64 n = count_of(xshape, dim);
  if (n == 0) return;
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    const u64 iy = tuple_to_index(t.data(), yshape, dim), iz = tuple_to_index(t.data(), zshape, dim);
    if (dtype == T_F64) {
      double* xx = static_cast<double*>(x);
      const double yv = static_cast<const double*>(y)[iy], zv = static_cast<const double*>(z)[iz];
      const double p = yv * xx[k];
      const double s = xx[k] + p;
      xx[k] = s - zv;
    } else {
      const float xv = float(load_as_double(x, k, dtype)), yv = float(load_as_double(y, iy, dtype)),
                  zv = float(load_as_double(z, iz, dtype));
      const float p = yv * xv;
      const float s = xv + p;
      const float r = s - zv;
      if (dtype == T_F32) static_cast<float*>(x)[k] = r;
      else if (dtype == T_BF16) static_cast<uint16_t*>(x)[k] = uint16_t(round_to_format(double(r), 8, -126, 127, 8));
      else static_cast<uint16_t*>(x)[k] = uint16_t(round_to_format(double(r), 11, -14, 15, 5));
    }
    advance_tuple(t.data(), xshape, dim);
  }
}

// Views of y starting at the tuple `ystart` (Section 4: the slice's flat index is the
// tensor's flat index of the start tuple -- its bias -- plus the flat index of the tuple
// within the slice, both by Horner's rule on y's own shape).  The tuples t walk x's shape
// (embed, crop) or the part of it that fits in y (product) with Algorithm 3.
void oracle_embed_at(int dtype, unsigned dim, const u64* xshape, const void* x, const u64* yshape,
                     void* y, const u64* ystart, int pad) {
  const size_t es = elem_size(dtype);
  if (pad) std::memset(y, 0, size_t(count_of(yshape, dim)) * es);
  const u64 n = count_of(xshape, dim);
  if (n == 0) return;
  const u64 bias = tuple_to_index(ystart, yshape, dim);
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    std::memcpy(static_cast<char*>(y) + (bias + tuple_to_index(t.data(), yshape, dim)) * es,
                static_cast<const char*>(x) + k * es, es);
    advance_tuple(t.data(), xshape, dim);
  }
}

void oracle_crop_at(int dtype, unsigned dim, const u64* xshape, void* x, const u64* yshape,
                    const void* y, const u64* ystart) {
  const size_t es = elem_size(dtype);
  const u64 n = count_of(xshape, dim);
  if (n == 0) return;
  const u64 bias = tuple_to_index(ystart, yshape, dim);
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    std::memcpy(static_cast<char*>(x) + k * es,
                static_cast<const char*>(y) + (bias + tuple_to_index(t.data(), yshape, dim)) * es, es);
    advance_tuple(t.data(), xshape, dim);
  }
}

void oracle_product_at(int dtype, unsigned dim, const u64* xshape, const void* x, const u64* yshape,
                       void* y, const u64* ystart) {
  std::vector<u64> I(dim);
  for (unsigned i = 0; i < dim; ++i) {
    const u64 room = yshape[i] - ystart[i];
    I[i] = xshape[i] < room ? xshape[i] : room;
  }
  const u64 n = count_of(I.data(), dim);
  if (n == 0) return;
  const u64 bias = tuple_to_index(ystart, yshape, dim);
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    multiply_into(y, bias + tuple_to_index(t.data(), yshape, dim), x,
                  tuple_to_index(t.data(), xshape, dim), dtype);
    advance_tuple(t.data(), I.data(), dim);
  }
}

// The moment of a product of tensors over the intersection I of their shapes (Algorithm
// 11 weights the tuple by x[t]*y[t]*z[t]; with two tensors the mass is benchmark 2's inner
// product over the tuples both shapes share, Section 3):
//   out[i]   = sum over t in I of w[t] * t_i,  i = 0..dim-1 (zero-based tuples),
//   out[dim] = sum over t in I of w[t],        w[t] = x_0[t] * x_1[t] * ... * x_{n-1}[t].
// w is formed left to right, each multiply rounded to nearest even in double for f64
// tensors and in float for f32, bf16 and f16 tensors (whose values float holds exactly).
// `shapes` holds n shapes of `dim` extents each, tensor k's at shapes[k*dim].  The tuples
// of I are walked with Algorithm 3 and each tensor is addressed by Horner's rule
// (Algorithm 2) with its own shape; sums are Neumaier-compensated in f64.
// Windows on both sides (Section 4: a view adds to every flat index the bias of its start
// tuple, both computed with its container's shape; views over the intersecting support let
// the product of two PMFs run without copies).  For every tuple t of the window extents
// `ext`:  copy:     y[ystart + t] = x[xstart + t]
//         product:  y[ystart + t] = y[ystart + t] * x[xstart + t]   (rounded as product)
// The caller guarantees that both windows lie inside their containers.
void oracle_copy_views(int dtype, unsigned dim, const u64* ext, const u64* xshape, const void* x,
                        const u64* xstart, const u64* yshape, void* y, const u64* ystart) {
  const size_t es = elem_size(dtype);
  const u64 n = count_of(ext, dim);
  if (n == 0) return;
  const u64 xbias = tuple_to_index(xstart, xshape, dim), ybias = tuple_to_index(ystart, yshape, dim);
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    std::memcpy(static_cast<char*>(y) + (ybias + tuple_to_index(t.data(), yshape, dim)) * es,
                static_cast<const char*>(x) + (xbias + tuple_to_index(t.data(), xshape, dim)) * es, es);
    advance_tuple(t.data(), ext, dim);
  }
}

void oracle_product_views(int dtype, unsigned dim, const u64* ext, const u64* xshape, const void* x,
                           const u64* xstart, const u64* yshape, void* y, const u64* ystart) {
  const u64 n = count_of(ext, dim);
  if (n == 0) return;
  const u64 xbias = tuple_to_index(xstart, xshape, dim), ybias = tuple_to_index(ystart, yshape, dim);
  std::vector<u64> t(dim, 0);
  for (u64 k = 0; k < n; ++k) {
    multiply_into(y, ybias + tuple_to_index(t.data(), yshape, dim), x,
                  xbias + tuple_to_index(t.data(), xshape, dim), dtype);
    advance_tuple(t.data(), ext, dim);
  }
}

// The nonzero bounding box of a product of tensors (Section 2: with the tuple visible to
// the operation, "the nonzero bounding box for the element-wise product of two tensors" is
// a plain loop).  Walks the tuples t of the intersection I of the shapes in order
// (Algorithm 3) and counts t when every factor x_k[t] is nonzero -- the support of the
// product of the tensors as real functions, so no rounding is involved; NaN and infinities
// count as nonzero, +0 and -0 do not.  out[2i] / out[2i+1]: the least and greatest t_i over
// the counted tuples, out[2 dim]: their number; with none counted, out[2i] = 0 and
// out[2i+1] = -1 (an empty range on every axis).
void oracle_nonzero_bbox(int dtype, unsigned dim, unsigned n, const u64* shapes,
                         const void* const* ptrs, int64_t* out) {
  for (unsigned i = 0; i < dim; ++i) {
    out[2 * i] = 0;
    out[2 * i + 1] = -1;
  }
  out[2 * dim] = 0;
  if (n == 0) return;
  std::vector<u64> I(dim);
  for (unsigned i = 0; i < dim; ++i) {
    I[i] = shapes[i];
    for (unsigned k = 1; k < n; ++k) I[i] = shapes[k * dim + i] < I[i] ? shapes[k * dim + i] : I[i];
  }
  const u64 count = count_of(I.data(), dim);
  std::vector<u64> t(dim, 0);
  int64_t found = 0;
  for (u64 c = 0; c < count; ++c) {
    bool nonzero = true;
    for (unsigned k = 0; k < n && nonzero; ++k)
      nonzero = load_as_double(ptrs[k], tuple_to_index(t.data(), shapes + k * dim, dim), dtype) != 0.0;
    if (nonzero) {
      for (unsigned i = 0; i < dim; ++i) {
        const int64_t v = int64_t(t[i]);
        if (found == 0 || v < out[2 * i]) out[2 * i] = v;
        if (found == 0 || v > out[2 * i + 1]) out[2 * i + 1] = v;
      }
      ++found;
    }
    advance_tuple(t.data(), I.data(), dim);
  }
  out[2 * dim] = found;
}

void oracle_moment_product(int dtype, unsigned dim, unsigned n, const u64* shapes,
                           const void* const* ptrs, double* out) {
  for (unsigned i = 0; i <= dim; ++i) out[i] = 0.0;
  if (n == 0) return;
  std::vector<u64> I(dim);
  for (unsigned i = 0; i < dim; ++i) {
    I[i] = shapes[i];
    for (unsigned k = 1; k < n; ++k) I[i] = shapes[k * dim + i] < I[i] ? shapes[k * dim + i] : I[i];
  }
  const u64 count = count_of(I.data(), dim);
  if (count == 0) return;
  std::vector<NeumaierSum> acc(dim + 1);
  std::vector<u64> t(dim, 0);
  for (u64 c = 0; c < count; ++c) {
    double w;
    if (dtype == T_F64) {
      w = load_as_double(ptrs[0], tuple_to_index(t.data(), shapes, dim), dtype);
      for (unsigned k = 1; k < n; ++k)
        w = w * load_as_double(ptrs[k], tuple_to_index(t.data(), shapes + k * dim, dim), dtype);
    } else {
      float wf = float(load_as_double(ptrs[0], tuple_to_index(t.data(), shapes, dim), dtype));
      for (unsigned k = 1; k < n; ++k)
        wf = wf * float(load_as_double(ptrs[k], tuple_to_index(t.data(), shapes + k * dim, dim), dtype));
      w = double(wf);
    }
    for (unsigned i = 0; i < dim; ++i) acc[i].add(w * double(t[i]));
    acc[dim].add(w);
    advance_tuple(t.data(), I.data(), dim);
  }
  for (unsigned i = 0; i <= dim; ++i) out[i] = acc[i].value();
}


// Naive multidimensional convolution by tuple iteration (Algorithm 14): for every pair of
// tuples (a of lhs, b of rhs) add lhs[a]*rhs[b] into result[a + b]; result shape is
// lhs.shape + rhs.shape - 1.  f64 only; plain (uncompensated) f64 adds in the paper's
// loop order.
void oracle_convolve_f64(unsigned dim, const u64* lshape, const double* lhs,
                         const u64* rshape, const double* rhs, double* result) {
  std::vector<u64> rs(dim);
  for (unsigned i = 0; i < dim; ++i) rs[i] = lshape[i] + rshape[i] - 1;
  const u64 nres = count_of(rs.data(), dim);
  for (u64 k = 0; k < nres; ++k) result[k] = 0.0;
  const u64 nl = count_of(lshape, dim), nr = count_of(rshape, dim);
  std::vector<u64> cl(dim, 0), cr(dim), cres(dim);
  for (u64 i = 0; i < nl; ++i, advance_tuple(cl.data(), lshape, dim)) {
    for (unsigned a = 0; a < dim; ++a) cr[a] = 0;
    for (u64 j = 0; j < nr; ++j, advance_tuple(cr.data(), rshape, dim)) {
      for (unsigned a = 0; a < dim; ++a) cres[a] = cl[a] + cr[a];
      result[tuple_to_index(cres.data(), rs.data(), dim)] += lhs[i] * rhs[j];
    }
  }
}

}  // extern "C"
