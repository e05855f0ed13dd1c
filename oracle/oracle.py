"""ctypes binding of the CPU oracle (oracle/triot_oracle.cpp) -- test infrastructure.

Arrays are numpy, C-contiguous.  bf16/f16 data travel as uint16 bit patterns
(np.uint16 views); f32/f64 as np.float32/np.float64.  Shapes are sequences of
non-negative ints.  Functions mirror the C entry points one to one; each C
function cites the passage of the paper it restates.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DTYPES = {"f64": 0, "f32": 1, "bf16": 2, "f16": 3}
NP_STORAGE = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16, "f16": np.uint16}
# (precision p incl. implicit bit, emin, emax, exponent bits)
FORMATS = {"f32": (24, -126, 127, 8), "bf16": (8, -126, 127, 8), "f16": (11, -14, 15, 5)}

_lib = None
_u64p = C.POINTER(C.c_uint64)


def load(path: str):
    """Open an oracle shared library at `path` and declare its C signatures."""
    L = C.CDLL(path)
    L.oracle_tuple_to_index.restype = C.c_uint64
    L.oracle_tuple_to_index.argtypes = [_u64p, _u64p, C.c_uint]
    L.oracle_advance_tuple.argtypes = [_u64p, _u64p, C.c_uint]
    L.oracle_reindex.restype = C.c_uint64
    L.oracle_reindex.argtypes = [C.c_uint64, _u64p, _u64p, C.c_uint]
    L.oracle_reindex_pow2.restype = C.c_uint64
    L.oracle_reindex_pow2.argtypes = [C.c_uint64, C.POINTER(C.c_uint), C.POINTER(C.c_uint), C.c_uint]
    L.oracle_enumerate.argtypes = [_u64p, C.c_uint, C.c_uint64, _u64p, _u64p]
    L.oracle_round_to_format.restype = C.c_uint32
    L.oracle_round_to_format.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, C.c_int]
    L.oracle_format_to_double.restype = C.c_double
    L.oracle_format_to_double.argtypes = [C.c_uint32, C.c_int, C.c_int]
    L.oracle_to_f64.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.c_void_p]
    L.oracle_from_f64.argtypes = [C.c_int, C.c_void_p, C.c_uint64, C.c_void_p]
    L.oracle_embed.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, C.c_int]
    L.oracle_crop.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, C.c_int]
    L.oracle_embed_window.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p,
                                      C.c_uint64, C.c_uint64, C.c_void_p]
    L.oracle_product.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, C.c_int]
    L.oracle_product_window.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p,
                                        C.c_uint64, C.c_uint64, C.c_void_p]
    L.oracle_moment.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, C.POINTER(C.c_double), C.c_int]
    L.oracle_apply_xpyxmz.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, _u64p,
                                      C.c_void_p]
    L.oracle_embed_at.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, _u64p, C.c_int]
    L.oracle_crop_at.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, _u64p]
    L.oracle_product_at.argtypes = [C.c_int, C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, _u64p]
    L.oracle_moment_product.argtypes = [C.c_int, C.c_uint, C.c_uint, _u64p, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_double)]
    L.oracle_convolve_f64.argtypes = [C.c_uint, _u64p, C.c_void_p, _u64p, C.c_void_p, C.c_void_p]
    L.oracle_copy_views.argtypes = [C.c_int, C.c_uint, _u64p, _u64p, C.c_void_p, _u64p, _u64p,
                                     C.c_void_p, _u64p]
    L.oracle_product_views.argtypes = [C.c_int, C.c_uint, _u64p, _u64p, C.c_void_p, _u64p, _u64p,
                                       C.c_void_p, _u64p]
    L.oracle_nonzero_bbox.argtypes = [C.c_int, C.c_uint, C.c_uint, _u64p, C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_int64)]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = load(_build.build())
    return _lib


def _shape(s) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(s), dtype=np.uint64))


def _p(a: np.ndarray):
    return a.ctypes.data_as(_u64p)


def _buf(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return C.c_void_p(a.ctypes.data)


def _check(a: np.ndarray, dtype: str, n: int):
    if a.dtype != NP_STORAGE[dtype]:
        raise TypeError(f"expected {NP_STORAGE[dtype]} storage for {dtype}, got {a.dtype}")
    if a.size != n:
        raise ValueError(f"expected {n} elements, got {a.size}")


# ------------------------------------------------------------ index arithmetic

def tuple_to_index(tup, shape) -> int:
    t, s = _shape(tup), _shape(shape)
    return int(lib().oracle_tuple_to_index(_p(t), _p(s), len(s)))


def advance_tuple(tup, shape) -> list:
    t, s = _shape(tup), _shape(shape)
    lib().oracle_advance_tuple(_p(t), _p(s), len(s))
    return [int(v) for v in t]


def reindex(index: int, shape, new_shape) -> int:
    s, n = _shape(shape), _shape(new_shape)
    return int(lib().oracle_reindex(index, _p(s), _p(n), len(s)))


def reindex_pow2(index: int, log_shape, new_log_shape) -> int:
    a = np.ascontiguousarray(np.asarray(log_shape, dtype=np.uint32))
    b = np.ascontiguousarray(np.asarray(new_log_shape, dtype=np.uint32))
    P = C.POINTER(C.c_uint)
    return int(lib().oracle_reindex_pow2(index, a.ctypes.data_as(P), b.ctypes.data_as(P), len(a)))


def enumerate_indices(shape, count=None):
    s = _shape(shape)
    n = int(np.prod([int(v) for v in shape])) if count is None else count
    idx = np.zeros(n, dtype=np.uint64)
    car = np.zeros(n, dtype=np.uint64)
    lib().oracle_enumerate(_p(s), len(s), n, _p(idx), _p(car))
    return idx, car


# ------------------------------------------------------------ formats

def round_to(v: float, fmt: str) -> int:
    p, emin, emax, eb = FORMATS[fmt]
    return int(lib().oracle_round_to_format(float(v), p, emin, emax, eb))


def format_to_double(bits: int, fmt: str) -> float:
    p, _, _, eb = FORMATS[fmt]
    return float(lib().oracle_format_to_double(int(bits), p, eb))


def to_f64(a: np.ndarray, dtype: str) -> np.ndarray:
    a = np.ascontiguousarray(a)
    out = np.empty(a.size, dtype=np.float64)
    lib().oracle_to_f64(DTYPES[dtype], _buf(a), a.size, _buf(out))
    return out.reshape(a.shape)


def from_f64(a: np.ndarray, dtype: str) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty(a.size, dtype=NP_STORAGE[dtype])
    lib().oracle_from_f64(DTYPES[dtype], _buf(a), a.size, _buf(out))
    return out.reshape(a.shape)


# ------------------------------------------------------------ operations

def embed(x: np.ndarray, xshape, yshape, dtype: str, nthreads: int = 1) -> np.ndarray:
    xs, ys = _shape(xshape), _shape(yshape)
    x = np.ascontiguousarray(x).reshape(-1)
    _check(x, dtype, int(np.prod(xs)) if len(xs) else 1)
    y = np.empty(int(np.prod(ys)), dtype=NP_STORAGE[dtype])
    lib().oracle_embed(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), nthreads)
    return y


def crop(y: np.ndarray, xshape, yshape, dtype: str, nthreads: int = 1) -> np.ndarray:
    xs, ys = _shape(xshape), _shape(yshape)
    y = np.ascontiguousarray(y).reshape(-1)
    _check(y, dtype, int(np.prod(ys)))
    x = np.empty(int(np.prod(xs)), dtype=NP_STORAGE[dtype])
    lib().oracle_crop(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), nthreads)
    return x


def embed_window(x: np.ndarray, xshape, yshape, begin: int, count: int, dtype: str) -> np.ndarray:
    xs, ys = _shape(xshape), _shape(yshape)
    x = np.ascontiguousarray(x).reshape(-1)
    out = np.empty(count, dtype=NP_STORAGE[dtype])
    lib().oracle_embed_window(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), begin, count, _buf(out))
    return out


def product(x: np.ndarray, xshape, y: np.ndarray, yshape, dtype: str, nthreads: int = 1) -> np.ndarray:
    """Returns a new array: y with y[t] *= x[t] over the shape intersection."""
    xs, ys = _shape(xshape), _shape(yshape)
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.array(y, copy=True).reshape(-1)
    _check(x, dtype, int(np.prod(xs)))
    _check(y, dtype, int(np.prod(ys)))
    lib().oracle_product(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), nthreads)
    return y


def product_inplace(x: np.ndarray, xshape, y: np.ndarray, yshape, dtype: str, nthreads: int = 1) -> None:
    xs, ys = _shape(xshape), _shape(yshape)
    assert y.flags["C_CONTIGUOUS"] and x.flags["C_CONTIGUOUS"]
    lib().oracle_product(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), nthreads)


def product_window(x: np.ndarray, xshape, ywin: np.ndarray, yshape, begin: int, dtype: str) -> np.ndarray:
    xs, ys = _shape(xshape), _shape(yshape)
    x = np.ascontiguousarray(x).reshape(-1)
    w = np.array(ywin, copy=True).reshape(-1)
    lib().oracle_product_window(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), begin, w.size, _buf(w))
    return w


def moment(p: np.ndarray, shape, dtype: str, nthreads: int = 1) -> np.ndarray:
    """Returns d+1 float64: [sum p*t_0, ..., sum p*t_{d-1}, sum p]."""
    s = _shape(shape)
    p = np.ascontiguousarray(p).reshape(-1)
    _check(p, dtype, int(np.prod(s)))
    out = np.zeros(len(s) + 1, dtype=np.float64)
    lib().oracle_moment(DTYPES[dtype], len(s), _p(s), _buf(p),
                        out.ctypes.data_as(C.POINTER(C.c_double)), nthreads)
    return out


def apply_xpyxmz(x: np.ndarray, xshape, y: np.ndarray, yshape, z: np.ndarray, zshape, dtype: str) -> np.ndarray:
    """Benchmark 3: a copy of x with x[t] <- x[t] + y[t] x[t] - z[t] over x's shape."""
    xs, ys, zs = _shape(xshape), _shape(yshape), _shape(zshape)
    x = np.ascontiguousarray(x).reshape(-1).copy()
    y = np.ascontiguousarray(y).reshape(-1)
    z = np.ascontiguousarray(z).reshape(-1)
    _check(x, dtype, int(np.prod(xs)))
    _check(y, dtype, int(np.prod(ys)))
    _check(z, dtype, int(np.prod(zs)))
    lib().oracle_apply_xpyxmz(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), _p(zs), _buf(z))
    return x


def embed_at(x: np.ndarray, xshape, yshape, ystart, dtype: str, y: np.ndarray | None = None) -> np.ndarray:
    """y[ystart + t] = x[t] over x's shape; the rest of y is +0 (or, given y, left as is)."""
    xs, ys, st = _shape(xshape), _shape(yshape), _shape(ystart)
    x = np.ascontiguousarray(x).reshape(-1)
    _check(x, dtype, int(np.prod(xs)))
    pad = y is None
    y = np.empty(int(np.prod(ys)), dtype=NP_STORAGE[dtype]) if pad else np.ascontiguousarray(y).reshape(-1).copy()
    lib().oracle_embed_at(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), _p(st), int(pad))
    return y


def crop_at(y: np.ndarray, xshape, yshape, ystart, dtype: str) -> np.ndarray:
    """x[t] = y[ystart + t] over x's shape."""
    xs, ys, st = _shape(xshape), _shape(yshape), _shape(ystart)
    y = np.ascontiguousarray(y).reshape(-1)
    _check(y, dtype, int(np.prod(ys)))
    x = np.empty(int(np.prod(xs)), dtype=NP_STORAGE[dtype])
    lib().oracle_crop_at(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), _p(st))
    return x


def product_at(x: np.ndarray, xshape, y: np.ndarray, yshape, ystart, dtype: str) -> np.ndarray:
    """A copy of y with y[ystart + t] *= x[t] over the tuples of x that fit in y."""
    xs, ys, st = _shape(xshape), _shape(yshape), _shape(ystart)
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1).copy()
    _check(x, dtype, int(np.prod(xs)))
    _check(y, dtype, int(np.prod(ys)))
    lib().oracle_product_at(DTYPES[dtype], len(xs), _p(xs), _buf(x), _p(ys), _buf(y), _p(st))
    return y


def _window_call(fn, ext, x, xshape, xstart, y, yshape, ystart, dtype):
    e, xs, ys = _shape(ext), _shape(xshape), _shape(yshape)
    xo, yo = _shape(xstart), _shape(ystart)
    x = np.ascontiguousarray(x).reshape(-1)
    y = np.ascontiguousarray(y).reshape(-1).copy()
    _check(x, dtype, int(np.prod(xs)))
    _check(y, dtype, int(np.prod(ys)))
    assert all(int(a) + int(b) <= int(c) for a, b, c in zip(xo, e, xs))
    assert all(int(a) + int(b) <= int(c) for a, b, c in zip(yo, e, ys))
    fn(DTYPES[dtype], len(e), _p(e), _p(xs), _buf(x), _p(xo), _p(ys), _buf(y), _p(yo))
    return y


def copy_views(ext, x, xshape, xstart, y, yshape, ystart, dtype: str) -> np.ndarray:
    """A copy of y with y[ystart + t] = x[xstart + t] for the tuples t of ext (Section 4)."""
    return _window_call(lib().oracle_copy_views, ext, x, xshape, xstart, y, yshape, ystart, dtype)


def product_views(ext, x, xshape, xstart, y, yshape, ystart, dtype: str) -> np.ndarray:
    """A copy of y with y[ystart + t] *= x[xstart + t] for the tuples t of ext (Section 4)."""
    return _window_call(lib().oracle_product_views, ext, x, xshape, xstart, y, yshape, ystart, dtype)


def moment_product(tensors, shapes, dtype: str) -> np.ndarray:
    """Moment of w = x_0 * x_1 * ... over the intersection of the shapes (Alg 11 with several
    weight tensors): d+1 float64 [sum w*t_0, ..., sum w*t_{d-1}, sum w]."""
    d = len(shapes[0])
    assert all(len(s) == d for s in shapes) and len(tensors) == len(shapes) >= 1
    flat = [np.ascontiguousarray(x).reshape(-1) for x in tensors]
    for x, s in zip(flat, shapes):
        _check(x, dtype, int(np.prod(s)))
    allshapes = np.ascontiguousarray(np.concatenate([_shape(s) for s in shapes]))
    ptrs = (C.c_void_p * len(flat))(*[x.ctypes.data for x in flat])
    out = np.zeros(d + 1, dtype=np.float64)
    lib().oracle_moment_product(DTYPES[dtype], d, len(flat), _p(allshapes), ptrs,
                                out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def nonzero_bbox(tensors, shapes, dtype: str) -> np.ndarray:
    """Nonzero bounding box of the product of the tensors over the intersection of their
    shapes: int64 [lo_0, hi_0, ..., lo_{d-1}, hi_{d-1}, count] (empty: lo 0, hi -1)."""
    d = len(shapes[0])
    assert all(len(s) == d for s in shapes) and len(tensors) == len(shapes) >= 1
    flat = [np.ascontiguousarray(x).reshape(-1) for x in tensors]
    for x, s in zip(flat, shapes):
        _check(x, dtype, int(np.prod(s)))
    allshapes = np.ascontiguousarray(np.concatenate([_shape(s) for s in shapes]))
    ptrs = (C.c_void_p * len(flat))(*[x.ctypes.data for x in flat])
    out = np.zeros(2 * d + 1, dtype=np.int64)
    lib().oracle_nonzero_bbox(DTYPES[dtype], d, len(flat), _p(allshapes), ptrs,
                              out.ctypes.data_as(C.POINTER(C.c_int64)))
    return out


def convolve_f64(lhs: np.ndarray, lshape, rhs: np.ndarray, rshape) -> np.ndarray:
    ls, rs = _shape(lshape), _shape(rshape)
    lhs = np.ascontiguousarray(lhs, dtype=np.float64).reshape(-1)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64).reshape(-1)
    outshape = [int(a) + int(b) - 1 for a, b in zip(lshape, rshape)]
    out = np.empty(int(np.prod(outshape)), dtype=np.float64)
    lib().oracle_convolve_f64(len(ls), _p(ls), _buf(lhs), _p(rs), _buf(rhs), _buf(out))
    return out.reshape(outshape)


def nproc() -> int:
    return os.cpu_count() or 1
