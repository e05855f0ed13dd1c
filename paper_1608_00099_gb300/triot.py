"""Python binding of the C ABI in include/triot.h (ctypes; argument marshalling only).

Every function here converts torch tensors to (rank, shape, device pointer, dtype
code, stream) and calls the entry point of the same name in libtriot.so; all
computation happens in the CUDA kernels behind that library.  If the library is
missing the first call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtriot.so")

MAX_RANK = 24
F64, F32, BF16, F16 = 0, 1, 2, 3
DTYPE_CODE = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
EMBED_NOPAD = 1
OP_EMBED, OP_CROP, OP_PRODUCT, OP_MOMENT, OP_BATCH = 0, 1, 2, 3, 4
BATCH_FUSED, BATCH_PHASED = 0, 1
MOMENT_MAX_WORKSPACE_PER_RANK = 16384 * 8

STATUS = {0: "OK", 1: "ERR_RANK", 2: "ERR_SHAPE", 3: "ERR_NULL", 4: "ERR_DTYPE", 5: "ERR_WORKSPACE",
          6: "ERR_ALIAS", 7: "ERR_CUDA", 8: "ERR_ARG", 9: "ERR_DEVICE"}


class TriotError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class BatchDesc(C.Structure):
    _fields_ = [("rank", C.c_int),
                ("xshape", C.c_int64 * MAX_RANK),
                ("yshape", C.c_int64 * MAX_RANK),
                ("x", C.c_void_p),
                ("y", C.c_void_p),
                ("moment_out", C.c_void_p)]


class Tune(C.Structure):
    _fields_ = [("threads", C.c_int), ("tile_elems", C.c_int), ("ctas_per_sm", C.c_int), ("unroll", C.c_int)]


_lib = None
_I64P = C.POINTER(C.c_int64)


def lib() -> C.CDLL:
    """Load libtriot.so (built by paper_1608_00099_gb300.build); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtriot.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, u, sz = C.c_void_p, C.c_int, C.c_uint, C.c_size_t
        sig = {
            "triot_last_error": (C.c_char_p, []),
            "triot_version": (C.c_char_p, []),
            "triot_embed": (i, [i, _I64P, vp, _I64P, vp, i, u, vp]),
            "triot_crop": (i, [i, _I64P, vp, _I64P, vp, i, vp]),
            "triot_product": (i, [i, _I64P, vp, _I64P, vp, i, vp]),
            "triot_moment_workspace_size": (i, [i, _I64P, i, C.POINTER(sz)]),
            "triot_moment": (i, [i, _I64P, vp, i, vp, vp, sz, vp]),
            "triot_moment_noalloc": (i, [i, _I64P, vp, i, vp, vp]),
            "triot_moment_plan": (i, [i, _I64P, i, C.POINTER(i), C.POINTER(i), _I64P, _I64P]),
            "triot_apply": (i, [i, i, _I64P, vp, _I64P, vp, _I64P, vp, i, vp]),
            "triot_convolve": (i, [i, _I64P, vp, _I64P, vp, vp, i, vp]),
            "triot_embed_at": (i, [i, _I64P, vp, _I64P, vp, _I64P, i, u, vp]),
            "triot_crop_at": (i, [i, _I64P, vp, _I64P, vp, _I64P, i, vp]),
            "triot_product_at": (i, [i, _I64P, vp, _I64P, vp, _I64P, i, vp]),
            "triot_copy_views": (i, [i, _I64P, _I64P, vp, _I64P, _I64P, vp, _I64P, i, vp]),
            "triot_product_views": (i, [i, _I64P, _I64P, vp, _I64P, _I64P, vp, _I64P, i, vp]),
            "triot_product_support": (i, [i, _I64P, vp, _I64P, _I64P, vp, _I64P, i, vp]),
            "triot_moment_product_workspace_size": (i, [i, i, C.POINTER(_I64P), i, C.POINTER(sz)]),
            "triot_moment_product": (i, [i, i, C.POINTER(_I64P), C.POINTER(vp), i, vp, vp, sz, vp]),
            "triot_nonzero_bbox_workspace_size": (i, [i, i, C.POINTER(_I64P), i, C.POINTER(sz)]),
            "triot_nonzero_bbox": (i, [i, i, C.POINTER(_I64P), C.POINTER(vp), i, vp, vp, sz, vp]),
            "triot_batch_plan_create": (i, [C.POINTER(BatchDesc), i, i, i, C.POINTER(Tune), C.POINTER(vp)]),
            "triot_batch_run": (i, [vp, vp]),
            "triot_batch_run_plain": (i, [vp, vp]),
            "triot_batch_plan_info": (i, [vp, C.POINTER(sz), _I64P]),
            "triot_batch_plan_destroy": (i, [vp]),
            "triot_batch_plan_geometry": (i, [vp, C.POINTER(Tune)]),
            "triot_batch_autotune": (i, [C.POINTER(BatchDesc), i, i, i, vp, C.POINTER(Tune)]),
            "triot_autotune": (i, [i, i, _I64P, vp, _I64P, vp, i, vp, sz, vp, C.POINTER(Tune)]),
            "triot_tune_get": (i, [i, i, _I64P, _I64P, i, C.POINTER(Tune)]),
            "triot_tune_set": (i, [i, i, _I64P, _I64P, i, C.POINTER(Tune)]),
            "triot_tune_save": (i, [C.c_char_p]),
            "triot_tune_load": (i, [C.c_char_p]),
            "triot_tune_clear": (i, []),
            "triot_canonicalize": (i, [i, i, _I64P, _I64P, C.POINTER(i), _I64P, _I64P, _I64P, _I64P,
                                       C.POINTER(i)]),
            "triot_fastdiv_check": (i, [C.c_uint32, C.POINTER(C.c_uint32), sz, C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint32)]),
            "triot_device_status": (i, []),
            "triot_selftest_wait_timeout": (i, [i, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != 0:
        raise TriotError(status, lib().triot_last_error().decode())


def _shape(s) -> C.Array:
    s = [int(v) for v in s]
    return (C.c_int64 * max(1, len(s)))(*s)


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dtype(t: torch.Tensor) -> int:
    try:
        return DTYPE_CODE[t.dtype]
    except KeyError:
        raise TriotError(4, f"unsupported dtype {t.dtype}") from None


def _dev(t: torch.Tensor) -> int:
    if not t.is_cuda:
        raise TriotError(3, "tensors must live on a CUDA device")
    if not t.is_contiguous():
        raise TriotError(8, "tensors must be contiguous")
    return t.data_ptr()


def version() -> str:
    return lib().triot_version().decode()


# ------------------------------------------------------------------ operations

def triot_embed(x: torch.Tensor, y: torch.Tensor, flags: int = 0, stream=None) -> torch.Tensor:
    """y <- 0; y[t] = x[t] over x's tuples (x at the origin of y)."""
    if x.dim() != y.dim():
        raise TriotError(1, "x and y must have the same rank")
    _check(lib().triot_embed(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _dtype(y),
                             flags, _stream(stream)))
    return y


def triot_crop(x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """x[t] = y[t] over x's tuples."""
    if x.dim() != y.dim():
        raise TriotError(1, "x and y must have the same rank")
    _check(lib().triot_crop(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _dtype(x),
                            _stream(stream)))
    return x


def triot_product(x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
    """y[t] *= x[t] over the intersection of the two shapes (in place on y)."""
    if x.dim() != y.dim():
        raise TriotError(1, "x and y must have the same rank")
    if x.dtype != y.dtype:
        raise TriotError(4, "x and y must share a dtype")
    _check(lib().triot_product(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _dtype(y),
                               _stream(stream)))
    return y


def triot_moment_workspace_size(shape, dtype: torch.dtype) -> int:
    n = C.c_size_t(0)
    _check(lib().triot_moment_workspace_size(len(shape), _shape(shape), DTYPE_CODE[dtype], C.byref(n)))
    return int(n.value)


def triot_moment(p: torch.Tensor, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                 stream=None) -> torch.Tensor:
    """out[i] = sum_t p[t] t_i (i < rank), out[rank] = sum_t p[t]; out is float64 on p's device."""
    rank = p.dim()
    if out is None:
        out = torch.empty(rank + 1, dtype=torch.float64, device=p.device)
    if workspace is None:
        nb = triot_moment_workspace_size(p.shape, p.dtype)
        workspace = torch.empty((nb + 15) // 16 * 2, dtype=torch.float64, device=p.device)
    if out.dtype != torch.float64 or out.numel() < rank + 1:
        raise TriotError(8, "out must hold rank + 1 float64 values")
    _check(lib().triot_moment(rank, _shape(p.shape), _dev(p), _dtype(p), _dev(out), _dev(workspace),
                              workspace.numel() * workspace.element_size(), _stream(stream)))
    return out


MOMENT_KERNELS = {0: "rows", 1: "blocks64", 2: "blocks32", 3: "warpblocks", 4: "marginals"}


def triot_moment_plan(shape, dtype: torch.dtype) -> dict:
    """The moment kernel triot_moment would launch for this shape and dtype."""
    k, g = C.c_int(0), C.c_int(0)
    r, c = C.c_int64(0), C.c_int64(0)
    _check(lib().triot_moment_plan(len(shape), _shape(shape), DTYPE_CODE[dtype], C.byref(k), C.byref(g),
                                   C.byref(r), C.byref(c)))
    return {"kernel": MOMENT_KERNELS[k.value], "grid": g.value, "rows": r.value, "cols": c.value}


def triot_convolve(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Naive multidimensional convolution of two f64 tensors of one rank; out has shape
    a.shape + b.shape - 1."""
    shape = [max(0, x + y - 1) for x, y in zip(a.shape, b.shape)]
    if out is None:
        out = torch.empty(shape, dtype=torch.float64, device=a.device)
    if list(out.shape) != shape:
        raise TriotError(8, f"out must have shape {shape}")
    _check(lib().triot_convolve(a.dim(), _shape(a.shape), _dev(a), _shape(b.shape), _dev(b), _dev(out),
                                _dtype(a), _stream(stream)))
    return out


APPLY_XPYXMZ = 1


def triot_apply_xpyxmz(x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, stream=None) -> torch.Tensor:
    """x[t] <- x[t] + y[t] * x[t] - z[t] over x's shape (y and z contain it), in place."""
    _check(lib().triot_apply(APPLY_XPYXMZ, x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y),
                             _shape(z.shape), _dev(z), _dtype(x), _stream(stream)))
    return x


def triot_embed_at(x: torch.Tensor, y: torch.Tensor, ystart, flags: int = 0, stream=None) -> torch.Tensor:
    """y[ystart + t] = x[t] over x's shape; the rest of y is +0 unless flags has EMBED_NOPAD."""
    _check(lib().triot_embed_at(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _shape(ystart),
                                _dtype(x), flags, _stream(stream)))
    return y


def triot_crop_at(x: torch.Tensor, y: torch.Tensor, ystart, stream=None) -> torch.Tensor:
    """x[t] = y[ystart + t] over x's shape."""
    _check(lib().triot_crop_at(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _shape(ystart),
                               _dtype(x), _stream(stream)))
    return x


def triot_product_at(x: torch.Tensor, y: torch.Tensor, ystart, stream=None) -> torch.Tensor:
    """y[ystart + t] *= x[t] over the tuples of x that fit in y."""
    _check(lib().triot_product_at(x.dim(), _shape(x.shape), _dev(x), _shape(y.shape), _dev(y), _shape(ystart),
                                  _dtype(x), _stream(stream)))
    return y


def triot_copy_views(ext, x: torch.Tensor, xstart, y: torch.Tensor, ystart, stream=None) -> torch.Tensor:
    """y[ystart + t] = x[xstart + t] for every tuple t of ext (windows of two containers)."""
    _check(lib().triot_copy_views(x.dim(), _shape(ext), _shape(x.shape), _dev(x), _shape(xstart),
                                  _shape(y.shape), _dev(y), _shape(ystart), _dtype(x), _stream(stream)))
    return y


def triot_product_views(ext, x: torch.Tensor, xstart, y: torch.Tensor, ystart, stream=None) -> torch.Tensor:
    """y[ystart + t] *= x[xstart + t] for every tuple t of ext (windows of two containers)."""
    _check(lib().triot_product_views(x.dim(), _shape(ext), _shape(x.shape), _dev(x), _shape(xstart),
                                     _shape(y.shape), _dev(y), _shape(ystart), _dtype(x), _stream(stream)))
    return y


def triot_product_support(x: torch.Tensor, xorigin, y: torch.Tensor, yorigin, stream=None) -> torch.Tensor:
    """y *= x over the tuples both cover when x sits at xorigin and y at yorigin of one grid."""
    _check(lib().triot_product_support(x.dim(), _shape(x.shape), _dev(x), _shape(xorigin), _shape(y.shape),
                                       _dev(y), _shape(yorigin), _dtype(x), _stream(stream)))
    return y


def _shape_table(shapes):
    arrs = [_shape(s) for s in shapes]
    table = (_I64P * len(arrs))(*[C.cast(a, _I64P) for a in arrs])
    return table, arrs          # keep the arrays alive with the table


def triot_moment_product_workspace_size(shapes, dtype: torch.dtype) -> int:
    table, _keep = _shape_table(shapes)
    n = C.c_size_t(0)
    _check(lib().triot_moment_product_workspace_size(len(shapes[0]), len(shapes), table, DTYPE_CODE[dtype],
                                                     C.byref(n)))
    return int(n.value)


def triot_moment_product(tensors, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                         stream=None) -> torch.Tensor:
    """Moment of w = x_0 * x_1 * ... over the intersection of the shapes (all tensors of one
    dtype and rank, on one device): out[i] = sum_t w[t] t_i, out[rank] = sum_t w[t]."""
    tensors = list(tensors)
    rank = tensors[0].dim()
    dev = tensors[0].device
    if out is None:
        out = torch.empty(rank + 1, dtype=torch.float64, device=dev)
    if out.dtype != torch.float64 or out.numel() < rank + 1:
        raise TriotError(8, "out must hold rank + 1 float64 values")
    shapes = [tuple(t.shape) for t in tensors]
    if workspace is None:
        nb = triot_moment_product_workspace_size(shapes, tensors[0].dtype)
        workspace = torch.empty((nb + 15) // 16 * 2, dtype=torch.float64, device=dev)
    table, _keep = _shape_table(shapes)
    ptrs = (C.c_void_p * len(tensors))(*[_dev(t) for t in tensors])
    _check(lib().triot_moment_product(rank, len(tensors), table, ptrs, _dtype(tensors[0]), _dev(out),
                                      _dev(workspace), workspace.numel() * workspace.element_size(),
                                      _stream(stream)))
    return out


def triot_nonzero_bbox_workspace_size(shapes, dtype: torch.dtype) -> int:
    n = C.c_size_t(0)
    table, _keep = _shape_table(shapes)
    _check(lib().triot_nonzero_bbox_workspace_size(len(shapes[0]), len(shapes), table, DTYPE_CODE[dtype],
                                                   C.byref(n)))
    return int(n.value)


def triot_nonzero_bbox(tensors, out: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
    """[lo_0, hi_0, .., lo_{d-1}, hi_{d-1}, count] of the nonzero entries of the tensors' product."""
    tensors = list(tensors)
    shapes = [tuple(t.shape) for t in tensors]
    rank = len(shapes[0])
    dev = tensors[0].device
    if out is None:
        out = torch.empty(2 * rank + 1, dtype=torch.int64, device=dev)
    if out.dtype != torch.int64 or out.numel() < 2 * rank + 1:
        raise TriotError(8, "out must hold 2 rank + 1 int64 values")
    if workspace is None:
        nb = triot_nonzero_bbox_workspace_size(shapes, tensors[0].dtype)
        workspace = torch.empty((nb + 15) // 16 * 2, dtype=torch.int64, device=dev)
    table, _keep = _shape_table(shapes)
    ptrs = (C.c_void_p * len(tensors))(*[_dev(t) for t in tensors])
    _check(lib().triot_nonzero_bbox(rank, len(tensors), table, ptrs, _dtype(tensors[0]), _dev(out),
                                    _dev(workspace), workspace.numel() * workspace.element_size(),
                                    _stream(stream)))
    return out


def triot_canonicalize(op: int, xshape, yshape=None) -> dict:
    """Host-only: the effective axes a call runs over."""
    d = C.c_int(0)
    ext = (C.c_int64 * MAX_RANK)()
    xs = (C.c_int64 * MAX_RANK)()
    ys = (C.c_int64 * MAX_RANK)()
    xb = (C.c_int64 * MAX_RANK)()
    orig = (C.c_int * MAX_RANK)()
    yarg = _shape(yshape) if yshape is not None else None
    _check(lib().triot_canonicalize(op, len(xshape), _shape(xshape), yarg, C.byref(d), ext, xs, ys, xb, orig))
    n = d.value
    return {"rank": n, "ext": list(ext[:n]), "xstride": list(xs[:n]), "ystride": list(ys[:n]),
            "xbound": list(xb[:n]), "orig": list(orig[:n])}


def triot_fastdiv_check(d: int, n) -> tuple:
    import numpy as np
    n = np.ascontiguousarray(np.asarray(n, dtype=np.uint32))
    q = np.empty_like(n)
    r = np.empty_like(n)
    P = C.POINTER(C.c_uint32)
    _check(lib().triot_fastdiv_check(d, n.ctypes.data_as(P), n.size, q.ctypes.data_as(P), r.ctypes.data_as(P)))
    return q, r


def triot_device_status() -> int:
    return int(lib().triot_device_status())


def triot_selftest_wait_timeout(limit: int = 16, stream=None) -> None:
    _check(lib().triot_selftest_wait_timeout(limit, _stream(stream)))


# ------------------------------------------------------------------ tuning

def _tune_dict(t: Tune) -> dict:
    return {"threads": t.threads, "tile_elems": t.tile_elems, "ctas_per_sm": t.ctas_per_sm, "unroll": t.unroll}


def triot_autotune(op: int, x: torch.Tensor, y: torch.Tensor | None = None, workspace: torch.Tensor | None = None,
                   stream=None) -> dict:
    best = Tune()
    rank = x.dim()
    yshape = _shape(y.shape) if y is not None else None
    ydev = _dev(y) if y is not None else None
    if op == OP_MOMENT and workspace is None:
        workspace = torch.empty(MOMENT_MAX_WORKSPACE_PER_RANK * (rank + 1) // 8, dtype=torch.float64,
                                device=x.device)
    ws = _dev(workspace) if workspace is not None else None
    wsb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check(lib().triot_autotune(op, rank, _shape(x.shape), _dev(x), yshape, ydev, _dtype(x), ws, wsb,
                                _stream(stream), C.byref(best)))
    return _tune_dict(best)


def triot_tune_get(op: int, xshape, yshape, dtype: torch.dtype) -> dict:
    t = Tune()
    _check(lib().triot_tune_get(op, len(xshape), _shape(xshape), _shape(yshape) if yshape else None,
                                DTYPE_CODE[dtype], C.byref(t)))
    return _tune_dict(t)


def triot_tune_set(op: int, xshape, yshape, dtype: torch.dtype, threads=0, tile_elems=0, ctas_per_sm=0,
                   unroll=0) -> None:
    t = Tune(threads, tile_elems, ctas_per_sm, unroll)
    _check(lib().triot_tune_set(op, len(xshape), _shape(xshape), _shape(yshape) if yshape else None,
                                DTYPE_CODE[dtype], C.byref(t)))


def triot_tune_save(path: str) -> None:
    _check(lib().triot_tune_save(path.encode()))


def triot_tune_load(path: str) -> None:
    _check(lib().triot_tune_load(path.encode()))


def triot_tune_clear() -> None:
    _check(lib().triot_tune_clear())


# ------------------------------------------------------------------ batched pipeline

def _batch_descs(xs, ys, outs):
    if not (len(xs) == len(ys) == len(outs)) or not xs:
        raise TriotError(8, "need matching, non-empty lists of x, y and out")
    dt = _dtype(xs[0])
    descs = (BatchDesc * len(xs))()
    for k, (x, y, o) in enumerate(zip(xs, ys, outs)):
        if x.dim() != y.dim() or _dtype(x) != dt or _dtype(y) != dt:
            raise TriotError(8, f"pair {k}: ranks or dtypes differ")
        d = descs[k]
        d.rank = x.dim()
        for a in range(x.dim()):
            d.xshape[a] = x.shape[a]
            d.yshape[a] = y.shape[a]
        d.x, d.y, d.moment_out = _dev(x), _dev(y), _dev(o)
    return descs, dt


def triot_batch_autotune(xs, ys, outs, mode: int = 0, stream=None) -> dict:
    """Time the batch's candidate geometries and cache the fastest (triot_batch_autotune)."""
    descs, dt = _batch_descs(xs, ys, outs)
    best = Tune()
    _check(lib().triot_batch_autotune(descs, len(xs), dt, mode, _stream(stream), C.byref(best)))
    return _tune_dict(best)


class BatchPlan:
    """Owns a triot_plan: embed -> product -> moment for many (x, y, out) triples."""

    def __init__(self, xs, ys, outs, mode: int = BATCH_FUSED, tile_elems: int = 0, ctas_per_sm: int = 0):
        descs, dt = _batch_descs(xs, ys, outs)
        self._keep = (xs, ys, outs)
        self._h = C.c_void_p(0)
        tune = Tune(0, tile_elems, ctas_per_sm, 0)
        _check(lib().triot_batch_plan_create(descs, len(xs), dt, mode, C.byref(tune), C.byref(self._h)))

    def run(self, stream=None) -> None:
        _check(lib().triot_batch_run(self._h, _stream(stream)))

    def run_plain(self, stream=None) -> None:
        _check(lib().triot_batch_run_plain(self._h, _stream(stream)))

    def info(self) -> dict:
        b = C.c_size_t(0)
        t = C.c_int64(0)
        _check(lib().triot_batch_plan_info(self._h, C.byref(b), C.byref(t)))
        return {"device_bytes": int(b.value), "tiles": int(t.value)}

    def geometry(self) -> dict:
        t = Tune()
        _check(lib().triot_batch_plan_geometry(self._h, C.byref(t)))
        return _tune_dict(t)

    def close(self) -> None:
        if self._h:
            lib().triot_batch_plan_destroy(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
