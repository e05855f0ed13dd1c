"""Host-side checks of the C ABI library (no GPU): it loads, exports every entry point
include/triot.h declares, runs the kernels' magic-number division exactly, canonicalises
shapes into an equivalent iteration, and rejects bad arguments before touching a GPU."""
import itertools
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def tr():
    from paper_1608_00099_gb300 import build, triot
    build.build()
    triot.lib()
    return triot


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "triot.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(triot_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function(tr):
    names = _declared_functions()
    assert len(names) >= 20
    L = tr.lib()
    for n in names:
        assert hasattr(L, n), n
    assert tr.version().startswith("triot-gb300")


def test_fastdiv_matches_integer_division(tr):
    rng = np.random.default_rng(1)
    edge = np.array([0, 1, 2, 3, 7, 8, 9, 2 ** 16, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 2, 2 ** 32 - 1],
                    dtype=np.uint64)
    divisors = list(range(1, 300)) + [2 ** k for k in range(31)] + [2 ** k + 1 for k in range(1, 31)] + \
        [2 ** k - 1 for k in range(2, 32)] + [int(v) for v in rng.integers(2, 2 ** 31, size=200)] + [3 ** 15, 9, 11, 10]
    for d in divisors:
        n = np.concatenate([edge, rng.integers(0, 2 ** 32, size=2000, dtype=np.uint64),
                            (np.arange(0, 50, dtype=np.uint64) * d) % (2 ** 32),
                            (np.arange(1, 50, dtype=np.uint64) * d - 1) % (2 ** 32)]).astype(np.uint32)
        q, r = tr.triot_fastdiv_check(d, n)
        n64 = n.astype(np.uint64)
        assert np.array_equal(q.astype(np.uint64), n64 // d), d
        assert np.array_equal(r.astype(np.uint64), n64 % d), d


def _iterate_canonical(c):
    """(x index, y index) of every iteration point, walking the canonical axes."""
    ext = c["ext"]
    for t in itertools.product(*[range(e) for e in ext]):
        xi = sum(a * s for a, s in zip(t, c["xstride"]))
        yi = sum(a * s for a, s in zip(t, c["ystride"]))
        inside = all(a < b for a, b in zip(t, c["xbound"]))
        yield xi, yi, inside


CANON_CASES = [((3, 4), (5, 4)), ((2, 3, 4), (2, 3, 4)), ((2, 1, 4), (3, 1, 4)), ((1, 1, 1), (1, 1, 1)),
               ((2, 2, 2), (3, 2, 2)), ((4, 3), (4, 5)), ((1, 5, 1, 2), (3, 5, 2, 2)), ((0, 3), (2, 3)),
               ((3, 1), (4, 6)), ((2, 3, 2), (2, 3, 5))]


@pytest.mark.parametrize("op", ["embed", "crop", "product"])
@pytest.mark.parametrize("case", CANON_CASES)
def test_canonical_form_addresses_the_same_elements(tr, op, case):
    xs, ys = case
    if op == "product":
        ys = tuple(max(1, b - (a % 2)) for a, b in zip(xs, ys))  # shapes that cross both ways
    code = {"embed": tr.OP_EMBED, "crop": tr.OP_CROP, "product": tr.OP_PRODUCT}[op]
    c = tr.triot_canonicalize(code, xs, ys)
    got = list(_iterate_canonical(c))
    # brute force over the original tuples (the oracle's addressing: Horner in each shape)
    if op == "embed":
        it = ys
    elif op == "crop":
        it = xs
    else:
        it = tuple(min(a, b) for a, b in zip(xs, ys))
    expect = []
    for t in itertools.product(*[range(e) for e in it]):
        inside = all(a < b for a, b in zip(t, xs))
        xi = int(np.ravel_multi_index(t, xs)) if inside and 0 not in xs else 0
        yi = int(np.ravel_multi_index(t, ys))
        expect.append((xi, yi, inside))
    if 0 in it:
        assert int(np.prod(c["ext"])) == 0 or not expect
        return
    assert len(got) == len(expect)
    for g, e in zip(got, expect):
        assert g[2] == e[2] or (op == "embed" and 0 in xs)
        if e[2]:
            assert g[0] == e[0]
        assert g[1] == e[1]


def test_canonical_form_of_the_workloads(tr):
    # f32 d=24: the last 9 axes merge into rows of 512 (x) inside rows of 768 (y)
    c = tr.triot_canonicalize(tr.OP_EMBED, (2,) * 24, (3,) * 16 + (2,) * 8)
    assert c["rank"] == 16 and c["ext"][-1] == 768 and c["xbound"][-1] == 512
    c = tr.triot_canonicalize(tr.OP_PRODUCT, (2,) * 24, (3,) * 16 + (2,) * 8)
    assert c["rank"] == 16 and c["ext"][-1] == 512 and c["ystride"][-2] == 768
    c = tr.triot_canonicalize(tr.OP_EMBED, (9,) * 8, (11, 10) * 4)
    assert c["rank"] == 8 and c["ext"] == [11, 10] * 4 and c["xbound"] == [9] * 8
    c = tr.triot_canonicalize(tr.OP_MOMENT, (1, 9, 1, 9))
    assert c["rank"] == 2 and c["ext"] == [9, 9] and c["orig"] == [1, 3]


def test_bad_arguments_fail_before_any_gpu_work(tr):
    import ctypes as C
    L = tr.lib()
    s3 = tr._shape((2, 3, 4))
    big = tr._shape((3, 3, 4))
    fake = C.c_void_p(0x1000)
    fake2 = C.c_void_p(0x100000)
    assert L.triot_embed(0, s3, fake, s3, fake2, 0, 0, None) == 1           # rank 0
    assert L.triot_embed(25, s3, fake, s3, fake2, 0, 0, None) == 1          # rank 25
    assert L.triot_embed(3, big, fake, s3, fake2, 0, 0, None) == 2          # x not inside y
    assert L.triot_embed(3, tr._shape((2, -1, 4)), fake, s3, fake2, 0, 0, None) == 2
    assert L.triot_embed(3, s3, fake, s3, fake2, 7, 0, None) == 4           # dtype
    assert L.triot_embed(3, s3, None, s3, fake2, 0, 0, None) == 3           # NULL x
    assert L.triot_embed(3, s3, fake, s3, fake, 0, 0, None) == 6            # aliasing
    assert L.triot_embed(3, s3, fake, s3, fake2, 0, 8, None) == 8           # unknown flag
    assert L.triot_crop(3, big, fake, s3, fake2, 1, None) == 2
    assert L.triot_product(3, s3, fake, s3, None, 1, None) == 3
    assert L.triot_moment(3, tr._shape((2, 2 ** 31, 1)), fake, 0, fake2, fake2, 1 << 20, None) == 2
    assert "must be < 2^31" in L.triot_last_error().decode()
    # the moment of a product: tensor count, extents and pointers are checked first
    shp = (tr._I64P * 2)(C.cast(s3, tr._I64P), C.cast(big, tr._I64P))
    ptrs = (C.c_void_p * 2)(fake, fake2)
    assert L.triot_moment_product(3, 0, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 8      # no tensors
    assert L.triot_moment_product(3, 5, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 8      # five
    assert L.triot_moment_product(0, 2, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 1      # rank 0
    assert L.triot_moment_product(3, 2, shp, ptrs, 9, fake2, fake2, 1 << 20, None) == 4      # dtype
    assert L.triot_moment_product(3, 2, None, ptrs, 0, fake2, fake2, 1 << 20, None) == 3     # NULL shapes
    neg = (tr._I64P * 2)(C.cast(s3, tr._I64P), C.cast(tr._shape((2, -1, 4)), tr._I64P))
    assert L.triot_moment_product(3, 2, neg, ptrs, 0, fake2, fake2, 1 << 20, None) == 2
    nbytes = C.c_size_t(0)
    assert L.triot_moment_product_workspace_size(3, 0, shp, 0, C.byref(nbytes)) == 8
    # windows on both sides: each window inside its container; support origins bounded
    e2 = tr._shape((2, 2))
    assert L.triot_copy_views(2, e2, tr._shape((2, 3)), fake, tr._shape((1, 0)), tr._shape((4, 4)), fake2,
                              tr._shape((0, 0)), 0, None) == 2
    assert L.triot_product_views(2, e2, tr._shape((2, 3)), fake, tr._shape((0, 0)), tr._shape((4, 4)), fake2,
                                 tr._shape((3, 0)), 0, None) == 2
    assert L.triot_product_views(2, e2, tr._shape((2, 3)), fake, tr._shape((0, 0)), tr._shape((4, 4)), fake,
                                 tr._shape((0, 0)), 0, None) == 6
    assert L.triot_product_views(2, e2, tr._shape((2, 3)), fake, tr._shape((0, 0)), tr._shape((4, 4)), fake2,
                                 tr._shape((0, 0)), 9, None) == 4
    assert L.triot_product_support(2, tr._shape((2, 3)), fake, tr._shape((1 << 62, 0)), tr._shape((4, 4)), fake2,
                                   tr._shape((0, 0)), 0, None) == 2
    assert L.triot_product_support(2, tr._shape((2, 3)), fake, None, tr._shape((4, 4)), fake2,
                                   tr._shape((0, 0)), 0, None) == 3
    # nonzero bounding box: tensor count, rank, dtype, shapes
    assert L.triot_nonzero_bbox(3, 0, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 8
    assert L.triot_nonzero_bbox(3, 5, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 8
    assert L.triot_nonzero_bbox(25, 2, shp, ptrs, 0, fake2, fake2, 1 << 20, None) == 1
    assert L.triot_nonzero_bbox(3, 2, shp, ptrs, 7, fake2, fake2, 1 << 20, None) == 4
    assert L.triot_nonzero_bbox(3, 2, None, ptrs, 0, fake2, fake2, 1 << 20, None) == 3
    assert L.triot_nonzero_bbox(3, 2, neg, ptrs, 0, fake2, fake2, 1 << 20, None) == 2
    assert L.triot_nonzero_bbox_workspace_size(3, 2, shp, 0, None) == 3
    # convolution: f64 only, rank, shapes
    assert L.triot_convolve(3, s3, fake, s3, fake2, fake, 1, None) == 4
    assert L.triot_convolve(0, s3, fake, s3, fake2, fake, 0, None) == 1
    assert L.triot_convolve(3, tr._shape((2, -1, 4)), fake, s3, fake2, fake, 0, None) == 2
    # apply: op code, shapes (y and z contain x)
    assert L.triot_apply(9, 3, s3, fake, s3, fake2, s3, fake2, 0, None) == 8
    assert L.triot_apply(1, 3, big, fake, s3, fake2, big, fake2, 0, None) == 2
    assert L.triot_apply(1, 3, s3, fake, s3, fake2, s3, fake2, 7, None) == 4
    assert L.triot_apply(1, 3, s3, None, s3, fake2, s3, fake2, 0, None) == 3
    # views: the window must fit (embed/crop) or start inside y (product)
    st = tr._shape((1, 1, 1))
    assert L.triot_crop_at(3, s3, fake, s3, fake2, st, 0, None) == 2            # 1 + 3 > 3
    assert L.triot_embed_at(3, s3, fake, big, fake2, tr._shape((0, 0, 1)), 0, 0, None) == 2
    assert L.triot_product_at(3, s3, fake, s3, fake2, tr._shape((0, 4, 0)), 0, None) == 2   # start > extent
    assert L.triot_crop_at(3, s3, fake, big, fake2, tr._shape((0, -1, 0)), 0, None) == 2
    assert L.triot_crop_at(3, s3, fake, big, fake2, None, 0, None) == 3
    assert L.triot_embed_at(3, s3, fake, big, fake2, tr._shape((1, 0, 0)), 0, 8, None) == 8  # flag
    # empty iterations are no-ops and succeed without touching the device
    assert L.triot_product(2, tr._shape((0, 3)), None, tr._shape((2, 3)), None, 0, None) == 0
    assert L.triot_crop(2, tr._shape((2, 0)), None, tr._shape((2, 3)), None, 0, None) == 0


def test_tune_cache_roundtrip_without_gpu(tr, tmp_path):
    # keys include the GPU name; without a GPU the calls still validate their input
    import ctypes as C
    L = tr.lib()
    bad = tr.Tune(33, 0, 0, 0)
    assert L.triot_tune_set(0, 2, tr._shape((2, 3)), tr._shape((4, 5)), 0, C.byref(bad)) == 8
    assert L.triot_tune_load(str(tmp_path / "missing.json").encode()) == 8


def _desc(tr, xs, ys, x=0x1000, y=0x10000000, out=0x20000000):
    d = tr.BatchDesc()
    d.rank = len(xs)
    for a, (e, f) in enumerate(zip(xs, ys)):
        d.xshape[a] = e
        d.yshape[a] = f
    d.x, d.y, d.moment_out = x, y, out
    return d


@pytest.mark.parametrize("case,code", [
    ("negative extent", 2), ("zero extent", 2), ("x larger than y", 2), ("extent 2^31", 2),
    ("rank 0", 1), ("rank 25", 1), ("rank -3", 1), ("null x", 3), ("null y", 3), ("null out", 3),
    ("x overlaps y", 6), ("too many elements", 2)])
def test_batch_plan_rejects_corrupted_descriptor(tr, case, code):
    """A corrupted descriptor anywhere in the list fails plan creation with its status code
    before any device memory is allocated (no GPU is present here)."""
    import ctypes as C
    L = tr.lib()
    good = [_desc(tr, (2, 3), (4, 5), x=0x1000 + k * 0x100000, y=0x40000000 + k * 0x100000) for k in range(5)]
    bad = _desc(tr, (2, 3), (4, 5), x=0x7000000, y=0x8000000)
    if case == "negative extent":
        bad.xshape[1] = -3
    elif case == "zero extent":
        bad.yshape[0] = 0
    elif case == "x larger than y":
        bad.xshape[0] = 9
    elif case == "extent 2^31":
        bad.xshape[1] = 1
        bad.yshape[1] = 1 << 31
    elif case == "rank 0":
        bad.rank = 0
    elif case == "rank 25":
        bad.rank = 25
    elif case == "rank -3":
        bad.rank = -3
    elif case == "null x":
        bad.x = None
    elif case == "null y":
        bad.y = None
    elif case == "null out":
        bad.moment_out = None
    elif case == "x overlaps y":
        bad.y = bad.x + 8
    elif case == "too many elements":
        bad.rank = 6
        for a in range(6):
            bad.xshape[a] = 2
            bad.yshape[a] = 1 << 20
    descs = (tr.BatchDesc * 6)(*(good[:3] + [bad] + good[3:]))
    plan = C.c_void_p(0)
    assert L.triot_batch_plan_create(descs, 6, 1, 0, None, C.byref(plan)) == code
    assert not plan.value
    assert "descriptor 3" in L.triot_last_error().decode()


def test_batch_plan_rejects_bad_arguments(tr):
    import ctypes as C
    L = tr.lib()
    descs = (tr.BatchDesc * 1)(_desc(tr, (2, 3), (4, 5)))
    plan = C.c_void_p(0)
    assert L.triot_batch_plan_create(descs, 0, 1, 0, None, C.byref(plan)) == 8        # no pairs
    assert L.triot_batch_plan_create(None, 1, 1, 0, None, C.byref(plan)) == 8
    assert L.triot_batch_plan_create(descs, 1, 7, 0, None, C.byref(plan)) == 4        # dtype
    assert L.triot_batch_plan_create(descs, 1, 1, 5, None, C.byref(plan)) == 8        # mode
    assert L.triot_batch_plan_create(descs, 1, 1, 0, None, None) == 3
    t = tr.Tune(0, -1, 0, 0)
    assert L.triot_batch_plan_create(descs, 1, 1, 0, C.byref(t), C.byref(plan)) == 8  # tile < 0
    t = tr.Tune(0, 0, 33, 0)
    assert L.triot_batch_plan_create(descs, 1, 1, 0, C.byref(t), C.byref(plan)) == 8  # ctas/SM
    assert L.triot_batch_autotune(None, 1, 1, 0, None, None) == 8
    assert not plan.value
