"""The oracle's pins are sensitive: plausible mistakes planted in a copy of the oracle
source (on the CPU, never in the GPU path) must each fail at least one pin."""
import os
import shutil
import subprocess

import pytest

from oracle import oracle as orc_mod

import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "triot_oracle.cpp")

# (description, text in the source, replacement, pins expected to catch it)
MUTANTS = [
    ("Horner multiplies by the wrong axis", "flat = flat * shape[axis] + tup[axis];",
     "flat = flat * shape[dim - 1 - axis] + tup[axis];",
     [lambda o: pins.test_worked_example_flat_index(o)]),
    ("carry test off by one", "tup[grow] + 1 == shape[grow]", "tup[grow] == shape[grow]",
     [lambda o: pins.test_advance_tuple_lexicographic(o, (2, 3, 4))]),
    ("reindex flattens with the old shape", "return tuple_to_index(tup.data(), new_shape, dim);",
     "return tuple_to_index(tup.data(), shape, dim);",
     [lambda o: pins.test_reindex_equals_unravel_ravel(o, ((3, 4), (5, 6)))]),
    ("ties round to odd", "std::fmod(fl, 2.0) != 0.0", "std::fmod(fl, 2.0) == 0.0",
     [lambda o: pins.test_round_to_f16_equals_numpy(o)]),
    ("embed addresses y with x's shape",
     "const u64 iy = tuple_to_index(t.data(), yshape, dim);\n      std::memcpy(ys + iy * es, xs + k * es, es);",
     "const u64 iy = tuple_to_index(t.data(), xshape, dim);\n      std::memcpy(ys + iy * es, xs + k * es, es);",
     [lambda o: pins.test_embed_crop_against_numpy_slicing(o, "f64", ((2, 3), (4, 5)))]),
    ("product adds instead of multiplying", "yy[iy] = yy[iy] * static_cast<const double*>(x)[ix];",
     "yy[iy] = yy[iy] + static_cast<const double*>(x)[ix];",
     [lambda o: pins.test_product_float_against_numpy(o, "f64", ((3, 4), (5, 2)))]),
    ("product misses the last slab of every axis",
     "I[i] = xshape[i] < yshape[i] ? xshape[i] : yshape[i];",
     "I[i] = (xshape[i] < yshape[i] ? xshape[i] : yshape[i]) - ((xshape[i] < yshape[i] ? xshape[i] : yshape[i]) > 1);",
     [lambda o: pins.test_product_properties_and_window(o)]),
    ("moment uses transposed axes", "acc[i].add(v * double(t[i]));", "acc[i].add(v * double(t[dim - 1 - i]));",
     [lambda o: pins.test_moment_point_mass_is_the_tuple(o, (3, 4))]),
    ("moment drops the mass term", "acc[dim].add(v);", "acc[dim].add(0.0);",
     [lambda o: pins.test_moment_constant_closed_form(o, (3, 4))]),
    ("product moment addresses every tensor with the first shape",
     "tuple_to_index(t.data(), shapes + k * dim, dim)", "tuple_to_index(t.data(), shapes, dim)",
     [lambda o: pins.test_moment_product_brute_force_f64(o, 0)]),
    ("view bias computed with x's shape", "const u64 bias = tuple_to_index(ystart, yshape, dim);",
     "const u64 bias = tuple_to_index(ystart, xshape, dim);",
     [lambda o: pins.test_views_against_numpy_slicing(o, "f64", 1)]),
    ("benchmark 3 reads z with y's shape",
     "const u64 iy = tuple_to_index(t.data(), yshape, dim), iz = tuple_to_index(t.data(), zshape, dim);",
     "const u64 iy = tuple_to_index(t.data(), yshape, dim), iz = tuple_to_index(t.data(), yshape, dim);",
     [lambda o: pins.test_apply_xpyxmz_against_numpy(o, "f64", 0)]),
    ("bounding box tests only the first factor",
     "for (unsigned k = 0; k < n && nonzero; ++k)", "for (unsigned k = 0; k < 1 && nonzero; ++k)",
     [lambda o: pins.test_nonzero_bbox_closed_forms(o)]),
    ("bounding box keeps the first tuple as the upper end",
     "if (found == 0 || v > out[2 * i + 1]) out[2 * i + 1] = v;", "if (found == 0) out[2 * i + 1] = v;",
     [lambda o: pins.test_nonzero_bbox_closed_forms(o)]),
    ("product window reads x with y's bias",
     "multiply_into(y, ybias + tuple_to_index(t.data(), yshape, dim), x,\n                  xbias + tuple_to_index",
     "multiply_into(y, ybias + tuple_to_index(t.data(), yshape, dim), x,\n                  ybias + tuple_to_index",
     [lambda o: pins.test_windows_both_sides_against_numpy_slicing(o, "f64", 1)]),
    ("bf16 product rounds with f16 parameters",
     "yy[iy] = uint16_t(round_to_format(exact, 8, -126, 127, 8));",
     "yy[iy] = uint16_t(round_to_format(exact, 11, -14, 15, 5));",
     [lambda o: pins.test_product_bf16_against_torch_and_tiny_values(o)]),
]


@pytest.mark.parametrize("mut", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, mut):
    desc, old, new, checks = mut
    src = open(SRC).read()
    assert src.count(old) >= 1, desc
    path = tmp_path / "mutant.cpp"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                    str(path), "-o", str(lib)], check=True)
    saved = orc_mod._lib
    orc_mod._lib = orc_mod.load(str(lib))
    try:
        caught = 0
        for chk in checks:
            try:
                chk(orc_mod)
            except AssertionError:
                caught += 1
        assert caught == len(checks), f"planted mistake not caught: {desc}"
    finally:
        orc_mod._lib = saved
