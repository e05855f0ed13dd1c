"""Host-side arithmetic of bench.py, on CPU: the algorithmic bytes behind every GB/s figure
(embed b(|x|+|y|), product 3b|I|, moment b|p| for the f64 d=8 step, written out from the
workload's shapes), the op entry arithmetic, and the rule that the recorded ncu traffic is
reported only while the hashed kernel sources are unchanged."""
import hashlib
import json
import os

import pytest

import bench
from paper_1608_00099_gb300 import synth


def test_step_bytes_f64_d8():
    cfg = synth.config_f64_d8()
    b = bench.step_bytes(cfg)
    nx = 9 ** 8                       # x 9^8
    ny = (11 * 10) ** 4               # y (11,10)x4
    ni = (9 * 8) ** 4                 # intersection of 9^8 and (12,8)x4
    assert b == {"embed": 8 * (nx + ny), "product": 3 * 8 * ni, "moment": 8 * nx}
    assert sum(b.values()) == 2_505_000_080  # the 2505.0 MB quoted for the step


def test_op_entry_arithmetic():
    e = bench.op_entry(1_000_000_000, 0.5, 5000.0, elems=250_000_000)
    assert e["gbs"] == pytest.approx(2000.0)
    assert e["us"] == pytest.approx(500.0)
    assert e["frac_measured"] == pytest.approx(0.4)
    assert e["frac_8tbs"] == pytest.approx(2000.0 / bench.NOMINAL_HBM_GBS)
    assert e["elem_per_s"] == pytest.approx(5e11)


def test_ncu_traffic_only_for_unchanged_sources(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_bytes(b"// a kernel\n")
    (tmp_path / "profiles").mkdir()
    rec = {"dram_bytes_per_launch": 123, "sources": ["kernel.cu"],
           "sources_sha256": hashlib.sha256(src.read_bytes()).hexdigest()}
    (tmp_path / "profiles" / "k.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("k") == 123
    src.write_bytes(b"// a changed kernel\n")
    assert bench.ncu_traffic("k") is None
    assert bench.ncu_traffic("absent") is None


def test_committed_embed_record():
    """The committed embed traffic record: close to the launch's algorithmic bytes (no
    re-reads), and reported by bench.py only while it hashes the files it names."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    rec = json.load(open(os.path.join(root, "profiles", "embed_f64_d8.json")))
    h = hashlib.sha256()
    for f in rec["sources"]:
        h.update(open(os.path.join(root, f), "rb").read())
    if h.hexdigest() != rec["sources_sha256"]:
        assert bench.ncu_traffic("embed_f64_d8") is None
        pytest.skip("the embed kernel changed since its ncu capture (bench.py reports null)")
    assert bench.ncu_traffic("embed_f64_d8") == rec["dram_bytes_per_launch"]
    algo = bench.step_bytes(synth.config_f64_d8())["embed"]
    assert 0.9 * algo <= rec["dram_bytes_per_launch"] <= 1.05 * algo


@pytest.mark.parametrize("dtype", ["bf16", "f16", "f32", "f64"])
def test_precision_errors_report(monkeypatch, dtype):
    """The precision workload's error report on CPU: outputs equal to the oracle's own give a
    bit-exact product and zero moment error; a planted product error shows up."""
    import numpy as np
    import torch
    from oracle import oracle as orc
    pc = synth.config_precision()
    I = tuple(min(a, b) for a, b in zip(pc.pshape, pc.qshape))

    def bits(a64):
        t = synth.to_storage(a64, dtype).contiguous()
        return t.view(torch.int16).numpy().view(np.uint16).reshape(-1) if dtype in ("bf16", "f16") \
            else t.numpy().reshape(-1)
    ph, qh = bits(pc.p64), bits(pc.q64)
    r = orc.product(qh, pc.qshape, orc.crop(ph, I, pc.pshape, dtype), I, dtype)
    m = orc.moment(r, I, dtype)
    rt = torch.from_numpy(r.view(np.int16).copy()).view({"bf16": torch.bfloat16, "f16": torch.float16}[dtype]) \
        if dtype in ("bf16", "f16") else torch.from_numpy(r.copy())
    monkeypatch.setattr(bench, "PRECISION_OUTPUTS", {dtype: (rt, m)})
    e = bench.precision_errors(synth)[dtype]
    assert e["product_bit_exact_vs_oracle"] and e["max_rel_err_moment"] == 0.0 and e["within_bounds"]
    assert e["max_rel_err_product"] <= bench.PRODUCT_BOUND[dtype]
    # a planted error: one result scaled by (1 + 4 bounds) is reported above the bound
    r2 = orc.to_f64(r, dtype)
    k = int(np.argmax(np.abs(r2)))
    r2[k] = r2[k] * (1 + 4 * bench.PRODUCT_BOUND[dtype]) if r2[k] >= 1e-4 else 0.5  # f16 results underflow
    bad = orc.from_f64(r2, dtype) if dtype in ("bf16", "f16") else r2.astype(r.dtype)
    rt2 = torch.from_numpy(bad.view(np.int16).copy()).view(rt.dtype) if dtype in ("bf16", "f16") \
        else torch.from_numpy(bad.copy())
    monkeypatch.setattr(bench, "PRECISION_OUTPUTS", {dtype: (rt2, m)})
    e = bench.precision_errors(synth)[dtype]
    assert not e["product_bit_exact_vs_oracle"] and not e["within_bounds"]
