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
