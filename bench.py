"""Benchmark of the TRIOT hot path on GB300: effective HBM GB/s per op and for a whole step.

A step is one pass of the path over the f64 d=8 workload: embed x (9^8, U(0,1)) into a
zero-padded y of shape (11,10)x4, y'[t] *= x[t] over the intersection with a U(0,1) y'
of shape (12,8)x4, and the tuple-weighted moment of p = x / sum(x) (with the mass).
`value` is the algorithmic bytes of those three ops divided by the device time of K
steps (inputs resident in HBM, every buffer larger than L2).  The JSON line also
carries per-op GB/s, the roofline of the dominant kernel (embed), an end-to-end figure
through the same C ABI with pinned host buffers copied in and out every step, SM clocks
sampled during the run, the CPU oracle timed on the host cores, and the batched
workload (4096 f32 pairs: one persistent graph launch vs per-pair plain launches).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

NOMINAL_HBM_GBS = 8000.0
TUNE_FILE = os.path.join(ROOT, "paper_1608_00099_gb300", "tune_gb300.json")
WORKLOAD = "f64_d8"
WORKLOAD_DESC = ("f64 d=8: embed x 9^8 U(0,1) -> (11,10)x4; product y*=x over (9,8)x4 into U(0,1) "
                 "(12,8)x4; moment of x/sum(x)")
METRIC = "effective HBM GB/s (frac of 8 TB/s) per op; batched vs plain launch elem/s"


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def step_bytes(cfg):
    nx = int(np.prod(cfg.xshape))
    ny = int(np.prod(cfg.embed_shape))
    I = int(np.prod([min(a, b) for a, b in zip(cfg.xshape, cfg.prod_shape)]))
    return {"embed": 8 * (nx + ny), "product": 3 * 8 * I, "moment": 8 * nx}


# ------------------------------------------------------------------ distributed plumbing

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    import torch
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend=backend)
    return rank, ws, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float, device=None) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        busy = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local, dist):
    import torch

    from paper_1608_00099_gb300 import build as tb
    from paper_1608_00099_gb300 import synth, triot

    tb.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = synth.config_f64_d8()
    xh = cfg.x_values()
    yph = cfg.yprod_values()
    ph = synth.normalise(xh)
    x = torch.from_numpy(xh.reshape(cfg.xshape)).to(dev)
    y1 = torch.empty(cfg.embed_shape, dtype=torch.float64, device=dev)
    y2 = torch.from_numpy(yph.reshape(cfg.prod_shape)).to(dev)
    p = torch.from_numpy(ph.reshape(cfg.xshape)).to(dev)
    out = torch.empty(len(cfg.xshape) + 1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    tuning = None
    if os.path.exists(TUNE_FILE) and not args.no_tune_file:
        triot.triot_tune_load(TUNE_FILE)
        tuning = {"loaded": os.path.relpath(TUNE_FILE, ROOT)}
    if args.autotune:
        tuning = {"autotuned": run_autotune(triot, cfg, x, y1, y2, p, dev, stream, args.autotune)}
    ws = torch.empty(triot.triot_moment_workspace_size(cfg.xshape, torch.float64) // 8 + 2,
                     dtype=torch.float64, device=dev)
    b = step_bytes(cfg)
    step_total = sum(b.values())

    def step():
        triot.triot_embed(x, y1, stream=stream)
        triot.triot_product(x, y2, stream=stream)
        triot.triot_moment(p, out=out, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # per-op events inside the timed region (recorded on the launching stream)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    # a short soak at the same work so the clock sampler sees the GPU under load
    t_soak = time.time()
    while time.time() - t_soak < args.soak:
        for _ in range(50):
            step()
        torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(args.steps):
        e = evs[k]
        e[0].record(stream)
        triot.triot_embed(x, y1, stream=stream)
        e[1].record(stream)
        triot.triot_product(x, y2, stream=stream)
        e[2].record(stream)
        triot.triot_moment(p, out=out, workspace=ws, stream=stream)
        e[3].record(stream)
    stop.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clocks = sampler.stop() if sampler else None
    ms = start.elapsed_time(stop)
    ms_max = max_over_ranks(dist, ms, dev)
    op_ms = {"embed": 0.0, "product": 0.0, "moment": 0.0}
    for e in evs:
        op_ms["embed"] += e[0].elapsed_time(e[1])
        op_ms["product"] += e[1].elapsed_time(e[2])
        op_ms["moment"] += e[2].elapsed_time(e[3])
    K = args.steps
    value = step_total * K * world / (ms_max * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    ops = {}
    for name, tot in op_ms.items():
        gbs = b[name] / (tot / K * 1e-3) / 1e9
        ops[name] = {"gbs": round(gbs, 1), "us": round(tot / K * 1e3, 2), "bytes": b[name],
                     "frac_8tbs": round(gbs / NOMINAL_HBM_GBS, 4), "frac_measured": round(gbs / peak, 4)}
    emb = ops["embed"]
    traffic = ncu_traffic("embed_f64_d8")
    roofline = {"bound": "hbm", "kernel": "rows_kernel<embed, f64, 7 outer axes>",
                "achieved": emb["gbs"], "peak": peak, "unit": "GB/s",
                "frac": round(emb["gbs"] / peak, 4), "peak_kind": peak_kind, "traffic": traffic}

    # end to end: pinned host buffers in, results out, every step through the same C ABI
    e2e = run_e2e(args, triot, cfg, xh, yph, ph, dev, stream, step_total)

    result = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_max / K, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (SplitMix64 seed 1002, U(0,1)); replicas only across GPUs",
        "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "bytes_per_step": step_total,
                   "frac_8tbs": round(value / world / NOMINAL_HBM_GBS, 4),
                   "l2": "every buffer is larger than L2 (smallest: x, 344 MB)",
                   "parallelism": f"replicas x{world}"},
        "ops": ops, "roofline": roofline, "e2e": e2e, "gpu_launches": 4 * K,
        "clocks": clocks,
    }
    result["tuning"] = tuning
    if not args.no_batch:
        result["batch"] = run_batch(args, triot, synth, dev, stream)
    if not args.no_extra:
        result["workloads"] = run_extra_workloads(args, triot, synth, dev, stream)
    if rank == 0 and world == 1 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(args, cfg, xh, yph, ph)
        if PRECISION_OUTPUTS and "workloads" in result:
            for name, e in precision_errors(synth).items():
                result["workloads"][f"precision_{name}"]["errors_vs_oracle"] = e
    return result


def ncu_traffic(name):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"{name}.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    h = hashlib.sha256()
    for f in rec.get("sources", []):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    if h.hexdigest() != rec.get("sources_sha256"):
        return None
    return rec.get("dram_bytes_per_launch")


def run_e2e(args, triot, cfg, xh, yph, ph, dev, stream, step_total):
    """Steps through the C ABI with every step's inputs copied in from pinned host memory and
    its results (y, y' and the moment) copied back.  Steps are pipelined over two sets of
    device buffers: the host-to-device copies of step k+1, the kernels of step k and the
    device-to-host copies of step k-1 run on three streams at once (the link is full duplex)."""
    import torch
    K = max(3, min(args.steps, args.e2e_steps))
    xp = torch.from_numpy(xh.reshape(cfg.xshape)).pin_memory()
    yp = torch.from_numpy(yph.reshape(cfg.prod_shape)).pin_memory()
    pp = torch.from_numpy(ph.reshape(cfg.xshape)).pin_memory()
    y1h = torch.empty(cfg.embed_shape, dtype=torch.float64).pin_memory()
    y2h = torch.empty(cfg.prod_shape, dtype=torch.float64).pin_memory()
    mh = torch.empty(len(cfg.xshape) + 1, dtype=torch.float64).pin_memory()
    sets = []
    for _ in range(2):
        sets.append({
            "x": torch.empty(cfg.xshape, dtype=torch.float64, device=dev),
            "y1": torch.empty(cfg.embed_shape, dtype=torch.float64, device=dev),
            "y2": torch.empty(cfg.prod_shape, dtype=torch.float64, device=dev),
            "p": torch.empty(cfg.xshape, dtype=torch.float64, device=dev),
            "out": torch.empty(len(cfg.xshape) + 1, dtype=torch.float64, device=dev),
            "ws": torch.empty(triot.triot_moment_workspace_size(cfg.xshape, torch.float64) // 8 + 2,
                              dtype=torch.float64, device=dev),
            "in": torch.cuda.Event(), "done": torch.cuda.Event(), "out_ev": torch.cuda.Event(),
            "used": False,
        })
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def step(k):
        b = sets[k % 2]
        with torch.cuda.stream(s_in):
            if b["used"]:
                s_in.wait_event(b["out_ev"])   # this set's previous results have left the device
            b["x"].copy_(xp, non_blocking=True)
            b["y2"].copy_(yp, non_blocking=True)
            b["p"].copy_(pp, non_blocking=True)
            b["in"].record(s_in)
        s_cmp.wait_event(b["in"])
        triot.triot_embed(b["x"], b["y1"], stream=s_cmp)
        triot.triot_product(b["x"], b["y2"], stream=s_cmp)
        triot.triot_moment(b["p"], out=b["out"], workspace=b["ws"], stream=s_cmp)
        b["done"].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(b["done"])
            y1h.copy_(b["y1"], non_blocking=True)
            y2h.copy_(b["y2"], non_blocking=True)
            mh.copy_(b["out"], non_blocking=True)
            b["out_ev"].record(s_out)
        b["used"] = True

    for k in range(2):
        step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        step(k)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h2d = 8 * (xp.numel() + yp.numel() + pp.numel())
    d2h = 8 * (y1h.numel() + y2h.numel() + mh.numel())
    return {"value": round(step_total * K / dt / 1e9, 1), "unit": "GB/s", "steps": K,
            "ms_per_step": round(dt / K * 1e3, 3), "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "pipelined": "copies in, kernels and copies out of consecutive steps overlap on three streams"}


def run_batch(args, triot, synth, dev, stream):
    """4096 f32 pairs: fused persistent graph launch, phased persistent, plain launches."""
    import torch
    pairs = synth.config_batch_shapes()
    xs_h = synth.batch_x_values(pairs)
    xs = [torch.from_numpy(v.astype(np.float32).reshape(pr.xshape)).to(dev) for pr, v in zip(pairs, xs_h)]
    ys = [torch.empty(pr.yshape, dtype=torch.float32, device=dev) for pr in pairs]
    outs = [torch.zeros(len(pr.xshape) + 1, dtype=torch.float64, device=dev) for pr in pairs]
    ny = sum(int(np.prod(pr.yshape)) for pr in pairs)
    nx = sum(int(np.prod(pr.xshape)) for pr in pairs)
    # launch geometry of each mode chosen by measurement (cached; the plans pick it up)
    tuned = {"fused": triot.triot_batch_autotune(xs, ys, outs, mode=triot.BATCH_FUSED, stream=stream),
             "phased": triot.triot_batch_autotune(xs, ys, outs, mode=triot.BATCH_PHASED, stream=stream)}
    fused = triot.BatchPlan(xs, ys, outs, mode=triot.BATCH_FUSED)
    phased = triot.BatchPlan(xs, ys, outs, mode=triot.BATCH_PHASED)

    def timed(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    res = {"workload": "4096 f32 pairs, rank U{2..10}, extents U{2..32}, |y| <= 2^22",
           "elements_y": ny, "elements_x": nx}
    ms_f = timed(lambda: fused.run(stream), args.batch_reps)
    ms_p = timed(lambda: phased.run(stream), args.batch_reps)
    ms_plain = timed(lambda: fused.run_plain(stream), max(2, args.batch_reps // 5))
    # the same plain launches captured in one CUDA graph (separates launch overhead)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        fused.run_plain(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=side):
            fused.run_plain(torch.cuda.current_stream())
    ms_pg = timed(lambda: g.replay(), max(2, args.batch_reps // 2))
    fused_bytes = 4 * (nx + ny)
    for name, ms in (("fused_graph", ms_f), ("phased_graph", ms_p), ("plain_launches", ms_plain),
                     ("plain_in_graph", ms_pg)):
        res[name] = {"ms": round(ms, 3), "elem_per_s": round(ny / (ms * 1e-3), 1),
                     "gbs_fused_bytes": round(fused_bytes / (ms * 1e-3) / 1e9, 1)}
    # kernels per run: fill, x-driven fused pass, combine / fill, embed, product, moment,
    # combine / per pair embed, product, moment, moment combine
    res["launches"] = {"fused_graph": 3, "phased_graph": 5, "plain_launches": 4 * len(pairs)}
    res["tuning"] = {"autotuned": tuned, "geometry_fused": fused.geometry(),
                     "geometry_phased": phased.geometry()}
    res["speedup_fused_vs_plain"] = round(ms_plain / ms_f, 2)
    fused.close()
    phased.close()
    return res


def time_op(fn, reps, stream):
    """Device time per call: the calls are captured once into a CUDA graph and the graph is
    replayed, so host launch overhead (ctypes, planning) is not in the measurement."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for k in range(2):
            fn(k, side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        for k in range(reps):
            fn(k, side)
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = 3
    a.record(stream)
    for _ in range(n):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / (n * reps)


def op_entry(nbytes, ms, peak, elems=None):
    gbs = nbytes / (ms * 1e-3) / 1e9
    d = {"us": round(ms * 1e3, 2), "bytes": int(nbytes), "gbs": round(gbs, 1),
         "frac_8tbs": round(gbs / NOMINAL_HBM_GBS, 4), "frac_measured": round(gbs / peak, 4)}
    if elems is not None:
        d["elem_per_s"] = round(elems / (ms * 1e-3), 1)
    return d


def run_extra_workloads(args, triot, synth, dev, stream):
    """Per-op figures on the other workloads (working sets under 4x L2 rotate copies)."""
    import torch
    peak, _ = measured_peak()
    l2 = torch.cuda.get_device_properties(dev).L2_cache_size
    res = {}
    # embed f64 d=6: 10 MB per call, rotated over enough copies to exceed 4x L2
    cfg = synth.config_embed_small()
    xh = cfg.x_values()
    per = 8 * (int(np.prod(cfg.xshape)) + int(np.prod(cfg.embed_shape)))
    ncopy = int(4 * l2 // per) + 1
    xs = [torch.from_numpy(xh.reshape(cfg.xshape)).to(dev) for _ in range(ncopy)]
    ys = [torch.empty(cfg.embed_shape, dtype=torch.float64, device=dev) for _ in range(ncopy)]
    ms = time_op(lambda k, st: triot.triot_embed(xs[k % ncopy], ys[k % ncopy], stream=st), 4 * ncopy, stream)
    res["embed_f64_d6"] = {"embed": op_entry(per, ms, peak, int(np.prod(cfg.embed_shape))), "copies_rotated": ncopy}
    x2 = [torch.empty_like(xs[0]) for _ in range(ncopy)]
    ms = time_op(lambda k, st: triot.triot_crop(x2[k % ncopy], ys[k % ncopy], stream=st), 4 * ncopy, stream)
    res["embed_f64_d6"]["crop"] = op_entry(2 * 8 * int(np.prod(cfg.xshape)), ms, peak)
    # single-launch latency: events around one plain call (host launch path included), median
    lat = []
    for k in range(21):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        triot.triot_embed(xs[k % ncopy], ys[k % ncopy], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1) * 1e3)
    res["embed_f64_d6"]["single_launch_us"] = round(sorted(lat)[len(lat) // 2], 2)
    del xs, ys, x2
    # f32 d=24: 44 GB embed target, product over the all-2 intersection, moment of x
    cfg = synth.config_f32_d24()
    ny = int(np.prod(cfg.embed_shape))
    free, _ = torch.cuda.mem_get_info(dev)
    xh = cfg.x_values().astype(np.float32)
    x = torch.from_numpy(xh.reshape(cfg.xshape)).to(dev)
    nx = xh.size
    r = {}
    if not args.no_big and free > 4 * ny + (8 << 30):
        y = torch.empty(ny, dtype=torch.float32, device=dev).view(cfg.embed_shape)
        ms = time_op(lambda k, st: triot.triot_embed(x, y, stream=st), 5, stream)
        r["embed"] = op_entry(4 * (nx + ny), ms, peak, ny)
        ms = time_op(lambda k, st: triot.triot_product(x, y, stream=st), 20, stream)
        r["product"] = op_entry(3 * 4 * nx, ms, peak, nx)
        del y
        torch.cuda.empty_cache()
    if True:
        # x (67 MB) is smaller than L2: rotate copies so that the moment reads HBM
        ncopy = max(1, -(-4 * l2 // (4 * nx)))
        xr = [x] + [x.clone() for _ in range(ncopy - 1)]
        out = torch.empty(25, dtype=torch.float64, device=dev)
        ws = torch.empty(triot.triot_moment_workspace_size(cfg.xshape, torch.float32) // 8 + 2,
                         dtype=torch.float64, device=dev)
        ms = time_op(lambda k, st: triot.triot_moment(xr[k % ncopy], out=out, workspace=ws, stream=st),
                     4 * ncopy, stream)
        r["moment"] = op_entry(4 * nx, ms, peak, nx)
        r["moment_copies_rotated"] = ncopy
        res["f32_d24"] = r
        del x, xr
        torch.cuda.empty_cache()
    # precision workload: crop p to the intersection, r *= q, moment of r; bf16 / f16 / f64
    pc = synth.config_precision()
    I = tuple(min(a, b) for a, b in zip(pc.pshape, pc.qshape))
    nI = int(np.prod(I))
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16, "f32": torch.float32, "f64": torch.float64}
    for name, dt in tdt.items():
        es = {"f64": 8, "f32": 4}.get(name, 2)
        pt = synth.to_storage(pc.p64, name).reshape(pc.pshape)
        qt = synth.to_storage(pc.q64, name).reshape(pc.qshape)
        per = es * (pt.numel() + qt.numel() + nI)
        ncopy = int(4 * l2 // per) + 1
        P = [pt.to(dev) for _ in range(ncopy)]
        Q = [qt.to(dev) for _ in range(ncopy)]
        R = [torch.empty(I, dtype=dt, device=dev) for _ in range(ncopy)]
        out = torch.empty(len(I) + 1, dtype=torch.float64, device=dev)
        ws = torch.empty(triot.triot_moment_workspace_size(I, dt) // 8 + 2, dtype=torch.float64, device=dev)
        r = {"copies_rotated": ncopy, "intersection": list(I)}
        ms = time_op(lambda k, st: triot.triot_crop(R[k % ncopy], P[k % ncopy], stream=st), 3 * ncopy, stream)
        r["crop"] = op_entry(2 * es * nI, ms, peak, nI)
        ms = time_op(lambda k, st: triot.triot_product(Q[k % ncopy], R[k % ncopy], stream=st), 3 * ncopy, stream)
        r["product"] = op_entry(3 * es * nI, ms, peak, nI)
        ms = time_op(lambda k, st: triot.triot_moment(R[k % ncopy], out=out, workspace=ws, stream=st), 3 * ncopy, stream)
        r["moment"] = op_entry(es * nI, ms, peak, nI)
        # the same pipeline fused: the moment of p*q over I, without writing r
        wsp = torch.empty(triot.triot_moment_product_workspace_size([pc.pshape, pc.qshape], dt) // 8 + 2,
                          dtype=torch.float64, device=dev)
        ms = time_op(lambda k, st: triot.triot_moment_product([P[k % ncopy], Q[k % ncopy]], out=out,
                                                              workspace=wsp, stream=st), 3 * ncopy, stream)
        r["moment_product"] = op_entry(2 * es * nI, ms, peak, nI)
        # one untimed pass whose results the CPU leg checks against the oracle
        triot.triot_crop(R[0], P[0], stream=stream)
        triot.triot_product(Q[0], R[0], stream=stream)
        m0 = triot.triot_moment(R[0], stream=stream)
        torch.cuda.synchronize()
        PRECISION_OUTPUTS[name] = (R[0].cpu().contiguous(), m0.cpu().numpy().copy())
        res[f"precision_{name}"] = r
        del P, Q, R
    torch.cuda.empty_cache()
    # benchmark 4 of Section 3: naive convolution of two (2^8, 2^3) f64 matrices; |a| |b|
    # multiply-adds (compute-bound: reported in GFLOP/s against the nominal FP64 rate)
    ca, cb = (2 ** 8, 2 ** 3), (2 ** 8, 2 ** 3)
    A4 = torch.from_numpy(synth.normal01(1010, 2048).reshape(ca)).to(dev)
    B4 = torch.from_numpy(synth.normal01(1011, 2048).reshape(cb)).to(dev)
    O4 = torch.empty([x + y - 1 for x, y in zip(ca, cb)], dtype=torch.float64, device=dev)
    ms = time_op(lambda k, st: triot.triot_convolve(A4, B4, out=O4, stream=st), 50, stream)
    flops = 2.0 * 2048 * 2048
    res["convolve_benchmark4_f64"] = {"convolve": {"us": round(ms * 1e3, 2), "gflops": round(flops / (ms * 1e-3) / 1e9, 1),
                                                   "frac_nominal_fp64": round(flops / (ms * 1e-3) / 1.25e12, 4)}}
    del A4, B4, O4
    # benchmark 3 of Section 3 on the paper's shapes, f64: x <- x + y x - z over x's shape;
    # 4 * 8 * |x| bytes per call, copies rotated so the touched data exceeds 4x L2
    bx = (2 ** 7 + 1, 2 ** 5, 2 ** 3 + 5, 2 ** 4)
    by = (2 ** 8 - 3, 2 ** 6, 2 ** 6, 2 ** 4 + 7)
    bz = (2 ** 8, 2 ** 5 + 7, 2 ** 6, 2 ** 5 + 1)
    nbx = int(np.prod(bx))
    per = 4 * 8 * nbx
    ncopy = int(4 * l2 // per) + 1
    X0 = torch.from_numpy(synth.normal01(1007, nbx).reshape(bx)).to(dev)
    Y0 = torch.from_numpy(synth.normal01(1008, int(np.prod(by))).reshape(by)).to(dev)
    Z0 = torch.from_numpy(synth.normal01(1009, int(np.prod(bz))).reshape(bz)).to(dev)
    XS = [X0.clone() for _ in range(ncopy)]
    YS = [Y0.clone() for _ in range(ncopy)]
    ZS = [Z0.clone() for _ in range(ncopy)]
    ms = time_op(lambda k, st: triot.triot_apply_xpyxmz(XS[k % ncopy], YS[k % ncopy], ZS[k % ncopy], stream=st),
                 2 * ncopy, stream)
    res["apply_benchmark3_f64"] = {"apply_xpyxmz": op_entry(per, ms, peak, nbx), "copies_rotated": ncopy}
    del X0, Y0, Z0, XS, YS, ZS
    torch.cuda.empty_cache()
    # views (Section 4's biased slices): the FFT-style centre pad of x (8)^6 into y (16)^6 at
    # (4)^6 and the extraction back; y (134 MB) is larger than L2
    xs6, ys6, st6 = (8,) * 6, (16,) * 6, (4,) * 6
    xv = torch.from_numpy(synth.normal01(1006, 8 ** 6).reshape(xs6)).to(dev)
    yv = [torch.empty(ys6, dtype=torch.float64, device=dev) for _ in range(2)]
    ms = time_op(lambda k, st: triot.triot_embed_at(xv, yv[k % 2], st6, stream=st), 6, stream)
    r = {"embed_at": op_entry(8 * (8 ** 6 + 16 ** 6), ms, peak, 16 ** 6)}
    xb = [torch.empty(xs6, dtype=torch.float64, device=dev) for _ in range(2)]
    ms = time_op(lambda k, st: triot.triot_crop_at(xb[k % 2], yv[k % 2], st6, stream=st), 6, stream)
    r["crop_at"] = op_entry(2 * 8 * 8 ** 6, ms, peak, 8 ** 6)
    res["fft_pad_f64_d6"] = r
    del xv, yv, xb
    # two PMFs on one grid (Section 4's product over the intersecting support): x (16)^6 at
    # the origin, y (16)^6 at (4)^6, y *= x over the shared (12)^6; 3 * 8 * 12^6 bytes,
    # copies rotated so the touched data exceeds 4x L2
    pm = (16,) * 6
    ni = 12 ** 6
    ncopy = int(4 * l2 // (3 * 8 * ni)) + 1
    xp = [torch.from_numpy(synth.uniform01(1012, 16 ** 6).reshape(pm)).to(dev) for _ in range(ncopy)]
    yp = [torch.from_numpy(synth.uniform01(1013, 16 ** 6).reshape(pm)).to(dev) for _ in range(ncopy)]
    ms = time_op(lambda k, st: triot.triot_product_support(xp[k % ncopy], (0,) * 6, yp[k % ncopy], (4,) * 6,
                                                           stream=st), 2 * ncopy, stream)
    res["pmf_support_f64_d6"] = {"product_support": op_entry(3 * 8 * ni, ms, peak, ni), "copies_rotated": ncopy,
                                 "intersection": [12] * 6}
    del xp, yp
    torch.cuda.empty_cache()
    # moment of the product of the f64 d=8 pair (x 9^8, y (12,8)x4) over I = (9,8)x4, fused:
    # 2 * 8 * |I| bytes read, against 4 * 8 * |I| for the product followed by the moment
    c8 = synth.config_f64_d8()
    I8 = tuple(min(a, b) for a, b in zip(c8.xshape, c8.prod_shape))
    n8 = int(np.prod(I8))
    x8 = torch.from_numpy(c8.x_values().reshape(c8.xshape)).to(dev)
    y8 = torch.from_numpy(c8.yprod_values().reshape(c8.prod_shape)).to(dev)
    out8 = torch.empty(len(I8) + 1, dtype=torch.float64, device=dev)
    ws8 = torch.empty(triot.triot_moment_product_workspace_size([c8.xshape, c8.prod_shape], torch.float64) // 8 + 2,
                      dtype=torch.float64, device=dev)
    ms = time_op(lambda k, st: triot.triot_moment_product([x8, y8], out=out8, workspace=ws8, stream=st), 20, stream)
    res["moment_product_f64_d8"] = {"moment_product": op_entry(2 * 8 * n8, ms, peak, n8),
                                    "unfused_bytes": 4 * 8 * n8, "intersection": list(I8)}
    # nonzero bounding box of the same pair's product (Section 2), y 99.9 % zeros: both
    # factors are read at every tuple of I (x has no zeros), 2 * 8 * |I| bytes
    yh = c8.yprod_values()
    yh[synth.uniform01(4242, yh.size) < 0.999] = 0.0
    ys8 = torch.from_numpy(yh.reshape(c8.prod_shape)).to(dev)
    bo = torch.empty(2 * len(I8) + 1, dtype=torch.int64, device=dev)
    bws = torch.empty(triot.triot_nonzero_bbox_workspace_size([c8.xshape, c8.prod_shape], torch.float64) // 8 + 2,
                      dtype=torch.int64, device=dev)
    ms = time_op(lambda k, st: triot.triot_nonzero_bbox([x8, ys8], out=bo, workspace=bws, stream=st), 20, stream)
    res["bbox_f64_d8"] = {"nonzero_bbox": op_entry(2 * 8 * n8, ms, peak, n8), "y_nonzero_fraction": 0.001}
    del x8, y8, ys8
    torch.cuda.empty_cache()
    return res


def run_autotune(triot, cfg, x, y1, y2, p, dev, stream, path):
    import torch
    ws = torch.empty(triot.MOMENT_MAX_WORKSPACE_PER_RANK * (len(cfg.xshape) + 1) // 8, dtype=torch.float64,
                     device=dev)
    t = {"embed": triot.triot_autotune(triot.OP_EMBED, x, y1, stream=stream),
         "product": triot.triot_autotune(triot.OP_PRODUCT, x, y2, stream=stream),
         "moment": triot.triot_autotune(triot.OP_MOMENT, p, None, workspace=ws, stream=stream)}
    if path:
        triot.triot_tune_save(path)
    return t


# ------------------------------------------------------------------ the oracle on the host

def oracle_step(cfg, xh, yph, ph, nt, slabs=None):
    from oracle import oracle as orc
    xs, es, ps = cfg.xshape, cfg.embed_shape, cfg.prod_shape
    x, yp, p = xh, yph, ph
    if slabs is not None:   # a bounded sample: the leading `slabs` slabs of the outermost axis
        xs = (slabs,) + tuple(xs[1:])
        es = (slabs,) + tuple(es[1:])
        ps = (slabs,) + tuple(ps[1:])
        x = xh[:int(np.prod(xs))]
        yp = yph[:int(np.prod(ps))]
        p = ph[:int(np.prod(xs))]
    t0 = time.perf_counter()
    orc.embed(x, xs, es, "f64", nthreads=nt)
    orc.product(x, xs, yp, ps, "f64", nthreads=nt)
    orc.moment(p, xs, "f64", nthreads=nt)
    dt = time.perf_counter() - t0
    nI = int(np.prod([min(a, b) for a, b in zip(xs, ps)]))
    nbytes = 8 * (int(np.prod(xs)) + int(np.prod(es))) + 24 * nI + 8 * int(np.prod(xs))
    return nbytes, dt


# outputs of the precision workload's GPU pass (dtype -> (r, moments)), checked by the CPU leg
PRECISION_OUTPUTS = {}
# error bounds the precision workload is held to: the product relative to the exact product
# of the rounded inputs (where that is a normal number of the format; half a subnormal step
# elsewhere), the moment relative to sum |r| t_i against the FP64 oracle
PRODUCT_BOUND = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11, "f32": 2.0 ** -24, "f64": 2.0 ** -53}
MOMENT_BOUND = {"bf16": 1e-5, "f16": 1e-5, "f32": 1e-5, "f64": 1e-12}
NONNORMAL_BOUND = {"bf16": 2.0 ** -134, "f16": 2.0 ** -25, "f32": 2.0 ** -150, "f64": 2.0 ** -1075}


def precision_errors(synth):
    """Per-result errors of the precision workload (d = 10, extents 3..7) against the oracle:
    the product r = crop(p) * q element by element, and the moment of r per component."""
    from oracle import oracle as orc
    pc = synth.config_precision()
    I = tuple(min(a, b) for a, b in zip(pc.pshape, pc.qshape))
    tiny = {"bf16": 2.0 ** -126, "f16": 2.0 ** -14, "f32": 2.0 ** -126, "f64": 2.0 ** -1022}
    out = {}
    for name, (rt, mg) in PRECISION_OUTPUTS.items():
        # the very inputs the GPU pass used (rounded by synth.to_storage)
        def bits(a64):
            t = synth.to_storage(a64, name).contiguous()
            return t.view(torch_int16()).numpy().view(np.uint16).reshape(-1) if name in ("bf16", "f16") \
                else t.numpy().reshape(-1)
        ph, qh = bits(pc.p64), bits(pc.q64)
        rp = orc.crop(ph, I, pc.pshape, name)
        rq = orc.crop(qh, I, pc.qshape, name)
        ref = orc.product(qh, pc.qshape, rp, I, name)
        got = rt.view(torch_int16()).numpy().view(np.uint16).reshape(-1) if name in ("bf16", "f16") \
            else rt.numpy().reshape(-1)
        exact = orc.to_f64(rp, name) * orc.to_f64(rq, name)
        g64 = orc.to_f64(got, name)
        normal = np.abs(exact) >= tiny[name]
        rel = np.abs(g64[normal] - exact[normal]) / np.abs(exact[normal]) if normal.any() else np.zeros(1)
        absn = np.abs(g64[~normal] - exact[~normal]) if (~normal).any() else np.zeros(1)
        mref = orc.moment(ref, I, name)
        scale = np.abs(orc.moment(np.abs(orc.to_f64(ref, name)), I, "f64"))
        merr = np.abs(mg - mref) / np.maximum(scale, 1e-300)
        out[name] = {"product_bit_exact_vs_oracle": bool(got.tobytes() == ref.tobytes()),
                     "max_rel_err_product": float(rel.max()), "product_normal_results": int(normal.sum()),
                     "max_abs_err_product_nonnormal": float(absn.max()),
                     "product_bound_rel": PRODUCT_BOUND[name], "product_bound_abs_nonnormal": NONNORMAL_BOUND[name],
                     "max_rel_err_moment": float(merr.max()), "moment_bound_rel": MOMENT_BOUND[name],
                     "within_bounds": bool(rel.max() <= PRODUCT_BOUND[name] and absn.max() <= NONNORMAL_BOUND[name]
                                           and merr.max() <= MOMENT_BOUND[name])}
    return out


def torch_int16():
    import torch
    return torch.int16


def cpu_baseline(args, cfg, xh, yph, ph):
    nt = os.cpu_count() or 1
    total_b, total_t, n = 0, 0.0, 0
    while total_t < args.cpu_seconds or n == 0:
        b, t = oracle_step(cfg, xh, yph, ph, nt, slabs=3)
        total_b += b
        total_t += t
        n += 1
    return {"value": round(total_b / total_t / 1e9, 3), "unit": "GB/s", "cores": nt, "kind": "oracle",
            "sample": f"{n} oracle steps on the leading 3 of 9 outer slabs of the f64 d=8 workload "
                      f"(embed+product+moment, outer-axis std::thread split), {total_t:.1f} s"}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, on this machine's host cores."""
    if rank != 0:
        return None
    from paper_1608_00099_gb300 import synth
    from oracle import build as ob
    ob.build()
    cfg = synth.config_f64_d8()
    xh = cfg.x_values()
    yph = cfg.yprod_values()
    ph = synth.normalise(xh)
    nt = os.cpu_count() or 1
    slabs = 1   # one of the 9 outer slabs per step keeps K steps within minutes
    for _ in range(args.warmup):
        oracle_step(cfg, xh, yph, ph, nt, slabs=slabs)
    tb, tt = 0, 0.0
    for _ in range(args.steps):
        b, t = oracle_step(cfg, xh, yph, ph, nt, slabs=slabs)
        tb += b
        tt += t
    value = tb / tt / 1e9
    sample = f"leading {slabs} of 9 outer slabs of the f64 d=8 workload per step (embed+product+moment)"
    return {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(tt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (SplitMix64 seed 1002, U(0,1))",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": nt, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_op(args):
    """A few calls of one op on its workload, for an ncu capture (no JSON line)."""
    import torch
    from paper_1608_00099_gb300 import build as tb
    from paper_1608_00099_gb300 import synth, triot
    tb.build()
    dev = torch.device("cuda", 0)
    n = max(1, args.steps)
    if args.profile_op == "moment_product_f64_d8":
        c8 = synth.config_f64_d8()
        x8 = torch.from_numpy(c8.x_values().reshape(c8.xshape)).to(dev)
        y8 = torch.from_numpy(c8.yprod_values().reshape(c8.prod_shape)).to(dev)
        out = torch.empty(len(c8.xshape) + 1, dtype=torch.float64, device=dev)
        ws = torch.empty(triot.triot_moment_product_workspace_size([c8.xshape, c8.prod_shape], torch.float64) // 8
                         + 2, dtype=torch.float64, device=dev)
        for _ in range(n):
            triot.triot_moment_product([x8, y8], out=out, workspace=ws)
    elif args.profile_op == "moment_product_bf16_d10":
        # the precision workload's fused crop -> product -> moment: p (pshape) and q (qshape)
        # in bf16, the moment of p * q over their intersection (rows of 3 elements)
        pc = synth.config_precision()
        P = synth.to_storage(pc.p64, "bf16").reshape(pc.pshape).to(dev)
        Q = synth.to_storage(pc.q64, "bf16").reshape(pc.qshape).to(dev)
        out = torch.empty(len(pc.pshape) + 1, dtype=torch.float64, device=dev)
        ws = torch.empty(triot.triot_moment_product_workspace_size([pc.pshape, pc.qshape], torch.bfloat16) // 8
                         + 2, dtype=torch.float64, device=dev)
        for _ in range(n):
            triot.triot_moment_product([P, Q], out=out, workspace=ws)
    elif args.profile_op == "bbox_f64_d8":
        # the bounding box workload: x 9^8 and y (12,8)x4 with 99.9 % zeros, over (9,8)x4
        c8 = synth.config_f64_d8()
        yh = c8.yprod_values()
        yh[synth.uniform01(4242, yh.size) < 0.999] = 0.0
        x8 = torch.from_numpy(c8.x_values().reshape(c8.xshape)).to(dev)
        y8 = torch.from_numpy(yh.reshape(c8.prod_shape)).to(dev)
        out = torch.empty(2 * len(c8.xshape) + 1, dtype=torch.int64, device=dev)
        ws = torch.empty(triot.triot_nonzero_bbox_workspace_size([c8.xshape, c8.prod_shape], torch.float64) // 8
                         + 2, dtype=torch.int64, device=dev)
        for _ in range(n):
            triot.triot_nonzero_bbox([x8, y8], out=out, workspace=ws)
    else:
        if args.profile_op == "moment_f64_d8":
            # the f64 d=8 step's moment: p = x / sum(x), x of shape 9^8, U(0,1)
            c8 = synth.config_f64_d8()
            p = torch.from_numpy(synth.normalise(c8.x_values()).reshape(c8.xshape)).to(dev)
        elif args.profile_op == "moment_f32_d24":
            # the f32 d=24 workload's moment: x of shape (2,)*24, U(0,1)
            c = synth.config_f32_d24()
            p = torch.from_numpy(c.x_values().astype(np.float32).reshape(c.xshape)).to(dev)
        else:
            # bf16 blocks of 16 under three axes of 200 (the chunked float block kernel)
            shape = (200, 200, 200, 16)
            v = synth.uniform01(1010, int(np.prod(shape))).astype(np.float32)
            p = torch.from_numpy(v.reshape(shape)).to(dev).to(torch.bfloat16)
        out = torch.empty(p.dim() + 1, dtype=torch.float64, device=dev)
        ws = torch.empty(triot.triot_moment_workspace_size(tuple(p.shape), p.dtype) // 8 + 2,
                         dtype=torch.float64, device=dev)
        for _ in range(n):
            triot.triot_moment(p, out=out, workspace=ws)
    torch.cuda.synchronize()
    print(f"{args.profile_op}: {n} calls done", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--soak", type=float, default=1.5, help="seconds of untimed load for the clock sampler")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--batch-reps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads' per-op figures")
    ap.add_argument("--no-big", action="store_true", help="skip the 44 GB f32 d=24 workload")
    ap.add_argument("--autotune", default="", help="autotune the three ops and save the cache here")
    ap.add_argument("--no-tune-file", action="store_true", help="ignore the committed tuning file")
    ap.add_argument("--profile-op", default="",
                    choices=["", "moment_product_f64_d8", "moment_f64_d8", "moment_f32_d24", "moment_bf16_blocks16",
                             "bbox_f64_d8", "moment_product_bf16_d10"],
                    help="only run one op a few times (the command the ncu summaries capture)")
    args = ap.parse_args()
    if args.profile_op:
        return profile_op(args)
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local, dist = dist_setup()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local, dist)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
