"""Benchmark: CSR nonzeros assembled per second by weighted-quadrature (WQ)
row-wise assembly on one GB300, next to Gauss (GQ) element-wise assembly on
the same GPU and the CPU oracle.

Workload (default): Poisson stiffness on a planar unstructured-spline domain
-- a 8 x 5 coarse quad core with 12 EPs of valence 3/5/6 (random interior
edge rotations), refined 4 times (10,240 elements) and wrapped in one passive
ring; kappa log-normal (sigma 0.5) on a 16 x 16 Fourier field.  All inputs are
seeded and synthetic.

One step = one assembly of the stiffness matrix for one coefficient field
(coefficients resident in HBM, weights and point tables precomputed -- the
paper's timing protocol, which excludes weight computation and basis
evaluation).  The rule build (point counts, placement, basis tables, Gauss
moments, truncated-SVD weights) runs once per mesh and is timed and reported
under "setup".  L2 is flushed (256 MB write) before every timed step; the
step's device time is taken with CUDA events on the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

# the oracle legs are timed single-threaded (reported as cores = 1)
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CSR nonzeros assembled/s (WQ, GPU) vs plain GQ on same GB300 at rel err ≤1e-6"
UNIT = "nnz/s"
WORKLOAD = "poisson_stiffness_rotated8x5_ep12_L4"


def make_mesh(seed=2001, levels=4):
    from wq_synth import meshes
    return meshes.rotated(nx=8, ny=5, n_ep=12, levels=levels, seed=seed)


def kappa_field(mesh, seed=2101):
    from wq_synth import meshes
    lo = mesh["xyz"].min(axis=0)
    hi = mesh["xyz"].max(axis=0)
    return meshes.LogNormalField(seed, lo, hi, nk=16, sigma=0.5)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join("/tmp", "wq_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def time_steps(fn, steps, warmup, flush):
    """Device time of `steps` calls of fn, each after an L2 flush; returns (ms list)."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in evs:
        flush()
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def aggregate(nnz, t_total, world, device):
    """Whole-job totals over ranks: nonzeros summed, timed region max over ranks
    (each rank assembles its own independent instance; no data-path collective)."""
    if world <= 1:
        return float(nnz), float(t_total)
    import torch
    import torch.distributed as dist
    v = torch.tensor([float(nnz)], dtype=torch.float64, device=device)
    dist.all_reduce(v)
    tt = torch.tensor([float(t_total)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(v.item()), float(tt.item())


def bench_ours(args, rank, world):
    import torch
    from paper_2605_29334_gb300 import wq
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    mesh = make_mesh(seed=2001 + rank)
    ctx = wq.Context(dev)
    basis = wq.Basis(ctx, mesh)
    host_ms = (time.perf_counter() - t0) * 1e3
    t1 = time.perf_counter()
    rule = wq.Rule(basis, comps=[wq.COMP_X, wq.COMP_Y])
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t1) * 1e3
    kap = kappa_field(mesh)
    xq = rule.points().cpu().numpy()
    xg = rule.gauss_points().cpu().numpy()
    coef = torch.tensor(kap(xq), device="cuda")
    coef_g = torch.tensor(kap(xg), device="cuda")
    nnz = rule.nnz
    flushbuf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush = lambda: flushbuf.fill_(1.0)
    out64 = torch.empty(nnz, dtype=torch.float64, device="cuda")
    out32 = torch.empty(nnz, dtype=torch.float32, device="cuda")
    outg = torch.empty(nnz, dtype=torch.float64, device="cuda")
    # accuracy of the FP32 paths against the FP64 path (same weights), per mode
    rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F64, out=out64)
    torch.cuda.synchronize()
    a64 = out64.cpu().numpy()
    rel = {}
    for name, pm in (("f32", wq.PREC_F32), ("f32_fast", wq.PREC_F32_FAST)):
        rule.assemble(wq.OP_STIFF, coef, prec=pm, out=out32)
        torch.cuda.synchronize()
        rel[name] = float(np.max(np.abs(out32.cpu().numpy().astype(np.float64) - a64)) / np.max(np.abs(a64)))
    modes = {"f64": wq.PREC_F64, "f32": wq.PREC_F32, "f32_fast": wq.PREC_F32_FAST}
    if args.prec == "auto":
        choice = "f32_fast" if rel["f32_fast"] <= 1e-6 else ("f32" if rel["f32"] <= 1e-6 else "f64")
    else:
        choice = args.prec
    prec = modes[choice]
    out = out64 if prec == wq.PREC_F64 else out32
    step = lambda: rule.assemble(wq.OP_STIFF, coef, prec=prec, out=out)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(dev)
    clk.start()
    ms = time_steps(step, args.steps, args.warmup, flush)
    clocks = clk.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_total = float(np.sum(ms)) / 1e3
    # comparators on the same GPU and protocol
    ms64 = time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F64, out=out64),
                      max(args.steps // 4, 10), args.warmup, flush)
    ms32 = {}
    for name in ("f32", "f32_fast"):
        pm = modes[name]
        ms32[name] = float(np.mean(time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=pm, out=out32),
                                              max(args.steps // 4, 10), args.warmup, flush)))
    msg = time_steps(lambda: rule.gq_assemble(wq.OP_STIFF, coef_g, out=outg), max(args.steps // 4, 10),
                     args.warmup, flush)
    # end to end through the C ABI with pinned host buffers
    h_coef = torch.tensor(kap(xq)).pin_memory()
    h_vals = torch.empty(nnz, dtype=torch.float64 if prec == wq.PREC_F64 else torch.float32).pin_memory()
    hc, hv = h_coef.numpy(), h_vals.numpy()
    for _ in range(args.warmup):
        rule.assemble_host(wq.OP_STIFF, hc, prec=prec, out=hv)
    n_e2e = max(args.steps // 4, 10)
    te = time.perf_counter()
    for _ in range(n_e2e):
        rule.assemble_host(wq.OP_STIFF, hc, prec=prec, out=hv)
    e2e_s = (time.perf_counter() - te) / n_e2e
    stats = {"nnz": nnz, "t": t_total, "t64": float(np.mean(ms64)) / 1e3, "tg": float(np.mean(msg)) / 1e3}
    tot_nnz, t_max = aggregate(nnz, t_total, world, "cuda")
    if rank != 0:
        return None
    value = tot_nnz * args.steps / t_max
    mean_s = t_total / args.steps
    ab = algorithmic_bytes_f(rule, basis, prec)
    gpu_launches = args.steps * (1 if prec == wq.PREC_F64 else 2)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    achieved = ab / mean_s / 1e9
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == wq.PREC_F64 else "f32", "precision_mode": choice, "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_functions": basis.n, "n_elements": basis.E, "nnz": nnz,
                   "n_points": rule.Q, "n_gauss": rule.G, "op": "stiffness", "l2": "flushed (256 MB write) before "
                   "every timed step; timed = the assembly kernel only", "parallelism": "independent instance per GPU"},
        "rel_err_vs_f64": rel,
        "gpu_launches": gpu_launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": None, "kernel": "k_rowasm_f64" if prec == wq.PREC_F64 else "k_chunk_f32",
                     "algorithmic_bytes": ab},
        "comparators": {
            "wq_f64_nnz_per_s": nnz / stats["t64"], "gq_f64_nnz_per_s": nnz / stats["tg"],
            "wq_f32_nnz_per_s": nnz / (ms32["f32"] / 1e3), "wq_f32_fast_nnz_per_s": nnz / (ms32["f32_fast"] / 1e3),
            "wq_f32_ms": ms32["f32"], "wq_f32_fast_ms": ms32["f32_fast"],
            "wq_f64_ms": stats["t64"] * 1e3, "gq_f64_ms": stats["tg"] * 1e3,
            "speedup_wq_over_gq_f64": stats["tg"] / stats["t64"]},
        "setup": {"host_basis_ms": host_ms, "rule_build_wall_ms": build_ms, "rule_build_device_ms": rule.info.setup_ms,
                  "n_truncated_x": rule.info.n_truncated[1], "n_z_identity_x": rule.info.n_z_identity[1]},
        "e2e": {"value": nnz / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(rule.Q * 8),
                "d2h_bytes_per_step": int(nnz * (8 if prec == wq.PREC_F64 else 4))},
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args)
    return res


def algorithmic_bytes_f(rule, basis, prec):
    """Algorithmic bytes of one stiffness assembly launch (2 weight/table components)."""
    E = basis.E
    side = basis.point_counts().astype(np.int64)
    m = np.array([basis.element(e)["fns"].size for e in range(E)], dtype=np.int64)
    P = side * side
    vb = 8  # FP64 value, or an FP32 (hi, lo) pair
    weights = rule.info.sum_r * 2 * vb
    tables = int(np.sum(P * m)) * 2 * vb
    coef = rule.Q * 8
    pos = int(np.sum(m * m)) * 2
    supp = int(np.sum(m)) * 4
    rows = (basis.n + 1) * (4 + 8 + 8)
    out = rule.nnz * (8 if prec == 0 else 4)
    return int(weights + tables + coef + pos + supp + rows + out)


def cpu_baseline(args, seconds=12.0):
    """The oracle's row-wise assembly, timed on the host on a bounded sample:
    the same coarse mesh refined twice (640 elements) instead of four times."""
    from oracle.basis import Basis
    from oracle import wq as owq
    mesh = make_mesh(levels=2)
    B = Basis(mesh)
    R = owq.Rule(B, ["x", "y"])
    R.compute_weights()
    kap = kappa_field(mesh)(R.x)
    nnz = len(R.col)
    t = time.perf_counter()
    reps = 0
    while True:
        R.assemble([("x", kap), ("y", kap)])
        reps += 1
        el = time.perf_counter() - t
        if el > seconds or reps >= 50:
            break
    return {"value": nnz * reps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "oracle row-wise assembly (NumPy, FP64) of the same workload family at refinement "
                      "level 2 (%d elements, %d nnz), %d passes in %.1f s" % (B.E, nnz, reps, el)}


def bench_reference(args, rank, world):
    """The oracle as it stands on the host cores, K timed steps of a bounded sample."""
    if rank != 0:
        return None
    from oracle.basis import Basis
    from oracle import wq as owq
    mesh = make_mesh(levels=2)
    B = Basis(mesh)
    R = owq.Rule(B, ["x", "y"])
    R.compute_weights()
    kap = kappa_field(mesh)(R.x)
    nnz = len(R.col)
    for _ in range(args.warmup):
        R.assemble([("x", kap), ("y", kap)])
    t = time.perf_counter()
    for _ in range(args.steps):
        R.assemble([("x", kap), ("y", kap)])
    el = time.perf_counter() - t
    v = nnz * args.steps / el
    sample = "oracle row-wise assembly of the workload family at refinement level 2 (%d elements, %d nnz)" % (B.E, nnz)
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "f32", "f32_fast", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        res = bench_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
        res = bench_ours(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if res is not None:
        print(json.dumps(res))


if __name__ == "__main__":
    main()
