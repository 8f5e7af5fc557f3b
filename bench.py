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
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # nvidia-smi takes a moment to start: wait (at most 3 s) for its first sample so
        # that the samples cover the timed region that follows
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.p.poll() is None:
            self.f.flush()
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

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


def rel_errors(a, ref):
    """Normwise errors of a matrix's CSR values against a reference: max|a - ref| / max|ref|
    and ||a - ref||_F / ||ref||_F (entry-wise relative errors mean little where stiffness
    rows sum to zero)."""
    d = np.asarray(a, dtype=np.float64) - ref
    return float(np.max(np.abs(d)) / np.max(np.abs(ref))), float(np.linalg.norm(d) / np.linalg.norm(ref))


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
    modes = {"f64": wq.PREC_F64, "f32": wq.PREC_F32, "f32_fast": wq.PREC_F32_FAST, "tc": wq.PREC_TC}
    # the library's autotuner: each float mode's error against FP64 on this workload, and
    # the fastest mode within the 1e-6 bar (else FP64)
    tune = rule.autotune(wq.OP_STIFF, coef, tol=1e-6, reps=50)
    rel = dict(zip(("tc", "f32", "f32_fast"), tune["err"]))
    if args.prec == "auto":
        choice = {wq.PREC_TC: "tc", wq.PREC_F32: "f32", wq.PREC_F32_FAST: "f32_fast"}.get(tune["chosen"], "f64")
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
    # per-kernel durations: the same K steps again, with the library recording CUDA
    # events around each of its kernels (kept out of the headline region: the extra
    # event records cost a few microseconds per step)
    rule.set_timing(args.steps)
    ms_inst = time_steps(step, args.steps, 0, flush)
    kt = rule.kernel_times(args.steps)
    rule.set_timing(0)
    clocks = clk.stop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t_total = float(np.sum(ms)) / 1e3
    # comparators on the same GPU and protocol
    nc = max(args.steps // 4, 10)
    comp_ms = {
        "wq_f64": time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F64, out=out64), nc,
                             args.warmup, flush),
        "wq_f32": time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F32, out=out32), nc,
                             args.warmup, flush),
        "wq_f32_fast": time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F32_FAST, out=out32), nc,
                                  args.warmup, flush),
        "gq_f64": time_steps(lambda: rule.gq_assemble(wq.OP_STIFF, coef_g, prec=wq.PREC_F64, out=outg), nc,
                             args.warmup, flush),
        "gq_f32": time_steps(lambda: rule.gq_assemble(wq.OP_STIFF, coef_g, prec=wq.PREC_F32, out=out32), nc,
                             args.warmup, flush),
        "wq_tc": time_steps(lambda: rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_TC, out=out32), nc,
                            args.warmup, flush),
        "gq_tc": time_steps(lambda: rule.gq_assemble(wq.OP_STIFF, coef_g, prec=wq.PREC_TC, out=out32), nc,
                            args.warmup, flush),
    }
    comp_ms = {k: float(np.mean(v)) for k, v in comp_ms.items()}
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
    tot_nnz, t_max = aggregate(nnz, t_total, world, "cuda")
    if rank != 0:
        return None
    value = tot_nnz * args.steps / t_max
    mean_s = t_total / args.steps
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    if "hbm_gbs" in peaks:
        hbm, hbm_src = float(peaks["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    else:
        hbm, hbm_src = 6800.0, "6.8 TB/s, the profiling recipe's fallback (of fallback; MEASURED_PEAKS.json absent)"
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    t_k1 = float(np.mean(kt[:, 0])) / 1e3 if len(kt) else float("nan")
    t_k2 = float(np.mean(kt[:, 1])) / 1e3 if len(kt) else float("nan")
    work = assembly_work(rule, basis, n_terms=2, value_bytes=8 if prec == wq.PREC_F64 else 4)
    variant = rule.variant(wq.OP_STIFF) if prec in (wq.PREC_F32, wq.PREC_F32_FAST) else -1
    kname, k2name = KERNELS.get((choice, variant), ("?", "?"))
    step_frac = work["step_bytes"] / mean_s / 1e9 / hbm
    if prec == wq.PREC_F64:
        # FP64 element blocks: one FMA (2 flops) per product; peak derived from the SM count
        # of this device x 2 FP64 FMA per cycle x 2 flops x max SM clock (not a measured peak)
        peak = n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12
        achieved = 2 * work["products"] / t_k1 / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s FP64", "frac": achieved / peak,
                "traffic": None, "kernel": kname, "second_kernel": k2name,
                "peak_source": "derived (not measured): %d SMs x 2 FP64 FMA/cycle x 2 x %.0f MHz" % (n_sm, sm_mhz),
                "kernel_ms": t_k1 * 1e3, "second_kernel_ms": t_k2 * 1e3,
                "step_algorithmic_bytes": work["step_bytes"], "step_hbm_frac": step_frac}
    else:
        # the binding roofline of the mixed path is HBM: the element kernel must read the
        # weights, the used table components and the coefficient once (algorithmic bytes,
        # FP64 sizes); slot buffers, index data and descriptors are overhead, in `traffic`
        achieved = work["kernel_bytes"] / t_k1 / 1e9
        traffic = ELEM_TRAFFIC.get(kname) if _kernel_source_sha1(kname) == ELEM_TRAFFIC.get(kname + ":sha1") else None
        per = 6 if prec == wq.PREC_F32 else 3
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": kname, "second_kernel": k2name, "peak_source": hbm_src,
                "kernel_algorithmic_bytes": work["kernel_bytes"], "kernel_ms": t_k1 * 1e3,
                "second_kernel_ms": t_k2 * 1e3, "instrumented_step_ms": float(np.mean(ms_inst)),
                "kernel_share_of_step": t_k1 / (float(np.mean(ms_inst)) / 1e3),
                "step_algorithmic_bytes": work["step_bytes"], "step_hbm_frac": step_frac,
                # diagnostic, not a roofline: FP32 lane-instructions of the products per second
                # against this device's SMs x 128 lanes x max clock
                "diag_lane_instruction_frac": (per * work["products"] / t_k1)
                / (n_sm * 128 * sm_mhz * 1e6) if prec != wq.PREC_TC else None}
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_s * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "tc": "bf16 (5-slice split operands, exact f32 level sums)"}.get(choice, "f32"),
        "precision_mode": choice, "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_functions": basis.n, "n_elements": basis.E, "nnz": nnz,
                   "n_points": rule.Q, "n_gauss": rule.G, "op": "stiffness", "l2": "flushed (256 MB write) before "
                   "every timed step; timed = the assembly call only", "parallelism": "independent instance per GPU"},
        "rel_err_vs_f64": rel,
        "precision_note": "value: the mixed mode wq_rule_autotune picks within 1e-6 of the same rule's GPU FP64 "
                          "result (rel_err_vs_f64); the GPU FP64 path is pinned to the FP64 oracle by "
                          "tests/test_gpu_fullsize.py at max(1e-11, 4x the oracle's LAPACK-driver spread); the "
                          "like-for-like FP64 WQ and GQ figures are comparators.wq_f64_* / gq_f64_*",
        "autotune_ms": dict(zip(("tc", "f32", "f32_fast"), tune["ms"])),
        "autotune_candidates": tune["candidates"], "kernel_variant": variant,
        "gpu_launches": args.steps * 2,
        "roofline": roof,
        "comparators": dict({k + "_ms": v for k, v in comp_ms.items()},
                            **{k + "_nnz_per_s": nnz / (v / 1e3) for k, v in comp_ms.items()},
                            speedup_wq_over_gq_f64=comp_ms["gq_f64"] / comp_ms["wq_f64"],
                            speedup_wq_over_gq_f32=comp_ms["gq_f32"] / comp_ms["wq_f32"],
                            speedup_wq_over_gq_tc=comp_ms["gq_tc"] / comp_ms["wq_tc"]),
        "setup": {"host_basis_ms": host_ms, "rule_build_wall_ms": build_ms, "rule_build_device_ms": rule.info.setup_ms,
                  "n_truncated_x": rule.info.n_truncated[1], "n_z_identity_x": rule.info.n_z_identity[1],
                  # truncated-SVD weight solves (a5): FP64 operations counted by the kernel against
                  # 152 SMs x 2 FP64 FMA per cycle x 2 x max SM clock
                  "tsvd_ms": rule.info.tsvd_ms, "tsvd_gflop": rule.info.tsvd_gflop,
                  "tsvd_fp64_tflops": rule.info.tsvd_gflop / max(rule.info.tsvd_ms, 1e-9),
                  "tsvd_fp64_frac": rule.info.tsvd_gflop / max(rule.info.tsvd_ms, 1e-9)
                  / (n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12),
                  "tsvd_fp64_peak_source": "derived (not measured): %d SMs x 2 FP64 FMA/cycle x 2 x %.0f MHz"
                  % (n_sm, sm_mhz)},
        "e2e": {"value": nnz / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(rule.Q * 8),
                "d2h_bytes_per_step": int(nnz * (8 if prec == wq.PREC_F64 else 4))},
        "clocks": clocks,
    }
    res["refine"] = refine_measure(wq, basis, mesh, flush, max(args.steps // 20, 20), args.warmup, hbm,
                                   n_sm * 2 * 2 * sm_mhz * 1e6 / 1e12)
    if not args.no_cpu_baseline and world == 1:   # CPU baselines: rank 0 at N = 1 only
        a64 = rule.assemble(wq.OP_STIFF, coef, prec=wq.PREC_F64).cpu().numpy()
        g64 = rule.gq_assemble(wq.OP_STIFF, coef_g, prec=wq.PREC_F64).cpu().numpy()
        res["cpu_ref"] = cpu_ref_measure(rule, basis, coef.cpu().numpy(), coef_g.cpu().numpy(), a64, g64)
    if not args.no_cpu_baseline and world == 1:
        res["cpu_baseline"] = cpu_baseline(args)
    if not args.no_configs and world == 1:
        res["other_configs"] = other_configs(ctx, flush, max(args.steps // 20, 20), args.warmup, hbm)
        res["other_configs"]["5_batched_%d_instances" % args.config5_instances] = config5_measure(
            ctx, flush, max(args.steps // 100, 10), args.warmup, hbm, args.config5_instances)
    return res


def config5_measure(ctx, flush, steps, warmup, hbm=6800.0, n_instances=256):
    """Batched assembly of many independent instances: n_instances planar meshes of
    500-50,000 elements (log-uniform target; each mesh is the refinement level nearest
    to it), 1-20 EPs of valence 3-8.  All rules are built by one call whose weight
    systems -- every row of the N, d_x and d_y components of every instance -- are
    solved in one persistent launch; the rules leave out the tensor-core and tile
    plans (device memory).  Mass + stiffness (coefficient kappa at the points) in
    compensated FP32: one batched launch pair per operator, against one call per
    instance and against per-instance Gauss assembly, same protocol (L2 flushed, CUDA
    events, median).  The FP32 error is measured against FP64 on the eight largest
    instances."""
    import gc
    import torch
    from paper_2605_29334_gb300 import wq
    from wq_synth import meshes
    t0 = time.perf_counter()
    ms = meshes.instances(5001, n_instances, 500, 50000, workers=max(1, min(16, os.cpu_count() or 1)))
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    bases = [wq.Basis(ctx, m) for m in ms]
    t_basis = time.perf_counter() - t0
    n_faces = [len(m["quads"]) for m in ms]
    del ms
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    t0 = time.perf_counter()
    rules = wq.build_rules(bases, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y],
                           skip_plans=wq.PLAN_NO_TC | wq.PLAN_NO_TILE)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    rule_bytes = free0 - torch.cuda.mem_get_info()[0]
    info = rules[0].info
    cqs = [torch.tensor(meshes.kappa_sines(rr.points().cpu().numpy()), device="cuda") for rr in rules]
    cgs = [torch.tensor(meshes.kappa_sines(rr.gauss_points().cpu().numpy()), device="cuda") for rr in rules]
    om = [torch.empty(rr.nnz, dtype=torch.float32, device="cuda") for rr in rules]
    ok = [torch.empty(rr.nnz, dtype=torch.float32, device="cuda") for rr in rules]
    batch = wq.Batch(rules)
    nnz = sum(rr.nnz for rr in rules)
    nnz5 = 2 * nnz                                   # mass + stiffness

    def b_wq():
        batch.assemble(wq.OP_MASS, cqs, prec=wq.PREC_F32, outs=om)
        batch.assemble(wq.OP_STIFF, cqs, prec=wq.PREC_F32, outs=ok)

    def per_wq():
        for rr, c, a, b in zip(rules, cqs, om, ok):
            rr.assemble(wq.OP_MASS, c, prec=wq.PREC_F32, out=a)
            rr.assemble(wq.OP_STIFF, c, prec=wq.PREC_F32, out=b)

    def per_gq():
        for rr, c, a, b in zip(rules, cgs, om, ok):
            rr.gq_assemble(wq.OP_MASS, c, prec=wq.PREC_F32, out=a)
            rr.gq_assemble(wq.OP_STIFF, c, prec=wq.PREC_F32, out=b)
    tb = float(np.median(time_steps(b_wq, steps, warmup, flush)))
    tp = float(np.median(time_steps(per_wq, steps, warmup, flush)))
    tq = float(np.median(time_steps(per_gq, steps, warmup, flush)))
    # FP32 error against FP64 on the largest instances
    errs = []
    for k in np.argsort([-rr.nnz for rr in rules])[:8]:
        rr, c = rules[int(k)], cqs[int(k)]
        for op in (wq.OP_MASS, wq.OP_STIFF):
            a64 = rr.assemble(op, c, prec=wq.PREC_F64)
            a32 = rr.assemble(op, c, prec=wq.PREC_F32).to(torch.float64)
            errs.append(float((a32 - a64).abs().max() / a64.abs().max()))
    # algorithmic HBM bytes of the batched step (sum_e m_e P_e = sum_i r_i): weights and
    # used table components 8 B per (weight row, term) each, the coefficient 8 B per point
    # per operator, the float values; mass 1 term, stiffness 2
    sum_r = sum(int(rr.info.sum_r) for rr in rules)
    n_pts = sum(int(rr.Q) for rr in rules)
    step_bytes = 2 * (sum_r * 3 * 8) + 2 * n_pts * 8 + nnz5 * 4
    achieved = step_bytes / (tb * 1e-3) / 1e9
    out = {"n_instances": len(rules), "n_faces": int(sum(n_faces)), "faces_min": int(min(n_faces)),
           "faces_max": int(max(n_faces)), "n_elements": int(sum(bb.E for bb in bases)),
           "n_functions": int(sum(bb.n for bb in bases)), "nnz_mass_plus_stiffness": int(nnz5),
           "n_weight_systems": 3 * int(sum(bb.n for bb in bases)),
           "wq_f32_batched_nnz_per_s": nnz5 / tb * 1e3, "wq_f32_per_instance_nnz_per_s": nnz5 / tp * 1e3,
           "gq_f32_per_instance_nnz_per_s": nnz5 / tq * 1e3, "batched_ms": tb, "per_instance_ms": tp,
           "gq_per_instance_ms": tq, "speedup_batched_over_per_instance": tp / tb,
           "speedup_batched_wq_over_gq": tq / tb, "f32_rel_err_vs_f64_max_largest8": max(errs),
           "roofline_wq_f32_batched_step": {"bound": "hbm", "algorithmic_bytes": int(step_bytes), "unit": "GB/s",
                                            "peak": hbm, "achieved": achieved, "frac": achieved / hbm},
           "setup": {"generate_s": t_gen, "host_basis_s": t_basis, "rule_build_wall_s": t_build,
                     "batched_tsvd_ms": info.tsvd_ms, "batched_tsvd_gflop": info.tsvd_gflop,
                     "batched_tsvd_fp64_tflops": info.tsvd_gflop / max(info.tsvd_ms, 1e-9),
                     "rule_device_bytes": int(rule_bytes)},
           "steps": steps}
    del batch, om, ok, cqs, cgs, rules, bases
    gc.collect()
    torch.cuda.empty_cache()
    return out


def _timed_pair(fn_wq, fn_gq, out_wq, out_gq, steps, warmup, flush):
    import torch
    t_wq = float(np.median(time_steps(lambda: fn_wq(out_wq), steps, warmup, flush)))
    t_gq = float(np.median(time_steps(lambda: fn_gq(out_gq), steps, warmup, flush)))
    torch.cuda.synchronize()
    return t_wq, t_gq


def other_configs(ctx, flush, steps, warmup, hbm=6800.0):
    """The other workloads of the method, same protocol (assembly only, L2 flushed, CUDA
    events, median): WQ against Gauss on the same GPU at FP32 (compensated) and FP64,
    with the FP32 error against the FP64 result (configs 1, 3 and 4; the batched
    instances are config5_measure)."""
    import torch
    from paper_2605_29334_gb300 import wq
    from wq_synth import meshes
    out = {}

    def one(name, mesh, comps, op, alpha, coef_fn, n_terms):
        t0 = time.perf_counter()
        b = wq.Basis(ctx, mesh)
        r = wq.Rule(b, comps=comps)
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        cq = torch.tensor(coef_fn(r.points().cpu().numpy()), device="cuda")
        cg = torch.tensor(coef_fn(r.gauss_points().cpu().numpy()), device="cuda")
        o32 = [torch.empty(r.nnz, dtype=torch.float32, device="cuda") for _ in range(2)]
        o64 = [torch.empty(r.nnz, dtype=torch.float64, device="cuda") for _ in range(2)]
        f32 = _timed_pair(lambda o: r.assemble(op, cq, alpha=alpha, prec=wq.PREC_F32, out=o),
                          lambda o: r.gq_assemble(op, cg, alpha=alpha, prec=wq.PREC_F32, out=o),
                          o32[0], o32[1], steps, warmup, flush)
        f64 = _timed_pair(lambda o: r.assemble(op, cq, alpha=alpha, prec=wq.PREC_F64, out=o),
                          lambda o: r.gq_assemble(op, cg, alpha=alpha, prec=wq.PREC_F64, out=o),
                          o64[0], o64[1], steps, warmup, flush)
        a64 = o64[0].cpu().numpy()
        err, err_fro = rel_errors(o32[0].cpu().numpy(), a64)
        tc = _timed_pair(lambda o: r.assemble(op, cq, alpha=alpha, prec=wq.PREC_TC, out=o),
                         lambda o: r.gq_assemble(op, cg, alpha=alpha, prec=wq.PREC_TC, out=o),
                         o32[0], o32[1], steps, warmup, flush)
        err_tc, err_tc_fro = rel_errors(o32[0].cpu().numpy(), a64)
        out[name] = {"n_elements": b.E, "nnz": r.nnz, "n_points": r.Q, "n_gauss": r.G,
                     "wq_f32_nnz_per_s": r.nnz / f32[0] * 1e3, "gq_f32_nnz_per_s": r.nnz / f32[1] * 1e3,
                     "wq_f64_nnz_per_s": r.nnz / f64[0] * 1e3, "gq_f64_nnz_per_s": r.nnz / f64[1] * 1e3,
                     "speedup_f32": f32[1] / f32[0], "speedup_f64": f64[1] / f64[0],
                     "f32_rel_err_vs_f64": err, "setup_s": setup_s,
                     "wq_tc_nnz_per_s": r.nnz / tc[0] * 1e3, "gq_tc_nnz_per_s": r.nnz / tc[1] * 1e3,
                     "speedup_tc": tc[1] / tc[0], "tc_rel_err_vs_f64": err_tc,
                     "f32_rel_err_fro_vs_f64": err_fro, "tc_rel_err_fro_vs_f64": err_tc_fro}
        # HBM roofline of the WQ FP32 step (both kernels): algorithmic bytes (weights, used
        # table components, coefficient, values) over the step's median device time
        wk = assembly_work(r, b, n_terms=n_terms, value_bytes=4)
        out[name]["roofline_wq_f32_step"] = {
            "bound": "hbm", "algorithmic_bytes": wk["step_bytes"], "unit": "GB/s", "peak": hbm,
            "achieved": wk["step_bytes"] / (f32[0] / 1e3) / 1e9,
            "frac": wk["step_bytes"] / (f32[0] / 1e3) / 1e9 / hbm}
        return b, r, cq

    disk = meshes.disk(mu=5, n=6)
    one("1_disk_mu5_mass_stiffness", disk, [wq.COMP_N, wq.COMP_X, wq.COMP_Y], wq.OP_HEAT_S, 1.0,
        meshes.kappa_sines, 3)
    sph = meshes.cube_sphere(pre=3, levels=3)
    one("3_sphere_biharmonic", sph, [wq.COMP_N, wq.COMP_LAP], wq.OP_BIHARM, 0.0,
        lambda x: 1.0 + 0.25 * x[:, 0] * x[:, 1] + 0.1 * x[:, 2], 1)
    heat = make_mesh(levels=5)
    u0 = meshes.gaussian_bumps(4001, heat["xyz"].min(0), heat["xyz"].max(0))
    b4, r4, _ = one("4_heat_tangent_L5", heat, [wq.COMP_N, wq.COMP_X, wq.COMP_Y], wq.OP_HEAT_S, 100.0,
                    lambda x: 1.0 + u0(x) ** 2, 3)
    # config 4: 20 Newton iterations (Sec. 5.2) on the 40,960-element mesh, u updated every
    # iteration; the re-assembly of each iteration (point fields, FP64 residual, tangent)
    # replays one CUDA graph, the correction is a BiCGSTAB solve outside it.  The exact
    # tangent in FP64 against the same tangent assembled in the mixed modes.  Time step
    # 1e-4: with 1e-2 and 3e-3 the iteration does not converge on this mesh family from
    # 2,560 elements up (for any tangent, with or without line search), while the same
    # code converges quadratically on 640 elements and matches the oracle there.
    from paper_2605_29334_gb300.newton import HeatNewton, boundary_fixed
    fixed = boundary_fixed(b4, heat)
    u0h = u0(b4.ctrl())
    runs = {"dt": 1e-4, "tangent": "exact (WQ_OP_HEAT_J)", "residual": "FP64"}
    for nm, p in (("f64", wq.PREC_F64), ("f32", wq.PREC_F32), ("tc", wq.PREC_TC)):
        nt = HeatNewton(r4, fixed, 1e-4, tangent=wq.OP_HEAT_J, prec=p)
        o = nt.run(u0h, iters=20)
        h = np.array(o["residual"]) / o["residual"][0]
        runs[nm] = {"relative_residual": h.tolist(),
                    "first_iteration_below_1e-8": int(np.argmax(h < 1e-8)) if np.any(h < 1e-8) else None,
                    "reassembly_graph_ms_median": float(np.median(o["reassembly_ms"])),
                    "linear_iterations": o["linear_iterations"], "wall_s": o["wall_s"]}
        del nt
    out["4_heat_tangent_L5"]["newton_20_iterations"] = runs
    return out


# DRAM bytes (read + write) of one launch of the element-block kernels on this workload,
# from `ncu --set full` (profiles/), valid for the kernel source they were taken on: the
# key "<kernel>:sha1" holds the SHA-1 of the kernel's own source text (see _KERNEL_TEXT),
# so that edits elsewhere in the file keep the measurement and edits of the kernel drop it.
ELEM_TRAFFIC = {"k_elem_f32<2,1,0,0,1>": 60644352, "k_elem_f32<2,1,0,0,1>:sha1": "1a3e2518c10271d66a893af1613b3e0eb6afa02a",
                "k_elem_tc<2,0>": 69611776, "k_elem_tc<2,0>:sha1": "3c5ca0106f23d6257452c245b034a1ca7f2d45f6"}
_KERNEL_TEXT = {"k_elem_f32": ("k_assemble.cu", "template <int NT, bool COMP, bool GAUSS, bool BATCH, int NP>\n__global__ void "
                               "__launch_bounds__(EL_NWARP * 32, 6)", "// Phase 2: one thread per two consecutive CSR entries."),
                "k_elem_tc": ("k_tc.cu", "template <int NT, bool GAUSS>\n__global__", "cudaError_t launch_elem_tc("),
                "k_tile_f32": ("k_tile.cu", "template <int NT, int V, bool COMP, bool BATCH, int NP>\n__global__",
                               "// ------------------------------------------------------------------ phase 2")}


def _kernel_source_sha1(kname):
    import hashlib
    base = kname.split("<")[0]
    if base not in _KERNEL_TEXT:
        return None
    name, begin, end = _KERNEL_TEXT[base]
    with open(os.path.join(ROOT, "paper_2605_29334_gb300", "csrc", name)) as f:
        s = f.read()
    try:
        s = s[s.index(begin):s.index(end)]
    except ValueError:
        return None
    return hashlib.sha1(s.encode()).hexdigest()


def refine_measure(wq, basis, mesh, flush, steps, warmup, hbm, fp64_tflops):
    """One global refinement of the workload's control mesh (Sec. 3) on the device:
    knot-insertion stencils for the vertex-based control points, de Casteljau splits of
    the enriched faces' nets for the face-based ones.  Algorithmic bytes: every coarse
    control point, stencil entry (4 B index + 8 B weight, 8 B row pointer), face job and
    non-zero term of a fine face-based point (the de Casteljau split folded into the
    Bezier coefficients; 4 B function id + 8 B value) read once, every fine control point
    written once.  FP64 work: 3 FMAs per stencil entry and per term."""
    import torch
    r = wq.Refine(basis)
    I = r.info
    x = torch.tensor(np.ascontiguousarray(mesh["xyz"], dtype=np.float64), device="cuda")
    fx = torch.tensor(basis.face_ctrl(), device="cuda").reshape(-1, 3)
    xf = torch.empty((I.n_vertices, 3), dtype=torch.float64, device="cuda")
    ff = torch.empty((I.n_face_xyz, 3), dtype=torch.float64, device="cuda")
    # the two launches replayed from a CUDA graph: the Python call costs more host time
    # than the kernels take on the device
    r.apply(x, fx, out=(xf, ff))
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        r.apply(x, fx, out=(xf, ff))
    ms = time_steps(graph.replay, steps, warmup, flush)
    t = float(np.mean(ms)) / 1e3
    byts = (24 * (I.n_coarse_vertices + I.n_coarse_face_xyz + I.n_vertices + I.n_face_xyz)
            + 12 * I.n_stencil + 8 * (I.n_vertices + 1) + 24 * I.n_face_jobs + 12 * I.n_face_terms)
    flops = 6 * (I.n_stencil + I.n_face_terms)
    return {"ms": t * 1e3, "coarse_vertices": I.n_coarse_vertices, "fine_vertices": I.n_vertices,
            "fine_faces": I.n_faces, "fine_face_points": I.n_face_xyz, "face_jobs": I.n_face_jobs,
            "face_coefficients_dense": I.n_face_coef, "face_terms_nonzero": I.n_face_terms,
            "algorithmic_bytes": byts, "achieved_gbs": byts / t / 1e9, "hbm_frac": byts / t / 1e9 / hbm,
            "fp64_gflop": flops / 1e9, "fp64_frac": flops / t / 1e12 / fp64_tflops,
            "fp64_peak_source": "derived (not measured): SMs x 2 FP64 FMA/cycle x 2 x max SM clock",
            "launches": 1, "timing": "CUDA-graph replay, L2 flushed before each"}


def assembly_work(rule, basis, n_terms, n_coef_rows=1, value_bytes=4):
    """Algorithmic work of one assembly of an operator with n_terms (weight component,
    table component) pairs: products = sum_e m_e^2 P_e n_terms (one per test x trial x
    point x term); algorithmic bytes (what must cross HBM once, FP64 storage): the
    weights sum_i r_i n_terms 8 (sum_i r_i = sum_e m_e P_e), the used table components
    sum_e m_e P_e n_terms 8, the coefficient rows Q n_coef_rows 8, and for the whole step
    the CSR values nnz value_bytes.  The element kernel's own algorithmic bytes are the
    first three (it reads them; the values are written by the per-row sums)."""
    E = basis.E
    side = basis.point_counts().astype(np.int64)
    m = np.array([basis.element(e)["fns"].size for e in range(E)], dtype=np.int64)
    P = side * side
    products = int(np.sum(m * m * P)) * n_terms
    weights = int(rule.info.sum_r) * n_terms * 8
    tables = int(np.sum(P * m)) * n_terms * 8
    coef = int(rule.Q) * n_coef_rows * 8
    values = int(rule.nnz) * value_bytes
    return {"products": products, "weights": weights, "tables": tables, "coef": coef, "values": values,
            "kernel_bytes": weights + tables + coef, "step_bytes": weights + tables + coef + values}


KERNELS = {  # (mode, variant) -> (element kernel, second kernel) of the stiffness operator (2 terms)
    ("f32", 2): ("k_elem_f32<2,1,0,0,1>", "k_gather_f32<1,0,1>"),
    ("f32_fast", 2): ("k_elem_f32<2,0,0,0,1>", "k_gather_f32<0,0,1>"),
    ("f32", 0): ("k_tile_f32<2,0,1,0,1>", "k_rowsum_f32<1,0,1>"),
    ("f32", 1): ("k_tile_f32<2,1,1,0,1>", "k_rowsum_f32<1,0,1>"),
    ("f32_fast", 0): ("k_tile_f32<2,0,0,0,1>", "k_rowsum_f32<0,0,1>"),
    ("f32_fast", 1): ("k_tile_f32<2,1,0,0,1>", "k_rowsum_f32<0,0,1>"),
    ("tc", -1): ("k_elem_tc<2,0>", "k_gather_f32<1,0,1>"),
    ("f64", -1): ("k_elem_f64<2,0>", "k_gather_f64"),
}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return ""


def cpu_ref_measure(rule, basis, kq, kg, a_wq64, a_gq64, seconds=6.0):
    """cpu_ref (C++/OpenMP, FP64) on the full workload and on every host core: row-wise
    WQ and element-wise Gauss stiffness assembly from the same precomputed inputs (the
    rule's weights and point tables, copied to the host as data), timed on the host."""
    import cpu_ref
    E = basis.E
    fl = [basis.element(e)["fns"] for e in range(E)]
    fn_ptr = np.concatenate([[0], np.cumsum([len(f) for f in fl])])
    fns = np.concatenate(fl)
    supp_ptr, supp, il = cpu_ref.supports(fn_ptr, fns, basis.n)
    rp, col = basis.pattern()
    comps = list(rule.comps)
    w = np.stack([rule.weights(c)[0].cpu().numpy() for c in comps], axis=1)
    t, g = rule.table(False), rule.table(True)
    pb = cpu_ref.Problem(row_ptr=rp, col=col, fn_ptr=fn_ptr, fns=fns, supp_ptr=supp_ptr, supp=supp, il=il,
                         w_ptr=rule.weights(comps[0])[1].cpu().numpy(), w=w, pt_ptr=t["pt_ptr"].cpu().numpy(),
                         tab_ptr=t["off"].cpu().numpy(), table=t["table"].cpu().numpy(),
                         gp_ptr=g["pt_ptr"].cpu().numpy(), gtab_ptr=g["off"].cpu().numpy(),
                         gtable=g["table"].cpu().numpy(), gw=g["gw"].cpu().numpy())
    nc = t["ncomp"]
    tw = [(comps.index(1), 1, 0, 1.0), (comps.index(2), 2, 0, 1.0)]      # (weight column, table comp, ...)
    tg = [(1, 1, 0, 1.0), (2, 2, 0, 1.0)]
    ncores = os.cpu_count() or 1
    cpu_ref.set_threads(ncores)
    kbuf = np.zeros(pb.kb_ptr[-1])

    def timed(fn):
        fn()
        n, t0 = 0, time.perf_counter()
        while True:
            r = fn()
            n += 1
            el = time.perf_counter() - t0
            if el > seconds / 2 or n >= 200:
                return r, el / n, n
    a_wq, t_wq, n_wq = timed(lambda: cpu_ref.wq_assemble(pb, nc, len(comps), tw, kq))
    a_gq, t_gq, n_gq = timed(lambda: cpu_ref.gq_assemble(pb, nc, tg, kg, kbuf))
    nnz = len(col)
    return {"kind": "cpu_ref", "wq_nnz_per_s": nnz / t_wq, "gq_nnz_per_s": nnz / t_gq, "unit": UNIT,
            "wq_ms": t_wq * 1e3, "gq_ms": t_gq * 1e3, "reps": [n_wq, n_gq], "threads": cpu_ref.threads(),
            "nproc": ncores, "cpu": _cpu_model(),
            "wq_rel_err_vs_gpu_f64": rel_errors(a_wq, a_wq64)[0], "gq_rel_err_vs_gpu_f64": rel_errors(a_gq, a_gq64)[0],
            "sample": "the full workload (%d elements, %d nnz), stiffness, FP64, precomputed weights and tables"
                      % (E, nnz)}


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
    ap.add_argument("--prec", default="auto", choices=["auto", "tc", "f32", "f32_fast", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads (configs 1, 3, 4, 5)")
    ap.add_argument("--config5-instances", type=int, default=256, help="instances of the batched workload")
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
