"""GPU path vs the FP64 oracle, step by step, through the C ABI.

a2 placement, a3 basis tables at WQ and Gauss points, a4 Gauss moments,
a5 truncated-SVD weights, a6 WQ assembly (FP64 to 1e-11 normwise -- the bar of
the FP64 path -- or, where the weight systems' conditioning makes that
unreachable for any two FP64 implementations, 4x the oracle's own spread
between two LAPACK SVD drivers, gesdd and gesvd; FP32 split-product path: 1e-6
against the GPU's FP64 result, and max(1e-6, the FP64 bar) against the oracle;
tensor-core slices: the same; every achieved error and bar is recorded as a test
property), a7
interpolation, a8 Gauss assembly.  Meshes cover one EP of valence 3..8 (m_e up to 37 > 32 lanes),
refined enriched regions, clustered EPs, an EP-free grid, a closed surface and
a mesh with a single active element.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu

COMP_ID = {"N": 0, "x": 1, "y": 2, "z": 3, "lap": 4}

CASES = {
    "disk5": (lambda: meshes.disk(mu=5, n=6), ["N", "x", "y", "lap"]),
    "disk8_L1": (lambda: meshes.disk(mu=8, n=4, levels=1), ["N", "x", "y"]),
    "disk3_L2": (lambda: meshes.disk(mu=3, n=3, levels=2), ["N", "x", "y", "lap"]),
    "rotated_L1": (lambda: meshes.rotated(levels=1), ["N", "x", "y"]),
    "sphere": (lambda: meshes.cube_sphere(pre=1, levels=1), ["N", "x", "y", "z", "lap"]),
    "grid1x1": (lambda: meshes.grid(1, 1), ["N", "x", "y"]),
}


def _kappa(x):
    x = np.asarray(x)
    return 1.0 + 0.5 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) + 0.25 * x[:, 2] ** 2


def nerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.fixture(scope="module")
def W():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return wq


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request, W):
    from oracle.basis import Basis
    from oracle import wq as owq
    make, comps = CASES[request.param]
    mesh = make()
    B = Basis(mesh)
    R = owq.Rule(B, comps)
    R.compute_weights()
    # the oracle's reproducibility floor: the same steps with LAPACK gesvd instead of gesdd
    R2 = owq.Rule(B, comps)
    R2.compute_weights(driver="gesvd")
    ctx = W.Context(0)
    b = W.Basis(ctx, mesh)
    r = W.Rule(b, comps=[COMP_ID[c] for c in comps])
    return {"name": request.param, "B": B, "R": R, "R2": R2, "ctx": ctx, "b": b, "r": r, "comps": comps}


def fp64_tol(spread, factor=4.0):
    """1e-11, or factor x the oracle's driver-to-driver spread where that is larger."""
    return max(1e-11, factor * spread)


def test_points(case):
    R, r = case["R"], case["r"]
    assert r.Q == R.Q
    assert np.max(np.abs(r.points().cpu().numpy() - R.x)) < 1e-14


def _oracle_block(d, comps_all):
    rows = [d["N"], d["grad"][..., 0], d["grad"][..., 1]]
    if comps_all == 5:
        rows.append(d["grad"][..., 2])
    rows.append(d["lap"])
    return np.stack(rows, axis=1)           # [m, nc, P]


def test_tables(case):
    from oracle.gq import gauss_data
    B, R, r = case["B"], case["R"], case["r"]
    for gauss in (False, True):
        t = r.table(gauss)
        tab = t["table"].cpu().numpy()
        off = t["off"].cpu().numpy()
        nc = t["ncomp"]
        worst = np.zeros(nc)
        scale = np.zeros(nc)
        for e in range(B.E):
            d = gauss_data(B, e) if gauss else R.data[e]
            ref = _oracle_block(d, nc)                       # [m, nc, P]
            m, P = ref.shape[0], ref.shape[2]
            got = tab[off[e]:off[e + 1]].reshape(P, nc, m).transpose(2, 1, 0)
            worst = np.maximum(worst, np.max(np.abs(got - ref), axis=(0, 2)))
            scale = np.maximum(scale, np.max(np.abs(ref), axis=(0, 2)))
            if gauss:
                gw = t["gw"].cpu().numpy()[t["pt_ptr"].cpu().numpy()[e]:t["pt_ptr"].cpu().numpy()[e + 1]]
                assert np.max(np.abs(gw - d["w"])) <= 1e-13 * np.max(d["w"])
        assert np.all(worst <= 1e-12 * scale), (gauss, worst / scale)


def test_moments(case):
    R, r = case["R"], case["r"]
    for c in case["comps"]:
        got = r.moments(COMP_ID[c]).cpu().numpy()
        assert nerr(got, R.moments[c]) < 1e-13, c


def test_weights(case, record_property):
    """The weights are an intermediate, unique only up to each system's conditioning
    (near-threshold singular values move them far more than the assembled matrices),
    so they are held to what defines them: per row, the exactness constraints
    A w = b (Sec. 4.3) on the oracle's own system, to the residual the oracle's weights
    leave (x 10, at least 1e-12 of |b|), the truncation counts, and -- recorded, not a
    bar -- their distance to the oracle's weights next to the driver spread."""
    R, r = case["R"], case["r"]
    for c in case["comps"]:
        w, wp = r.weights(COMP_ID[c])
        w = w.cpu().numpy()
        assert np.array_equal(wp.cpu().numpy(), R.w_ptr)
        record_property("weights_%s_dist_to_oracle" % c, nerr(w, R.weights[c]))
        record_property("weights_%s_driver_spread" % c, nerr(case["R2"].weights[c], R.weights[c]))
        worst = 0.0
        for i in range(R.basis.n):
            A, _ = R.local_system(i, c)
            b = R.moments[c][R.row_ptr[i]:R.row_ptr[i + 1]]
            sl = slice(R.w_ptr[i], R.w_ptr[i + 1])
            bs = max(np.max(np.abs(b)), 1e-300)
            res_gpu = np.max(np.abs(A @ w[sl] - b)) / bs
            res_ora = np.max(np.abs(A @ R.weights[c][sl] - b)) / bs
            worst = max(worst, res_gpu)
            assert res_gpu <= max(1e-12, 10.0 * res_ora), (c, i, res_gpu, res_ora)
        record_property("weights_%s_exactness_residual" % c, worst)
        n_trunc = int(np.sum(R.rank[c] < np.diff(R.row_ptr)))
        assert r.info.n_truncated[COMP_ID[c]] == n_trunc, c


def _ops(case, kap, alpha):
    comps = case["comps"]
    grads = [c for c in ("x", "y", "z") if c in comps]
    ops = {}
    if "N" in comps:
        ops[0] = [("N", kap)]
        if len(grads) >= 2:
            ops[3] = [("N", alpha * np.ones_like(kap))] + [(g, kap) for g in grads]
    if len(grads) >= 2:
        ops[1] = [(g, kap) for g in grads]
    if "lap" in comps:
        ops[2] = [("lap", kap)]
    return ops


def test_assembly_f64_and_f32(case, W, record_property):
    import torch
    R, r = case["R"], case["r"]
    kap = _kappa(R.x)
    alpha = 7.5
    kd = torch.tensor(kap, device="cuda")
    for op, terms in _ops(case, kap, alpha).items():
        ref = R.assemble(terms)
        spread = nerr(case["R2"].assemble(terms), ref)
        tol = fp64_tol(spread)
        got = r.assemble(op, kd, alpha=alpha, prec=W.PREC_F64).cpu().numpy()
        record_property("op%d_fp64_err_vs_oracle" % op, nerr(got, ref))
        record_property("op%d_driver_spread" % op, spread)
        record_property("op%d_fp64_bar" % op, tol)
        print(case["name"], "op", op, "FP64 error vs oracle %.3e, bar %.3e (driver spread %.3e)"
              % (nerr(got, ref), tol, spread))
        assert nerr(got, ref) < tol, (op, nerr(got, ref), tol)
        got32 = r.assemble(op, kd, alpha=alpha, prec=W.PREC_F32).cpu().numpy()
        assert nerr(got32, got) < 1e-6, (op, nerr(got32, got))
        assert nerr(got32, ref) < max(1e-6, tol), (op, nerr(got32, ref))
        assert np.array_equal(got32, r.assemble(op, kd, alpha=alpha, prec=W.PREC_F32).cpu().numpy())
        # plain FP32 sums: error grows with the cancellation in the rows (stated, not 1e-6)
        gotf = r.assemble(op, kd, alpha=alpha, prec=W.PREC_F32_FAST).cpu().numpy()
        assert nerr(gotf, got) < 2e-5, (op, nerr(gotf, got))
        # tensor cores, bf16 slices with exact integer sums: the mixed-precision bar
        gott = r.assemble(op, kd, alpha=alpha, prec=W.PREC_TC).cpu().numpy()
        assert nerr(gott, got) < 1e-6, (op, nerr(gott, got))
        assert nerr(gott, ref) < max(1e-6, tol), (op, nerr(gott, ref))
        assert np.array_equal(gott, r.assemble(op, kd, alpha=alpha, prec=W.PREC_TC).cpu().numpy())
    # constant coefficient reproduces the Gauss moments (exactness, Sec. 4.3)
    if "x" in case["comps"]:
        ones = torch.ones(R.Q, dtype=torch.float64, device="cuda")
        K1 = r.assemble(1, ones).cpu().numpy()
        G = sum(R.moments[c] for c in case["comps"] if c in ("x", "y", "z"))
        assert nerr(K1, G) < 1e-11


def test_gauss_assembly(case, W):
    import torch
    from oracle import gq
    B, R, r = case["B"], case["R"], case["r"]
    gx = r.gauss_points().cpu().numpy()
    kg = torch.tensor(_kappa(gx), device="cuda")
    comps = case["comps"]
    grads = [c for c in ("x", "y", "z") if c in comps]
    checks = {0: ["N"], 1: grads}
    if "lap" in comps:
        checks[2] = ["lap"]
    for op, cc in checks.items():
        ref = gq.assemble(B, cc, coef=_kappa, row_ptr=R.row_ptr, col=R.col)
        got = r.gq_assemble(op, kg).cpu().numpy()
        assert nerr(got, ref) < 1e-12, op
        # element-major FP32 (split products, TwoSum): Gauss systems are well conditioned
        got32 = r.gq_assemble(op, kg, prec=W.PREC_F32).cpu().numpy().astype(np.float64)
        assert nerr(got32, ref) < 1e-6, op
        again = r.gq_assemble(op, kg, prec=W.PREC_F32).cpu().numpy().astype(np.float64)
        assert np.array_equal(got32, again)
        gott = r.gq_assemble(op, kg, prec=W.PREC_TC).cpu().numpy().astype(np.float64)
        assert nerr(gott, ref) < 1e-6, (op, nerr(gott, ref))


def test_interp(case):
    import torch
    R, r = case["R"], case["r"]
    rng = np.random.Generator(np.random.PCG64(4))
    u = rng.normal(size=R.basis.n)
    uq, gr = r.interp(torch.tensor(u, device="cuda"))
    ruq, rgr = R.interp(u)
    assert nerr(uq.cpu().numpy(), ruq) < 1e-13
    assert nerr(gr.cpu().numpy(), rgr) < 1e-12


def test_assemble_host_roundtrip(case, W):
    import torch
    R, r = case["R"], case["r"]
    if "x" not in case["comps"]:
        pytest.skip("no stiffness weights")
    kap = _kappa(R.x)
    dev = r.assemble(1, torch.tensor(kap, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    host = r.assemble_host(1, kap)
    assert np.array_equal(dev, host)
    # page-locked output buffers, both precisions
    for prec, dt in ((W.PREC_F32, torch.float32), (W.PREC_F64, torch.float64)):
        pinned = torch.full((r.nnz,), float("nan"), dtype=dt).pin_memory()
        r.assemble_host(1, kap, prec=prec, out=pinned.numpy())
        ref = r.assemble(1, torch.tensor(kap, device="cuda"), prec=prec).cpu().numpy()
        assert np.array_equal(pinned.numpy(), ref), prec


def _dk(d):
    """Smooth stand-ins for the rows k'(u) d_d u of the exact heat tangent."""
    return lambda x: 0.3 * np.sin(1.7 * x[:, d] + 0.4 * d) + 0.2 * np.cos(x[:, (d + 1) % 3])


def test_heat_tangent_operator(case, W):
    """WQ_OP_HEAT_J (Sec. 5.2): alpha * mass + stiffness(k) + sum_d (w^d, N; k' d_d u),
    the exact Newton tangent of the WQ heat residual, against the oracle's mixed
    terms (WQ) and Gauss mixed integrals (GQ), FP64 and FP32."""
    import torch
    from oracle import gq
    comps = case["comps"]
    grads = [c for c in ("x", "y", "z") if c in comps]
    if "N" not in comps or len(grads) < 2:
        pytest.skip("needs N and gradient weights")
    R, r = case["R"], case["r"]
    alpha = 7.5
    dks = [_dk(d) for d in range(len(grads))]
    kap_q = _kappa(R.x)
    terms = ([("N", "N", np.full(R.Q, alpha))] + [(g, g, kap_q) for g in grads]
             + [(g, "N", dks[d](R.x)) for d, g in enumerate(grads)])
    ref = R.assemble(terms)
    spread = nerr(case["R2"].assemble(terms), ref)
    coef = torch.tensor(np.stack([kap_q] + [f(R.x) for f in dks]), device="cuda")
    got = r.assemble(W.OP_HEAT_J, coef, alpha=alpha, prec=W.PREC_F64).cpu().numpy()
    assert nerr(got, ref) < fp64_tol(spread), (nerr(got, ref), fp64_tol(spread))
    got32 = r.assemble(W.OP_HEAT_J, coef, alpha=alpha, prec=W.PREC_F32).cpu().numpy()
    assert nerr(got32, got) < 1e-6, nerr(got32, got)
    gott = r.assemble(W.OP_HEAT_J, coef, alpha=alpha, prec=W.PREC_TC).cpu().numpy()
    assert nerr(gott, got) < 1e-6, nerr(gott, got)
    # the same operator by Gauss quadrature
    gx = r.gauss_points().cpu().numpy()
    gterms = ([("N", "N", lambda x: np.full(len(x), alpha))] + [(g, g, _kappa) for g in grads]
              + [(g, "N", dks[d]) for d, g in enumerate(grads)])
    gref = gq.assemble_terms(R.basis, gterms, row_ptr=R.row_ptr, col=R.col)
    gcoef = torch.tensor(np.stack([_kappa(gx)] + [f(gx) for f in dks]), device="cuda")
    ggot = r.gq_assemble(W.OP_HEAT_J, gcoef, alpha=alpha, prec=W.PREC_F64).cpu().numpy()
    assert nerr(ggot, gref) < 1e-12, nerr(ggot, gref)
    ggot32 = r.gq_assemble(W.OP_HEAT_J, gcoef, alpha=alpha, prec=W.PREC_F32).cpu().numpy()
    assert nerr(ggot32, gref) < 1e-6, nerr(ggot32, gref)
    # five terms on 64-point irregular elements: K = 320, two exact segments
    ggott = r.gq_assemble(W.OP_HEAT_J, gcoef, alpha=alpha, prec=W.PREC_TC).cpu().numpy()
    assert nerr(ggott, gref) < 1e-6, nerr(ggott, gref)
