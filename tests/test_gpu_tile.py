"""Tile engine (bulk-copied element blocks, then per-row sums) against the slot-map
engine and the FP64 path, through the C ABI.

The two float engines run the same arithmetic per element block (split (hi, lo)
products, extraction-compensated sums) and add each CSR entry's element contributions
in the same (support) order; they differ in the extraction constants (the tile engine
bounds |T| over the whole element from a set-up table, the slot-map kernel per chunk)
and, for Gauss items, in the test side (the Gauss weight folded in at set-up).  The
constants only move the rounding at ~2^-48 of each tile's scale, so the WQ values agree
to a few FP32 ulps of the matrix scale (held to 2e-7 normwise), and every variant is
held to the 1e-6 bar against the FP64 result; each variant reproduces itself bit for
bit.  Meshes cover elements with more than 16 and more than 32 functions
(several column blocks per element), P = 4, 9, 16 points, a closed surface (3
gradient components, 4- and 7-term operators) and a single active element.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu

CASES = {
    "disk5": lambda: meshes.disk(mu=5, n=6),
    "disk8_L1": lambda: meshes.disk(mu=8, n=4, levels=1),
    "disk3_L2": lambda: meshes.disk(mu=3, n=3, levels=2),
    "rotated_L2": lambda: meshes.rotated(levels=2),
    "sphere": lambda: meshes.cube_sphere(pre=1, levels=1),
    "grid1x1": lambda: meshes.grid(1, 1),
}


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
def rule(request, W):
    mesh = CASES[request.param]()
    ctx = W.Context(0)
    b = W.Basis(ctx, mesh)
    dim = 3 if request.param == "sphere" else 2
    comps = [W.COMP_N, W.COMP_X, W.COMP_Y] + ([W.COMP_Z] if dim == 3 else []) + [W.COMP_LAP]
    r = W.Rule(b, comps=comps)
    return {"name": request.param, "ctx": ctx, "b": b, "r": r, "dim": dim}


def _coef(x, rows, seed):
    rng = np.random.default_rng(seed)
    x = np.asarray(x)
    k = 1.0 + 0.5 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) + 0.25 * x[:, 2] ** 2
    if rows == 1:
        return k
    return np.stack([k] + [0.3 * rng.standard_normal(len(k)) for _ in range(rows - 1)])


def test_tile_engine_against_slot_map(rule, W):
    import torch
    r, dim = rule["r"], rule["dim"]
    ops = [(W.OP_MASS, 0.0), (W.OP_STIFF, 0.0), (W.OP_BIHARM, 0.0), (W.OP_HEAT_S, 37.0), (W.OP_HEAT_J, 11.0)]
    worst = {}
    for op, alpha in ops:
        rows = 1 + dim if op == W.OP_HEAT_J else 1
        for gauss in (False, True):
            x = (r.gauss_points() if gauss else r.points()).cpu().numpy()
            c = torch.tensor(_coef(x, rows, 7 + op), device="cuda")
            run = (lambda p: r.gq_assemble(op, c, alpha=alpha, prec=p)) if gauss else \
                (lambda p: r.assemble(op, c, alpha=alpha, prec=p))
            a64 = run(W.PREC_F64).cpu().numpy()
            out = {}
            for v in (W.VARIANT_SLOTMAP, W.VARIANT_TILE12, W.VARIANT_TILE16):
                r.set_variant(op, v, gauss=gauss)
                for prec in (W.PREC_F32, W.PREC_F32_FAST):
                    out[v, prec] = run(prec).cpu().numpy()
            r.set_variant(op, -1, gauss=gauss)
            torch.cuda.synchronize()
            if not gauss:
                d = nerr(out[W.VARIANT_TILE12, W.PREC_F32], out[W.VARIANT_SLOTMAP, W.PREC_F32])
                assert d <= 2e-7, (rule["name"], op, d)
            for v in (W.VARIANT_SLOTMAP, W.VARIANT_TILE12, W.VARIANT_TILE16):
                e = nerr(out[v, W.PREC_F32], a64)
                worst[(op, gauss, v)] = e
                assert e <= 1e-6, (rule["name"], op, gauss, v, e)
            assert r.variant(op, gauss=gauss) == W.VARIANT_SLOTMAP   # the default before any autotune
    print(rule["name"], "worst compensated-FP32 error vs FP64: %.2e" % max(worst.values()))


def test_tile_engine_without_coefficient(rule, W):
    """coef = null means c = 1: the WQ stiffness then reproduces the Gauss stiffness
    (exactness, Sec. 4.3) up to the FP32 rounding."""
    r = rule["r"]
    a = r.assemble(W.OP_STIFF, None, prec=W.PREC_F32).cpu().numpy()
    g = r.gq_assemble(W.OP_STIFF, None, prec=W.PREC_F32).cpu().numpy()
    g64 = r.gq_assemble(W.OP_STIFF, None, prec=W.PREC_F64).cpu().numpy()
    assert nerr(g, g64) <= 1e-6
    assert nerr(a, g64) <= 1e-6


def test_tile_engine_workload_bitwise(W):
    """The 10,240-element benchmark mesh: WQ stiffness of the engines against each other
    and FP64; each variant reproduces itself bit for bit."""
    import torch
    mesh = meshes.rotated(nx=8, ny=5, n_ep=12, levels=4, seed=2001)
    ctx = W.Context(0)
    b = W.Basis(ctx, mesh)
    r = W.Rule(b, comps=[W.COMP_X, W.COMP_Y])
    x = r.points().cpu().numpy()
    kap = meshes.LogNormalField(2101, mesh["xyz"].min(axis=0), mesh["xyz"].max(axis=0), nk=16, sigma=0.5)
    c = torch.tensor(kap(x), device="cuda")
    r.set_variant(W.OP_STIFF, W.VARIANT_SLOTMAP)
    a2 = r.assemble(W.OP_STIFF, c, prec=W.PREC_F32).cpu().numpy()
    a64 = r.assemble(W.OP_STIFF, c, prec=W.PREC_F64).cpu().numpy()
    for v in (W.VARIANT_TILE12, W.VARIANT_TILE16):
        r.set_variant(W.OP_STIFF, v)
        a0 = r.assemble(W.OP_STIFF, c, prec=W.PREC_F32).cpu().numpy()
        a0b = r.assemble(W.OP_STIFF, c, prec=W.PREC_F32).cpu().numpy()
        assert np.array_equal(a0, a0b)
        assert nerr(a0, a2) <= 2e-7
        assert nerr(a0, a64) <= 1e-6
