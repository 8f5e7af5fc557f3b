"""Tensor-core mode (WQ_PREC_TC) on the ill-conditioned operators of the larger
workloads, against the GPU's own FP64 path (itself pinned to the oracle in
test_gpu_parity / test_gpu_fullsize).

The slicing error is relative to each tile's largest |s| |T| K, not to each entry, and
the weights of ill-conditioned rows span several decades with cancelling signs.  On
the closed-surface bilaplacian (cube-sphere, 24,576 elements) four slices (2^-32) gave
1e-5 normwise; five slices must keep it, and the heat operator at 40,960 elements,
within the mixed-precision bar of 1e-6 -- as close to FP64 as the compensated FP32
path (both then sit at the final FP32 rounding of the values).
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


def _nerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def W():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available()
    return wq


@pytest.mark.parametrize("case", ["sphere_bilaplacian", "heat_L5"])
def test_tc_on_ill_conditioned_operators(W, case):
    import torch
    ctx = W.Context(0)
    if case == "sphere_bilaplacian":
        mesh = meshes.cube_sphere(pre=3, levels=3)
        comps, op, alpha = [W.COMP_N, W.COMP_LAP], W.OP_BIHARM, 0.0
        cf = lambda x: 1.0 + 0.25 * x[:, 0] * x[:, 1] + 0.1 * x[:, 2]
    else:
        mesh = meshes.rotated(nx=8, ny=5, n_ep=12, levels=5, seed=2001)
        u0 = meshes.gaussian_bumps(4001, mesh["xyz"].min(0), mesh["xyz"].max(0))
        comps, op, alpha = [W.COMP_N, W.COMP_X, W.COMP_Y], W.OP_HEAT_S, 100.0
        cf = lambda x: 1.0 + u0(x) ** 2
    b = W.Basis(ctx, mesh)
    r = W.Rule(b, comps=comps)
    cq = torch.tensor(cf(r.points().cpu().numpy()), device="cuda")
    cg = torch.tensor(cf(r.gauss_points().cpu().numpy()), device="cuda")
    a64 = r.assemble(op, cq, alpha=alpha, prec=W.PREC_F64).cpu().numpy()
    a32 = r.assemble(op, cq, alpha=alpha, prec=W.PREC_F32).cpu().numpy()
    atc = r.assemble(op, cq, alpha=alpha, prec=W.PREC_TC).cpu().numpy()
    e32, etc = _nerr(a32, a64), _nerr(atc, a64)
    assert e32 < 1e-6 and etc < 1e-6, (case, e32, etc)
    assert etc < 4 * e32, (case, e32, etc)        # at the FP32 rounding, like the SIMT path
    g64 = r.gq_assemble(op, cg, alpha=alpha, prec=W.PREC_F64).cpu().numpy()
    gtc = r.gq_assemble(op, cg, alpha=alpha, prec=W.PREC_TC).cpu().numpy()
    assert _nerr(gtc, g64) < 1e-6, (case, _nerr(gtc, g64))
