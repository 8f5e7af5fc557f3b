"""Edge cases of the assembly through the C ABI.

* The smallest meshes: one active element (a 1 x 1 core in its passive ring: 16
  functions, every row's support a single element) and two; every precision mode
  against the oracle.
* A zero coefficient: every mode returns exact zeros (the compensated sums start
  from their extraction constant and must give it back exactly).
* A coefficient spanning 14 decades: the float modes stay within the metric's 1e-6
  of FP64 normwise, the tile-level extraction constant notwithstanding.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


def nerr(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.float64) - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def W():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available()
    return wq


@pytest.mark.parametrize("nx, ny", [(1, 1), (2, 1)])
def test_smallest_meshes_against_oracle(W, nx, ny):
    import torch
    from oracle.basis import Basis
    from oracle import wq as owq
    mesh = meshes.grid(nx, ny)
    ctx = W.Context(0)
    b = W.Basis(ctx, mesh)
    r = W.Rule(b, comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    B = Basis(mesh)
    R = owq.Rule(B, ["N", "x", "y"])
    R.compute_weights()
    assert (b.E, b.n, r.Q) == (B.E, B.n, R.Q)
    kap = meshes.kappa_sines(R.x)
    kd = torch.tensor(meshes.kappa_sines(r.points().cpu().numpy()), device="cuda")
    for op, terms in ((W.OP_MASS, [("N", kap)]), (W.OP_STIFF, [("x", kap), ("y", kap)])):
        ref = R.assemble(terms)
        assert nerr(r.assemble(op, kd, prec=W.PREC_F64).cpu().numpy(), ref) < 1e-11
        for prec in (W.PREC_F32, W.PREC_TC):
            assert nerr(r.assemble(op, kd, prec=prec).cpu().numpy(), ref) < 1e-6, (op, prec)
        assert nerr(r.gq_assemble(op, torch.tensor(meshes.kappa_sines(r.gauss_points().cpu().numpy()),
                                                   device="cuda"), prec=W.PREC_F64).cpu().numpy(),
                    owq.gq_assemble(B, [t[0] for t in terms], coef=meshes.kappa_sines, row_ptr=R.row_ptr,
                                    col=R.col)) < 1e-12


def test_zero_coefficient_gives_exact_zeros(W):
    import torch
    mesh = meshes.disk(mu=5, n=6)
    r = W.Rule(W.Basis(W.Context(0), mesh), comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    zq = torch.zeros(r.Q, dtype=torch.float64, device="cuda")
    zg = torch.zeros(r.G, dtype=torch.float64, device="cuda")
    for op in (W.OP_MASS, W.OP_STIFF):
        for prec in (W.PREC_F64, W.PREC_F32, W.PREC_F32_FAST, W.PREC_TC):
            assert not torch.any(r.assemble(op, zq, prec=prec) != 0), (op, prec)
            assert not torch.any(r.gq_assemble(op, zg, prec=prec) != 0), (op, prec)


def test_coefficient_over_fourteen_decades(W):
    import torch
    mesh = meshes.rotated(nx=8, ny=5, n_ep=12, levels=2, seed=2001)
    r = W.Rule(W.Basis(W.Context(0), mesh), comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    x = r.points().cpu().numpy()
    span = np.log(10.0) * 7.0
    g = (x[:, 0] - x[:, 0].mean()) / np.ptp(x[:, 0]) + (x[:, 1] - x[:, 1].mean()) / np.ptp(x[:, 1])
    kd = torch.tensor(np.exp(span * g), device="cuda")            # about 1e-7 .. 1e7
    assert float(kd.max() / kd.min()) > 1e13
    for op in (W.OP_MASS, W.OP_STIFF):
        ref = r.assemble(op, kd, prec=W.PREC_F64).cpu().numpy()
        for prec in (W.PREC_F32, W.PREC_TC):
            got = r.assemble(op, kd, prec=prec).cpu().numpy()
            assert nerr(got, ref) < 1e-6, (op, prec, nerr(got, ref))
