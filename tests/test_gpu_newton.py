"""Newton iterations of the nonlinear heat problem (Sec. 5.2, theta = 1) with the
re-assembly of every iteration replayed from one CUDA graph, through the C ABI.

k(u) = 1 + u^2, f = 0, homogeneous Dirichlet data on the functions of boundary
vertices, u0 a sum of 8 Gaussian bumps (amplitude 0.5), dt = 1e-2 on the 640-element
mesh (from 2,560 elements up this step is too long for Newton from u_old; the
40,960-element run uses dt = 1e-4).  The residual is
always FP64; the tangent is the exact derivative of the WQ residual (WQ_OP_HEAT_J) in
FP64, or assembled in a mixed mode (compensated FP32, tensor-core bf16 slices with FP32
sums).  Checks: the FP64 tangent converges quadratically; every tangent drives the
relative residual below 1e-8 within 20 iterations; the converged solution is the
oracle's (its own Newton iteration with its exact tangent) to 1e-8.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu

DT = 1e-2


@pytest.fixture(scope="module")
def problem():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from paper_2605_29334_gb300 import build, wq
    from paper_2605_29334_gb300.newton import boundary_fixed
    from oracle.basis import Basis
    from oracle import wq as owq
    build.build()
    mesh = meshes.rotated(nx=8, ny=5, n_ep=12, levels=2, seed=2001)
    u0f = meshes.gaussian_bumps(4001, mesh["xyz"].min(0), mesh["xyz"].max(0))
    ctx = wq.Context(0)
    b = wq.Basis(ctx, mesh)
    r = wq.Rule(b, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y])
    fixed = boundary_fixed(b, mesh)
    # the oracle's converged solution (its exact tangent, 8 iterations)
    B = Basis(mesh)
    R = owq.Rule(B, ["N", "x", "y"])
    R.compute_weights()
    kap, dkap = (lambda v: 1.0 + v * v), (lambda v: 2.0 * v)
    u_old = u0f(B.ctrl)
    u_old[fixed] = 0.0
    u = u_old.copy()
    free = np.nonzero(~fixed)[0]
    for _ in range(8):
        res = R.heat_residual(u, u_old, DT, kap)
        res[fixed] = 0.0
        J = sp.csr_matrix((R.assemble(R.heat_tangent(u, DT, kap, dkap, exact=True)), R.col, R.row_ptr),
                          shape=(B.n, B.n))
        d = np.zeros(B.n)
        d[free] = spla.spsolve(J[free][:, free].tocsc(), -res[free])
        u = u + d
    return wq, r, fixed, u0f(b.ctrl()), u


@pytest.mark.parametrize("prec", ["f64", "f32", "tc"])
def test_newton_converges_to_the_oracle_solution(problem, prec, record_property):
    from paper_2605_29334_gb300.newton import HeatNewton
    wq, r, fixed, u0, u_ref = problem
    p = {"f64": wq.PREC_F64, "f32": wq.PREC_F32, "tc": wq.PREC_TC}[prec]
    nt = HeatNewton(r, fixed, DT, tangent=wq.OP_HEAT_J, prec=p)
    out = nt.run(u0, iters=20)
    h = np.array(out["residual"]) / out["residual"][0]
    k8 = int(np.argmax(h < 1e-8)) if np.any(h < 1e-8) else -1
    record_property("iteration_below_1e-8", k8)
    record_property("final_relative_residual", float(nt.residual_norm() / out["residual"][0]))
    print(prec, "relative residuals", " ".join("%.1e" % v for v in h[:10]), "| first below 1e-8:", k8)
    assert 0 < k8 <= 10
    if prec == "f64":
        # quadratic: once below 1e-2 each step squares the error (up to a modest constant)
        for k in range(1, k8):
            if h[k - 1] < 1e-2:
                assert h[k] <= 50.0 * h[k - 1] ** 2, (k, h[k - 1], h[k])
    u = nt.u.cpu().numpy()
    assert np.max(np.abs(u - u_ref)) <= 1e-8 * np.max(np.abs(u_ref))


def test_newton_graph_replay_matches_eager(problem):
    """The captured re-assembly reproduces the eager one bit for bit."""
    import torch
    from paper_2605_29334_gb300.newton import HeatNewton
    wq, r, fixed, u0, _ = problem
    nt = HeatNewton(r, fixed, DT, tangent=wq.OP_HEAT_J, prec=wq.PREC_F32)
    nt.u.copy_(torch.tensor(u0, device="cuda"))
    nt.u_old.copy_(nt.u * 0.9)
    nt.capture()
    nt.graph.replay()
    torch.cuda.synchronize()
    g = (nt.res.clone(), nt.vals.clone())
    nt._reassemble()
    torch.cuda.synchronize()
    assert torch.equal(g[0], nt.res) and torch.equal(g[1], nt.vals)
