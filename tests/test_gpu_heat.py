"""Nonlinear heat transfer (paper Sec. 5): Newton iterations with WQ residual
and WQ symmetric tangent S, on the GPU through the C ABI, against the oracle's
own Newton iterations.

kappa(u) = 1 + u^2, f = 0, one backward-Euler step (theta = 1), homogeneous
Dirichlet data on the functions of boundary vertices, u0 a sum of 8 Gaussian
bumps.  The GPU side: wq_heat_fields -> wq_apply (residual) -> wq_assemble
(WQ_OP_HEAT_S) -> linear solve (harness) -> update; the re-assembly part of one
iteration is also captured in a CUDA graph and replayed.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu

DT = 1e-2


def _setup_mesh():
    mesh = meshes.rotated(nx=8, ny=5, n_ep=12, levels=2, seed=2001)
    u0f = meshes.gaussian_bumps(4001, mesh["xyz"].min(0), mesh["xyz"].max(0))
    bnd = set()
    q = mesh["quads"]
    from collections import Counter
    cnt = Counter()
    for f in q:
        for k in range(4):
            a, b = int(f[k]), int(f[(k + 1) % 4])
            cnt[(min(a, b), max(a, b))] += 1
    for (a, b), c in cnt.items():
        if c == 1:
            bnd.update((a, b))
    return mesh, u0f, bnd


def _oracle_newton(mesh, u0f, bnd, iters):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from oracle.basis import Basis
    from oracle import wq as owq
    B = Basis(mesh)
    R = owq.Rule(B, ["N", "x", "y"])
    R.compute_weights()
    fixed = np.array([rid < len(mesh["xyz"]) and rid in bnd for rid in B.raw_ids])
    u_old = u0f(B.ctrl)
    u_old[fixed] = 0.0
    u = u_old.copy()
    hist = []
    for _ in range(iters):
        res = R.heat_residual(u, u_old, DT, lambda v: 1.0 + v * v)
        res[fixed] = 0.0
        hist.append(np.linalg.norm(res))
        uq, _g = R.interp(u)
        kq = 1.0 + uq * uq
        vals = R.assemble([("N", np.full(R.Q, 1.0 / DT)), ("x", kq), ("y", kq)])
        S = sp.csr_matrix((vals, R.col, R.row_ptr), shape=(B.n, B.n))
        free = np.nonzero(~fixed)[0]
        d = np.zeros(B.n)
        d[free] = spla.spsolve(S[free][:, free].tocsc(), -res[free])
        u = u + d
    return u, np.array(hist), fixed


def test_newton_matches_oracle_and_graph_replay():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    mesh, u0f, bnd = _setup_mesh()
    iters = 7
    u_ref, hist_ref, fixed = _oracle_newton(mesh, u0f, bnd, iters)

    ctx = wq.Context(0)
    b = wq.Basis(ctx, mesh)
    r = wq.Rule(b, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y])
    raw = b.raw_ids()
    fixed_g = np.array([rid < len(mesh["xyz"]) and rid in bnd for rid in raw])
    assert np.array_equal(fixed_g, fixed)
    ctrl = b.ctrl()
    u_old_h = u0f(ctrl)
    u_old_h[fixed_g] = 0.0
    u_old = torch.tensor(u_old_h, device="cuda")
    u = u_old.clone()
    free = torch.tensor(np.nonzero(~fixed_g)[0], device="cuda")
    rp, col = r.pattern()
    crow, ccol = rp.to(torch.int64), col.to(torch.int64)
    kappa = torch.empty(r.Q, dtype=torch.float64, device="cuda")
    g = torch.empty((3, r.Q), dtype=torch.float64, device="cuda")
    res = torch.empty(r.n, dtype=torch.float64, device="cuda")
    vals = torch.empty(r.nnz, dtype=torch.float64, device="cuda")

    def reassemble():
        r.heat_fields(u, u_old, DT, 1.0, 1.0, 0.0, kappa=kappa, g=g)
        r.apply([wq.COMP_N, wq.COMP_X, wq.COMP_Y], g, out=res)
        r.assemble(wq.OP_HEAT_S, kappa, alpha=1.0 / DT, out=vals)

    hist = []
    for _ in range(iters):
        reassemble()
        res[torch.tensor(fixed_g, device="cuda")] = 0.0
        hist.append(float(torch.linalg.norm(res)))
        S = torch.sparse_csr_tensor(crow, ccol, vals, size=(r.n, r.n)).to_dense()
        d = torch.zeros(r.n, dtype=torch.float64, device="cuda")
        d[free] = torch.linalg.solve(S[free][:, free], -res[free])
        u += d
    hist = np.array(hist)
    # same Newton history and solution as the oracle (FP64 path)
    assert np.max(np.abs(hist - hist_ref) / hist_ref[0]) < 1e-9
    assert np.max(np.abs(u.cpu().numpy() - u_ref)) < 1e-9 * np.max(np.abs(u_ref))
    assert hist[-1] < 1e-8 * hist[0]

    # the re-assembly of one iteration, captured in a CUDA graph, replays to the same values
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        reassemble()
    torch.cuda.current_stream().wait_stream(s)
    eager = (res.clone(), vals.clone(), kappa.clone())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        reassemble()
    res.zero_(), vals.zero_(), kappa.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(res, eager[0]) and torch.equal(vals, eager[1]) and torch.equal(kappa, eager[2])


def test_exact_tangent_newton_on_surface():
    """NEXT-1: nonlinear heat on a closed surface (cube-sphere, 8 valence-3 EPs,
    surface gradients with three components), Newton with the exact tangent
    WQ_OP_HEAT_J (the derivative of the WQ residual, Sec. 5.2): the GPU history
    matches the oracle's, and convergence is quadratic where the symmetric S alone
    converges only linearly."""
    import torch
    from oracle.basis import Basis
    from oracle import wq as owq
    from paper_2605_29334_gb300 import build, wq
    build.build()
    mesh = meshes.cube_sphere(pre=2, levels=1)
    u0f = meshes.gaussian_bumps(4101, mesh["xyz"].min(0), mesh["xyz"].max(0), amp=0.8)
    dt = 0.05
    kap = lambda v: 1.0 + v * v
    dkap = lambda v: 2.0 * v
    # oracle Newton, exact tangent
    B = Basis(mesh)
    R = owq.Rule(B, ["N", "x", "y", "z"])
    R.compute_weights()
    u_old = u0f(B.ctrl)
    u = u_old.copy()
    hist_ref = []
    for _ in range(5):
        res = R.heat_residual(u, u_old, dt, kap)
        hist_ref.append(np.linalg.norm(res))
        J = gq_dense(B.n, R.row_ptr, R.col, R.assemble(R.heat_tangent(u, dt, kap, dkap, exact=True)))
        u = u - np.linalg.solve(J, res)
    hist_ref = np.array(hist_ref)
    # GPU Newton, exact tangent
    ctx = wq.Context(0)
    b = wq.Basis(ctx, mesh)
    r = wq.Rule(b, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y, wq.COMP_Z])
    ug = torch.tensor(u0f(b.ctrl()), device="cuda")
    uo = ug.clone()
    rp, col = r.pattern()
    crow, ccol = rp.to(torch.int64), col.to(torch.int64)
    hist = []
    for _ in range(5):
        kc, g = r.heat_fields(ug, uo, dt, 1.0, 1.0, 0.0, jacobian=True)
        res = r.apply([wq.COMP_N, wq.COMP_X, wq.COMP_Y, wq.COMP_Z], g)
        hist.append(float(torch.linalg.norm(res)))
        vals = r.assemble(wq.OP_HEAT_J, kc, alpha=1.0 / dt)
        Jg = torch.sparse_csr_tensor(crow, ccol, vals, size=(r.n, r.n)).to_dense()
        ug = ug - torch.linalg.solve(Jg, res)
    hist = np.array(hist)
    assert np.max(np.abs(hist - hist_ref) / hist_ref[0]) < 1e-9, (hist, hist_ref)
    # quadratic convergence: each step at most ~ the square of the previous (relative)
    rel = hist / hist[0]
    assert rel[1] < 0.5 and rel[4] < 1e-8, rel
    assert rel[3] < 10 * rel[2] ** 2 and rel[4] < 10 * rel[3] ** 2 + 1e-14, rel
    # the symmetric S alone converges linearly on the same problem
    us = torch.tensor(u0f(b.ctrl()), device="cuda")
    hs = []
    for _ in range(5):
        kc, g = r.heat_fields(us, uo, dt, 1.0, 1.0, 0.0)
        res = r.apply([wq.COMP_N, wq.COMP_X, wq.COMP_Y, wq.COMP_Z], g)
        hs.append(float(torch.linalg.norm(res)))
        vals = r.assemble(wq.OP_HEAT_S, kc, alpha=1.0 / dt)
        Sg = torch.sparse_csr_tensor(crow, ccol, vals, size=(r.n, r.n)).to_dense()
        us = us - torch.linalg.solve(Sg, res)
    assert hs[4] / hs[0] > 1e3 * rel[4], (hs, hist)


def gq_dense(n, row_ptr, col, vals):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[row_ptr[i]:row_ptr[i + 1]]] = vals[row_ptr[i]:row_ptr[i + 1]]
    return A
