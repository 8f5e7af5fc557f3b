"""cpu_ref (the multi-core FP64 CPU baseline) against the oracle, on the oracle's own
precomputed data: the WQ row-wise assembly reproduces the oracle's WQ matrices and the
element-wise Gauss assembly its Gauss matrices, to FP64 rounding, for one and for several
threads (the result does not depend on the thread count)."""
import os

import numpy as np
import pytest

from wq_synth import meshes


def nerr(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def data():
    from oracle.basis import Basis
    from oracle import wq as owq
    from oracle.gq import gauss_data
    import cpu_ref
    B = Basis(meshes.disk(mu=5, n=6))
    R = owq.Rule(B, ["N", "x", "y"])
    R.compute_weights()

    def block(d):                     # [P][comp][m] with comp = N, d_x, d_y, lap
        return np.stack([d["N"], d["grad"][..., 0], d["grad"][..., 1], d["lap"]], axis=1).transpose(2, 1, 0)

    fn_ptr = np.concatenate([[0], np.cumsum([len(B.elem_fns[e]) for e in range(B.E)])])
    fns = np.concatenate([B.elem_fns[e] for e in range(B.E)])
    supp_ptr, supp, il = cpu_ref.supports(fn_ptr, fns, B.n)
    assert all(np.array_equal(supp[supp_ptr[i]:supp_ptr[i + 1]], B.supp[i]) for i in range(B.n))
    wq_blocks = [block(R.data[e]).ravel() for e in range(B.E)]
    gdat = [gauss_data(B, e) for e in range(B.E)]
    g_blocks = [block(d).ravel() for d in gdat]
    pb = cpu_ref.Problem(
        row_ptr=R.row_ptr, col=R.col, fn_ptr=fn_ptr, fns=fns, supp_ptr=supp_ptr, supp=supp, il=il, w_ptr=R.w_ptr,
        w=np.stack([R.weights[c] for c in ("N", "x", "y")], axis=1), pt_ptr=R.pt_ptr,
        tab_ptr=np.concatenate([[0], np.cumsum([b.size for b in wq_blocks])]), table=np.concatenate(wq_blocks),
        gp_ptr=np.concatenate([[0], np.cumsum([d["w"].size for d in gdat])]),
        gtab_ptr=np.concatenate([[0], np.cumsum([b.size for b in g_blocks])]), gtable=np.concatenate(g_blocks),
        gw=np.concatenate([d["w"] for d in gdat]))
    gx = np.concatenate([d["x"] for d in gdat])
    return B, R, pb, gx


def test_cpu_ref_wq_matches_oracle(data):
    import cpu_ref
    B, R, pb, _ = data
    kap = meshes.kappa_sines(R.x)
    K = cpu_ref.wq_assemble(pb, 4, 3, [(1, 1, 0, 1.0), (2, 2, 0, 1.0)], kap)
    assert nerr(K, R.assemble([("x", kap), ("y", kap)])) < 1e-13
    M = cpu_ref.wq_assemble(pb, 4, 3, [(0, 0, -1, 2.5)])
    assert nerr(M, R.assemble([("N", np.full(R.Q, 2.5))])) < 1e-13


def test_cpu_ref_gauss_matches_oracle(data):
    import cpu_ref
    from oracle import gq
    B, R, pb, gx = data
    kg = meshes.kappa_sines(gx)
    K = cpu_ref.gq_assemble(pb, 4, [(1, 1, 0, 1.0), (2, 2, 0, 1.0)], kg)
    ref = gq.assemble(B, ["x", "y"], coef=meshes.kappa_sines, row_ptr=R.row_ptr, col=R.col)
    assert nerr(K, ref) < 1e-13


def test_cpu_ref_thread_count_does_not_change_the_result(data):
    import cpu_ref
    B, R, pb, gx = data
    kap = meshes.kappa_sines(R.x)
    kg = meshes.kappa_sines(gx)
    t0 = cpu_ref.threads()
    res = []
    for t in (1, 4):
        cpu_ref.set_threads(t)
        assert cpu_ref.threads() == t
        res.append((cpu_ref.wq_assemble(pb, 4, 3, [(1, 1, 0, 1.0), (2, 2, 0, 1.0)], kap),
                    cpu_ref.gq_assemble(pb, 4, [(1, 1, 0, 1.0), (2, 2, 0, 1.0)], kg)))
    cpu_ref.set_threads(t0)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
