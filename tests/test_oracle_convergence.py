"""Approximation order of the refined spaces (Sec. 3 refinement, Sec. 6.1: bicubic
ASUTS converge at the optimal rate, 4 in L2, and WQ does not compromise it).

The L2 projection of a smooth function onto the space of a mesh refined three
times by the oracle's refinement (Sec. 3) is computed twice: with the Gauss mass
matrix and load vector, and with the WQ ones (weights from the oracle's truncated
SVD, load vector sum_q w_iq f(x_q)).  Bicubic splines approximate smooth functions
to O(h^4) in L2, so halving h divides the error by 16: the observed rate must
approach 4 on both, and the WQ error must stay within a few percent of the Gauss
one.  This pins the approximation power of the refined spaces (the enrichment and
D-patch construction on meshes produced by the refinement: a function missing from
the space or a broken partition of unity stops the convergence) and that the WQ
projection, a Petrov-Galerkin projection with the point functionals
sum_q w_iq (.)(x_q), keeps it.  It is not a fine check of the weights themselves:
both sides of that projection use the same weights, and random relative errors of
1e-2 in them leave the rate and the ratio within the bars (the exactness and KKT
pins in test_oracle_wq.py check the weights).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from wq_synth import meshes
from oracle.basis import Basis
from oracle.refine import refine
from oracle import gq, wq


def _f(x):
    return np.sin(2.0 * x[:, 0] + 0.5) * np.cos(1.5 * x[:, 1]) + 0.3 * x[:, 0] ** 2


def _projection_errors(B):
    rp, col = gq.pattern(B)
    gd = [gq.gauss_data(B, e) for e in range(B.E)]
    M = sp.csr_matrix((gq.assemble(B, ["N"], row_ptr=rp, col=col, gdata=gd), col, rp), shape=(B.n, B.n))
    b = np.zeros(B.n)
    for e in range(B.E):
        b[B.elem_fns[e]] += gd[e]["N"] @ (gd[e]["w"] * _f(gd[e]["x"]))
    R = wq.Rule(B, ["N"])
    R.compute_weights(gdata=gd)
    Mw = sp.csr_matrix((R.assemble([("N", np.ones(R.Q))]), R.col, R.row_ptr), shape=(B.n, B.n))
    bw = np.array([R.weights["N"][R.w_ptr[i]:R.w_ptr[i + 1]] @ _f(R.x[R.row_points(i)]) for i in range(B.n)])

    def l2(c):
        return np.sqrt(sum(np.sum(gd[e]["w"] * (c[B.elem_fns[e]] @ gd[e]["N"] - _f(gd[e]["x"])) ** 2)
                           for e in range(B.E)))
    return l2(sla.spsolve(M.tocsc(), b)), l2(sla.spsolve(Mw.tocsc(), bw))


@pytest.mark.parametrize("mu", [3, 5])
def test_projection_converges_at_order_four(mu):
    m = meshes.disk(mu=mu, n=4)
    eg, ew = [], []
    for level in range(4):
        a, b = _projection_errors(Basis(m))
        eg.append(a)
        ew.append(b)
        if level < 3:
            m = refine(m)
    rg = np.log2(np.array(eg[:-1]) / np.array(eg[1:]))
    rw = np.log2(np.array(ew[:-1]) / np.array(ew[1:]))
    assert np.all(np.diff(rg) > 0) and rg[-1] > 3.8, rg       # pre-asymptotic, rising towards 4
    assert np.all(np.diff(rw) > 0) and rw[-1] > 3.8, rw
    assert ew[-1] < 1.05 * eg[-1], (ew[-1], eg[-1])
