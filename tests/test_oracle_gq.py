"""Pins of the oracle's Gauss assembly (paper Sec. 6 reference, Table 2 GQ column).

* the 4-point rule equals numpy's Gauss-Legendre (a library routine) and is
  exact for degree 7;
* sum of all mass entries = area (partition of unity; det J has degree <= 5 per
  direction so 4 points are exact), cross-checked by Green's theorem on the
  boundary curve;
* stiffness row sums vanish (gradient of the partition of unity);
* symmetry;
* a single affine element: the closed-form Bernstein Gram matrix
  int_0^1 B^3_a B^3_b = C(3,a) C(3,b) / (7 C(6, a+b)), tensor product, mapped
  through the element's extraction;
* Table 3 arithmetic: GQ points = 16 E + 48 I reproduces the printed GQ column
  with E = 252 * 4^l and I = 8 (64 Gauss points per irregular element).
"""
import os
from math import comb

import numpy as np
import pytest

from wq_synth import meshes
from oracle.basis import Basis
from oracle.geometry import eval_element
from oracle import gq

HERE = os.path.dirname(__file__)


def test_gauss_rule_vs_library():
    x, w = gq.gauss4()
    t, wl = np.polynomial.legendre.leggauss(4)
    assert np.max(np.abs(x - 0.5 * (t + 1))) < 1e-15
    assert np.max(np.abs(w - 0.5 * wl)) < 1e-15
    for deg in range(8):
        assert abs(np.sum(w * x ** deg) - 1.0 / (deg + 1)) < 1e-15
    assert abs(np.sum(w * x ** 8) - 1.0 / 9) > 1e-8


def _area_green(B):
    """Area of the active domain from its boundary curve: 1/2 closed integral (x dy - y dx)."""
    T = B.topo
    e_of = {f: e for e, f in enumerate(B.elements)}
    t, wl = np.polynomial.legendre.leggauss(6)
    s, ws = 0.5 * (t + 1), 0.5 * wl
    UV = np.array([(0, 0), (1, 0), (1, 1), (0, 1)], dtype=float)
    area = 0.0
    for f, e in e_of.items():
        for k in range(4):
            nb = T.nb[f][k]
            if nb is not None and nb[0] in e_of:
                continue
            th = UV[k][None] + s[:, None] * (UV[(k + 1) % 4] - UV[k])[None]
            d = eval_element(B, e, theta=th)
            # tangent by the chain rule of the boundary parametrisation, finite-free:
            # differentiate the bicubic along the edge with a complex step
            h = 1e-20
            thc = th.astype(complex) + 1j * h * (UV[(k + 1) % 4] - UV[k])[None]
            from oracle.geometry import bernstein3
            sub = np.zeros(len(s), dtype=int)
            net = B.geom[e]
            if net.shape[0] == 4:
                raise RuntimeError("boundary edge on a split element")
            Bu = np.stack([(1 - thc[:, 0]) ** 3, 3 * thc[:, 0] * (1 - thc[:, 0]) ** 2,
                           3 * thc[:, 0] ** 2 * (1 - thc[:, 0]), thc[:, 0] ** 3], -1)
            Bv = np.stack([(1 - thc[:, 1]) ** 3, 3 * thc[:, 1] * (1 - thc[:, 1]) ** 2,
                           3 * thc[:, 1] ** 2 * (1 - thc[:, 1]), thc[:, 1] ** 3], -1)
            X = B.geom_ref[e][None, :] + np.einsum("ijk,pi,pj->pk", net[0], Bu, Bv)
            dx = X.imag / h
            x = d["x"]
            area += 0.5 * np.sum(ws * (x[:, 0] * dx[:, 1] - x[:, 1] * dx[:, 0]))
    return area


@pytest.mark.parametrize("make", [lambda: meshes.disk(mu=5, n=6), lambda: meshes.rotated(levels=1),
                                  lambda: meshes.grid(4, 3, jitter=0.1)])
def test_mass_sum_is_area(make):
    B = Basis(make())
    M = gq.assemble(B, ["N"])
    area = _area_green(B)
    assert abs(M.sum() - area) < 1e-12 * area


@pytest.mark.parametrize("make", [lambda: meshes.disk(mu=5, n=6), lambda: meshes.disk(mu=3, n=4, levels=1)])
def test_stiffness_rowsum_and_symmetry(make):
    B = Basis(make())
    rp, col = gq.pattern(B)
    for comps in (["x", "y"], ["x"], ["lap"]):
        K = gq.assemble(B, comps, row_ptr=rp, col=col)
        Kd = gq.to_dense(B.n, rp, col, K)
        assert np.max(np.abs(Kd - Kd.T)) <= 1e-15 * np.max(np.abs(Kd)) * 4
        assert np.max(np.abs(Kd.sum(1))) < 1e-11 * np.max(np.abs(Kd))
    Md = gq.to_dense(B.n, rp, col, gq.assemble(B, ["N"], row_ptr=rp, col=col))
    assert np.max(np.abs(Md - Md.T)) <= 4e-16 * np.max(np.abs(Md))


def test_affine_element_closed_form():
    B = Basis(meshes.grid(6, 6))
    G1 = np.array([[comb(3, a) * comb(3, b) / (7.0 * comb(6, a + b)) for b in range(4)] for a in range(4)])
    G2 = np.kron(G1, G1)            # index a*4+b  <->  (i along u, j along v)
    checked = 0
    for e in range(B.E):
        C = B.elem_coef[e][:, 0].reshape(B.m(e), 16)
        d = gq.gauss_data(B, e)
        if np.ptp(d["dA"]) > 1e-14 * np.max(d["dA"]):
            continue                     # not an affine element (clamped boundary layer)
        checked += 1
        area = np.sum(d["w"])
        Ke = (d["N"] * d["w"]) @ d["N"].T
        assert np.max(np.abs(Ke - area * C @ G2 @ C.T)) < 1e-16 + 1e-14 * np.max(np.abs(Ke))
    assert checked >= 4


def test_table3_gauss_count_identity():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "table3_points.txt")) if l[0] != "#"]
    for lvl, _wq, gqn in rows:
        E = 252 * 4 ** int(lvl)
        assert 16 * E + 48 * 8 == int(gqn)
    # the oracle's Gauss count on a mesh with I irregular elements follows the same rule
    B = Basis(meshes.disk(mu=5, n=6))
    nsub = np.array([B.elem_coef[e].shape[1] for e in range(B.E)])
    I = int(np.sum(B.topo.irregular[B.elements]))
    assert int(np.sum(16 * nsub)) == 16 * B.E + 48 * I


def test_mixed_terms_pin():
    """assemble_terms: a (c, c) term equals assemble([c]); swapping the test and
    trial components of a mixed term gives the transposed matrix (on the
    symmetric pattern S_i)."""
    from oracle.basis import Basis
    from oracle import gq
    B = Basis(meshes.disk(mu=5, n=4))
    rp, col = gq.pattern(B)
    kap = lambda x: 1.0 + 0.5 * np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1])
    a = gq.assemble(B, ["x"], coef=kap, row_ptr=rp, col=col)
    b = gq.assemble_terms(B, [("x", "x", kap)], row_ptr=rp, col=col)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(a))
    xn = gq.to_dense(B.n, rp, col, gq.assemble_terms(B, [("x", "N", kap)], row_ptr=rp, col=col))
    nx = gq.to_dense(B.n, rp, col, gq.assemble_terms(B, [("N", "x", kap)], row_ptr=rp, col=col))
    assert np.max(np.abs(xn - nx.T)) <= 1e-14 * np.max(np.abs(xn))
    assert np.max(np.abs(xn - xn.T)) > 1e-3 * np.max(np.abs(xn))      # genuinely non-symmetric
