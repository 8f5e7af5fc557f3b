"""Pins of the oracle's spline space against facts the paper and mathematics fix.

* Table 1 of the paper (functions per element type), every valence 3..8 and
  refinement level 0, 1, 2 (golden file tests/golden/table1_counts.txt).
* Partition of unity and geometric reproduction (Sec. 3: ASUTS has polynomial
  partition of unity; x = sum_j P_j N_j).
* EP-free meshes: the Bezier-net rule equals tensor-product clamped cubic
  B-splines evaluated by Cox-de Boor (scipy), i.e. the paper's "bicubic
  B-splines in regular elements" with zero knot spans at the boundary (Sec. 3).
* C1 across edges away from EPs, C0 everywhere.
* The Laplace-Beltrami form of Eq. 17 equals the planar chain rule on planar
  domains; on a surface, grad_G x = I - n n^T and lap_G x is normal.
* Linear independence (mass matrix positive definite).
"""
import os

import numpy as np
import pytest

from wq_synth import meshes
from oracle.basis import Basis
from oracle.topology import TYPE_NAMES, Topology, MeshError
from oracle.geometry import eval_element, planar_derivatives, locate
from oracle import gq

HERE = os.path.dirname(__file__)


def _table1():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "table1_counts.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, *cols = line.split()
        rows[t] = cols
    return rows


def _expected(entry, mu):
    if entry == "NA":
        return None
    out = set()
    for tok in entry.split("/"):
        out.add(eval(tok.replace("mu", "*%d" % mu).replace("3*", "3*")) if "mu" in tok else int(tok))
    return out


@pytest.mark.parametrize("mu", [3, 5, 6, 7, 8])
@pytest.mark.parametrize("level", [0, 1, 2])
def test_table1_counts(mu, level):
    B = Basis(meshes.disk(mu=mu, n=5, levels=level))
    found = {}
    for e in range(B.E):
        found.setdefault(TYPE_NAMES[B.etype[e]], set()).add(B.m(e))
    col = min(level, 2)
    table = _table1()
    for t, vals in found.items():
        exp = _expected(table[t][col], mu)
        assert exp is not None, (t, level)
        assert vals <= exp, (t, mu, level, vals, exp)
    # every type that must exist at this level does
    assert "irregular" in found and "regular" in found and "transition" in found
    if level >= 1:
        assert "enriched_transition" in found
    if level >= 2:
        assert "enriched_regular" in found


def _rand_theta(rng, P):
    return rng.uniform(0.02, 0.98, size=(P, 2))


@pytest.mark.parametrize("mesh", ["disk5", "disk3_L1", "rotated"])
def test_partition_of_unity_and_reproduction(mesh):
    m = {"disk5": lambda: meshes.disk(mu=5, n=6),
         "disk3_L1": lambda: meshes.disk(mu=3, n=4, levels=1),
         "rotated": lambda: meshes.rotated(levels=1)}[mesh]()
    B = Basis(m)
    rng = np.random.Generator(np.random.PCG64(7))
    for e in range(0, B.E, max(1, B.E // 60)):
        d = eval_element(B, e, theta=_rand_theta(rng, 6))
        assert np.max(np.abs(d["N"].sum(0) - 1.0)) < 1e-13
        assert np.max(np.abs(d["grad"].sum(0))) < 1e-10
        assert np.max(np.abs(d["lap"].sum(0))) < 1e-7 * (1 + np.max(np.abs(d["lap"])))
        P = B.ctrl[B.elem_fns[e]]
        assert np.max(np.abs(np.einsum("mk,mp->pk", P, d["N"]) - d["x"])) < 1e-13
        # grad x = I on the plane; lap x = 0
        G = np.einsum("mk,mpl->pkl", P[:, :2], d["grad"][..., :2])
        assert np.max(np.abs(G - np.eye(2))) < 1e-9
        L = np.einsum("mk,mp->pk", P[:, :2], d["lap"])
        scale = np.max(np.abs(d["lap"])) + 1
        assert np.max(np.abs(L)) < 1e-9 * scale


def test_cox_de_boor_on_grid():
    from scipy.interpolate import BSpline
    nx, ny = 5, 4
    m = meshes.grid(nx, ny)
    B = Basis(m)
    assert not B.topo.is_ep.any()
    xyz = m["xyz"]
    ab = np.rint(xyz[:, :2] * nx).astype(int) + 1           # wrap column/row -> 0
    Tu = np.r_[[0, 0, 0], np.arange(nx + 1), [nx, nx, nx]].astype(float)
    Tv = np.r_[[0, 0, 0], np.arange(ny + 1), [ny, ny, ny]].astype(float)
    rng = np.random.Generator(np.random.PCG64(3))
    raw = B.raw_ids
    for e, f in enumerate(B.elements):
        q = m["quads"][f]
        i0, j0 = ab[q[0]] - 1
        th = _rand_theta(rng, 5)
        d = eval_element(B, e, theta=th)
        u, v = i0 + th[:, 0], j0 + th[:, 1]
        for k, fn in enumerate(B.elem_fns[e]):
            a, b = ab[raw[fn]]
            Bu = BSpline.basis_element(Tu[a:a + 5], extrapolate=False)(u)
            Bv = BSpline.basis_element(Tv[b:b + 5], extrapolate=False)(v)
            ref = np.nan_to_num(Bu) * np.nan_to_num(Bv)
            assert np.max(np.abs(d["N"][k] - ref)) < 1e-14
        # every function active on the element shows up
        assert B.m(e) == 16


UV = np.array([(0, 0), (1, 0), (1, 1), (0, 1)], dtype=float)


def _edge_points(k, s):
    return UV[k][None] + s[:, None] * (UV[(k + 1) % 4] - UV[k])[None]


@pytest.mark.parametrize("mu,level", [(5, 1), (3, 0), (7, 2)])
def test_continuity_across_edges(mu, level):
    m = meshes.disk(mu=mu, n=4, levels=level)
    B = Basis(m)
    T = B.topo
    e_of = {f: e for e, f in enumerate(B.elements)}
    s = np.array([0.13, 0.37, 0.62, 0.88])
    worst_c0, worst_c1 = 0.0, 0.0
    for f in B.elements:
        for k in range(4):
            nb = T.nb[f][k]
            if nb is None or nb[0] not in e_of or nb[0] < f:
                continue
            g, kg = nb
            ef, eg = e_of[f], e_of[g]
            da = eval_element(B, ef, theta=_edge_points(k, s))
            db = eval_element(B, eg, theta=_edge_points(kg, 1 - s))
            assert np.max(np.abs(da["x"] - db["x"])) < 1e-13
            fa, fb = list(B.elem_fns[ef]), list(B.elem_fns[eg])
            for j in set(fa) | set(fb):
                va = da["N"][fa.index(j)] if j in fa else 0.0
                vb = db["N"][fb.index(j)] if j in fb else 0.0
                worst_c0 = max(worst_c0, np.max(np.abs(va - vb)))
                near_ep = T.irregular[f] or T.irregular[g]
                if not near_ep:
                    ga = da["grad"][fa.index(j)] if j in fa else 0.0
                    gb = db["grad"][fb.index(j)] if j in fb else 0.0
                    worst_c1 = max(worst_c1, np.max(np.abs(ga - gb)))
    assert worst_c0 < 1e-13
    assert worst_c1 < 1e-9


def test_planar_laplacian_two_routes():
    B = Basis(meshes.disk(mu=5, n=6))
    rng = np.random.Generator(np.random.PCG64(11))
    for e in range(0, B.E, 9):
        th = _rand_theta(rng, 3)
        d = eval_element(B, e, theta=th)
        g2, l2 = planar_derivatives(B, e, th)
        assert np.max(np.abs(d["grad"][..., :2] - g2)) < 1e-10 * (1 + np.max(np.abs(g2)))
        assert np.max(np.abs(d["lap"] - l2)) < 1e-9 * (1 + np.max(np.abs(l2)))


def test_surface_identities():
    m = meshes.cube_sphere(pre=1, levels=1)
    B = Basis(m)
    assert B.topo.is_ep.sum() == 8 and not B.topo.passive.any()
    rng = np.random.Generator(np.random.PCG64(5))
    for e in range(0, B.E, 5):
        th = _rand_theta(rng, 4)
        d = eval_element(B, e, theta=th)
        P = B.ctrl[B.elem_fns[e]]
        sub, xi = locate(B.elem_coef[e].shape[1], th)
        from oracle.geometry import _tensor_derivs
        _, Xu, Xv, _, _, _ = [a[0] for a in _tensor_derivs(B.geom[e][None], sub, xi)]
        n = np.cross(Xu, Xv)
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        G = np.einsum("mk,mpl->pkl", P, d["grad"])
        Pt = np.eye(3)[None] - n[:, :, None] * n[:, None, :]
        assert np.max(np.abs(G - Pt)) < 1e-9
        L = np.einsum("mk,mp->pk", P, d["lap"])
        tang = L - np.sum(L * n, axis=1, keepdims=True) * n
        assert np.max(np.abs(tang)) < 1e-7 * (1 + np.max(np.abs(L)))


def test_linear_independence():
    B = Basis(meshes.disk(mu=5, n=6))
    rp, col = gq.pattern(B)
    Mv = gq.assemble(B, ["N"], row_ptr=rp, col=col)
    Md = gq.to_dense(B.n, rp, col, Mv)
    assert np.min(np.linalg.eigvalsh(Md)) > 1e-10


def test_ep_near_boundary_rejected():
    # with one face ring per sector every face touches the boundary, so the EP
    # is a vertex of a passive element (not allowed, Sec. 3 assumptions)
    m = meshes.disk(mu=5, n=1)
    with pytest.raises(MeshError):
        Topology(m["xyz"], m["quads"], m["level0_face"])
