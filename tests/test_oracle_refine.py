"""Pins of the oracle's global refinement (paper Sec. 3: knot insertion for
vertex-based control points, de Casteljau for face-based ones, the enriched
region keeping its size, nested or nearly nested spaces).

* One-dimensional insertion against scipy's FITPACK ``insert`` on clamped knot
  vectors (the zero spans of the passive ring) and on non-uniform spans.
* The uniform interior case against the Catmull-Clark masks of a bicubic
  B-spline (vertex 1/64 [1 6 1; 6 36 6; 1 6 1], edge 1/16 [1 6 1] x [1 1],
  face 1/4).
* EP-free grid with its passive ring: every fine control point equals the
  tensor product of the FITPACK insertions.
* Random control points (a random element of the space): the fine geometry
  equals the coarse geometry at the same parameters on every face without an EP
  corner and on the child of an irregular face opposite its EP, and stays close
  on the children that touch a spoke; twice in a row.
* Refined meshes reproduce Table 1's function counts per element type.
"""
import os

import numpy as np
import pytest

from wq_synth import meshes
from oracle.basis import Basis
from oracle.geometry import eval_element
from oracle.refine import insert_midpoints_1d, refine
from oracle.topology import TYPE_NAMES

HERE = os.path.dirname(__file__)


def _fitpack_refinement(knots):
    """Matrix R [n', n] with fine coefficients = R @ coarse, inserting the midpoint
    of every non-zero span of the clamped cubic knot vector ``knots``."""
    from scipy.interpolate import insert
    n = len(knots) - 4
    mids = [0.5 * (a + b) for a, b in zip(knots[:-1], knots[1:]) if b > a]
    cols = []
    for j in range(n):
        c = np.zeros(n)
        c[j] = 1.0
        tck = (np.asarray(knots, dtype=float), np.r_[c, np.zeros(4)], 3)
        for x in mids:
            tck = insert(x, tck)
        cols.append(np.asarray(tck[1])[:len(tck[0]) - 4])
    return np.stack(cols, axis=1)


def _rule_refinement(vknots):
    """The same matrix from insert_midpoints_1d, one fine point at a time.
    vknots[j] = knot of control point d_j (clamped: repeated at both ends)."""
    n = len(vknots)
    span = np.diff(vknots)                       # span[j] = t_{j+1} - t_j
    get = lambda j: float(span[j]) if 0 <= j < n - 1 else 0.0
    rows = []
    for j in range(n):
        wV, wE = insert_midpoints_1d((get(j - 2), get(j - 1), get(j), get(j + 1)))
        r = np.zeros(n)
        for o, w in zip((-1, 0, 1), wV):
            if w != 0.0:
                r[j + o] += w
        rows.append(r)
        if wE is not None:
            r = np.zeros(n)
            r[j], r[j + 1] = wE
            rows.append(r)
    return np.stack(rows)


@pytest.mark.parametrize("spans", [
    [1, 1, 1, 1, 1],
    [1, 2, 0.5, 1.5, 1, 3],
    [0.3, 1.7, 2.2, 0.9],
])
def test_insertion_matches_fitpack(spans):
    inner = np.r_[0.0, np.cumsum(spans)]
    knots = np.r_[[inner[0]] * 3, inner, [inner[-1]] * 3]
    R_ref = _fitpack_refinement(knots)
    # control point d_j of the clamped spline belongs to knot knots[j + 2]
    vknots = knots[2:len(knots) - 2]
    R = _rule_refinement(vknots)
    assert R.shape == R_ref.shape
    assert np.max(np.abs(R - R_ref)) < 1e-14


def _random_xyz(m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = dict(m)
    out["xyz"] = rng.uniform(-1.0, 1.0, size=m["xyz"].shape)
    return out


def test_catmull_clark_masks_on_uniform_interior():
    m = meshes.grid(8, 8)
    mr = _random_xyz(m, 11)
    fine = refine(mr)
    X, Xc = fine["xyz"], mr["xyz"]
    ab = np.rint(m["xyz"][:, :2] * 8).astype(int) + 1
    vid = {tuple(a): i for i, a in enumerate(ab)}
    # coarse vertex (5, 5): deep in the interior (all spans 1 within two rings)
    P = lambda a, b: Xc[vid[(a, b)]]
    v = vid[(5, 5)]
    cc = (36 * P(5, 5) + 6 * (P(4, 5) + P(6, 5) + P(5, 4) + P(5, 6))
          + P(4, 4) + P(6, 4) + P(4, 6) + P(6, 6)) / 64
    assert np.max(np.abs(X[v] - cc)) < 1e-15
    # edge (5,5)-(6,5) and face (5,5)-(6,6): find their fine vertices by position
    mf = refine(m)
    pos = lambda a, b: (np.array([a, b]) - 1) / 8.0
    def fine_at(p):
        d = np.linalg.norm(mf["xyz"][:, :2] - p[None], axis=1)
        i = int(np.argmin(d))
        assert d[i] < 1e-12
        return i
    e = fine_at(0.5 * (pos(5, 5) + pos(6, 5)))
    ce = (6 * (P(5, 5) + P(6, 5)) + P(5, 4) + P(6, 4) + P(5, 6) + P(6, 6)) / 16
    assert np.max(np.abs(X[e] - ce)) < 1e-15
    f = fine_at(0.25 * (pos(5, 5) + pos(6, 5) + pos(6, 6) + pos(5, 6)))
    cf = (P(5, 5) + P(6, 5) + P(6, 6) + P(5, 6)) / 4
    assert np.max(np.abs(X[f] - cf)) < 1e-15


def _greville(knots):
    return np.array([(knots[k + 1] + knots[k + 2] + knots[k + 3]) / 3.0 for k in range(len(knots) - 4)])


def _refined_knots(knots):
    mids = [0.5 * (a + b) for a, b in zip(knots[:-1], knots[1:]) if b > a]
    return np.sort(np.r_[knots, mids])


def test_grid_with_passive_ring_is_tensor_fitpack():
    nx, ny = 5, 4
    m = meshes.grid(nx, ny)
    h = 1.0 / nx
    Tu = np.r_[[0, 0, 0], np.arange(nx + 1), [nx, nx, nx]].astype(float)
    Tv = np.r_[[0, 0, 0], np.arange(ny + 1), [ny, ny, ny]].astype(float)
    cab = np.rint(m["xyz"][:, :2] / h).astype(int) + 1          # passive ring -> 0 and n + 2
    # fine grid indices: refine the Greville abscissae (knot insertion keeps linear
    # functions), whose fine values are the fine Greville abscissae
    gu, gv = _greville(Tu), _greville(Tv)
    mg = dict(m)
    mg["xyz"] = np.stack([gu[cab[:, 0]], gv[cab[:, 1]], np.zeros(len(cab))], axis=1)
    fg = refine(mg)["xyz"]
    fu, fv = _greville(_refined_knots(Tu)), _greville(_refined_knots(Tv))
    iu = {round(x, 9): i for i, x in enumerate(fu)}
    iv = {round(x, 9): i for i, x in enumerate(fv)}
    fab = np.array([(iu[round(x, 9)], iv[round(y, 9)]) for x, y in fg[:, :2]])
    mr = _random_xyz(m, 5)
    fine = refine(mr)
    C = np.zeros((nx + 3, ny + 3, 3))
    C[cab[:, 0], cab[:, 1]] = mr["xyz"]
    Ru, Rv = _fitpack_refinement(Tu), _fitpack_refinement(Tv)
    Cf = np.einsum("ia,abk,jb->ijk", Ru, C, Rv)
    # the fine mesh has every fine tensor index but the two missing corners of each
    # passive corner face (zero spans both ways: the corner face stays whole)
    assert len({tuple(a) for a in fab}) == len(fab)
    got = fine["xyz"]
    assert np.max(np.abs(got - Cf[fab[:, 0], fab[:, 1]])) < 1e-14


def _expected_exact(T, f, child):
    """Children reproduced exactly: any child of a face without an EP corner; the
    child opposite the EP of an irregular face."""
    eps = [c for c in range(4) if T.is_ep[T.quads[f][c]]]
    return all(child == (c + 2) % 4 for c in eps)


def _child_index(fine, fp):
    """Child position (coarse corner contained) of fine face fp."""
    off = fine["child_off"][fp]
    sc = fine["child_scale"][fp]
    if sc[0] == 0.5 and sc[1] == 0.5:
        return {(0.0, 0.0): 0, (0.5, 0.0): 1, (0.5, 0.5): 2, (0.0, 0.5): 3}[tuple(off)]
    return -1


def _check_reproduction(coarse, seed):
    Bc = Basis(coarse)
    fine = refine(coarse)
    Bf = Basis(fine)
    T = Bc.topo
    eidx = {f: e for e, f in enumerate(Bc.elements)}
    rng = np.random.Generator(np.random.PCG64(seed))
    scale = np.max(np.abs(Bc.raw_xyz))
    n_exact = n_near = 0
    worst_near = 0.0
    for ef, fp in enumerate(Bf.elements):
        f = int(fine["parent"][fp])
        th = rng.uniform(0.0, 1.0, size=(6, 2))
        xf = eval_element(Bf, ef, theta=th)["x"]
        xc = eval_element(Bc, eidx[f], theta=fine["child_off"][fp] + fine["child_scale"][fp] * th)["x"]
        err = np.max(np.abs(xf - xc)) / scale
        if _expected_exact(T, f, _child_index(fine, fp)):
            assert err < 1e-13, (f, fp, err)
            n_exact += 1
        else:
            worst_near = max(worst_near, err)
            n_near += 1
    return fine, n_exact, n_near, worst_near


@pytest.mark.parametrize("name", ["disk5", "disk3", "rotated", "grid", "sphere"])
def test_geometry_reproduced_twice(name):
    m = {"disk5": lambda: meshes.disk(mu=5, n=4),
         "disk3": lambda: meshes.disk(mu=3, n=4),
         "rotated": lambda: meshes.rotated(levels=1),
         "grid": lambda: meshes.grid(4, 3),
         "sphere": lambda: meshes.cube_sphere(pre=1, levels=1)}[name]()     # closed surface, 8 EPs
    coarse = _random_xyz(m, 21)
    fine, n_exact, n_near, worst = _check_reproduction(coarse, 1)
    n_irr = int(Basis(coarse).topo.irregular.sum())
    assert n_near == 3 * n_irr
    assert n_exact > 0
    assert worst < 1.0            # nearly nested: the spoke children move by a fraction of the data
    fine2, n_exact2, n_near2, _ = _check_reproduction(fine, 2)
    assert n_near2 == 3 * int(Basis(fine).topo.irregular.sum())


def test_fine_topology_counts():
    m = meshes.rotated(levels=0)
    Bc = Basis(m)
    fine = refine(m)
    Bf = Basis(fine)
    T, Tf = Bc.topo, Bf.topo
    assert Bf.E == 4 * Bc.E
    assert int(Tf.enriched.sum()) == 4 * int(T.enriched.sum())
    assert int(Tf.is_ep.sum()) == int(T.is_ep.sum())
    # one irregular child per EP corner of every irregular face
    assert int(Tf.irregular.sum()) == int(T.is_ep[T.quads].sum())
    assert len(fine["face_xyz"]) == 4 * int(Tf.enriched.sum())
    # passive ring: 1 x 2 per edge face, corner faces whole
    n_corner = int(((T.span[:, 0] == 0) & (T.span[:, 1] == 0)).sum())
    n_pass = int(T.passive.sum())
    assert int(Tf.passive.sum()) == 2 * (n_pass - n_corner) + n_corner


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
        out.add(eval(tok.replace("mu", "*%d" % mu)) if "mu" in tok else int(tok))
    return out


@pytest.mark.parametrize("mu", [3, 5, 6])
def test_table1_counts_on_refined_meshes(mu):
    m = meshes.disk(mu=mu, n=5)
    table = _table1()
    for level in (1, 2):
        m = refine(m)
        B = Basis(m)
        found = {}
        for e in range(B.E):
            found.setdefault(TYPE_NAMES[B.etype[e]], set()).add(B.m(e))
        for t, vals in found.items():
            exp = _expected(table[t][level], mu)
            assert exp is not None and vals <= exp, (t, level, vals, exp)
        assert "enriched_transition" in found
        if level == 2:
            assert "enriched_regular" in found
