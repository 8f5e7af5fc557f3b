"""One global refinement of a bicubic ASUTS control mesh (paper Sec. 3, Fig. 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3 gives the refinement in words: the irregular (enriched) region keeps its
size, vertex-based control points come from classical knot insertion and
face-based control points from de Casteljau's algorithm, so that the spaces are
nested or nearly nested.  The reading used here:

Topology
  * a face is halved in every direction whose knot span (Sec. 3: 1, or 0 across
    edges perpendicular to the boundary) is non-zero: active faces 2 x 2, faces of
    the passive ring 1 x 2 along the boundary, the passive corner faces (zero
    spans both ways) stay whole;
  * fine vertices: the coarse vertices [0, V); then one per split edge, in the
    order the edges are first met scanning faces f = 0..F-1 and their edges
    k = 0..3 (edge k joins corners k and k+1); then one per 2 x 2-split face, at
    its centre, in face order;
  * fine faces in coarse face order; the children of a 2 x 2 split are listed by
    the coarse corner they contain (0, 1, 2, 3), those of a 1 x 2 split by
    increasing coordinate; every child keeps its parent's orientation and
    inherits ``level0_face`` (the coarse face index when the coarse mesh is an
    initial mesh), so the enriched faces of the fine mesh are the children of the
    coarse enriched faces and the enriched region keeps its size.

Vertex-based control points: knot insertion
  Around the parent of a fine vertex (coarse vertex, edge or face) the mesh is a
  tensor-product chart: the two lines through a valence-4 vertex are its pairs
  of opposite edges, the knot spans along a line are its edge spans, and the
  spans beyond the chart are the cross spans of the neighbouring faces (0 beyond
  the boundary).  A cubic control point d_j belongs to the knot t_j (local knots
  t_{j-2} .. t_{j+2}).  In each direction the midpoints of the non-zero spans
  next to the parent are inserted with Boehm's algorithm, one knot at a time,
  and the fine control point is the tensor product of the two one-dimensional
  results.  A vertex of the outer boundary loop has zero spans on both sides
  across the boundary, so only the insertion along the loop acts on it.
  At an EP there is no tensor chart: the fine control point keeps the coarse
  position (the EP function is eliminated at every level, so the value enters
  no fine function).

Face-based control points: de Casteljau
  For every child of an enriched face, its four inner Bezier points: the
  parent's 4 x 4 Bezier net split at 1/2 in both directions by de Casteljau's
  algorithm (a split irregular parent: its four sub-nets after the D-patch
  treatment, which are the children's nets).

Consequence (pinned): where the coarse geometry is a bicubic spline with the
C1 averaging rules of the Bezier nets (every face without an EP corner), the
fine geometry equals the coarse geometry; the children of an irregular face that
touch one of its spokes are only nearly reproduced (their common corner on the
spoke is re-averaged).

Parity: pinned in tests/test_oracle_refine.py -- one-dimensional insertion
against scipy's FITPACK knot insertion on clamped knot vectors with zero spans,
the Catmull-Clark masks of the uniform bicubic case, exact reproduction of the
geometry (random control points) on every face that the reading above says is
reproduced, and Table 1's function counts on refined meshes.
"""
from __future__ import annotations

import numpy as np

from .basis import Basis, CORNER_UV
from .topology import MeshError, Topology


# ----------------------------------------------------------------------------
# one-dimensional knot insertion (Boehm), on a window d_{-2} .. d_2
# ----------------------------------------------------------------------------

def _boehm(P, tau, tbar):
    """Insert knot tbar into the cubic spline (control points P [n, ...], knots
    tau [n + 4], P_k supported on [tau_k, tau_{k+4}]).  Returns (P', tau')."""
    l = int(np.searchsorted(tau, tbar, side="right")) - 1       # tau_l <= tbar < tau_{l+1}
    n = len(P)
    out = []
    for k in range(n + 1):
        if k <= l - 3:
            out.append(P[k])
        elif k <= l:
            a = (tbar - tau[k]) / (tau[k + 3] - tau[k])
            out.append((1.0 - a) * P[k - 1] + a * P[k])
        else:
            out.append(P[k - 1])
    return np.array(out), np.insert(tau, l + 1, tbar)


def insert_midpoints_1d(spans):
    """Knot insertion around the control point d_0 of a cubic spline.

    spans = (D_{-2}, D_{-1}, D_0, D_1): the knot spans t_{j+1} - t_j for
    j = -2 .. 1 (d_j belongs to knot t_j).  The midpoints of D_{-1} and D_0 are
    inserted when non-zero.  Returns (wV, wE): the weights of (d_{-1}, d_0, d_1)
    in the fine control point at t_0, and of (d_0, d_1) in the fine control
    point at the midpoint of D_0 (None when D_0 = 0).
    """
    Dm2, Dm1, D0, D1 = (float(s) for s in spans)
    t = {0: 0.0, -1: -Dm1, 1: D0}
    t[-2] = t[-1] - Dm2
    t[2] = t[1] + D1
    # pads beyond the window: they reach only fine points that are not read
    t[-3], t[-4] = t[-2] - 1.0, t[-2] - 2.0
    t[3], t[4] = t[2] + 1.0, t[2] + 2.0
    P = np.eye(5)                          # P_k = d_{k-2}, k = 0..4, as weight vectors
    tau = np.array([t[j] for j in range(-4, 5)])   # tau_{k+2} = t_{k-2}
    i0 = 2                                 # index of d_0
    if Dm1 > 0:
        P, tau = _boehm(P, tau, 0.5 * (t[-1] + t[0]))
        i0 += 1
    iE = None
    if D0 > 0:
        P, tau = _boehm(P, tau, 0.5 * (t[0] + t[1]))
        iE = i0 + 1
    wV = P[i0]
    assert abs(wV[0]) < 1e-15 and abs(wV[4]) < 1e-15
    wE = None
    if iE is not None:
        wE = P[iE]
        assert abs(wE[0]) < 1e-15 and abs(wE[1]) < 1e-15 and abs(wE[4]) < 1e-15
        wE = wE[2:4]
    return wV[1:4], wE


# ----------------------------------------------------------------------------
# de Casteljau split of a 4 x 4 net at 1/2 in both directions -> 7 x 7
# ----------------------------------------------------------------------------

def _split_curve(b):
    b0, b1, b2, b3 = b
    b01, b12, b23 = 0.5 * (b0 + b1), 0.5 * (b1 + b2), 0.5 * (b2 + b3)
    b012, b123 = 0.5 * (b01 + b12), 0.5 * (b12 + b23)
    return [b0, b01, b012, 0.5 * (b012 + b123), b123, b23, b3]


def split_net(net):
    """net [4][4] (points) -> [7][7]; net[i][j], i along u, j along v."""
    cols = [_split_curve([net[i][j] for j in range(4)]) for i in range(4)]     # cols[i][y]
    out = [[None] * 7 for _ in range(7)]
    for y in range(7):
        row = _split_curve([cols[i][y] for i in range(4)])
        for x in range(7):
            out[x][y] = row[x]
    return out


# ----------------------------------------------------------------------------
# the refinement
# ----------------------------------------------------------------------------

def refine(mesh):
    """One global refinement of ``mesh`` (a ``wq_synth`` mesh dict, optionally with
    ``face_xyz``).  Returns the fine mesh dict (``xyz``, ``quads``,
    ``level0_face``, ``face_xyz``, ``dim``) plus, per fine face, ``parent``,
    ``child_off`` [2] and ``child_scale`` [2] (parent coordinates
    theta = child_off + child_scale * theta_child)."""
    B = Basis(mesh)
    T = B.topo
    q = T.quads
    V, F = T.V, T.F
    raw = B.raw_xyz
    xyz = raw[:V]

    # ---------------------------------------------------------------- topology
    esplit = {}
    for f in range(F):
        for k in range(4):
            a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
            key = (min(a, b), max(a, b))
            sp = float(T.span[f][k % 2])
            if key in esplit:
                if (esplit[key][1] > 0) != (sp > 0):
                    raise MeshError("edge (%d, %d) has inconsistent knot spans" % key)
                continue
            esplit[key] = (f, sp)
    mid = {}
    nv = V
    edge_parent = []                       # (face, edge k) of every edge midpoint
    for f in range(F):
        for k in range(4):
            a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
            key = (min(a, b), max(a, b))
            if esplit[key][1] > 0 and key not in mid:
                mid[key] = nv
                edge_parent.append((f, k))
                nv += 1
    centre = {}
    for f in range(F):
        if T.span[f][0] > 0 and T.span[f][1] > 0:
            centre[f] = nv
            nv += 1

    def m(f, k):
        a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
        return mid[(min(a, b), max(a, b))]

    l0_in = mesh.get("level0_face")
    quads, level0, parent, off, scale = [], [], [], [], []
    for f in range(F):
        c = [int(x) for x in q[f]]
        su, sv = T.span[f][0] > 0, T.span[f][1] > 0
        if su and sv:
            z = centre[f]
            kids = [((c[0], m(f, 0), z, m(f, 3)), (0.0, 0.0)), ((m(f, 0), c[1], m(f, 1), z), (0.5, 0.0)),
                    ((z, m(f, 1), c[2], m(f, 2)), (0.5, 0.5)), ((m(f, 3), z, m(f, 2), c[3]), (0.0, 0.5))]
            sc = (0.5, 0.5)
        elif su:
            kids = [((c[0], m(f, 0), m(f, 2), c[3]), (0.0, 0.0)), ((m(f, 0), c[1], c[2], m(f, 2)), (0.5, 0.0))]
            sc = (0.5, 1.0)
        elif sv:
            kids = [((c[0], c[1], m(f, 1), m(f, 3)), (0.0, 0.0)), ((m(f, 3), m(f, 1), c[2], c[3]), (0.0, 0.5))]
            sc = (1.0, 0.5)
        else:
            kids = [(tuple(c), (0.0, 0.0))]
            sc = (1.0, 1.0)
        for quad, o in kids:
            quads.append(quad)
            level0.append(int(l0_in[f]) if l0_in is not None else f)
            parent.append(f)
            off.append(o)
            scale.append(sc)

    # ------------------------------------------- vertex-based control points
    X = np.zeros((nv, 3))

    def nbr_cycle(v):
        """(neighbours n_k, diagonal g_k between n_k and n_{k+1}, fan faces) of interior v."""
        fan = T.fan(v)
        n = [int(q[f][(c + 1) % 4]) for f, c in fan]
        g = [int(q[f][(c + 2) % 4]) for f, c in fan]
        return n, g, fan

    def span_of(a, b):
        return esplit[(min(a, b), max(a, b))][1]

    # boundary loop neighbours (edges of one face)
    nface = {}
    for f in range(F):
        for k in range(4):
            a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
            key = (min(a, b), max(a, b))
            nface[key] = nface.get(key, 0) + 1
    bloop = {}
    for (a, b), cnt in nface.items():
        if cnt == 1:
            bloop.setdefault(a, []).append(b)
            bloop.setdefault(b, []).append(a)
    for v, lst in bloop.items():
        if len(lst) != 2:
            raise MeshError("boundary vertex %d has %d boundary edges" % (v, len(lst)))

    for v in range(V):
        if not (q == v).any():
            X[v] = xyz[v]
            continue
        if T.is_bnd_vertex[v]:
            # along the boundary loop; across it both spans are zero
            p, n = bloop[v]
            pp = [w for w in bloop[p] if w != v][0]
            nn = [w for w in bloop[n] if w != v][0]
            wV, _ = insert_midpoints_1d((span_of(pp, p), span_of(p, v), span_of(v, n), span_of(n, nn)))
            X[v] = wV[0] * xyz[p] + wV[1] * xyz[v] + wV[2] * xyz[n]
            continue
        if T.is_ep[v]:
            X[v] = xyz[v]
            continue
        n, g, fan = nbr_cycle(v)
        # beyond n_k along the line v -> n_k: cross span of fan face k across its edge (c+1)
        beyond = [T.cross_span(f, (c + 1) % 4) for f, c in fan]
        span = [span_of(v, n[k]) for k in range(4)]
        a, _ = insert_midpoints_1d((beyond[2], span[2], span[0], beyond[0]))   # (n2, v, n0)
        b, _ = insert_midpoints_1d((beyond[3], span[3], span[1], beyond[1]))   # (n3, v, n1)
        grid = {(0, 0): v, (1, 0): n[0], (0, 1): n[1], (-1, 0): n[2], (0, -1): n[3],
                (1, 1): g[0], (-1, 1): g[1], (-1, -1): g[2], (1, -1): g[3]}
        X[v] = sum(a[i + 1] * b[j + 1] * xyz[grid[(i, j)]] for i in (-1, 0, 1) for j in (-1, 0, 1))

    for (f, k) in edge_parent:
        w = mid[tuple(sorted((int(q[f][k]), int(q[f][(k + 1) % 4]))))]
        a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
        _, lam = insert_midpoints_1d((0.0, T.cross_span(f, (k + 3) % 4), float(T.span[f][k % 2]),
                                      T.cross_span(f, (k + 1) % 4)))
        rows = {0: (a, b), 1: (int(q[f][(k + 3) % 4]), int(q[f][(k + 2) % 4]))}
        nb = T.nb[f][k]
        across_g, beyond_g = 0.0, 0.0
        if nb is not None:
            g, kg = nb
            rows[-1] = (int(q[g][(kg + 2) % 4]), int(q[g][(kg + 3) % 4]))
            across_g = float(T.span[g][(kg + 1) % 2])
            beyond_g = T.cross_span(g, (kg + 2) % 4)
        beta, _ = insert_midpoints_1d((beyond_g, across_g, float(T.span[f][(k + 1) % 2]),
                                       T.cross_span(f, (k + 2) % 4)))
        val = np.zeros(3)
        for r in (-1, 0, 1):
            if beta[r + 1] == 0.0:
                continue
            if r not in rows:
                raise MeshError("edge (%d, %d): knot insertion needs a missing row" % (a, b))
            ra, rb = rows[r]
            val += beta[r + 1] * (lam[0] * xyz[ra] + lam[1] * xyz[rb])
        X[w] = val

    for f, z in centre.items():
        _, lu = insert_midpoints_1d((0.0, T.cross_span(f, 3), float(T.span[f][0]), T.cross_span(f, 1)))
        _, lv = insert_midpoints_1d((0.0, T.cross_span(f, 0), float(T.span[f][1]), T.cross_span(f, 2)))
        c = [int(x) for x in q[f]]
        X[z] = (lu[0] * lv[0] * xyz[c[0]] + lu[1] * lv[0] * xyz[c[1]] + lu[1] * lv[1] * xyz[c[2]]
                + lu[0] * lv[1] * xyz[c[3]])

    # --------------------------------------------- face-based control points
    fine_face_xyz = []
    for f in range(F):
        if not T.enriched[f]:
            continue
        if not (T.span[f][0] > 0 and T.span[f][1] > 0):
            raise MeshError("enriched face %d is not split 2 x 2" % f)
        if f in B.split_nets:
            C = [[_pos(B.split_nets[f][x][y], raw) for y in range(7)] for x in range(7)]
        else:
            C = split_net([[_pos(B.nets[f][i][j], raw) for j in range(4)] for i in range(4)])
        for cc in range(4):                  # children in corner order
            cu, cv = CORNER_UV[cc]
            for c2 in range(4):              # inner point nearest each corner of the child
                du, dv = CORNER_UV[c2]
                fine_face_xyz.append(C[3 * cu + 1 + du][3 * cv + 1 + dv])

    out = {"xyz": X, "quads": np.array(quads, dtype=np.int32),
           "level0_face": np.array(level0, dtype=np.int32),
           "face_xyz": np.array(fine_face_xyz, dtype=np.float64).reshape(-1, 3),
           "dim": int(mesh.get("dim", 2)),
           "parent": np.array(parent, dtype=np.int64), "child_off": np.array(off),
           "child_scale": np.array(scale)}
    return out


def _pos(lin, raw):
    """Point of a net entry (raw control variable -> weight)."""
    p = np.zeros(3)
    for k, w in lin.items():
        p += w * raw[k]
    return p
