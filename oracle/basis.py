"""The bicubic unstructured spline space, written element by element (paper Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper describes the analysis space of bicubic ASUTS in words (Sec. 3,
Figs. 1-2) and defers the formulas to its references.  This module is the
reading used here; every rule is a plain statement about Bezier control
points, and each function N_j is the set of Bezier nets obtained by setting its
control variable to 1 and all others to 0.

Control variables ("DOFs")
  * one per mesh vertex (vertex-based bicubic B-splines, Sec. 3);
  * four per enriched face, one near each corner (face-based C1 bicubic
    B-splines with doubled knots, Sec. 3, Fig. 1).

Bezier net of a face (4 x 4 points b[i][j], i along corner0->corner1, j along
corner0->corner3):
  * inner points b11, b21, b22, b12 -- for an enriched face, its face DOF at that
    corner; otherwise the B-spline "leg division" of the face's four vertex
    DOFs with ratio  span_left : span : span_right  (knot spans of Sec. 3:
    1, or 0 across edges perpendicular to the boundary);
  * edge points -- the span-weighted mean of the two inner points facing each
    other across the edge (C1 join), weights = the other face's span;
  * corner points -- the tensor span-weighted mean of the four inner points
    around a valence-4 vertex; the plain mean of the mu inner points around an
    EP.
  With all faces non-enriched this is exactly Boehm's B-spline-to-Bezier
  conversion of bicubic B-splines (pinned against Cox-de Boor in the tests);
  with enriched faces the vertex functions lose their inner points there, which
  is the truncation that restores the partition of unity (Sec. 3); EP vertex
  DOFs appear in enriched faces only, so the EP splines are eliminated.

Irregular faces (Sec. 3, Fig. 2)
  * split 2 x 2 by de Casteljau at 1/2 (7 x 7 net, four 4 x 4 sub-nets);
  * at every EP of valence mu, in the sub-net touching the EP (local index
    d[i][j], i along the spoke shared with the clockwise neighbour, j along the
    other spoke): "squares" d10 = d01 = d00 = p (collapsed at the EP);
    "triangles" d20 on every spoke are replaced by their projection onto the
    first Fourier mode around the EP, t_k <- p + cos(2 pi k/mu) X + sin(2 pi k/mu) Y
    (a common plane through p), and d11 <- (t_k + t_{k+1})/2 (coplanar).
  The remaining coefficients are the de Casteljau values.

With this reading, the number of functions on each element type reproduces
Table 1 for every entry (tests/test_oracle_basis.py).  The construction is a
partition of unity and C1 across every edge except inside the sub-elements
touching an EP (C0 there, with a common tangent plane at the EP).

Positions of the control variables: vertex DOFs sit at the mesh vertices; the
face DOFs of enriched faces are given by the mesh (``face_xyz`` [4 per enriched
face, ascending face id, corner order], e.g. computed by a refinement, Sec. 3) or,
when absent, placed at the B-spline inner Bezier points of the face's four
vertices (the legs divided in the ratio of the knot spans, (4 near + 2 + 2 +
1 far)/9 with unit spans; a generator choice for initial meshes, which makes
the geometry away from EPs the bicubic B-spline of the vertex DOFs).

Function numbering: raw id = vertex index for vertex DOFs, V + 4 * (rank of the
enriched face) + corner for face DOFs; functions with no non-zero coefficient
(|c| > 1e-12) on an active element are dropped and the rest renumbered in
raw-id order.
"""
from __future__ import annotations

import numpy as np

from .topology import Topology

COEF_TOL = 1e-12
CORNER_UV = [(0, 0), (1, 0), (1, 1), (0, 1)]


def _lin(*terms):
    """Sparse linear combination: _lin((a, dictA), (b, dictB), ...)."""
    out = {}
    for w, d in terms:
        if w == 0.0:
            continue
        for k, v in d.items():
            out[k] = out.get(k, 0.0) + w * v
    return out


def _split_1d(b):
    """de Casteljau split at 1/2 of 4 control points -> 7 points."""
    b0, b1, b2, b3 = b
    return [b0,
            _lin((0.5, b0), (0.5, b1)),
            _lin((0.25, b0), (0.5, b1), (0.25, b2)),
            _lin((0.125, b0), (0.375, b1), (0.375, b2), (0.125, b3)),
            _lin((0.25, b1), (0.5, b2), (0.25, b3)),
            _lin((0.5, b2), (0.5, b3)),
            b3]


def _dmap(c, i, j):
    """Index in the 7x7 net of entry d[i][j] of the EP sub-net when the EP is corner c."""
    if c == 0:
        return i, j
    if c == 1:
        return 6 - j, i
    if c == 2:
        return 6 - i, 6 - j
    return j, 6 - i


class Basis:
    """Element-wise Bezier form of every spline function on the active elements."""

    def __init__(self, mesh, topo=None):
        xyz = mesh["xyz"]
        self.dim = int(mesh.get("dim", 2))
        self.topo = topo or Topology(xyz, mesh["quads"], mesh.get("level0_face"))
        T = self.topo
        V = T.V
        enr = np.nonzero(T.enriched)[0]
        self.erank = -np.ones(T.F, dtype=np.int64)
        self.erank[enr] = np.arange(len(enr))
        self.n_raw = V + 4 * len(enr)
        self._inner_cache = {}
        nets = {}
        for f in range(T.F):
            if T.active[f]:
                nets[f] = self._net(f)
        # split irregular faces
        split = {}
        for f in nets:
            if T.irregular[f]:
                rows = [_split_1d([nets[f][i][j] for i in range(4)]) for j in range(4)]  # rows[j][x]
                C = [[None] * 7 for _ in range(7)]
                for x in range(7):
                    col = _split_1d([rows[j][x] for j in range(4)])
                    for y in range(7):
                        C[x][y] = col[y]
                split[f] = C
        # D-patch treatment around every EP
        for v in np.nonzero(T.is_ep)[0]:
            self._dpatch(int(v), split)
        # gather per active element: raw dof -> coefficient array [nsub, 4, 4]
        self.elements = []   # list of active face ids
        elem_raw = []
        for f in range(T.F):
            if not T.active[f]:
                continue
            if f in split:
                C = split[f]
                subs = []
                for sv in range(2):
                    for su in range(2):
                        subs.append([[C[3 * su + i][3 * sv + j] for j in range(4)] for i in range(4)])
            else:
                subs = [nets[f]]
            coefs = {}
            for s, net in enumerate(subs):
                for i in range(4):
                    for j in range(4):
                        for k, val in net[i][j].items():
                            if k not in coefs:
                                coefs[k] = np.zeros((len(subs), 4, 4))
                            coefs[k][s, i, j] += val
            coefs = {k: a for k, a in coefs.items() if np.max(np.abs(a)) > COEF_TOL}
            self.elements.append(f)
            elem_raw.append(coefs)
        used = sorted({k for c in elem_raw for k in c})
        self.raw_ids = np.array(used, dtype=np.int64)
        rid2fn = {k: i for i, k in enumerate(used)}
        self.n = len(used)
        self.E = len(self.elements)
        self.elem_fns = []
        self.elem_coef = []
        for coefs in elem_raw:
            keys = sorted(coefs, key=lambda k: rid2fn[k])
            self.elem_fns.append(np.array([rid2fn[k] for k in keys], dtype=np.int64))
            self.elem_coef.append(np.stack([coefs[k] for k in keys]) if keys else np.zeros((0, 1, 4, 4)))
        self.nsub = np.array([c.shape[1] for c in self.elem_coef], dtype=np.int64)
        self.etype = T.etype[self.elements]
        # positions of every control variable: vertices, then the face-based points
        # (given by the mesh, e.g. by a refinement, else the generator's choice below)
        raw_xyz = np.zeros((self.n_raw, 3))
        raw_xyz[:V] = xyz
        fx = mesh.get("face_xyz")
        if fx is not None:
            fx = np.asarray(fx, dtype=np.float64).reshape(-1, 3)
            if len(fx) != 4 * len(enr):
                raise ValueError("face_xyz holds %d points, the mesh has %d enriched faces"
                                 % (len(fx), len(enr)))
            raw_xyz[V:] = fx
        else:
            for r, f in enumerate(enr):
                for c in range(4):
                    raw_xyz[V + 4 * r + c] = sum(w * xyz[k] for k, w in self.leg(int(f), c).items())
        self.raw_xyz = raw_xyz
        self.nets = nets            # active face -> 4 x 4 net (raw id -> weight)
        self.split_nets = split     # irregular face -> 7 x 7 net after the D-patch treatment
        # control points of the functions
        P = raw_xyz[np.asarray(used, dtype=np.int64)] if used else np.zeros((0, 3))
        self.ctrl = P
        # geometry Bezier nets per element relative to a reference control point
        # (the element's first function): x = ref + sum_j c_j (P_j - ref), the same map
        # (partition of unity) without the cancellation of absolute coordinates
        self.geom_ref = [P[fns[0]] for fns in self.elem_fns]
        self.geom = [np.einsum("msij,mk->sijk", c, P[fns] - P[fns[0]])
                     for c, fns in zip(self.elem_coef, self.elem_fns)]
        # supports (as active-element index lists)
        self.supp = [[] for _ in range(self.n)]
        for e, fns in enumerate(self.elem_fns):
            for j in fns:
                self.supp[j].append(e)

    # ------------------------------------------------------------- net rules
    def fdof(self, f, c):
        return self.topo.V + 4 * int(self.erank[f]) + c

    def inner(self, f, c):
        key = (f, c)
        if key in self._inner_cache:
            return self._inner_cache[key]
        T = self.topo
        out = {self.fdof(f, c): 1.0} if T.enriched[f] else self.leg(f, c)
        self._inner_cache[key] = out
        return out

    def leg(self, f, c):
        """B-spline inner Bezier point of face f next to corner c, as weights of its
        four vertex DOFs: each leg divided in the ratio of the knot spans around it."""
        T = self.topo
        du, dv = T.span[f]
        dum, dup = T.cross_span(f, 3), T.cross_span(f, 1)
        dvm, dvp = T.cross_span(f, 0), T.cross_span(f, 2)
        su, sv = dum + du + dup, dvm + dv + dvp
        if su <= 0 or sv <= 0:
            raise ValueError("degenerate knot spans around face %d" % f)
        cu, cv = CORNER_UV[c]
        a = (dum + (du if cu else 0.0)) / su
        b = (dvm + (dv if cv else 0.0)) / sv
        q = T.quads[f]
        out = {}
        for cc, w in ((0, (1 - a) * (1 - b)), (1, a * (1 - b)), (2, a * b), (3, (1 - a) * b)):
            if w != 0.0:
                out[int(q[cc])] = out.get(int(q[cc]), 0.0) + w
        return out

    def edge_point(self, f, k, c):
        """Point on edge k of f next to corner c (c in {k, k+1})."""
        T = self.topo
        g, kg = T.nb[f][k]
        df = T.span[f][(k + 1) % 2]
        dg = T.span[g][(kg + 1) % 2]
        v = int(T.quads[f][c])
        return _lin((dg / (df + dg), self.inner(f, c)), (df / (df + dg), self.inner(g, T.corner_of(g, v))))

    def corner_point(self, f, c):
        T = self.topo
        v = int(T.quads[f][c])
        if T.is_bnd_vertex[v]:
            raise ValueError("corner point requested at boundary vertex %d" % v)
        if T.is_ep[v] or T.valence[v] != 4:
            fan = T.vfaces[v]
            return _lin(*[(1.0 / len(fan), self.inner(h, ch)) for h, ch in fan])
        ka, kb = (c + 3) % 4, c
        ga, kga = T.nb[f][ka]
        gb, kgb = T.nb[f][kb]
        others = [h for h, _ in T.vfaces[v] if h not in (f, ga, gb)]
        d = others[0]
        dxp, dxm = T.span[f][(ka + 1) % 2], T.span[ga][(kga + 1) % 2]
        dyp, dym = T.span[f][(kb + 1) % 2], T.span[gb][(kgb + 1) % 2]
        den = (dxm + dxp) * (dym + dyp)
        return _lin((dxm * dym / den, self.inner(f, c)),
                    (dxp * dym / den, self.inner(ga, T.corner_of(ga, v))),
                    (dxm * dyp / den, self.inner(gb, T.corner_of(gb, v))),
                    (dxp * dyp / den, self.inner(d, T.corner_of(d, v))))

    def _net(self, f):
        b = [[None] * 4 for _ in range(4)]
        b[0][0], b[3][0] = self.corner_point(f, 0), self.corner_point(f, 1)
        b[3][3], b[0][3] = self.corner_point(f, 2), self.corner_point(f, 3)
        b[1][1], b[2][1] = self.inner(f, 0), self.inner(f, 1)
        b[2][2], b[1][2] = self.inner(f, 2), self.inner(f, 3)
        b[1][0], b[2][0] = self.edge_point(f, 0, 0), self.edge_point(f, 0, 1)
        b[3][1], b[3][2] = self.edge_point(f, 1, 1), self.edge_point(f, 1, 2)
        b[2][3], b[1][3] = self.edge_point(f, 2, 2), self.edge_point(f, 2, 3)
        b[0][2], b[0][1] = self.edge_point(f, 3, 3), self.edge_point(f, 3, 0)
        return b

    def _dpatch(self, v, split):
        T = self.topo
        fan = T.fan(v)
        mu = len(fan)
        C0 = split[fan[0][0]]
        x0, y0 = _dmap(fan[0][1], 0, 0)
        p = C0[x0][y0]
        t = []
        for f, c in fan:
            x, y = _dmap(c, 2, 0)
            t.append(split[f][x][y])
        ang = 2.0 * np.pi * np.arange(mu) / mu
        dt = [_lin((1.0, tk), (-1.0, p)) for tk in t]
        X = _lin(*[(2.0 / mu * np.cos(ang[k]), dt[k]) for k in range(mu)])
        Y = _lin(*[(2.0 / mu * np.sin(ang[k]), dt[k]) for k in range(mu)])
        tn = [_lin((1.0, p), (np.cos(ang[k]), X), (np.sin(ang[k]), Y)) for k in range(mu)]
        for k, (f, c) in enumerate(fan):
            C = split[f]
            for (i, j), val in (((1, 0), p), ((0, 1), p), ((2, 0), tn[k]), ((0, 2), tn[(k + 1) % mu]),
                                ((1, 1), _lin((0.5, tn[k]), (0.5, tn[(k + 1) % mu])))):
                x, y = _dmap(c, i, j)
                C[x][y] = val

    # --------------------------------------------------------------- queries
    def m(self, e):
        return len(self.elem_fns[e])
