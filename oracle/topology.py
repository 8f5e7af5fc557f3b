"""Control-mesh terminology and element classification (paper Sec. 3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed (paper Sec. 3, itemised terminology list):

* valence: number of edges sharing a vertex;
* extraordinary point (EP): interior vertex of valence != 4, or boundary vertex
  of valence > 3;
* irregular element: a face with an EP corner;
* enriched element: the irregular faces of the initial mesh and all their
  descendants (the input gives, per face, the initial face it descends from);
* transition point: a vertex shared by an enriched and a non-enriched face;
  transition element: a face with a transition-point corner;
* n-ring neighbourhood of the boundary; passive boundary elements = 1-ring of
  the boundary, boundary elements = 2nd ring;
* regular element: not enriched, transition or boundary.

Assumptions checked (Sec. 3, assumption list): no EP in the 1-ring
neighbourhood of the boundary; knot spans are 1 except on edges perpendicular
to the boundary, which get 0 (an edge with exactly one boundary end point;
opposite edges of a face share their span).

Parity: pinned by hand-built meshes in ``tests/test_oracle_topology.py``
(type counts of the disk and grid meshes, EP detection, assumption errors).
"""
from __future__ import annotations

import numpy as np

PASSIVE, BOUNDARY, IRREGULAR, ENR_TRANSITION, TRANSITION, ENR_REGULAR, REGULAR = range(7)
TYPE_NAMES = ["passive", "boundary", "irregular", "enriched_transition", "transition",
              "enriched_regular", "regular"]


class MeshError(ValueError):
    pass


class Topology:
    def __init__(self, xyz, quads, level0_face=None):
        self.xyz = np.asarray(xyz, dtype=np.float64)
        self.quads = np.asarray(quads, dtype=np.int64)
        F = len(self.quads)
        V = len(self.xyz)
        self.F, self.V = F, V
        e2f = {}
        for f in range(F):
            q = self.quads[f]
            if len(set(q.tolist())) != 4:
                raise MeshError("face %d is not a quad with 4 distinct vertices" % f)
            for k in range(4):
                a, b = int(q[k]), int(q[(k + 1) % 4])
                e2f.setdefault((min(a, b), max(a, b)), []).append((f, k))
        self.nb = [[None] * 4 for _ in range(F)]
        bverts = set()
        nbr = [set() for _ in range(V)]
        for (a, b), lst in e2f.items():
            nbr[a].add(b)
            nbr[b].add(a)
            if len(lst) > 2:
                raise MeshError("non-manifold edge (%d, %d)" % (a, b))
            if len(lst) == 1:
                bverts.add(a)
                bverts.add(b)
            else:
                (f, k), (g, kg) = lst
                self.nb[f][k] = (g, kg)
                self.nb[g][kg] = (f, k)
        self.is_bnd_vertex = np.zeros(V, dtype=bool)
        self.is_bnd_vertex[list(bverts)] = True
        self.valence = np.array([len(s) for s in nbr], dtype=np.int64)
        self.vfaces = [[] for _ in range(V)]
        for f in range(F):
            for c in range(4):
                self.vfaces[int(self.quads[f][c])].append((f, c))
        used = np.zeros(V, dtype=bool)
        used[self.quads.ravel()] = True
        self.is_ep = used & (((~self.is_bnd_vertex) & (self.valence != 4)) |
                             (self.is_bnd_vertex & (self.valence > 3)))
        self._classify(level0_face)
        self._spans()

    # ------------------------------------------------------------------ types
    def _classify(self, level0_face):
        F, q = self.F, self.quads
        self.passive = np.array([bool(self.is_bnd_vertex[q[f]].any()) for f in range(F)])
        # EPs must not lie in the 1-ring neighbourhood of the boundary
        for f in np.nonzero(self.passive)[0]:
            if self.is_ep[q[f]].any():
                raise MeshError("EP in the 1-ring neighbourhood of the boundary (face %d)" % f)
        passive_verts = set(q[self.passive].ravel().tolist())
        self.boundary = np.array([(not self.passive[f]) and any(int(v) in passive_verts for v in q[f])
                                  for f in range(F)])
        self.irregular = np.array([bool(self.is_ep[q[f]].any()) for f in range(F)])
        if level0_face is None:
            self.enriched = self.irregular.copy()
        else:
            l0 = np.asarray(level0_face, dtype=np.int64)
            irr_groups = set(l0[self.irregular & (l0 >= 0)].tolist())
            self.enriched = np.array([l0[f] >= 0 and int(l0[f]) in irr_groups for f in range(F)])
            self.enriched |= self.irregular
        self.transition_pt = np.zeros(self.V, dtype=bool)
        for v in range(self.V):
            fs = [f for f, _ in self.vfaces[v]]
            if fs:
                e = self.enriched[fs]
                self.transition_pt[v] = bool(e.any() and (~e).any())
        self.transition = np.array([bool(self.transition_pt[q[f]].any()) for f in range(F)])
        et = np.full(F, REGULAR, dtype=np.int64)
        for f in range(F):
            if self.passive[f]:
                et[f] = PASSIVE
            elif self.boundary[f]:
                et[f] = BOUNDARY
            elif self.irregular[f]:
                et[f] = IRREGULAR
            elif self.enriched[f] and self.transition[f]:
                et[f] = ENR_TRANSITION
            elif self.transition[f]:
                et[f] = TRANSITION
            elif self.enriched[f]:
                et[f] = ENR_REGULAR
        self.etype = et
        self.active = ~self.passive

    # ------------------------------------------------------------------ spans
    def _spans(self):
        """span[f][d]: knot span of the pair of opposite edges (d, d+2) of face f."""
        q, bnd = self.quads, self.is_bnd_vertex
        self.span = np.ones((self.F, 2))
        for f in range(self.F):
            for d in range(2):
                for k in (d, d + 2):
                    a, b = int(q[f][k]), int(q[f][(k + 1) % 4])
                    if bnd[a] != bnd[b]:
                        self.span[f][d] = 0.0

    def cross_span(self, f, k):
        """Span, across edge k of f, of the face on the other side (0 beyond the boundary)."""
        nb = self.nb[f][k]
        if nb is None:
            return 0.0
        g, kg = nb
        return float(self.span[g][(kg + 1) % 2])

    def corner_of(self, f, v):
        return int(np.nonzero(self.quads[f] == v)[0][0])

    def fan(self, v):
        """Faces around interior vertex v in counter-clockwise order: [(f, corner), ...]."""
        f, c = self.vfaces[v][0]
        out = [(f, c)]
        while True:
            nb = self.nb[f][(c + 3) % 4]
            if nb is None:
                raise MeshError("vertex %d is not interior" % v)
            g = nb[0]
            cg = self.corner_of(g, v)
            if g == out[0][0]:
                break
            out.append((g, cg))
            f, c = g, cg
            if len(out) > 64:
                raise MeshError("fan of vertex %d does not close" % v)
        if len(out) != len(self.vfaces[v]):
            raise MeshError("vertex %d has a non-manifold fan" % v)
        return out
