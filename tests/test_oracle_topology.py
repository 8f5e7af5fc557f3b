"""Pins of the oracle's mesh terminology and classification (paper Sec. 3).

Expected counts are derived by hand from the definitions, not from the code:

* grid(nx, ny): the core is an nx x ny grid wrapped in one ring of quads (one per
  boundary edge, one per convex corner), so passive = 2 (nx + ny) + 4 (the whole
  ring), boundary = the core's outer ring 2 (nx + ny) - 4, regular = (nx - 2)(ny - 2);
  every passive face has one zero span (two for a corner face), every active face
  spans (1, 1).
* disk(mu, n): mu sectors of n x n faces (i, j) around the EP at (0, 0).  Passive:
  the outermost ring max(i, j) = n - 1 (2 n - 1 faces a sector); boundary: the next
  ring (2 n - 3); irregular: the face (0, 0) of each sector; transition: the three
  faces sharing a vertex with it, (1, 0), (0, 1), (1, 1); regular: the rest.
* disk refined once (N = 2 n faces a sector side): the enriched region is the
  2 x 2 block of children of every initial irregular face; irregular 1, enriched
  transition 3 (the other block faces) and transition 5 ((2, 0), (2, 1), (2, 2),
  (0, 2), (1, 2)) per sector.
* EP detection: one interior vertex of valence mu; an EP in the 1-ring of the
  boundary, or a boundary vertex of valence > 3, is rejected.
"""
import numpy as np
import pytest

from wq_synth import meshes
from oracle.topology import MeshError, TYPE_NAMES, Topology


def _counts(m):
    T = Topology(m["xyz"], m["quads"], m.get("level0_face"))
    return T, {TYPE_NAMES[k]: int((T.etype == k).sum()) for k in range(7)}


@pytest.mark.parametrize("nx,ny", [(5, 4), (3, 3), (6, 2)])
def test_grid_counts_and_spans(nx, ny):
    T, c = _counts(meshes.grid(nx, ny))
    assert c["passive"] == 2 * (nx + ny) + 4
    assert c["boundary"] == 2 * (nx + ny) - 4
    assert c["regular"] == (nx - 2) * (ny - 2)
    assert sum(c.values()) == T.F and not T.is_ep.any()
    for f in range(T.F):
        zeros = int((T.span[f] == 0).sum())
        if T.passive[f]:
            assert zeros in (1, 2)
        else:
            assert zeros == 0
    assert int(((T.span[:, 0] == 0) & (T.span[:, 1] == 0)).sum()) == 4


@pytest.mark.parametrize("mu", [3, 5, 7])
@pytest.mark.parametrize("n", [5, 6])
def test_disk_counts(mu, n):
    T, c = _counts(meshes.disk(mu=mu, n=n))
    assert c["passive"] == mu * (2 * n - 1)
    assert c["boundary"] == mu * (2 * n - 3)
    assert c["irregular"] == mu
    assert c["transition"] == 3 * mu
    assert c["enriched_transition"] == 0 and c["enriched_regular"] == 0
    assert c["regular"] == mu * (n * n - (2 * n - 1) - (2 * n - 3) - 4)
    assert int(T.is_ep.sum()) == 1
    v = int(np.nonzero(T.is_ep)[0][0])
    assert T.valence[v] == mu and not T.is_bnd_vertex[v]


@pytest.mark.parametrize("mu", [3, 5])
def test_disk_refined_once_keeps_the_enriched_region(mu):
    n = 6
    T, c = _counts(meshes.disk(mu=mu, n=n, levels=1))
    N = 2 * n
    assert int(T.enriched.sum()) == 4 * mu
    assert c["irregular"] == mu
    assert c["enriched_transition"] == 3 * mu
    assert c["transition"] == 5 * mu
    assert c["passive"] == mu * (2 * N - 1) and c["boundary"] == mu * (2 * N - 3)


def test_rejections():
    # an EP next to the boundary: the valence-5 disk without its outer rings
    m = meshes.disk(mu=5, n=1)
    with pytest.raises(MeshError, match="EP in the 1-ring"):
        Topology(m["xyz"], m["quads"])
    # a boundary vertex of valence 4 (two rows of quads meeting at a boundary vertex
    # from three sides) is an EP, and it lies on the boundary
    xyz = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0], [1, 1, 0], [2, 1, 0], [1, 2, 0], [2, 2, 0]],
                   dtype=float)
    quads = np.array([[0, 1, 4, 3], [1, 2, 5, 4], [4, 5, 7, 6]])
    with pytest.raises(MeshError, match="EP in the 1-ring"):
        Topology(xyz, quads)
    # a repeated vertex
    with pytest.raises(MeshError, match="4 distinct vertices"):
        Topology(xyz, np.array([[0, 1, 1, 3]]))
