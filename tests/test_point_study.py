"""Point-count ablation (min-max rule vs Table 2's fixed values) and the point
reduction of WQ against Gauss quadrature across refinement levels (the analogue
of the paper's Table 3, Sec. 6.1), from the library's host set-up (no GPU).

The Gauss count is 16 per element plus 48 per irregular element (its 2 x 2
split needs 64 points, Sec. 4.2).  On a 14 x 18 core with 4 EPs (252 elements,
like the paper's unit square) the WQ reduction grows with the level as in
Table 3 (56 % -> 71 %); both counting modes give well-posed rules.
"""
import numpy as np
import pytest

from wq_synth import meshes


@pytest.fixture(scope="module")
def wq():
    from paper_2605_29334_gb300 import build, wq
    build.build()
    return wq


def _study(wq, mk, levels):
    ctx = wq.Context(-1)
    rows = []
    for lev in levels:
        b = wq.Basis(ctx, mk(lev))
        types = np.array([b.element(e)["type"] for e in range(b.E)])
        irregular = int(np.sum(types == 2))
        gq = 16 * b.E + 48 * irregular
        w = [int(np.sum(b.point_counts(mode).astype(np.int64) ** 2)) for mode in (0, 1)]
        rows.append((lev, b.E, irregular, gq, w[0], w[1]))
    return rows


def test_reduction_grows_with_level(wq):
    rows = _study(wq, lambda lev: meshes.rotated(nx=14, ny=18, n_ep=4, levels=lev, seed=2001), range(4))
    assert rows[0][1] == 252
    red = [(gq - w) / gq for _, _, _, gq, w, _ in rows]
    assert all(0.5 < r < 0.75 for r in red)
    assert all(red[k + 1] > red[k] for k in range(3)), red
    red_t2 = [(gq - w) / gq for _, _, _, gq, _, w in rows]
    assert all(red_t2[k + 1] > red_t2[k] for k in range(3)), red_t2


def test_modes_agree_on_single_ep_disk(wq):
    rows = _study(wq, lambda lev: meshes.disk(mu=5, n=6, levels=lev), range(2))
    for lev, E, irr, gq, w_mm, w_t2 in rows:
        assert w_mm == w_t2 and irr == 5
