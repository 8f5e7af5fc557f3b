"""The C-ABI library on the host (no GPU): it loads, exports every declared
symbol, and its host set-up (classification, spline space, pattern S_i,
min-max point counts) equals the oracle's; errors come back as status codes."""
import os
import re

import numpy as np
import pytest

from wq_synth import meshes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def wq():
    from paper_2605_29334_gb300 import build, wq as W
    build.build()
    return W


def test_exports_every_declared_symbol(wq):
    hdr = open(os.path.join(ROOT, "include", "wq.h")).read()
    names = set(re.findall(r"^\s*(?:wq_status|void|const char\*)\s+(wq_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 20
    L = wq.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    assert names <= set(wq.EXPORTS)


MESHES = {
    "disk5": lambda: meshes.disk(mu=5, n=6),
    "disk8_L1": lambda: meshes.disk(mu=8, n=4, levels=1),
    "disk3_L2": lambda: meshes.disk(mu=3, n=4, levels=2),
    "rotated_L1": lambda: meshes.rotated(levels=1),
    "grid": lambda: meshes.grid(5, 3, jitter=0.1),
    "sphere": lambda: meshes.cube_sphere(pre=1, levels=1),
}


@pytest.mark.parametrize("name", sorted(MESHES))
def test_host_setup_matches_oracle(wq, name):
    from oracle.basis import Basis
    from oracle import gq, wq as owq
    m = MESHES[name]()
    ctx = wq.Context(-1)
    b = wq.Basis(ctx, m)
    B = Basis(m)
    assert (b.n, b.E) == (B.n, B.E)
    for e in range(b.E):
        el = b.element(e)
        assert el["face"] == B.elements[e]
        assert el["type"] == B.etype[e]
        assert np.array_equal(el["fns"], B.elem_fns[e])
        assert np.max(np.abs(el["coef"] - B.elem_coef[e])) < 1e-15
    assert np.max(np.abs(b.ctrl() - B.ctrl)) == 0.0
    rp, col = b.pattern()
    rp2, col2 = gq.pattern(B)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    assert np.array_equal(b.point_counts(), owq.point_counts(B, rp2))
    assert np.array_equal(b.point_counts(1), owq.point_counts(B, rp2, "table2"))


def test_type_counts_and_info(wq):
    ctx = wq.Context(-1)
    b = wq.Basis(ctx, meshes.disk(mu=5, n=6))
    tc = list(b.info.type_count)
    assert tc[0] == 55 and sum(tc) == 180 and tc[2] == 5
    assert b.info.n_irregular == 5 and b.info.max_m == 28


def test_errors_are_status_codes(wq):
    ctx = wq.Context(-1)
    with pytest.raises(wq.WQError) as ei:
        wq.Basis(ctx, meshes.disk(mu=5, n=1))
    assert ei.value.code == wq.WQ_ERR_MESH and "boundary" in str(ei.value)
    bad = meshes.disk(mu=5, n=4)
    bad["quads"] = bad["quads"].copy()
    bad["quads"][3, 1] = bad["quads"][3, 0]
    with pytest.raises(wq.WQError) as ei:
        wq.Basis(ctx, bad)
    assert ei.value.code == wq.WQ_ERR_MESH
    bad2 = meshes.disk(mu=5, n=4)
    bad2["dim"] = 4
    with pytest.raises(wq.WQError) as ei:
        wq.Basis(ctx, bad2)
    assert ei.value.code == wq.WQ_ERR_ARG
    b = wq.Basis(ctx, meshes.disk(mu=5, n=4))
    with pytest.raises(wq.WQError) as ei:
        wq.Rule(b)
    assert ei.value.code == wq.WQ_ERR_NO_DEVICE


def test_binding_refuses_host_tensors(wq):
    """The binding checks tensors before the library dereferences their pointers."""
    import torch
    r = wq.Rule.__new__(wq.Rule)
    r.Q, r.G, r.n, r.nnz, r.basis_dim, r.h, r.ctx = 10, 20, 5, 30, 2, None, None
    host = torch.zeros(30, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        r.assemble(wq.OP_MASS, torch.zeros(10, dtype=torch.float64), out=host)
    with pytest.raises(ValueError, match="CUDA tensor"):
        r.gq_assemble(wq.OP_MASS, None, out=host)
    with pytest.raises(ValueError, match="CUDA tensor"):
        r.interp(torch.zeros(5, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA tensor"):
        wq._need([1.0], "x", torch.float64, 1)
