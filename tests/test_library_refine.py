"""The library's refinement plan on the host (no GPU): the fine topology equals
the oracle's bit for bit, and its knot-insertion stencils applied to the coarse
vertices give the oracle's fine vertex control points; the default face-based
control points equal the oracle's; the face-based control points of a refined
mesh are accepted by the basis and checked for their count; applying on a
host-only context is refused."""
import numpy as np
import pytest

from wq_synth import meshes

MESHES = {
    "disk5": lambda: meshes.disk(mu=5, n=4),
    "disk3_L1": lambda: meshes.disk(mu=3, n=4, levels=1),
    "rotated_L0": lambda: meshes.rotated(levels=0),       # faces with several EPs
    "rotated_L1": lambda: meshes.rotated(levels=1),
    "grid": lambda: meshes.grid(4, 3),
    "grid1x1": lambda: meshes.grid(1, 1),                 # one active element
    "sphere": lambda: meshes.cube_sphere(pre=1, levels=1),
}


@pytest.fixture(scope="module")
def wq():
    from paper_2605_29334_gb300 import build, wq as W
    build.build()
    return W


def _apply_stencils(ptr, src, w, xyz):
    out = np.zeros((len(ptr) - 1, 3))
    for v in range(len(ptr) - 1):
        s = slice(ptr[v], ptr[v + 1])
        out[v] = (w[s, None] * xyz[src[s]]).sum(0)
    return out


@pytest.mark.parametrize("name", sorted(MESHES))
def test_plan_matches_oracle(wq, name):
    from oracle.basis import Basis
    from oracle.refine import refine
    m = MESHES[name]()
    ctx = wq.Context(-1)
    b = wq.Basis(ctx, m)
    r = wq.Refine(b)
    o = refine(m)
    q, l0 = r.mesh()
    assert r.info.n_vertices == len(o["xyz"]) and r.info.n_faces == len(o["quads"])
    assert np.array_equal(q, o["quads"]) and np.array_equal(l0, o["level0_face"])
    assert r.info.n_face_xyz == len(o["face_xyz"])
    ptr, src, w = r.stencils()
    assert ptr[-1] == r.info.n_stencil
    X = _apply_stencils(ptr, src, w, np.asarray(m["xyz"], dtype=np.float64))
    scale = np.max(np.abs(m["xyz"]))
    assert np.max(np.abs(X - o["xyz"])) <= 4e-16 * 9 * scale
    # default face-based control points
    fc = b.face_ctrl()
    ob = Basis(m)
    assert fc.shape == (r.info.n_coarse_face_xyz, 3)
    if len(fc):
        assert np.max(np.abs(fc - ob.raw_xyz[ob.topo.V:])) <= 1e-15 * scale
    # the device's term lists of the fine face-based points: 16 points per coarse enriched
    # face, an even number of (padded) terms each, no more non-zero terms than the dense
    # coefficients of the 16 points would give with the split folded in (m x 16 per face)
    I = r.info
    assert I.n_face_xyz == 16 * I.n_face_jobs
    assert I.n_face_ell % 32 == 0 and I.n_face_ell >= I.n_face_terms
    assert (I.n_face_jobs == 0) == (I.n_face_terms == 0)
    assert I.n_face_terms <= 16 * I.n_face_fns


def test_refined_mesh_builds_and_checks_face_points(wq):
    from oracle.basis import Basis
    from oracle.refine import refine
    ctx = wq.Context(-1)
    fine = refine(meshes.disk(mu=5, n=4))
    b = wq.Basis(ctx, fine)
    ob = Basis(fine)
    assert (b.n, b.E) == (ob.n, ob.E)
    assert np.max(np.abs(b.ctrl() - ob.ctrl)) < 1e-15
    bad = dict(fine)
    bad["face_xyz"] = fine["face_xyz"][:-1]
    with pytest.raises(wq.WQError) as ei:
        wq.Basis(ctx, bad)
    assert ei.value.code == wq.WQ_ERR_ARG


def test_apply_needs_a_device(wq):
    import torch
    ctx = wq.Context(-1)
    r = wq.Refine(wq.Basis(ctx, meshes.disk(mu=5, n=4)))
    x = torch.zeros((r.info.n_coarse_vertices, 3), dtype=torch.float64)
    f = torch.zeros((r.info.n_coarse_face_xyz, 3), dtype=torch.float64)
    with pytest.raises(wq.WQError) as ei:
        r.apply(x, f, stream=0)
    assert ei.value.code == wq.WQ_ERR_NO_DEVICE


def test_null_arguments_are_status_codes(wq):
    import ctypes as C
    L = wq.lib()
    h = C.c_void_p()
    assert L.wq_refine_create(None, C.byref(h)) == wq.WQ_ERR_ARG
    assert L.wq_refine_info_get(None, None) == wq.WQ_ERR_ARG
    assert L.wq_refine_apply(None, None, None, None, None, None) == wq.WQ_ERR_ARG
    ctx = wq.Context(-1)
    r = wq.Refine(wq.Basis(ctx, meshes.disk(mu=5, n=4)))
    assert L.wq_refine_mesh(r.h, None, None) == wq.WQ_OK          # NULL arrays are skipped
    assert L.wq_refine_stencils(r.h, None, None, None) == wq.WQ_OK
