"""Device refinement (wq_refine_apply: the knot-insertion stencils of the
vertex-based control points and the de Casteljau splits of the enriched faces'
Bezier nets) against the oracle's refinement (Sec. 3), on the meshes' own control
points and on random ones (the map is linear), once and twice in a row; the
twice-refined mesh then goes through the whole WQ rule on the device (c = 1 mass
matrix equal to the Gauss one, the exactness of Sec. 2)."""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu

MESHES = {
    "disk5": lambda: meshes.disk(mu=5, n=4),
    "disk8_L1": lambda: meshes.disk(mu=8, n=3, levels=1),
    "rotated_L0": lambda: meshes.rotated(levels=0),
    "rotated_L1": lambda: meshes.rotated(levels=1),
    "grid": lambda: meshes.grid(4, 3),
    "sphere": lambda: meshes.cube_sphere(pre=1, levels=1),
}

# Bars: a vertex point is a sum of at most 9 products (FP64, order may differ from
# the oracle's): 1e-14 of the data's scale.  A face point sums the element's
# Bezier coefficients times control points; the library drops coefficients below
# 1e-12 (rounding residues of the D-patch combinations), the oracle keeps them:
# 1e-12 of the scale.
TOL_V, TOL_F = 1e-14, 1e-12


@pytest.fixture(scope="module")
def W():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return wq


def _device_refine(W, ctx, mesh, xyz, fxyz):
    import torch
    b = W.Basis(ctx, mesh)
    r = W.Refine(b)
    xf, ff = r.apply(torch.tensor(xyz, device="cuda"), torch.tensor(fxyz, device="cuda").reshape(-1, 3))
    torch.cuda.synchronize()
    return r, xf.cpu().numpy(), ff.cpu().numpy()


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("data", ["mesh", "random"])
def test_apply_matches_oracle(W, name, data):
    from oracle.basis import Basis
    from oracle.refine import refine
    m = dict(MESHES[name]())
    ob = Basis(m)
    if data == "random":
        rng = np.random.Generator(np.random.PCG64(17))
        m["xyz"] = rng.uniform(-1.0, 1.0, size=m["xyz"].shape)
        m["face_xyz"] = rng.uniform(-1.0, 1.0, size=(ob.n_raw - ob.topo.V, 3))
    o = refine(m)
    ctx = W.Context(0)
    b = W.Basis(ctx, m)
    fx = b.face_ctrl()
    r, xf, ff = _device_refine(W, ctx, m, np.asarray(m["xyz"], dtype=np.float64), fx)
    q, l0 = r.mesh()
    assert np.array_equal(q, o["quads"]) and np.array_equal(l0, o["level0_face"])
    scale = max(np.max(np.abs(m["xyz"])), np.max(np.abs(fx)) if len(fx) else 0.0)
    assert xf.shape == o["xyz"].shape and ff.shape == o["face_xyz"].shape
    assert np.max(np.abs(xf - o["xyz"])) <= TOL_V * scale
    if len(ff):
        assert np.max(np.abs(ff - o["face_xyz"])) <= TOL_F * scale


def test_two_levels_then_rule(W):
    import torch
    from oracle.refine import refine
    ctx = W.Context(0)
    m0 = meshes.disk(mu=5, n=3)
    fine = W.refine_mesh(ctx, m0, levels=2)
    o = refine(refine(m0))
    assert np.array_equal(fine["quads"], o["quads"]) and np.array_equal(fine["level0_face"], o["level0_face"])
    scale = np.max(np.abs(m0["xyz"]))
    assert np.max(np.abs(fine["xyz"] - o["xyz"])) <= 4 * TOL_V * scale
    assert np.max(np.abs(fine["face_xyz"] - o["face_xyz"])) <= 4 * TOL_F * scale
    b = W.Basis(ctx, fine)
    r = W.Rule(b, comps=[W.COMP_N])
    M = r.assemble(W.OP_MASS, torch.ones(r.Q, dtype=torch.float64, device="cuda")).cpu().numpy()
    Mg = r.gq_assemble(W.OP_MASS, torch.ones(r.G, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.max(np.abs(M - Mg)) <= 1e-10 * np.max(np.abs(Mg))
    assert b.E == 16 * W.Basis(ctx, m0).E
