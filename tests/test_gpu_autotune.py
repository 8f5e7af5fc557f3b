"""wq_rule_autotune / WQ_PREC_AUTO: the library measures the float modes and kernel variants on the
rule's own data (error against its FP64 result, then device time of the modes within
the tolerance) and WQ_PREC_AUTO assembles with the fastest of them."""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    ctx = wq.Context(0)
    b = wq.Basis(ctx, meshes.rotated(levels=2))
    r = wq.Rule(b, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y])
    cq = torch.tensor(meshes.kappa_sines(r.points().cpu().numpy()), device="cuda")
    cg = torch.tensor(meshes.kappa_sines(r.gauss_points().cpu().numpy()), device="cuda")
    return wq, r, cq, cg


@pytest.mark.parametrize("gauss", [False, True])
@pytest.mark.parametrize("op", ["STIFF", "HEAT_S"])
def test_autotune_picks_a_measured_mode(setup, op, gauss):
    import torch
    wq, r, cq, cg = setup
    opc = getattr(wq, "OP_" + op)
    coef = cg if gauss else cq
    res = r.autotune(opc, coef, alpha=3.0, gauss=gauss, tol=1e-6, reps=5)
    modes = [wq.PREC_TC, wq.PREC_F32, wq.PREC_F32_FAST]
    assert res["chosen"] in modes
    k = modes.index(res["chosen"])
    assert 0.0 <= res["err"][k] <= 1e-6 and res["ms"][k] > 0.0
    # the choice is the fastest of the modes within the tolerance
    timed = [m for m, e, t in zip(range(3), res["err"], res["ms"]) if 0.0 <= e <= 1e-6]
    assert all(res["ms"][k] <= res["ms"][j] for j in timed)
    asm = r.gq_assemble if gauss else r.assemble
    got = asm(opc, coef, alpha=3.0, prec=wq.PREC_AUTO)
    ref = asm(opc, coef, alpha=3.0, prec=res["chosen"])
    assert got.dtype == torch.float32 and torch.equal(got, ref)


def test_autotune_without_an_eligible_mode(setup):
    import torch
    wq, r, cq, _ = setup
    res = r.autotune(wq.OP_MASS, cq, tol=0.0, reps=2)
    assert res["chosen"] == -1 and all(t == -1.0 for t in res["ms"])
    assert torch.equal(r.assemble(wq.OP_MASS, cq, prec=wq.PREC_AUTO), r.assemble(wq.OP_MASS, cq, prec=wq.PREC_F32))


@pytest.mark.parametrize("gauss", [False, True])
def test_autotune_chooses_mode_and_kernel_variant(setup, gauss):
    """The candidates are the tensor-core mode and each SIMT mode with each kernel variant;
    the recorded choice is the fastest timed candidate, WQ_PREC_AUTO reproduces it bit
    for bit, and an explicit variant overrides it until reset."""
    import torch
    wq, r, cq, cg = setup
    coef = cg if gauss else cq
    res = r.autotune(wq.OP_STIFF, coef, gauss=gauss, tol=1e-6, reps=5)
    cands = res["candidates"]
    assert len(cands) == 7
    pairs = {(c["mode"], c["variant"]) for c in cands}
    for mode in (wq.PREC_F32, wq.PREC_F32_FAST):
        for v in (wq.VARIANT_SLOTMAP, wq.VARIANT_TILE12, wq.VARIANT_TILE16):
            assert (mode, v) in pairs
    timed = [c for c in cands if c["ms"] > 0.0]
    assert timed and all(0.0 <= c["err"] <= 1e-6 for c in timed)
    best = min(timed, key=lambda c: c["ms"])
    assert res["chosen"] == best["mode"]
    if best["mode"] != wq.PREC_TC:
        assert res["variant"] == best["variant"]
    asm = r.gq_assemble if gauss else r.assemble
    got = asm(wq.OP_STIFF, coef, prec=wq.PREC_AUTO)
    r.set_variant(wq.OP_STIFF, res["variant"], gauss=gauss)
    ref = asm(wq.OP_STIFF, coef, prec=res["chosen"])
    r.set_variant(wq.OP_STIFF, -1, gauss=gauss)
    assert torch.equal(got, ref)
    assert r.variant(wq.OP_STIFF, gauss=gauss) == res["variant"]
