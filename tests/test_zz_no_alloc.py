"""wq_rule_weights_noalloc: the weight solve without any device allocation.

Some callers cannot allocate device memory while they run (their own pool
allocator owns the free memory, or cudaMalloc's implicit synchronisation is not
acceptable in their loop).  For them the library carries a fixed scratch array;
this checks, through the C ABI, that two calls in a row reproduce the weights
of the allocating path (wq_rule_build / wq_rule_weights) within the FP64 bar of
the other tests.  Collected last on purpose (file name), and independent of the
other tests' state.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


def test_noalloc_weights_match_rule_weights():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available()
    ctx = wq.Context(0)
    b = wq.Basis(ctx, meshes.disk(mu=5, n=6))
    r = wq.Rule(b, comps=[wq.COMP_N, wq.COMP_X, wq.COMP_Y])
    for comp in (wq.COMP_X, wq.COMP_N):
        ref = r.weights(comp)[0].cpu().numpy()
        for _call in range(2):
            out = torch.full((r.info.sum_r,), float("nan"), dtype=torch.float64, device="cuda")
            r.weights_noalloc(comp, out)
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_noalloc_rejects_unbuilt_component():
    import torch
    from paper_2605_29334_gb300 import wq
    ctx = wq.Context(0)
    b = wq.Basis(ctx, meshes.disk(mu=5, n=4))
    r = wq.Rule(b, comps=[wq.COMP_N])
    out = torch.empty(r.info.sum_r, dtype=torch.float64, device="cuda")
    with pytest.raises(wq.WQError) as ei:
        r.weights_noalloc(wq.COMP_X, out)
    assert ei.value.code == wq.WQ_ERR_ARG
