"""wq_rule_weights_noalloc: the weight solve without any device allocation.

Some callers cannot allocate device memory while they run (their own pool
allocator owns the free memory, or cudaMalloc's implicit synchronisation is not
acceptable in their loop).  For them the library carries a fixed scratch array;
this checks, through the C ABI, that two calls in a row reproduce the weights
of the allocating path (wq_rule_build / wq_rule_weights) bit for bit (the same
solve kernel on the same inputs; a difference would mean a workspace-layout
fault), and that neither call changes the device's free memory (the array is
committed when the context is created).  Collected last on purpose (file name),
and independent of the other tests' state.
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
        out = torch.full((r.info.sum_r,), float("nan"), dtype=torch.float64, device="cuda")
        for _call in range(2):
            out.fill_(float("nan"))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            r.weights_noalloc(comp, out)
            torch.cuda.synchronize()
            assert torch.cuda.mem_get_info()[0] == free0
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got))
            assert np.array_equal(got, ref)


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
