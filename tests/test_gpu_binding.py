"""The binding refuses, before any library call, device tensors of the wrong type,
size or layout (the library reads them through raw pointers with implied sizes),
and the checked calls still run."""
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


def test_binding_checks_device_tensors():
    import torch
    from paper_2605_29334_gb300 import build, wq as W
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    ctx = W.Context(0)
    r = W.Rule(W.Basis(ctx, meshes.disk(mu=5, n=4)), comps=[W.COMP_N])
    good = torch.ones(r.Q, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError, match="coef must be torch.float64"):
        r.assemble(W.OP_MASS, good.float())
    with pytest.raises(ValueError, match="needed"):
        r.assemble(W.OP_MASS, good[:-1])
    with pytest.raises(ValueError, match="contiguous"):
        r.assemble(W.OP_MASS, torch.ones(2 * r.Q, dtype=torch.float64, device="cuda")[::2])
    with pytest.raises(ValueError, match="out must be torch.float32"):
        r.assemble(W.OP_MASS, good, prec=W.PREC_F32, out=torch.empty(r.nnz, dtype=torch.float64, device="cuda"))
    out = r.assemble(W.OP_MASS, good)
    torch.cuda.synchronize()
    assert out.shape == (r.nnz,) and bool(torch.isfinite(out).all())
