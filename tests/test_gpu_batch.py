"""Batched assembly of independent instances and rule checkpoints, through the C ABI.

* wq_batch_create / wq_assemble_batched: eight planar instances of uneven size
  (rotated cores with up to 20 EPs of valence 3/5/6, disks around one EP of
  valence 3..8), assembled by one launch per kernel; every instance must be
  bitwise equal to its own wq_assemble (same arithmetic, same summation order),
  the FP64 mode falls back to per-rule calls, the batched call replays from a
  CUDA graph, and one instance is anchored to the oracle.
* wq_rule_build_batched: the same instances' weight systems in one launch, bitwise
  equal to separate builds; rules built without the optional assembly plans.
* wq_rule_save / wq_rule_load: a loaded rule reproduces weights, moments and
  assembled matrices bitwise; a file saved for another mesh, or cut short, is
  refused with WQ_ERR_ARG.
"""
import numpy as np
import pytest

from wq_synth import meshes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    from paper_2605_29334_gb300 import build, wq
    build.build()
    assert torch.cuda.is_available()
    return wq


@pytest.fixture(scope="module")
def batch_case(W):
    import torch
    ms = meshes.instances(5001, 8, 100, 2000)
    ctx = W.Context(0)
    bases = [W.Basis(ctx, m) for m in ms]
    rules = [W.Rule(b, comps=[W.COMP_N, W.COMP_X, W.COMP_Y]) for b in bases]
    coefs = [torch.tensor(meshes.kappa_sines(r.points().cpu().numpy()), device="cuda") for r in rules]
    return {"meshes": ms, "ctx": ctx, "bases": bases, "rules": rules, "coefs": coefs, "batch": W.Batch(rules)}


def test_batched_equals_per_rule(W, batch_case):
    import torch
    rules, coefs, batch = batch_case["rules"], batch_case["coefs"], batch_case["batch"]
    assert len({r.nnz for r in rules}) > 4          # uneven sizes
    for op, alpha in ((W.OP_MASS, 0.0), (W.OP_STIFF, 0.0), (W.OP_HEAT_S, 5.0)):
        for prec in (W.PREC_F32, W.PREC_F32_FAST, W.PREC_F64):
            outs = batch.assemble(op, coefs, alpha=alpha, prec=prec)
            for r, c, o in zip(rules, coefs, outs):
                assert torch.equal(o, r.assemble(op, c, alpha=alpha, prec=prec)), (op, prec)


def test_batched_against_oracle(W, batch_case):
    from oracle.basis import Basis
    from oracle import wq as owq
    k = int(np.argmin([r.nnz for r in batch_case["rules"]]))
    mesh, rule = batch_case["meshes"][k], batch_case["rules"][k]
    B = Basis(mesh)
    R = owq.Rule(B, ["N", "x", "y"])
    R.compute_weights()
    kap = meshes.kappa_sines(R.x)
    ref = R.assemble([("x", kap), ("y", kap)])
    outs = batch_case["batch"].assemble(W.OP_STIFF, batch_case["coefs"], prec=W.PREC_F32)
    got = outs[k].cpu().numpy().astype(np.float64)
    f64 = rule.assemble(W.OP_STIFF, batch_case["coefs"][k], prec=W.PREC_F64).cpu().numpy()
    scale = np.max(np.abs(ref))
    # the FP64 path's own bar (with the conditioning floor) is checked in test_gpu_parity;
    # here the oracle anchors the batched instance to the method
    assert np.max(np.abs(f64 - ref)) / scale < 1e-8
    assert np.max(np.abs(got - f64)) / scale < 1e-6


def test_batched_rule_build_equals_separate_builds(W, batch_case):
    """wq_rule_build_batched: the weight systems of all eight instances and three
    components, solved in one persistent launch in order of estimated work, give the
    weights, moments, weight statistics and matrices of eight separate builds, bit for
    bit (each system is solved by the same code, whatever CTA takes it)."""
    import torch
    rules, coefs = batch_case["rules"], batch_case["coefs"]
    built = W.build_rules(batch_case["bases"], comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    assert len(built) == len(rules)
    for r, b, c in zip(rules, built, coefs):
        for comp in (W.COMP_N, W.COMP_X, W.COMP_Y):
            assert torch.equal(r.weights(comp)[0], b.weights(comp)[0]), comp
            assert torch.equal(r.moments(comp), b.moments(comp)), comp
        assert list(r.info.n_truncated) == list(b.info.n_truncated)
        assert list(r.info.n_z_identity) == list(b.info.n_z_identity)
        assert b.info.tsvd_ms > 0.0 and b.info.tsvd_gflop > 0.0
        for op in (W.OP_MASS, W.OP_STIFF):
            for prec in (W.PREC_F32, W.PREC_F64):
                assert torch.equal(r.assemble(op, c, prec=prec), b.assemble(op, c, prec=prec)), (op, prec)
    # one instance alone through the batched call
    one = W.build_rules(batch_case["bases"][:1], comps=[W.COMP_N, W.COMP_X, W.COMP_Y])[0]
    assert torch.equal(one.weights(W.COMP_X)[0], rules[0].weights(W.COMP_X)[0])


def test_rule_without_tensor_core_and_tile_plans(W, batch_case):
    """skip_plans: a rule without the tensor-core and tile-engine plans assembles the
    same FP32 and FP64 matrices, refuses WQ_PREC_TC and the tile variants with
    WQ_ERR_ARG, and the autotuner picks among the modes it has."""
    import torch
    b, r, c = batch_case["bases"][0], batch_case["rules"][0], batch_case["coefs"][0]
    lean = W.Rule(b, comps=[W.COMP_N, W.COMP_X, W.COMP_Y], skip_plans=W.PLAN_NO_TC | W.PLAN_NO_TILE)
    for op in (W.OP_MASS, W.OP_STIFF):
        for prec in (W.PREC_F32, W.PREC_F64):
            assert torch.equal(lean.assemble(op, c, prec=prec), r.assemble(op, c, prec=prec)), (op, prec)
    with pytest.raises(W.WQError) as e:
        lean.assemble(W.OP_STIFF, c, prec=W.PREC_TC)
    assert e.value.code == 1
    with pytest.raises(W.WQError):
        lean.set_variant(W.OP_STIFF, W.VARIANT_TILE12)
    res = lean.autotune(W.OP_STIFF, c, tol=1e-6, reps=3)
    assert res["chosen"] in (W.PREC_F32, W.PREC_F32_FAST)
    assert res["err"][0] < 0.0                          # no tensor-core candidate


def test_batched_graph_replay(W, batch_case):
    import torch
    rules, coefs, batch = batch_case["rules"], batch_case["coefs"], batch_case["batch"]
    outs = [torch.empty(r.nnz, dtype=torch.float32, device="cuda") for r in rules]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.assemble(W.OP_STIFF, coefs, prec=W.PREC_F32, outs=outs)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.assemble(W.OP_STIFF, coefs, prec=W.PREC_F32, outs=outs)
    for o in outs:
        o.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(outs, eager))


def test_batch_rejects_mixed_rules(W, batch_case):
    r0 = batch_case["rules"][0]
    other = W.Rule(batch_case["bases"][1], comps=[W.COMP_X, W.COMP_Y])
    with pytest.raises(W.WQError):
        W.Batch([r0, other])


def test_rule_save_load_roundtrip(W, tmp_path):
    import torch
    ctx = W.Context(0)
    mesh = meshes.disk(mu=5, n=6)
    b = W.Basis(ctx, mesh)
    r = W.Rule(b, comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    path = str(tmp_path / "disk5.wqrule")
    r.save(path)
    r2 = W.Rule(b, path=path)
    assert r2.comps == r.comps and r2.Q == r.Q and r2.nnz == r.nnz
    assert list(r2.info.n_truncated) == list(r.info.n_truncated)
    for c in r.comps:
        assert torch.equal(r.weights(c)[0].clone(), r2.weights(c)[0].clone())
        assert torch.equal(r.moments(c), r2.moments(c))
    kap = torch.tensor(meshes.kappa_sines(r.points().cpu().numpy()), device="cuda")
    for prec in (W.PREC_F64, W.PREC_F32):
        for op in (W.OP_MASS, W.OP_STIFF):
            assert torch.equal(r.assemble(op, kap, prec=prec), r2.assemble(op, kap, prec=prec))
    # another mesh (same topology, other jitter) is refused
    b3 = W.Basis(ctx, meshes.disk(mu=5, n=6, seed=7))
    with pytest.raises(W.WQError):
        W.Rule(b3, path=path)
    # a truncated file is refused
    data = open(path, "rb").read()
    cut = str(tmp_path / "cut.wqrule")
    with open(cut, "wb") as f:
        f.write(data[: len(data) // 2])
    with pytest.raises(W.WQError):
        W.Rule(b, path=cut)


def test_handles_destroyed_in_any_order(W):
    """A context destroyed before its rule (Python's cyclic collector finalises in any
    order) leaves the rule's teardown and every later call working."""
    import torch
    L = W.lib()
    ctx = W.Context(0)
    b = W.Basis(ctx, meshes.disk(mu=5, n=4))
    r = W.Rule(b, comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    batch = W.Batch([r])
    L.wq_destroy(ctx.h)
    ctx.h = None
    L.wq_batch_destroy(batch.h)
    batch.h = None
    L.wq_rule_destroy(r.h)
    r.h = None
    L.wq_basis_destroy(b.h)
    b.h = None
    ctx2 = W.Context(0)
    b2 = W.Basis(ctx2, meshes.disk(mu=5, n=4))
    r2 = W.Rule(b2, comps=[W.COMP_N, W.COMP_X, W.COMP_Y])
    kap = torch.tensor(meshes.kappa_sines(r2.points().cpu().numpy()), device="cuda")
    v = r2.assemble(W.OP_STIFF, kap, prec=W.PREC_F32)
    torch.cuda.synchronize()
    assert torch.isfinite(v).all()
