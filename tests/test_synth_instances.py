"""The batched workload's instance generator (wq_synth.meshes.instances): every random
draw happens in instance_specs, so the meshes are the same whether they are built in one
process or in spawned workers; sizes follow the drawn targets (nearest refinement level)."""
import numpy as np

from wq_synth import meshes


def test_specs_are_deterministic_and_in_range():
    a = meshes.instance_specs(5001, 64, 500, 50000)
    b = meshes.instance_specs(5001, 64, 500, 50000)
    assert a == b
    for sp in a:
        if sp[0] == "rotated":
            _, nx, ny, n_ep, levels, _ = sp
            assert 4 <= nx <= 10 and 4 <= ny <= 10 and n_ep % 2 == 0 and 0 <= n_ep <= 20 and 0 <= levels <= 6
        else:
            _, mu, n, levels, _ = sp
            assert 3 <= mu <= 8 and 3 <= n <= 6 and 0 <= levels <= 6


def test_parallel_build_equals_serial():
    serial = meshes.instances(5001, 6, 100, 2000)
    parallel = meshes.instances(5001, 6, 100, 2000, workers=2)
    assert len(serial) == len(parallel) == 6
    for x, y in zip(serial, parallel):
        assert np.array_equal(x["quads"], y["quads"]) and np.array_equal(x["xyz"], y["xyz"])
        assert np.array_equal(x["level0_face"], y["level0_face"])


def test_sizes_track_the_targets():
    specs = meshes.instance_specs(5001, 12, 100, 2000)
    for sp, m in zip(specs, meshes.instances(5001, 12, 100, 2000)):
        base = sp[1] * sp[2] if sp[0] == "rotated" else sp[1] * sp[2] * sp[2]
        levels = sp[4] if sp[0] == "rotated" else sp[3]
        core = base * 4 ** levels
        assert core <= len(m["quads"]) <= core + 8 * int(np.sqrt(core)) + 64   # plus one passive ring
