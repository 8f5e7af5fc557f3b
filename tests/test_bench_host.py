"""Host-side helpers of bench.py (no GPU)."""
import numpy as np


def test_rel_errors_closed_form():
    import bench
    ref = np.array([1.0, 2.5, -3.0])
    mx, fro = bench.rel_errors(np.array([1.0, 2.0, -3.0], dtype=np.float32), ref)
    assert abs(mx - 0.5 / 3.0) < 1e-15
    assert abs(fro - 0.5 / np.sqrt(1.0 + 6.25 + 9.0)) < 1e-15
    assert bench.rel_errors(ref, ref) == (0.0, 0.0)
