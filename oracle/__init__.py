"""Plain FP64 CPU oracle for weighted quadrature (WQ) on bicubic unstructured splines.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` leg / ``--impl reference`` arm of ``bench.py`` may import or
run anything in this package.  The product library never calls it, and it
never calls the product library: the two share no code; both read meshes from
``wq_synth`` only.

The oracle follows the paper (Sheng, Wei, Chen, "Weighted Quadrature on
Unstructured Splines") step by step, slowly and in FP64:

* ``topology``  -- terminology and element classification (Sec. 3).
* ``basis``     -- the spline space: bicubic B-splines on knot spans, face-based
                   C1 enrichment, truncation, 2x2 split and D-patch treatment of
                   irregular elements (Sec. 3, Table 1).
* ``geometry``  -- Bernstein evaluation and physical / surface derivatives
                   (Sec. 4.1, Eqs. 13-17).
* ``gq``        -- 4x4 Gauss-Legendre element-wise assembly (the GQ reference,
                   Table 2 right column) and the moments b (Sec. 2, Eq. 5).
* ``wq``        -- point counts (Eq. qp_allocation), placement (Sec. 4.1),
                   exactness sets (Eq. 10), truncated-SVD weights (Sec. 4.3)
                   and row-wise WQ assembly (Eqs. 9, 11, 12, S).

Parity status of every function is stated in its module header.
"""
