"""Pins of the oracle's WQ steps (paper Sec. 4).

* Table 2: the min-max rule gives 2x2 regular, 4x4 boundary, 4x4 irregular and
  3x3 non-enriched transition points on the valence-5 disk;
* well-posedness r_i >= n_i for every test function (Sec. 4.2);
* TSVD weights: planted SVD with known rank; full rank => Eq. w0 / Eq. QR;
  exactness A w = b; KKT (Z^-2 w in range(V_t)); brute force in rationals;
* assembly: c = 1 gives the Gauss matrix (the exactness constraints, which is
  what Sec. 6 measures to ~1e-12), c = k gives k times it, stiffness row sums
  vanish for any coefficient, sum_j M_ij = sum_q w_iq c_q, and every operator
  reproduces the coordinates (sum_j A_ij P_j = sum_q w_iq c_q D x(x_q)) for any
  coefficient.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from wq_synth import meshes
from oracle.basis import Basis
from oracle.topology import TYPE_NAMES
from oracle import wq, gq

HERE = os.path.dirname(__file__)


@pytest.fixture(scope="module")
def disk_rule():
    B = Basis(meshes.disk(mu=5, n=6))
    R = wq.Rule(B, ["N", "x", "y", "lap"])
    R.compute_weights()
    return R


def test_table2_counts_on_disk(disk_rule):
    R = disk_rule
    tab = {}
    for line in open(os.path.join(HERE, "golden", "table2_points.txt")):
        if line[0] == "#" or not line.strip():
            continue
        t, s, _ = line.split()
        tab[t] = {int(v) for v in s.split("/")}
    seen = {}
    for e in range(R.basis.E):
        seen.setdefault(TYPE_NAMES[R.basis.etype[e]], set()).add(int(R.side[e]))
    assert seen["regular"] == {2} and seen["boundary"] == {4} and seen["irregular"] == {4}
    assert seen["transition"] == {3}
    for t, s in seen.items():
        assert s <= tab[t]


@pytest.mark.parametrize("make", [lambda: meshes.disk(mu=5, n=6), lambda: meshes.disk(mu=7, n=5, levels=1),
                                  lambda: meshes.rotated(levels=1), lambda: meshes.disk(mu=3, n=5, levels=2)])
def test_well_posed(make):
    B = Basis(make())
    rp, _ = gq.pattern(B)
    side = wq.point_counts(B, rp)
    for i in range(B.n):
        assert sum(int(side[k]) ** 2 for k in B.supp[i]) >= rp[i + 1] - rp[i]


def test_tsvd_planted():
    rng = np.random.Generator(np.random.PCG64(1))
    n, r = 7, 12
    U, _ = np.linalg.qr(rng.normal(size=(n, n)))
    V, _ = np.linalg.qr(rng.normal(size=(r, r)))
    sig = np.array([3.0, 1.0, 0.1, 1e-3, 1e-6, 1e-15, 1e-17])
    A = U @ np.diag(sig) @ V[:, :n].T
    z = rng.uniform(0.2, 1.0, size=r)
    b = U[:, :5] @ rng.normal(size=5)         # in range of the kept part
    w, t = wq.tsvd_weights(A, z, b)
    assert t == 5
    Vt = V[:, :5]
    Z2 = np.diag(z ** 2)
    ref = Z2 @ Vt @ np.linalg.inv(Vt.T @ Z2 @ Vt) @ np.diag(1 / sig[:5]) @ U[:, :5].T @ b
    assert np.max(np.abs(w - ref)) < 1e-9 * np.max(np.abs(ref))
    # kept condition number s_1/s_5 = 3e6: residual bound ~ 3e6 * eps
    assert np.max(np.abs(A @ w - b)) < 1e-10 * np.max(np.abs(b))


def test_tsvd_full_rank_equals_w0_and_qr():
    rng = np.random.Generator(np.random.PCG64(2))
    A = rng.normal(size=(6, 10))
    z = rng.uniform(0.3, 1.0, size=10)
    b = rng.normal(size=6)
    w, t = wq.tsvd_weights(A, z, b)
    assert t == 6
    Z2 = np.diag(z ** 2)
    w0 = Z2 @ A.T @ np.linalg.solve(A @ Z2 @ A.T, b)                   # Eq. w0
    Q, R = np.linalg.qr((A * z).T)
    wqr = z * (Q @ np.linalg.solve(R.T, b))                            # Eq. QR (Z read for Z^-1)
    assert np.max(np.abs(w - w0)) < 1e-12 * np.max(np.abs(w0))
    assert np.max(np.abs(w - wqr)) < 1e-12 * np.max(np.abs(w0))


def test_tsvd_brute_force_rationals():
    """Tiny full-rank case: KKT system of min |Z^-1 w|^2 s.t. A w = b solved exactly."""
    A = [[1, 2, 0, 1], [0, 1, 3, 1]]
    z = [1, Fraction(1, 2), 2, 1]
    b = [1, 2]
    n, r = 2, 4
    # KKT: Z^-2 w = A^T lam, A w = b  ->  (A Z^2 A^T) lam = b
    M = [[sum(Fraction(A[i][q]) * z[q] ** 2 * A[j][q] for q in range(r)) for j in range(n)] for i in range(n)]
    det = M[0][0] * M[1][1] - M[0][1] * M[1][0]
    lam = [(M[1][1] * b[0] - M[0][1] * b[1]) / det, (M[0][0] * b[1] - M[1][0] * b[0]) / det]
    wex = [z[q] ** 2 * sum(A[i][q] * lam[i] for i in range(n)) for q in range(r)]
    w, t = wq.tsvd_weights(np.array(A, float), np.array([float(x) for x in z]), np.array(b, float))
    assert t == 2
    assert np.max(np.abs(w - np.array([float(x) for x in wex]))) < 1e-14


def test_exactness_and_kkt(disk_rule):
    R = disk_rule
    for c in R.comps:
        for i in range(0, R.basis.n, 7):
            A, z = R.local_system(i, c)
            b = R.moments[c][R.row_ptr[i]:R.row_ptr[i + 1]]
            w = R.weights[c][R.w_ptr[i]:R.w_ptr[i + 1]]
            assert np.max(np.abs(A @ w - b)) <= 1e-12 * np.max(np.abs(b)) + 1e-18
            if np.all(z != 0):
                _, S, Vt = np.linalg.svd(A, full_matrices=False)
                t = R.rank[c][i]
                y = w / z ** 2
                resid = y - Vt[:t].T @ (Vt[:t] @ y)
                assert np.max(np.abs(resid)) < 1e-8 * np.max(np.abs(y))


def test_assembly_constant_coefficient_is_gauss(disk_rule):
    R = disk_rule
    ones = np.ones(R.Q)
    for c in R.comps:
        G = R.moments[c]
        A1 = R.assemble([(c, ones)])
        assert np.max(np.abs(A1 - G)) <= 1e-12 * np.max(np.abs(G))
        A3 = R.assemble([(c, 3.0 * ones)])
        assert np.max(np.abs(A3 - 3 * G)) <= 1e-12 * np.max(np.abs(3 * G))


def test_assembly_rowsums_and_mass_sums(disk_rule):
    R = disk_rule
    kap = meshes.kappa_sines(R.x)
    K = R.assemble([("x", kap), ("y", kap)])
    rs = np.add.reduceat(K, R.row_ptr[:-1])
    assert np.max(np.abs(rs)) < 1e-12 * np.max(np.abs(K))
    Mw = R.assemble([("N", kap)])
    for i in range(0, R.basis.n, 5):
        q = R.row_points(i)
        lhs = Mw[R.row_ptr[i]:R.row_ptr[i + 1]].sum()
        rhs = R.weights["N"][R.w_ptr[i]:R.w_ptr[i + 1]] @ kap[q]
        assert abs(lhs - rhs) < 1e-14


def test_assembly_linear_reproduction_any_coefficient(disk_rule):
    """x = sum_j P_j N_j reproduces the coordinates, so for any coefficient c and every
    component d: sum_j A^d_ij P_j,k = sum_q w^d_iq c_q D_d x_k(x_q), with D_d x_k = delta_dk
    for the gradient components, 0 for the planar Laplacian and x_k(x_q) for values."""
    R = disk_rule
    kap = meshes.kappa_sines(R.x)
    P = R.basis.ctrl
    col = R.col
    for d, g in (("x", (1.0, 0.0)), ("y", (0.0, 1.0)), ("lap", (0.0, 0.0)), ("N", None)):
        A = R.assemble([(d, kap)])
        for i in range(0, R.basis.n, 3):
            s = slice(R.row_ptr[i], R.row_ptr[i + 1])
            lhs = A[s] @ P[col[s], :2]
            q = R.row_points(i)
            wk = R.weights[d][R.w_ptr[i]:R.w_ptr[i + 1]] * kap[q]
            rhs = wk @ R.x[q, :2] if g is None else wk.sum() * np.array(g)
            scale = np.abs(R.weights[d][R.w_ptr[i]:R.w_ptr[i + 1]]).sum() * np.max(np.abs(kap)) * (1 + np.max(np.abs(P)))
            assert np.max(np.abs(lhs - rhs)) <= 1e-11 * scale, (d, i)


def test_heat_tangent_is_the_residual_derivative(disk_rule):
    """The exact tangent (Sec. 5.2) is the derivative of the WQ residual: pinned by
    central differences of heat_residual, column by column (the residual itself is
    a plain sum of weights times point data).  With exact=False the non-symmetric
    k'(u) part is missing, so the same check fails by the size of that part."""
    R = disk_rule
    B = R.basis
    rng = np.random.Generator(np.random.PCG64(31))
    u = 0.5 + 0.3 * rng.standard_normal(B.n)
    u_old = u + 0.05 * rng.standard_normal(B.n)
    dt = 0.1
    kap = lambda v: 1.0 + v * v
    dkap = lambda v: 2.0 * v
    J = R.assemble(R.heat_tangent(u, dt, kap, dkap, exact=True))
    S = R.assemble(R.heat_tangent(u, dt, kap, dkap, exact=False))
    h = 1e-6
    worst_J = worst_S = 0.0
    for j in range(0, B.n, 23):
        e = np.zeros(B.n)
        e[j] = h
        col = (R.heat_residual(u + e, u_old, dt, kap) - R.heat_residual(u - e, u_old, dt, kap)) / (2 * h)
        for i in np.nonzero(col)[0]:
            r0, r1 = R.row_ptr[i], R.row_ptr[i + 1]
            k = r0 + np.searchsorted(R.col[r0:r1], j)
            assert k < r1 and R.col[k] == j          # the derivative lives on the pattern S_i
            worst_J = max(worst_J, abs(J[k] - col[i]))
            worst_S = max(worst_S, abs(S[k] - col[i]))
    scale = np.max(np.abs(J))
    assert worst_J < 1e-7 * scale, worst_J / scale
    assert worst_S > 1e-4 * scale


def test_table2_mode_on_disk_and_well_posed():
    """Table 2 mode: on the valence-5 disk (one EP, no clustering) it gives the
    same sides as the min-max rule (Table 2's values); on meshes with clustered
    or high-valence EPs it uses 4 x 4 there, and every test function stays well
    posed (r_i >= n_i, Sec. 4.2)."""
    B = Basis(meshes.disk(mu=5, n=6))
    rp, _ = gq.pattern(B)
    assert np.array_equal(wq.point_counts(B, rp, "table2"), wq.point_counts(B, rp))
    for mesh in (meshes.disk(mu=8, n=4, levels=1), meshes.rotated(levels=1)):
        B = Basis(mesh)
        rp, _ = gq.pattern(B)
        side = wq.point_counts(B, rp, "table2")
        for i in range(B.n):
            assert sum(int(side[k]) ** 2 for k in B.supp[i]) >= rp[i + 1] - rp[i]
        assert set(np.unique(side)) <= {2, 3, 4, 5, 6}


def test_heat_residual_identity_with_assembled_matrices(disk_rule):
    """The discrete heat residual (Sec. 5.1, theta = 1) through the assembled WQ matrices:
    R = M (u - u_old) / dt + K(k(u_h)) u - M(f) 1, with M the WQ mass matrix (c = 1),
    K(k) the WQ stiffness with coefficient k(u_h(x_q)) and M(f) 1 = sum_q w_iq f_q
    (partition of unity).  A non-zero, non-constant source f and u != u_old make a
    wrong sign or a dropped term of the transient or source part fail (the tangent test
    pins only the part that depends on u)."""
    R = disk_rule
    B = R.basis
    rng = np.random.Generator(np.random.PCG64(47))
    u = 0.4 + 0.3 * rng.standard_normal(B.n)
    u_old = u + 0.2 * rng.standard_normal(B.n)
    dt = 0.05
    kap = lambda v: 1.0 + v * v
    f = 2.0 + np.sin(3.0 * R.x[:, 0]) * np.cos(2.0 * R.x[:, 1])
    res = R.heat_residual(u, u_old, dt, kap, f=f)

    def matvec(vals, v):
        y = np.zeros(B.n)
        for i in range(B.n):
            r0, r1 = R.row_ptr[i], R.row_ptr[i + 1]
            y[i] = vals[r0:r1] @ v[R.col[r0:r1]]
        return y

    uq, _ = R.interp(u)
    M = R.assemble([("N", np.ones(R.Q))])
    K = R.assemble([("x", kap(uq)), ("y", kap(uq))])
    Mf = R.assemble([("N", f)])
    ref = matvec(M, (u - u_old) / dt) + matvec(K, u) - matvec(Mf, np.ones(B.n))
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(res - ref)) <= 1e-12 * scale
    # the source and transient parts are each large enough to be seen
    assert np.max(np.abs(matvec(Mf, np.ones(B.n)))) > 1e-3 * scale
    assert np.max(np.abs(matvec(M, (u - u_old) / dt))) > 1e-3 * scale
