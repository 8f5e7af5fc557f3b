"""Weighted quadrature on the unstructured spline space (paper Sec. 4, Sec. 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Steps, in the paper's order:

1. Point counts per element (Sec. 4.2, Eq. qp_allocation, Table 2).
   Regular elements 2 x 2 and boundary elements 4 x 4 (kept from standard WQ).
   For every test function N_i and every element k of its support that is not
   regular/boundary:  r_ik = m_k / sum_{l in supp N_i \\ R} m_l * (n_i - 4 e^r_i - 16 e^b_i),
   then r_k = max_i r_ik.  Reading (the paper's tables list square grids):
   the side of element k is the smallest integer s >= 2 with s^2 >= r_ik
   (computed exactly in integers: s^2 * sum m_l >= m_k * numerator), maximised
   over i; then while some N_i has sum_k s_k^2 < n_i, the side of its
   non-regular element with the most functions (lowest id on ties) is raised
   by one -- the fallback the paper gives after Table 2.
2. Placement (Sec. 4.1): points evenly spaced in each element's parametric
   domain at cell centres ((k + 1/2)/s, (l + 1/2)/s), mapped to the physical
   domain; a split irregular element is spaced over its parent domain.
3. Exactness set S_i (Eq. 10) = CSR pattern row i; the points of N_i are those of
   the elements in supp N_i, in ascending element order.
4. Moments b^(i),c_j = Gauss value of int D_c N_i D_c N_j (gq.assemble with c = 1).
5. Weights per test function and component (Sec. 4.3): A = [D_c N_j(x_q)]
   (rows j in S_i, columns q), Z = diag(N_i(x_q)) for every operator (the
   paper: "the treatment is identical for different kinds of matrices"), or
   Z = I when N_i vanishes identically on the sub-element of one of its points
   (then V_t^T Z^2 V_t is singular); SVD A = U S V^T (LAPACK
   via numpy), keep singular values s_k >= tol * s_max (tol = 1e-12), and
   w = Z^2 V_t (V_t^T Z^2 V_t)^-1 S_t^-1 U_t^T b.  The inverse of
   V_t^T Z^2 V_t = G^T G (G = Z V_t) is applied through the QR factorisation of
   G, as in Sec. 2 (Eq. QR, with the Z^-1 printed there read as Z: the
   substitution v = Z^-1 w gives w = Z v):  w = Z Q R^-T S_t^-1 U_t^T b.
6. Row-wise assembly (Eqs. 9, 11, 12, S): A_ij = sum_q sum_c w^c_iq coef^c_q D_c N_j(x_q).
7. Nonlinear heat (Sec. 5): interpolation u(x_q), grad u(x_q) and the residual
   R_A = sum_q w_Aq (u_q - u^n_q)/dt + sum_q sum_d w^d_Aq k(u_q) d_d u_q - sum_q w_Aq f_q.

Parity: steps 1-3 pinned by Table 2 / well-posedness tests; step 5 pinned by
planted-SVD and full-rank (Eq. w0) special cases and exactness; step 6 by
"c = 1 gives the Gauss matrix" and, for any coefficient, by identities that follow
from x = sum_j P_j N_j and the partition of unity: zero stiffness row sums,
sum_j M_ij = sum_q w_iq c_q, and sum_j A_ij P_j = sum_q w_iq c_q D x(x_q) for every
component (tests/test_oracle_wq.py).  For non-constant coefficients the entries
themselves have no closed form; those identities are their pins.
"""
from __future__ import annotations

import numpy as np

from .geometry import eval_element
from .gq import pattern, assemble as gq_assemble, comp_values
from .topology import REGULAR, BOUNDARY, IRREGULAR, ENR_TRANSITION, TRANSITION, ENR_REGULAR

TSVD_TOL = 1e-12


# ---------------------------------------------------------------- 1. counts
def table2_counts(basis):
    """Table 2's fixed sides: regular 2, boundary 4, irregular 4, enriched
    transition 4, non-enriched transition and enriched regular 3, or 4 next to
    high-valence (>= 7) or clustered EPs.  Reading of "clustered": at least two
    EPs among the vertices of the elements in the union of the supports of the
    functions active on the element (the note under Table 2)."""
    T = basis.topo
    E = basis.E
    et = basis.etype
    side = np.zeros(E, dtype=np.int64)
    fixed = {REGULAR: 2, BOUNDARY: 4, IRREGULAR: 4, ENR_TRANSITION: 4}
    for e in range(E):
        t = int(et[e])
        if t in fixed:
            side[e] = fixed[t]
            continue
        region = set()
        for i in basis.elem_fns[e]:
            region.update(int(k) for k in basis.supp[i])
        verts = set()
        for k in region:
            verts.update(int(v) for v in T.quads[basis.elements[k]])
        eps = [v for v in verts if T.is_ep[v]]
        high = any(T.valence[v] >= 7 for v in eps)
        side[e] = 4 if (len(eps) >= 2 or high) else 3
    return side


def point_counts(basis, row_ptr=None, mode="minmax"):
    """Sides of the per-element point grids (Sec. 4.2).  mode "minmax": the
    min-max rule of eq. qp_allocation; mode "table2": Table 2's fixed values.
    Both end with the same repair (raise the non-regular element with most
    functions while some test function has fewer points than n_i), which the
    paper prescribes when the table's numbers are not well posed."""
    if row_ptr is None:
        row_ptr, _ = pattern(basis)
    if mode == "table2":
        return _repair(basis, row_ptr, table2_counts(basis))
    if mode != "minmax":
        raise ValueError("unknown count mode")
    E = basis.E
    et = basis.etype
    isR = (et == REGULAR) | (et == BOUNDARY)
    m = np.array([basis.m(e) for e in range(E)], dtype=np.int64)
    side = np.zeros(E, dtype=np.int64)
    side[et == REGULAR] = 2
    side[et == BOUNDARY] = 4
    side[~isR] = 2
    n_i = np.diff(row_ptr)
    for i in range(basis.n):
        supp = basis.supp[i]
        nonR = [k for k in supp if not isR[k]]
        if not nonR:
            continue
        er = sum(1 for k in supp if et[k] == REGULAR)
        eb = sum(1 for k in supp if et[k] == BOUNDARY)
        num = int(n_i[i]) - 4 * er - 16 * eb
        den = int(sum(m[k] for k in nonR))
        if num <= 0:
            continue
        for k in nonR:
            s = 2
            while s * s * den < int(m[k]) * num:
                s += 1
            side[k] = max(side[k], s)
    return _repair(basis, row_ptr, side)


def _repair(basis, row_ptr, side):
    et = basis.etype
    isR = (et == REGULAR) | (et == BOUNDARY)
    m = np.array([basis.m(e) for e in range(basis.E)], dtype=np.int64)
    n_i = np.diff(row_ptr)
    side = np.asarray(side, dtype=np.int64).copy()
    changed = True
    while changed:
        changed = False
        for i in range(basis.n):
            supp = basis.supp[i]
            if sum(int(side[k]) ** 2 for k in supp) < n_i[i]:
                nonR = [k for k in supp if not isR[k]]
                if not nonR:
                    raise ValueError("row %d cannot be made well-posed" % i)
                k = sorted(nonR, key=lambda kk: (-m[kk], kk))[0]
                side[k] += 1
                changed = True
    return side


# ------------------------------------------------------------- 2. placement
def local_points(s):
    c = (np.arange(s) + 0.5) / s
    return np.array([(c[k], c[l]) for l in range(s) for k in range(s)])


class Rule:
    """Everything the weight computation and assembly need, built from a Basis."""

    def __init__(self, basis, comps, tol=TSVD_TOL, side=None, count_mode="minmax"):
        self.basis = basis
        self.comps = list(comps)
        self.row_ptr, self.col = pattern(basis)
        self.side = point_counts(basis, self.row_ptr, count_mode) if side is None else np.asarray(side)
        E = basis.E
        self.pt_ptr = np.zeros(E + 1, dtype=np.int64)
        self.pt_ptr[1:] = np.cumsum(self.side ** 2)
        self.Q = int(self.pt_ptr[-1])
        self.theta = np.zeros((self.Q, 2))
        self.x = np.zeros((self.Q, 3))
        self.data = []
        for e in range(E):
            th = local_points(int(self.side[e]))
            d = eval_element(basis, e, theta=th)
            self.theta[self.pt_ptr[e]:self.pt_ptr[e + 1]] = th
            self.x[self.pt_ptr[e]:self.pt_ptr[e + 1]] = d["x"]
            self.data.append(d)
        self.tol = tol
        self.weights = None

    def row_points(self, i):
        return np.concatenate([np.arange(self.pt_ptr[e], self.pt_ptr[e + 1]) for e in self.basis.supp[i]])

    def local_system(self, i, comp):
        """A (n_i x r_i), z (r_i) of test function i for component comp."""
        B = self.basis
        cols = self.col[self.row_ptr[i]:self.row_ptr[i + 1]]
        blocks, zs = [], []
        for e in B.supp[i]:
            d = self.data[e]
            fns = B.elem_fns[e]
            D = comp_values(d, comp)                 # [m_e, P_e]
            blk = np.zeros((len(cols), D.shape[1]))
            blk[np.searchsorted(cols, fns)] = D
            blocks.append(blk)
            zs.append(d["N"][int(np.nonzero(fns == i)[0][0])])
        return np.concatenate(blocks, axis=1), np.concatenate(zs)

    # ---------------------------------------------------- 4-5. moments, TSVD
    def compute_weights(self, gdata=None, driver="gesdd", perturb_seed=None, perturb_ulps=16):
        """Moments and TSVD weights of every row.  perturb_seed (test use only): multiply
        every input of the weight solves (A, z, b) by 1 + perturb_ulps 2^-52 u, u ~ U(-1, 1)
        seeded -- the spread this causes measures the conditioning of the solves at FP64
        for inputs that agree to a few ulps (as two FP64 evaluations of the basis do)."""
        self.moments = {c: gq_assemble(self.basis, [c], row_ptr=self.row_ptr, col=self.col, gdata=gdata)
                        for c in self.comps}
        self.w_ptr = np.zeros(self.basis.n + 1, dtype=np.int64)
        self.w_ptr[1:] = np.cumsum([len(self.row_points(i)) for i in range(self.basis.n)])
        self.weights = {c: np.zeros(int(self.w_ptr[-1])) for c in self.comps}
        self.rank = {c: np.zeros(self.basis.n, dtype=np.int64) for c in self.comps}
        rng = None if perturb_seed is None else np.random.Generator(np.random.PCG64(perturb_seed))
        for c in self.comps:
            for i in range(self.basis.n):
                A, z = self.local_system(i, c)
                b = self.moments[c][self.row_ptr[i]:self.row_ptr[i + 1]]
                if rng is not None:
                    u = perturb_ulps * 2.0 ** -52
                    A = A * (1 + u * rng.uniform(-1, 1, A.shape))
                    z = z * (1 + u * rng.uniform(-1, 1, z.shape))
                    b = b * (1 + u * rng.uniform(-1, 1, b.shape))
                w, t = tsvd_weights(A, z, b, self.tol, driver)
                self.weights[c][self.w_ptr[i]:self.w_ptr[i + 1]] = w
                self.rank[c][i] = t
        return self.weights

    # ----------------------------------------------------------- 6. assembly
    def assemble(self, terms):
        """terms: list of (comp, coef [Q]) or (test comp, trial comp, coef [Q]) -> CSR
        values on the S_i pattern:  A_ij = sum_terms sum_q w^{test}_iq coef_q D_{trial} N_j(x_q)
        (Sec. 4.1; a 2-tuple uses the same component on both sides)."""
        B = self.basis
        vals = np.zeros(len(self.col))
        terms = [t if len(t) == 3 else (t[0], t[0], t[1]) for t in terms]
        for i in range(B.n):
            r0, r1 = self.row_ptr[i], self.row_ptr[i + 1]
            cols = self.col[r0:r1]
            acc = np.zeros(r1 - r0)
            off = self.w_ptr[i]
            for e in B.supp[i]:
                p0, p1 = self.pt_ptr[e], self.pt_ptr[e + 1]
                P = p1 - p0
                pos = np.searchsorted(cols, B.elem_fns[e])
                for wcomp, tcomp, coef in terms:
                    wc = self.weights[wcomp][off:off + P] * coef[p0:p1]
                    acc[pos] += comp_values(self.data[e], tcomp) @ wc
                off += P
            vals[r0:r1] = acc
        return vals

    # -------------------------------------------------------- 7. heat helpers
    def interp(self, u):
        """u_h and grad u_h at every WQ point: ([Q], [Q, 3])."""
        uq = np.zeros(self.Q)
        gq = np.zeros((self.Q, 3))
        for e in range(self.basis.E):
            d = self.data[e]
            ue = u[self.basis.elem_fns[e]]
            uq[self.pt_ptr[e]:self.pt_ptr[e + 1]] = ue @ d["N"]
            gq[self.pt_ptr[e]:self.pt_ptr[e + 1]] = np.einsum("m,mpk->pk", ue, d["grad"])
        return uq, gq

    def heat_residual(self, u, u_old, dt, kappa, f=None):
        """R_i = Q_i((u - u_old)/dt) + sum_d Q^d_i(k(u) d_d u) - Q_i(f)."""
        uq, gq = self.interp(u)
        uo, _ = self.interp(u_old)
        src = (uq - uo) / dt - (0.0 if f is None else f)
        R = np.zeros(self.basis.n)
        grads = [c for c in self.comps if c in "xyz"]
        for i in range(self.basis.n):
            q = self.row_points(i)
            sl = slice(self.w_ptr[i], self.w_ptr[i + 1])
            R[i] = self.weights["N"][sl] @ src[q]
            for c in grads:
                R[i] += self.weights[c][sl] @ (kappa(uq[q]) * gq[q, "xyz".index(c)])
        return R


    def heat_tangent(self, u, dt, kappa, dkappa, exact=True):
        """Newton tangent of heat_residual at u (Sec. 5.2, theta = 1) as assembly terms.

        dR_i/du_j = Q_i(N_j)/dt + sum_d Q^d_i(k(u) d_d N_j) + sum_d Q^d_i(k'(u) d_d u N_j):
        the derivative of the WQ residual itself (weights fixed), so Newton on the WQ
        system converges quadratically.  exact=False drops the last (non-symmetric)
        sum, which leaves the paper's S (eq. S)."""
        uq, gq = self.interp(u)
        k = kappa(uq)
        terms = [("N", "N", np.full(self.Q, 1.0 / dt))]
        grads = [c for c in self.comps if c in "xyz"]
        for c in grads:
            terms.append((c, c, k))
        if exact:
            dk = dkappa(uq)
            for c in grads:
                terms.append((c, "N", dk * gq[:, "xyz".index(c)]))
        return terms


def tsvd_weights(A, z, b, tol=TSVD_TOL, driver="gesdd"):
    """Truncated-SVD weights (Sec. 4.3) -> (w, t).

    driver: LAPACK SVD routine (gesdd, numpy's default, or gesvd via scipy);
    the two give the same weights up to the conditioning of the system, which
    is how the tests measure the reproducibility floor of FP64 weights.

    Reading for a test function that vanishes identically on the sub-element of
    some of its points (z_q == 0 exactly, so V_t^T Z^2 V_t is singular): that
    row uses Z = I, i.e. the plain minimum-norm truncated solution."""
    if driver == "gesdd":
        U, S, Vt = np.linalg.svd(A, full_matrices=False)
    else:
        import scipy.linalg
        U, S, Vt = scipy.linalg.svd(A, full_matrices=False, lapack_driver=driver)
    if S.size == 0 or S[0] == 0.0:
        return np.zeros(A.shape[1]), 0
    if np.any(z == 0.0):
        z = np.ones_like(z)
    t = int(np.sum(S >= tol * S[0]))
    g = (U[:, :t].T @ b) / S[:t]
    G = z[:, None] * Vt[:t].T
    Qm, R = np.linalg.qr(G)
    y = np.linalg.solve(R.T, g)
    return z * (Qm @ y), t
