"""Element-wise Gauss quadrature (GQ) assembly and the moments b (paper Secs. 2, 4.2, 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* 4-point Gauss-Legendre rule per direction, written from its closed form:
  nodes +-sqrt(3/7 -+ (2/7) sqrt(6/5)), weights (18 +- sqrt 30)/36 on [-1, 1],
  mapped to [0, 1].  4 x 4 points per element and per sub-element of a split
  irregular element, i.e. 64 on an irregular element (Table 2, right column;
  the remark after Table 2).
* Component matrices  G^c_ij = sum_g w_g dA_g c(x_g) D_c N_i(x_g) D_c N_j(x_g)
  for D_c in {N, d_x, d_y, d_z, Laplace-Beltrami}; an operator is a sum of
  components (mass: N; stiffness: d_x + d_y (+ d_z), Eq. 11; biharmonic: lap,
  Eq. 12).
* The moments of WQ are these matrices with c = 1 (Sec. 2: "the entries of b
  are precomputed"; Sec. 6 uses GQ as the reference): b^(i),c_j = G^c_ij.

Values are returned on the CSR pattern rows = i, columns = S_i sorted (Eq. 10).

Parity: pinned in tests/test_oracle_gq.py (Gauss rule vs polynomial exactness,
mass sum = area by Green's theorem, zero stiffness row sums, symmetry, the
closed-form Bernstein Gram matrix on one affine element, brute-force 20 x 20
Gauss on a curved element).
"""
from __future__ import annotations

import numpy as np

from .geometry import eval_element

COMP_N, COMP_X, COMP_Y, COMP_Z, COMP_LAP = "N", "x", "y", "z", "lap"


def gauss4():
    """4-point Gauss-Legendre nodes and weights on [0, 1]."""
    s = 2.0 / 7.0 * np.sqrt(6.0 / 5.0)
    t = np.array([-np.sqrt(3.0 / 7.0 + s), -np.sqrt(3.0 / 7.0 - s),
                  np.sqrt(3.0 / 7.0 - s), np.sqrt(3.0 / 7.0 + s)])
    w = np.array([(18 - np.sqrt(30)) / 36, (18 + np.sqrt(30)) / 36,
                  (18 + np.sqrt(30)) / 36, (18 - np.sqrt(30)) / 36])
    return 0.5 * (t + 1.0), 0.5 * w


def gauss_points_local():
    """16 local points [16, 2] (u fastest) and weights [16] of the 4 x 4 rule."""
    x, w = gauss4()
    xi = np.array([(x[a], x[b]) for b in range(4) for a in range(4)])
    ww = np.array([w[a] * w[b] for b in range(4) for a in range(4)])
    return xi, ww


def pattern(basis):
    """CSR pattern of S_i (Eq. 10): j in row i iff supp N_i and supp N_j share an element."""
    n = basis.n
    rows = [set() for _ in range(n)]
    for fns in basis.elem_fns:
        for i in fns:
            rows[i].update(fns.tolist())
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols = []
    for i in range(n):
        c = sorted(rows[i])
        cols.extend(c)
        row_ptr[i + 1] = row_ptr[i] + len(c)
    return row_ptr, np.array(cols, dtype=np.int64)


def comp_values(data, comp):
    if comp == COMP_N:
        return data["N"]
    if comp == COMP_LAP:
        return data["lap"]
    return data["grad"][..., "xyz".index(comp)]


def gauss_data(basis, e):
    """Basis data at the Gauss points of element e (all sub-elements), with weights w*dA."""
    xi, ww = gauss_points_local()
    nsub = basis.elem_coef[e].shape[1]
    sub = np.repeat(np.arange(nsub), 16)
    xis = np.tile(xi, (nsub, 1))
    d = eval_element(basis, e, sub=sub, xi=xis)
    d["w"] = np.tile(ww, nsub) * d["dA"]
    return d


def assemble(basis, comps, coef=None, row_ptr=None, col=None, gdata=None):
    """sum_c G^c (Gauss), coefficient c(x) given as a callable of physical x [P,3]
    (or None for c = 1).  Returns CSR values on the S_i pattern."""
    if row_ptr is None:
        row_ptr, col = pattern(basis)
    pos = _positions(basis, row_ptr, col)
    vals = np.zeros(len(col))
    for e in range(basis.E):
        d = gdata[e] if gdata is not None else gauss_data(basis, e)
        c = np.ones(len(d["w"])) if coef is None else coef(d["x"])
        wc = d["w"] * c
        K = np.zeros((basis.m(e), basis.m(e)))
        for comp in comps:
            D = comp_values(d, comp)          # [m, P]
            K += (D * wc) @ D.T
        vals[pos[e]] += K.ravel()
    return vals


def assemble_terms(basis, terms, row_ptr=None, col=None, gdata=None):
    """sum over terms (test comp, trial comp, coef) of the Gauss integrals
    int coef(x) D_test N_i D_trial N_j (coef a callable of physical x [P,3], or None
    for 1) on the S_i pattern: the mixed form needed by the exact heat tangent
    (Sec. 5.2), where the test side carries a gradient and the trial side a value."""
    if row_ptr is None:
        row_ptr, col = pattern(basis)
    pos = _positions(basis, row_ptr, col)
    vals = np.zeros(len(col))
    for e in range(basis.E):
        d = gdata[e] if gdata is not None else gauss_data(basis, e)
        K = np.zeros((basis.m(e), basis.m(e)))
        for test, trial, coef in terms:
            c = np.ones(len(d["w"])) if coef is None else coef(d["x"])
            K += (comp_values(d, test) * (d["w"] * c)) @ comp_values(d, trial).T
        vals[pos[e]] += K.ravel()
    return vals


def _positions(basis, row_ptr, col):
    """For each element, flat CSR positions of its m x m local pairs (i, j)."""
    out = []
    for fns in basis.elem_fns:
        p = np.empty((len(fns), len(fns)), dtype=np.int64)
        for a, i in enumerate(fns):
            seg = col[row_ptr[i]:row_ptr[i + 1]]
            p[a] = row_ptr[i] + np.searchsorted(seg, fns)
        out.append(p.ravel())
    return out


def to_dense(n, row_ptr, col, vals):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[row_ptr[i]:row_ptr[i + 1]]] = vals[row_ptr[i]:row_ptr[i + 1]]
    return A
