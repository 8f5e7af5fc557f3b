"""Evaluation of the spline functions and their physical derivatives (paper Sec. 4.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The contravariant base vectors are evaluated through the normal n = a_1 x a_2
(a^1 = (a_2 x n)/|n|^2, a^2 = (n x a_1)/|n|^2, |n|^2 = det a_ab), which is the
same quantity as inverting the metric but avoids the cancellation in
a_11 a_22 - a_12^2 on skewed elements.

On an element (or one of the four sub-elements of a split irregular element)
each function is a bicubic Bernstein polynomial in the local coordinates
xi = (u, v) in [0, 1]^2; the geometry is x(xi) = sum_j P_j N_j(xi).

Derivatives follow the paper's surface formulas (Eqs. 13-17):
  tangents a_alpha = dx/dxi^alpha, covariant metric a_ab = a_a . a_b,
  contravariant metric [a^ab] = [a_ab]^-1,
  surface gradient  grad N = a_a a^ab N_,b,
  Laplace-Beltrami  lap N = a^ab (N_,ab - Gamma^g_ab N_,g),
                    Gamma^g_ab = a^gd a_d . a_a,b,
which is the expansion of (1/J) d_a (J a^ab d_b N) with J = sqrt(det a_ab)
(reading: the paper calls J the determinant of the metric; the square root
is the standard form and the only one that makes the two forms equal).
For planar domains these are the flat gradient and Laplacian; the tests pin
that against the direct route J^-T grad and the chain rule for the Hessian
(``planar_derivatives``).

A point at parent coordinate theta of a split element lies in sub-element
(theta_u >= 1/2, theta_v >= 1/2) with xi = 2 theta - sub.
"""
from __future__ import annotations

import numpy as np


def bernstein3(t):
    """Cubic Bernstein values and first/second derivatives at t (shape [..., 4])."""
    t = np.asarray(t, dtype=np.float64)
    s = 1.0 - t
    B = np.stack([s ** 3, 3 * t * s ** 2, 3 * t ** 2 * s, t ** 3], axis=-1)
    dB = np.stack([-3 * s ** 2, 3 * s ** 2 - 6 * t * s, 6 * t * s - 3 * t ** 2, 3 * t ** 2], axis=-1)
    ddB = np.stack([6 * s, -12 + 18 * t, 6 - 18 * t, 6 * t], axis=-1)
    return B, dB, ddB


def locate(nsub, theta):
    """Parent coordinates theta [P, 2] -> (sub index [P], local xi [P, 2])."""
    theta = np.asarray(theta, dtype=np.float64)
    if nsub == 1:
        return np.zeros(len(theta), dtype=np.int64), theta.copy()
    su = (theta[:, 0] >= 0.5).astype(np.int64)
    sv = (theta[:, 1] >= 0.5).astype(np.int64)
    xi = np.stack([2 * theta[:, 0] - su, 2 * theta[:, 1] - sv], axis=1)
    return su + 2 * sv, xi


def _tensor_derivs(coef, sub, xi):
    """coef [m, nsub, 4, 4(, k)] -> value and d_u, d_v, d_uu, d_uv, d_vv at each point."""
    Bu, dBu, ddBu = bernstein3(xi[:, 0])
    Bv, dBv, ddBv = bernstein3(xi[:, 1])
    c = coef[:, sub]                      # [m, P, 4, 4, ...]
    f = lambda a, b: np.einsum("mpij...,pi,pj->mp...", c, a, b)
    return f(Bu, Bv), f(dBu, Bv), f(Bu, dBv), f(ddBu, Bv), f(dBu, dBv), f(Bu, ddBv)


def eval_element(basis, e, theta=None, sub=None, xi=None):
    """Basis data of active element e at parent coordinates theta [P, 2]
    (or at explicit sub-element / local coordinates).

    Returns dict with x [P,3], dA [P] (area element sqrt(det a_ab) of the local
    chart), N [m,P], grad [m,P,3], lap [m,P].
    """
    coef = basis.elem_coef[e]
    geom = basis.geom[e]
    if theta is not None:
        sub, xi = locate(coef.shape[1], theta)
    N, Nu, Nv, Nuu, Nuv, Nvv = _tensor_derivs(coef, sub, xi)
    X, Xu, Xv, Xuu, Xuv, Xvv = [a[0] for a in _tensor_derivs(geom[None], sub, xi)]   # [P, 3]
    X = basis.geom_ref[e][None, :] + X          # nets are stored relative to a control point
    a1, a2 = Xu, Xv
    # contravariant base vectors a^alpha = a^{alpha beta} a_beta, written with the
    # normal n = a_1 x a_2 (|n|^2 = det a_ab):  a^1 = (a_2 x n)/|n|^2, a^2 = (n x a_1)/|n|^2
    nrm = np.cross(a1, a2)
    det = np.sum(nrm * nrm, -1)
    A1 = np.cross(a2, nrm) / det[:, None]
    A2 = np.cross(nrm, a1) / det[:, None]
    i11 = np.sum(A1 * A1, -1); i12 = np.sum(A1 * A2, -1); i22 = np.sum(A2 * A2, -1)
    grad = Nu[..., None] * A1[None] + Nv[..., None] * A2[None]
    # Christoffel symbols Gamma^g_ab = a^g . a_{a,b}
    G1 = [np.sum(A1 * Xuu, -1), np.sum(A1 * Xuv, -1), np.sum(A1 * Xvv, -1)]
    G2 = [np.sum(A2 * Xuu, -1), np.sum(A2 * Xuv, -1), np.sum(A2 * Xvv, -1)]
    luu = Nuu - G1[0] * Nu - G2[0] * Nv
    luv = Nuv - G1[1] * Nu - G2[1] * Nv
    lvv = Nvv - G1[2] * Nu - G2[2] * Nv
    lap = i11 * luu + 2 * i12 * luv + i22 * lvv
    return {"x": X, "dA": np.sqrt(det), "N": N, "grad": grad, "lap": lap,
            "sub": sub, "xi": xi}


def planar_derivatives(basis, e, theta):
    """Flat gradient and Laplacian by the planar chain rule (independent route for pins):
    grad N = J^-T grad_xi N,  H_x N = J^-T (H_xi N - sum_k (grad N)_k H_xi x_k) J^-1."""
    coef = basis.elem_coef[e]
    sub, xi = locate(coef.shape[1], theta)
    N, Nu, Nv, Nuu, Nuv, Nvv = _tensor_derivs(coef, sub, xi)
    X, Xu, Xv, Xuu, Xuv, Xvv = [a[0][:, :2] for a in _tensor_derivs(basis.geom[e][None], sub, xi)]
    P = len(xi)
    grad = np.zeros(N.shape + (2,))
    lap = np.zeros(N.shape)
    for p in range(P):
        J = np.column_stack([Xu[p], Xv[p]])
        Jinv = np.linalg.inv(J)
        for m in range(N.shape[0]):
            g = Jinv.T @ np.array([Nu[m, p], Nv[m, p]])
            H = np.array([[Nuu[m, p], Nuv[m, p]], [Nuv[m, p], Nvv[m, p]]])
            for k in range(2):
                Hx = np.array([[Xuu[p, k], Xuv[p, k]], [Xuv[p, k], Xvv[p, k]]])
                H = H - g[k] * Hx
            Hphys = Jinv.T @ H @ Jinv
            grad[m, p] = g
            lap[m, p] = np.trace(Hphys)
    return grad, lap
