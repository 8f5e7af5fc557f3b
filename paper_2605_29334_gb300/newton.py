"""Newton iterations of the nonlinear heat problem (Sec. 5) on the device.

One backward-Euler step (theta = 1) of  du/dt = div(k(u) grad u) + f  with
k(u) = k0 + k2 u^2 and homogeneous Dirichlet data on a set of fixed functions:
the WQ residual R(u) (Eq. heat_residual_discrete, FP64: wq_heat_fields + wq_apply)
and a tangent (wq_assemble of WQ_OP_HEAT_J -- the exact derivative of the WQ
residual -- or of WQ_OP_HEAT_S, the paper's symmetric S) are re-assembled every
iteration by replaying one CUDA graph; the correction solves  T d = -R  on the free
functions and u += d, by Jacobi-preconditioned BiCGSTAB on the device (the default;
the WQ matrices are not symmetric) or by a sparse LU factorisation of the free-free
block on the host (SuperLU through SciPy; seconds per solve beyond 10^5 functions).  Once the residual is at the FP64 rounding
of its first value the correction is zero and no solve is done; the re-assembly still
runs every iteration.  The tangent may be assembled in a float
mode (WQ_PREC_F32, WQ_PREC_TC): with the residual kept in FP64 the iteration still
converges to the FP64 solution, at the rate the tangent's error allows.
"""
from __future__ import annotations

import time

import numpy as np

from . import wq


def _bicgstab(matvec, b, dinv, tol=1e-12, max_iter=2000):
    """Right-preconditioned BiCGSTAB for A x = b (torch FP64 vectors); returns (x, iters)."""
    import torch
    x = torch.zeros_like(b)
    r = b.clone()
    bn = float(torch.linalg.norm(b))
    if bn == 0.0:
        return x, 0
    rh = r.clone()
    rho = alpha = omega = 1.0
    v = torch.zeros_like(b)
    p = torch.zeros_like(b)
    for it in range(1, max_iter + 1):
        rho_n = float(torch.dot(rh, r))
        if rho_n == 0.0:
            break
        beta = (rho_n / rho) * (alpha / omega) if it > 1 else 0.0
        p = r + beta * (p - omega * v) if it > 1 else r.clone()
        ph = dinv * p
        v = matvec(ph)
        alpha = rho_n / float(torch.dot(rh, v))
        s = r - alpha * v
        if float(torch.linalg.norm(s)) <= tol * bn:
            x += alpha * ph
            return x, it
        sh = dinv * s
        t = matvec(sh)
        omega = float(torch.dot(t, s)) / float(torch.dot(t, t))
        x += alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_n
        if float(torch.linalg.norm(r)) <= tol * bn:
            return x, it
    return x, max_iter


class HeatNewton:
    """Newton driver for one rule (built with COMP_N and the gradient components)."""

    def __init__(self, rule, fixed, dt, k0=1.0, k2=1.0, f=0.0, tangent=wq.OP_HEAT_J, prec=wq.PREC_F64,
                 solver="bicgstab"):
        import torch
        self.r, self.dt, self.k0, self.k2, self.f = rule, float(dt), float(k0), float(k2), float(f)
        self.tangent, self.prec, self.solver = int(tangent), int(prec), solver
        n, Q = rule.n, rule.Q
        dim = rule.basis_dim
        self.grads = [wq.COMP_X, wq.COMP_Y] + ([wq.COMP_Z] if dim == 3 else [])
        self.fixed = torch.tensor(np.asarray(fixed, dtype=bool), device="cuda")
        self.free = (~self.fixed).to(torch.float64)
        rp, col = rule.pattern()
        self.crow, self.ccol = rp.to(torch.int64), col.to(torch.int64)
        rows = torch.repeat_interleave(torch.arange(n, device="cuda"), self.crow[1:] - self.crow[:-1])
        self.diag_pos = torch.nonzero(rows == self.ccol).flatten()
        assert len(self.diag_pos) == n, "the pattern S_i holds every diagonal entry"
        jac = self.tangent == wq.OP_HEAT_J
        self.u = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.u_old = torch.zeros(n, dtype=torch.float64, device="cuda")
        self.kappa = torch.empty(((1 + dim) if jac else 1, Q), dtype=torch.float64, device="cuda")
        self.g = torch.empty((1 + dim, Q), dtype=torch.float64, device="cuda")
        self.res = torch.empty(n, dtype=torch.float64, device="cuda")
        vt = torch.float64 if self.prec == wq.PREC_F64 else torch.float32
        self.vals = torch.empty(rule.nnz, dtype=vt, device="cuda")
        self.graph = None
        self.free_idx = np.nonzero(~np.asarray(fixed, dtype=bool))[0]
        self.crow_h, self.ccol_h = self.crow.cpu().numpy(), self.ccol.cpu().numpy()

    def _solve(self, res):
        """Correction d with T d = -res on the free functions (d = 0 on the fixed ones)."""
        import torch
        n = self.r.n
        if self.solver == "splu":
            import scipy.sparse as sp
            import scipy.sparse.linalg as spla
            T = sp.csr_matrix((self.vals.to(torch.float64).cpu().numpy(), self.ccol_h, self.crow_h), shape=(n, n))
            f = self.free_idx
            d = np.zeros(n)
            d[f] = spla.splu(T[f][:, f].tocsc()).solve(-res.cpu().numpy()[f])
            return torch.tensor(d, device="cuda"), 1
        A = torch.sparse_csr_tensor(self.crow, self.ccol, self.vals.to(torch.float64), size=(n, n))
        diag = self.vals[self.diag_pos].to(torch.float64)
        dinv = torch.where(self.fixed, torch.ones_like(diag), 1.0 / diag)
        free = self.free

        def matvec(x):
            return free * (A @ (free * x)) + (1.0 - free) * x
        d, it = _bicgstab(matvec, -res, dinv)
        return free * d, it

    def _reassemble(self):
        r = self.r
        r.heat_fields(self.u, self.u_old, self.dt, self.k0, self.k2, self.f, kappa=self.kappa, g=self.g,
                      jacobian=self.tangent == wq.OP_HEAT_J)
        r.apply([wq.COMP_N] + self.grads, self.g, out=self.res)
        r.assemble(self.tangent, self.kappa, alpha=1.0 / self.dt, prec=self.prec, out=self.vals)

    def capture(self):
        """Capture one iteration's re-assembly (point fields, residual, tangent) in a graph."""
        import torch
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._reassemble()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._reassemble()
        torch.cuda.synchronize()

    def run(self, u_old, iters=20, line_search=False):
        """`iters` Newton iterations from u = u_old.  line_search: halve the step (up to 10
        times) until |R| decreases.  Returns a dict: the residual norms |R(u_k)| (free
        functions) before each update, the linear iterations, the step lengths, the
        re-assembly times (graph replay, CUDA events, ms) and the wall time."""
        import torch
        if self.graph is None:
            self.capture()
        self.u_old.copy_(torch.as_tensor(u_old, dtype=torch.float64, device="cuda"))
        self.u_old[self.fixed] = 0.0
        self.u.copy_(self.u_old)
        hist, lin, t_re, steps = [], [], [], []
        n = self.r.n
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        for _ in range(iters):
            e0.record()
            self.graph.replay()
            e1.record()
            e1.synchronize()
            t_re.append(e0.elapsed_time(e1))
            res = self.res * self.free
            hist.append(float(torch.linalg.norm(res)))
            if hist[-1] <= 64 * 2.0 ** -52 * hist[0]:   # converged to the FP64 rounding: d = 0
                lin.append(0)
                continue
            d, it = self._solve(res)
            lin.append(it)
            lam = 1.0
            if line_search:
                u0 = self.u.clone()
                for _k in range(10):
                    self.u.copy_(u0 + lam * d)
                    if self.residual_norm() < hist[-1]:
                        break
                    lam *= 0.5
                self.u.copy_(u0)
            steps.append(lam)
            self.u += lam * d
        torch.cuda.synchronize()
        return {"residual": hist, "linear_iterations": lin, "steps": steps, "reassembly_ms": t_re,
                "wall_s": time.perf_counter() - t0}

    def residual_norm(self):
        """|R(u)| on the free functions at the current u (one eager re-assembly)."""
        import torch
        self._reassemble()
        return float(torch.linalg.norm(self.res * self.free))


def boundary_fixed(basis, mesh):
    """The functions of boundary vertices (the homogeneous Dirichlet set)."""
    from collections import Counter
    cnt = Counter()
    for f in np.asarray(mesh["quads"]):
        for k in range(4):
            a, b = int(f[k]), int(f[(k + 1) % 4])
            cnt[(min(a, b), max(a, b))] += 1
    bnd = set()
    for (a, b), c in cnt.items():
        if c == 1:
            bnd.update((a, b))
    nv = len(mesh["xyz"])
    return np.array([rid < nv and rid in bnd for rid in basis.raw_ids()])
