"""Python binding of the WQ C ABI (include/wq.h) -- argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module loads
``lib/libwq.so`` (built in-tree by ``paper_2605_29334_gb300.build``) and fails
loudly if it is missing.  Device buffers are torch tensors (the caller's
memory) or zero-copy torch views of library-owned memory; streams are torch
streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libwq.so")

WQ_OK, WQ_ERR_ARG, WQ_ERR_MESH, WQ_ERR_ILLPOSED, WQ_ERR_NOT_CONVERGED, WQ_ERR_NONFINITE, WQ_ERR_CUDA, \
    WQ_ERR_OOM, WQ_ERR_NO_DEVICE = range(9)
OP_MASS, OP_STIFF, OP_BIHARM, OP_HEAT_S, OP_HEAT_J = range(5)
COMP_N, COMP_X, COMP_Y, COMP_Z, COMP_LAP = range(5)
PREC_F64, PREC_F32, PREC_F32_FAST, PREC_TC, PREC_AUTO = 0, 1, 2, 3, 4
VARIANT_TILE12, VARIANT_TILE16, VARIANT_SLOTMAP = 0, 1, 2
PLAN_NO_TC, PLAN_NO_TILE = 1, 2
TYPE_NAMES = ["passive", "boundary", "irregular", "enriched_transition", "transition", "enriched_regular", "regular"]


class WQError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("wq status %d: %s" % (code, msg))
        self.code = code


class _Mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("n_faces", C.c_int64), ("quads", C.POINTER(C.c_int32)), ("level0_face", C.POINTER(C.c_int32)),
                ("n_face_xyz", C.c_int64), ("face_xyz", C.POINTER(C.c_double))]


class BasisInfo(C.Structure):
    _fields_ = [("n_functions", C.c_int64), ("n_elements", C.c_int64), ("n_irregular", C.c_int64),
                ("nnz", C.c_int64), ("max_m", C.c_int32), ("max_n_i", C.c_int32), ("type_count", C.c_int64 * 7)]


class RuleOpts(C.Structure):
    _fields_ = [("comps", C.c_uint32), ("count_mode", C.c_int32), ("tsvd_rel_tol", C.c_double),
                ("max_sweeps", C.c_int32), ("stream", C.c_void_p), ("skip_plans", C.c_uint32)]


class RuleInfo(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_gauss", C.c_int64), ("sum_r", C.c_int64), ("max_r", C.c_int32),
                ("n_truncated", C.c_int32 * 5), ("n_z_identity", C.c_int32 * 5), ("setup_ms", C.c_double),
                ("tsvd_ms", C.c_double), ("tsvd_gflop", C.c_double)]


class RefineInfo(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_faces", C.c_int64), ("n_face_xyz", C.c_int64),
                ("n_coarse_vertices", C.c_int64), ("n_coarse_face_xyz", C.c_int64), ("n_stencil", C.c_int64),
                ("n_face_jobs", C.c_int64), ("n_face_fns", C.c_int64), ("n_face_coef", C.c_int64),
                ("n_face_terms", C.c_int64), ("n_face_ell", C.c_int64)]


EXPORTS = {
    "wq_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "wq_destroy": (None, [C.c_void_p]),
    "wq_last_error": (C.c_char_p, [C.c_void_p]),
    "wq_build_basis": (C.c_int, [C.c_void_p, C.POINTER(_Mesh), C.POINTER(C.c_void_p)]),
    "wq_basis_destroy": (None, [C.c_void_p]),
    "wq_basis_info_get": (C.c_int, [C.c_void_p, C.POINTER(BasisInfo)]),
    "wq_basis_element": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_void_p, C.c_void_p]),
    "wq_basis_ctrl": (C.c_int, [C.c_void_p, C.c_void_p]),
    "wq_basis_pattern": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_point_counts": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "wq_rule_build": (C.c_int, [C.c_void_p, C.POINTER(RuleOpts), C.POINTER(C.c_void_p)]),
    "wq_rule_build_batched": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p), C.POINTER(RuleOpts),
                                        C.POINTER(C.c_void_p)]),
    "wq_rule_destroy": (None, [C.c_void_p]),
    "wq_rule_info_get": (C.c_int, [C.c_void_p, C.POINTER(RuleInfo)]),
    "wq_rule_points": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "wq_rule_gauss_points": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "wq_pattern": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                             C.POINTER(C.c_void_p)]),
    "wq_rule_weights": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "wq_rule_table": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int32)]),
    "wq_moments": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "wq_assemble": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]),
    "wq_gq_assemble": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                 C.c_void_p]),
    "wq_interp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_assemble_host": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p,
                                   C.c_void_p]),
    "wq_rule_weights_noalloc": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "wq_apply": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_heat_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                 C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_basis_functions": (C.c_int, [C.c_void_p, C.c_void_p]),
    "wq_rule_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "wq_rule_set_variant": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "wq_rule_get_variant": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]),
    "wq_rule_autotune_report": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_rule_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "wq_batch_create": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "wq_batch_destroy": (None, [C.c_void_p]),
    "wq_assemble_batched": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_void_p), C.c_double, C.c_int32,
                                      C.POINTER(C.c_void_p), C.c_void_p]),
    "wq_rule_load": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_void_p)]),
    "wq_rule_autotune": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_double,
                                   C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p]),
    "wq_rule_kernel_times": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]),
    "wq_basis_face_ctrl": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "wq_refine_create": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "wq_refine_destroy": (None, [C.c_void_p]),
    "wq_refine_info_get": (C.c_int, [C.c_void_p, C.POINTER(RefineInfo)]),
    "wq_refine_mesh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_refine_stencils": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "wq_refine_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def lib():
    """Load the library (raises ImportError when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("WQ library not built: %s missing (run __graft_entry__.build())" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class _CAI:
    """Zero-copy __cuda_array_interface__ wrapper of library-owned device memory."""

    def __init__(self, ptr, shape, typestr, strides=None, owner=None):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": strides}
        self._owner = owner


def _dev_view(ptr, shape, dtype, strides=None, owner=None):
    import torch
    typestr = {"f8": "<f8", "f4": "<f4", "i4": "<i4", "i8": "<i8"}[dtype]
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype={"f8": torch.float64, "f4": torch.float32, "i4": torch.int32,
                                         "i8": torch.int64}[dtype], device="cuda")
    return torch.as_tensor(_CAI(ptr, shape, typestr, strides, owner), device="cuda")


def _need(t, name, dtype, min_numel):
    """The library reads and writes through raw device pointers with implied sizes:
    refuse, before the call, a tensor that is not a contiguous CUDA tensor of the
    expected type holding at least min_numel elements."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, not %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() < min_numel:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), min_numel))
    return t


def _stream_handle(stream):
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return C.c_void_p(0)
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    def __init__(self, device=0):
        h = C.c_void_p()
        st = lib().wq_create(int(device), C.byref(h))
        if st != WQ_OK:
            raise WQError(st, "wq_create(%d) failed" % device)
        self.h = h
        self.device = device

    def check(self, st):
        if st != WQ_OK:
            raise WQError(st, lib().wq_last_error(self.h).decode(errors="replace"))

    def __del__(self):
        if getattr(self, "h", None):
            lib().wq_destroy(self.h)
            self.h = None


class Basis:
    """wq_build_basis on a mesh dict {xyz, quads, level0_face, dim, face_xyz (optional)}."""

    def __init__(self, ctx, mesh):
        self.ctx = ctx
        self._xyz = np.ascontiguousarray(mesh["xyz"], dtype=np.float64)
        self._quads = np.ascontiguousarray(mesh["quads"], dtype=np.int32)
        l0 = mesh.get("level0_face")
        self._l0 = None if l0 is None else np.ascontiguousarray(l0, dtype=np.int32)
        fx = mesh.get("face_xyz")
        self._fx = None if fx is None else np.ascontiguousarray(fx, dtype=np.float64).reshape(-1, 3)
        md = _Mesh(int(mesh.get("dim", 2)), len(self._xyz), self._xyz.ctypes.data_as(C.POINTER(C.c_double)),
                   len(self._quads), self._quads.ctypes.data_as(C.POINTER(C.c_int32)),
                   None if self._l0 is None else self._l0.ctypes.data_as(C.POINTER(C.c_int32)),
                   0 if self._fx is None else len(self._fx),
                   None if self._fx is None else self._fx.ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        ctx.check(lib().wq_build_basis(ctx.h, C.byref(md), C.byref(h)))
        self.h = h
        info = BasisInfo()
        ctx.check(lib().wq_basis_info_get(h, C.byref(info)))
        self.info = info
        self.n, self.E, self.nnz = info.n_functions, info.n_elements, info.nnz
        self.dim = int(mesh.get("dim", 2))

    def element(self, e):
        face, typ, m, ns = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self.ctx.check(lib().wq_basis_element(self.h, e, C.byref(face), C.byref(typ), C.byref(m), C.byref(ns),
                                              None, None))
        fns = np.zeros(m.value, dtype=np.int32)
        coef = np.zeros((m.value, ns.value, 4, 4))
        self.ctx.check(lib().wq_basis_element(self.h, e, None, None, None, None, _ptr(fns), _ptr(coef)))
        return {"face": face.value, "type": typ.value, "fns": fns, "coef": coef}

    def ctrl(self):
        out = np.zeros((self.n, 3))
        self.ctx.check(lib().wq_basis_ctrl(self.h, _ptr(out)))
        return out

    def pattern(self):
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(self.nnz, dtype=np.int32)
        self.ctx.check(lib().wq_basis_pattern(self.h, _ptr(rp), _ptr(col)))
        return rp, col

    def raw_ids(self):
        out = np.zeros(self.n, dtype=np.int64)
        self.ctx.check(lib().wq_basis_functions(self.h, _ptr(out)))
        return out

    def face_ctrl(self):
        """Face-based control points [4 per enriched face, 3] (wq_basis_face_ctrl)."""
        n = C.c_int64()
        self.ctx.check(lib().wq_basis_face_ctrl(self.h, C.byref(n), None))
        out = np.zeros((n.value, 3))
        self.ctx.check(lib().wq_basis_face_ctrl(self.h, C.byref(n), _ptr(out)))
        return out

    def point_counts(self, mode=0):
        """Sides of the per-element point grids (wq_count_mode: 0 min-max, 1 Table 2)."""
        side = np.zeros(self.E, dtype=np.int32)
        self.ctx.check(lib().wq_point_counts(self.h, int(mode), _ptr(side)))
        return side

    def __del__(self):
        if getattr(self, "h", None):
            lib().wq_basis_destroy(self.h)
            self.h = None


class Refine:
    """One global refinement of a basis's control mesh (wq_refine_*)."""

    def __init__(self, basis):
        self.ctx = basis.ctx
        self.dim = basis.dim
        h = C.c_void_p()
        self.ctx.check(lib().wq_refine_create(basis.h, C.byref(h)))
        self.h = h
        info = RefineInfo()
        self.ctx.check(lib().wq_refine_info_get(h, C.byref(info)))
        self.info = info

    def mesh(self):
        """Fine topology: (quads [n_faces, 4] int32, level0_face [n_faces] int32)."""
        q = np.zeros((self.info.n_faces, 4), dtype=np.int32)
        l0 = np.zeros(self.info.n_faces, dtype=np.int32)
        self.ctx.check(lib().wq_refine_mesh(self.h, _ptr(q), _ptr(l0)))
        return q, l0

    def stencils(self):
        ptr = np.zeros(self.info.n_vertices + 1, dtype=np.int64)
        src = np.zeros(self.info.n_stencil, dtype=np.int32)
        w = np.zeros(self.info.n_stencil)
        self.ctx.check(lib().wq_refine_stencils(self.h, _ptr(ptr), _ptr(src), _ptr(w)))
        return ptr, src, w

    def apply(self, xyz, face_xyz, out=None, stream=None):
        """Coarse control points (CUDA float64 tensors [Vc, 3], [n_coarse_face_xyz, 3]) ->
        fine ones ([n_vertices, 3], [n_face_xyz, 3]; new tensors unless out = (xyz_fine,
        face_xyz_fine) is given)."""
        import torch
        xyz = xyz.contiguous()
        face_xyz = face_xyz.contiguous()
        if out is None:
            fine = torch.empty((self.info.n_vertices, 3), dtype=torch.float64, device=xyz.device)
            ffine = torch.empty((self.info.n_face_xyz, 3), dtype=torch.float64, device=xyz.device)
        else:
            fine, ffine = out
        if self.ctx.device >= 0:
            _need(xyz, "xyz", torch.float64, 3 * self.info.n_coarse_vertices)
            _need(face_xyz, "face_xyz", torch.float64, 3 * self.info.n_coarse_face_xyz)
            _need(fine, "xyz_fine", torch.float64, 3 * self.info.n_vertices)
            _need(ffine, "face_xyz_fine", torch.float64, 3 * self.info.n_face_xyz)
        self.ctx.check(lib().wq_refine_apply(self.h, C.c_void_p(xyz.data_ptr()), C.c_void_p(face_xyz.data_ptr()),
                                             C.c_void_p(fine.data_ptr()), C.c_void_p(ffine.data_ptr()),
                                             _stream_handle(stream)))
        return fine, ffine

    def __del__(self):
        if getattr(self, "h", None):
            lib().wq_refine_destroy(self.h)
            self.h = None


def refine_mesh(ctx, mesh, levels=1):
    """Refine a mesh dict ``levels`` times on the device: returns the fine mesh dict
    (xyz, quads, level0_face, face_xyz, dim) with host arrays."""
    import torch
    for _ in range(levels):
        b = Basis(ctx, mesh)
        r = Refine(b)
        x = torch.tensor(np.ascontiguousarray(mesh["xyz"], dtype=np.float64), device="cuda")
        fx = torch.tensor(b.face_ctrl(), device="cuda").reshape(-1, 3)
        xf, fxf = r.apply(x, fx)
        q, l0 = r.mesh()
        torch.cuda.synchronize()
        mesh = {"xyz": xf.cpu().numpy(), "quads": q, "level0_face": l0, "face_xyz": fxf.cpu().numpy(),
                "dim": b.dim}
    return mesh


def _rule_opts(comps, count_mode, tol, max_sweeps, stream, skip_plans):
    mask = 0
    for c in comps:
        mask |= 1 << int(c)
    return RuleOpts(mask, int(count_mode), float(tol), int(max_sweeps), _stream_handle(stream), int(skip_plans))


def build_rules(bases, comps=(COMP_N, COMP_X, COMP_Y), tol=1e-12, max_sweeps=0, stream=None, count_mode=0,
                skip_plans=0):
    """wq_rule_build_batched: the rules of several bases (one device), with every
    truncated-SVD system of all of them solved in one persistent launch."""
    bases = list(bases)
    k = len(bases)
    hb = (C.c_void_p * k)(*[b.h.value if isinstance(b.h, C.c_void_p) else b.h for b in bases])
    out = (C.c_void_p * k)()
    opts = _rule_opts(comps, count_mode, tol, max_sweeps, stream, skip_plans)
    bases[0].ctx.check(lib().wq_rule_build_batched(k, hb, C.byref(opts), out))
    return [Rule(b, comps=comps, _handle=C.c_void_p(out[i])) for i, b in enumerate(bases)]


class Rule:
    """wq_rule_build: placement, basis tables, Gauss moments and TSVD weights on the device."""

    def __init__(self, basis, comps=(COMP_N, COMP_X, COMP_Y), tol=1e-12, max_sweeps=0, stream=None, path=None,
                 count_mode=0, skip_plans=0, _handle=None):
        """Build the rule, or (path given) load weights and moments saved by save().
        skip_plans: PLAN_NO_TC | PLAN_NO_TILE leave those assembly plans out."""
        self.basis = basis
        self.ctx = basis.ctx
        h = C.c_void_p()
        if _handle is not None:                 # built by build_rules
            h = _handle
            self.h = h
        elif path is not None:
            self.ctx.check(lib().wq_rule_load(basis.h, os.fsencode(path), C.byref(h)))
            self.h = h
        else:
            opts = _rule_opts(comps, count_mode, tol, max_sweeps, stream, skip_plans)
            self.ctx.check(lib().wq_rule_build(basis.h, C.byref(opts), C.byref(h)))
            self.h = h
        info = RuleInfo()
        self.ctx.check(lib().wq_rule_info_get(h, C.byref(info)))
        self.info = info
        if path is not None:
            comps = [c for c in range(5) if self._has_comp(c)]
        self.comps = tuple(comps)
        self.Q, self.G, self.n, self.nnz = info.n_points, info.n_gauss, basis.n, basis.nnz
        self.basis_dim = basis.dim

    def _has_comp(self, c):
        w, wp = C.c_void_p(), C.c_void_p()
        return lib().wq_rule_weights(self.h, int(c), C.byref(w), C.byref(wp)) == 0

    def save(self, path):
        """Write the weights, moments and weight statistics (wq_rule_save)."""
        self.ctx.check(lib().wq_rule_save(self.h, os.fsencode(path)))

    def points(self):
        p, q = C.c_void_p(), C.c_int64()
        self.ctx.check(lib().wq_rule_points(self.h, C.byref(p), C.byref(q)))
        return _dev_view(p.value, (q.value, 3), "f8", owner=self)

    def gauss_points(self):
        p, q = C.c_void_p(), C.c_int64()
        self.ctx.check(lib().wq_rule_gauss_points(self.h, C.byref(p), C.byref(q)))
        return _dev_view(p.value, (q.value, 3), "f8", owner=self)

    def pattern(self):
        n, nnz, rp, col = C.c_int64(), C.c_int64(), C.c_void_p(), C.c_void_p()
        self.ctx.check(lib().wq_pattern(self.h, C.byref(n), C.byref(nnz), C.byref(rp), C.byref(col)))
        return (_dev_view(rp.value, (n.value + 1,), "i4", owner=self),
                _dev_view(col.value, (nnz.value,), "i4", owner=self))

    def weights(self, comp):
        w, wp = C.c_void_p(), C.c_void_p()
        self.ctx.check(lib().wq_rule_weights(self.h, int(comp), C.byref(w), C.byref(wp)))
        nwc = len(self.comps)
        return (_dev_view(w.value, (self.info.sum_r,), "f8", strides=(8 * nwc,), owner=self),
                _dev_view(wp.value, (self.n + 1,), "i8", owner=self))

    def table(self, gauss=False):
        t, off, pp, gw, nc = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_int32()
        self.ctx.check(lib().wq_rule_table(self.h, int(gauss), C.byref(t), C.byref(off), C.byref(pp), C.byref(gw),
                                           C.byref(nc)))
        E = self.basis.E
        offs = _dev_view(off.value, (E + 1,), "i8", owner=self)
        total = int(offs[-1].item())
        out = {"table": _dev_view(t.value, (total,), "f8", owner=self), "off": offs,
               "pt_ptr": _dev_view(pp.value, (E + 1,), "i8", owner=self), "ncomp": nc.value}
        if gauss:
            out["gw"] = _dev_view(gw.value, (self.G,), "f8", owner=self)
        return out

    def moments(self, comp, stream=None):
        import torch
        out = torch.empty(self.nnz, dtype=torch.float64, device="cuda")
        self.ctx.check(lib().wq_moments(self.h, int(comp), C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def _coef_rows(self, op):
        return 1 + (3 if self.basis_dim == 3 else 2) if int(op) == OP_HEAT_J else 1

    def assemble(self, op, coef, alpha=0.0, prec=PREC_F64, out=None, stream=None):
        import torch
        vt = torch.float64 if prec == PREC_F64 else torch.float32
        if out is None:
            out = torch.empty(self.nnz, dtype=vt, device="cuda")
        _need(out, "out", vt, self.nnz)
        if coef is not None:
            _need(coef, "coef", torch.float64, self._coef_rows(op) * self.Q)
        cp = C.c_void_p(coef.data_ptr()) if coef is not None else C.c_void_p(0)
        self.ctx.check(lib().wq_assemble(self.h, int(op), cp, float(alpha), int(prec), C.c_void_p(out.data_ptr()),
                                         _stream_handle(stream)))
        return out

    def gq_assemble(self, op, coef_gauss, alpha=0.0, prec=PREC_F64, out=None, stream=None):
        import torch
        vt = torch.float64 if prec == PREC_F64 else torch.float32
        if out is None:
            out = torch.empty(self.nnz, dtype=vt, device="cuda")
        _need(out, "out", vt, self.nnz)
        if coef_gauss is not None:
            _need(coef_gauss, "coef_gauss", torch.float64, self._coef_rows(op) * self.G)
        cp = C.c_void_p(coef_gauss.data_ptr()) if coef_gauss is not None else C.c_void_p(0)
        self.ctx.check(lib().wq_gq_assemble(self.h, int(op), cp, float(alpha), int(prec),
                                            C.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def interp(self, u, stream=None):
        import torch
        _need(u, "u", torch.float64, self.n)
        uq = torch.empty(self.Q, dtype=torch.float64, device="cuda")
        gr = torch.empty((self.Q, 3), dtype=torch.float64, device="cuda")
        self.ctx.check(lib().wq_interp(self.h, C.c_void_p(u.data_ptr()), C.c_void_p(uq.data_ptr()),
                                       C.c_void_p(gr.data_ptr()), _stream_handle(stream)))
        return uq, gr

    def apply(self, comps, g, out=None, stream=None):
        """y_i = sum_t sum_q w^{comps[t]}_iq g[t][q]; g: device tensor [len(comps), Q]."""
        import torch
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        hc = np.ascontiguousarray(comps, dtype=np.int32)
        _need(out, "out", torch.float64, self.n)
        _need(g, "g", torch.float64, len(hc) * self.Q)
        self.ctx.check(lib().wq_apply(self.h, len(hc), _ptr(hc), C.c_void_p(g.data_ptr()), C.c_void_p(out.data_ptr()),
                                      _stream_handle(stream)))
        return out

    def heat_fields(self, u, u_old, dt, k0=1.0, k2=1.0, f=0.0, kappa=None, g=None, jacobian=False, stream=None):
        """kappa(u) = k0 + k2 u^2 at the WQ points ([Q], or [1 + dim, Q] with the rows
        k'(u) d_d u when jacobian) and the residual point data g [1 + dim, Q]."""
        import torch
        ng = 1 + (3 if self.basis_dim == 3 else 2)
        if kappa is None:
            kappa = torch.empty((ng, self.Q) if jacobian else self.Q, dtype=torch.float64, device="cuda")
        if g is None:
            g = torch.empty((ng, self.Q), dtype=torch.float64, device="cuda")
        _need(u, "u", torch.float64, self.n)
        _need(u_old, "u_old", torch.float64, self.n)
        _need(kappa, "kappa", torch.float64, (ng if jacobian else 1) * self.Q)
        _need(g, "g", torch.float64, ng * self.Q)
        self.ctx.check(lib().wq_heat_fields(self.h, C.c_void_p(u.data_ptr()), C.c_void_p(u_old.data_ptr()),
                                            float(dt), float(k0), float(k2), float(f), int(bool(jacobian)),
                                            C.c_void_p(kappa.data_ptr()), C.c_void_p(g.data_ptr()),
                                            _stream_handle(stream)))
        return kappa, g

    def assemble_host(self, op, h_coef, alpha=0.0, prec=PREC_F64, out=None, stream=None):
        h_coef = np.ascontiguousarray(h_coef, dtype=np.float64)
        if out is None:
            out = np.zeros(self.nnz, dtype=np.float64 if prec == PREC_F64 else np.float32)
        # plain integer addresses: ctypes.data_as costs microseconds per call on this end-to-end path
        self.ctx.check(lib().wq_assemble_host(self.h, int(op), h_coef.ctypes.data, float(alpha), int(prec),
                                              out.ctypes.data, _stream_handle(stream)))
        return out

    def weights_noalloc(self, comp, out, stream=None):
        """Recompute the weights of comp into the caller's device tensor out [sum_r]
        using the library's fixed scratch array (no device allocation)."""
        import torch
        _need(out, "out", torch.float64, self.info.sum_r)
        self.ctx.check(lib().wq_rule_weights_noalloc(self.h, int(comp), C.c_void_p(out.data_ptr()),
                                                     _stream_handle(stream)))
        return out

    def autotune(self, op, coef, alpha=0.0, gauss=False, tol=1e-6, reps=20, stream=None):
        """wq_rule_autotune: pick the fastest float mode within tol for (op, gauss) by
        measurement; later calls with prec=PREC_AUTO use it.  Returns {"chosen": mode
        or -1, "err": [TC, F32, F32_FAST], "ms": [...]} (-1: not available / not timed)."""
        import torch
        if coef is not None:
            _need(coef, "coef", torch.float64, self._coef_rows(op) * (self.G if gauss else self.Q))
        chosen = C.c_int32(0)
        err = np.zeros(3, dtype=np.float64)
        ms = np.zeros(3, dtype=np.float32)
        cp = C.c_void_p(coef.data_ptr()) if coef is not None else C.c_void_p(0)
        self.ctx.check(lib().wq_rule_autotune(self.h, int(op), cp, float(alpha), int(bool(gauss)),
                                              float(tol), int(reps), _stream_handle(stream), C.byref(chosen),
                                              _ptr(err), _ptr(ms)))
        return {"chosen": chosen.value, "err": err.tolist(), "ms": ms.tolist(),
                "variant": self.variant(op, gauss=gauss), "candidates": self.autotune_report(op, gauss=gauss)}

    def autotune_report(self, op, gauss=False):
        """Every candidate of the last autotune: list of {mode, variant, err, ms}."""
        n = C.c_int32(0)
        cap = 16
        mode = np.zeros(cap, dtype=np.int32)
        var = np.zeros(cap, dtype=np.int32)
        err = np.zeros(cap, dtype=np.float64)
        ms = np.zeros(cap, dtype=np.float32)
        self.ctx.check(lib().wq_rule_autotune_report(self.h, int(op), int(bool(gauss)), cap, C.byref(n), _ptr(mode),
                                                     _ptr(var), _ptr(err), _ptr(ms)))
        k = min(n.value, cap)
        return [{"mode": int(mode[i]), "variant": int(var[i]), "err": float(err[i]), "ms": float(ms[i])}
                for i in range(k)]

    def set_variant(self, op, variant, gauss=False):
        """wq_rule_set_variant: kernel variant of the float modes for (op, gauss); -1 = the
        autotuner's choice."""
        self.ctx.check(lib().wq_rule_set_variant(self.h, int(op), int(bool(gauss)), int(variant)))

    def variant(self, op, gauss=False):
        v = C.c_int32(0)
        self.ctx.check(lib().wq_rule_get_variant(self.h, int(op), int(bool(gauss)), C.byref(v)))
        return v.value

    def set_timing(self, capacity):
        """Record per-kernel CUDA events for the next `capacity` assembly calls (0: off)."""
        self.ctx.check(lib().wq_rule_set_timing(self.h, int(capacity)))

    def kernel_times(self, max_calls=1 << 20):
        """[calls, 2] durations (ms) of the two kernels of each recorded assembly call."""
        max_calls = max(0, min(int(max_calls), 1 << 24))
        buf = np.zeros(2 * max(max_calls, 1), dtype=np.float32)
        n = C.c_int32(0)
        self.ctx.check(lib().wq_rule_kernel_times(self.h, max_calls, _ptr(buf), C.byref(n)))
        return buf[:2 * n.value].reshape(n.value, 2)

    def __del__(self):
        if getattr(self, "h", None):
            lib().wq_rule_destroy(self.h)
            self.h = None


class Batch:
    """wq_batch_create: several rules assembled by one launch per kernel."""

    def __init__(self, rules):
        self.rules = list(rules)
        self.ctx = self.rules[0].ctx
        arr = (C.c_void_p * len(self.rules))(*[r.h for r in self.rules])
        h = C.c_void_p()
        self.ctx.check(lib().wq_batch_create(len(self.rules), arr, C.byref(h)))
        self.h = h

    def assemble(self, op, coefs, alpha=0.0, prec=PREC_F32, outs=None, stream=None):
        import torch
        k = len(self.rules)
        if outs is None:
            dt = torch.float64 if prec == PREC_F64 else torch.float32
            outs = [torch.empty(r.nnz, dtype=dt, device="cuda") for r in self.rules]
        cp = (C.c_void_p * k)(*[c.data_ptr() if c is not None else None for c in coefs])
        vp = (C.c_void_p * k)(*[o.data_ptr() for o in outs])
        self.ctx.check(lib().wq_assemble_batched(self.h, int(op), cp, float(alpha), int(prec), vp,
                                                 _stream_handle(stream)))
        return outs

    def __del__(self):
        if getattr(self, "h", None):
            lib().wq_batch_destroy(self.h)
            self.h = None

