"""cpu_ref: multi-core CPU baseline of the WQ and Gauss assembly (FP64, OpenMP).

``build()`` compiles ``libcpu_ref.so`` from ``cpu_ref.cpp`` (g++ -O3 -fopenmp); the
functions below take host arrays of precomputed inputs -- weights, point tables,
coefficients (the data, not the code, of whichever implementation produced them) --
and return the CSR values.  A timing baseline for the host cores, used by
``bench.py``; it shares no code with the GPU library or with the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpu_ref.cpp")
LIB = os.path.join(HERE, "libcpu_ref.so")
_lib = None


def build(force=False):
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        subprocess.run(["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", SRC, "-o", LIB], check=True)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        L.cpu_ref_threads.restype = C.c_int
        L.cpu_ref_set_threads.restype = None
        L.cpu_ref_wq.restype = None
        L.cpu_ref_gq.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Problem:
    """Host arrays of one mesh and quadrature rule:
    row_ptr [n+1], col [nnz] (int64 / int32); per element fn_ptr [E+1], fns (ascending);
    per row supp_ptr [n+1], supp (ascending), il (local index of the row's function);
    WQ: w_ptr [n+1], w [sum_r][nwc], pt_ptr [E+1], tab_ptr [E+1], table ([P][nc][m] per
    element); Gauss: gp_ptr, gtab_ptr, gtable, gw."""

    def __init__(self, **kw):
        conv = {"row_ptr": np.int64, "col": np.int32, "fn_ptr": np.int64, "fns": np.int32, "supp_ptr": np.int64,
                "supp": np.int32, "il": np.uint8, "w_ptr": np.int64, "w": np.float64, "pt_ptr": np.int64,
                "tab_ptr": np.int64, "table": np.float64, "gp_ptr": np.int64, "gtab_ptr": np.int64,
                "gtable": np.float64, "gw": np.float64}
        for k, v in kw.items():
            setattr(self, k, np.ascontiguousarray(v, dtype=conv[k]) if k in conv else v)
        self.n = len(self.row_ptr) - 1
        self.E = len(self.fn_ptr) - 1
        m = np.diff(self.fn_ptr)
        self.kb_ptr = np.concatenate([[0], np.cumsum(m * m)]).astype(np.int64)


def supports(fn_ptr, fns, n):
    """supp_ptr, supp (ascending elements), il of every function from the element lists."""
    E = len(fn_ptr) - 1
    cnt = np.zeros(n + 1, dtype=np.int64)
    np.add.at(cnt, np.asarray(fns) + 1, 1)
    supp_ptr = np.cumsum(cnt)
    supp = np.zeros(supp_ptr[-1], dtype=np.int32)
    il = np.zeros(supp_ptr[-1], dtype=np.uint8)
    cur = supp_ptr[:-1].copy()
    for e in range(E):
        for a, j in enumerate(fns[fn_ptr[e]:fn_ptr[e + 1]]):
            supp[cur[j]] = e
            il[cur[j]] = a
            cur[j] += 1
    return supp_ptr, supp, il


def _terms(terms):
    nt = len(terms)
    a = np.array([t[0] for t in terms], dtype=np.int32)
    b = np.array([t[1] for t in terms], dtype=np.int32)
    cr = np.array([t[2] for t in terms], dtype=np.int32)
    sc = np.array([t[3] for t in terms], dtype=np.float64)
    return nt, a, b, cr, sc


def wq_assemble(pb, nc, nwc, terms, coef=None):
    """terms: (weight column, table component, coefficient row or -1, constant scale)."""
    nt, wc, tc, cr, sc = _terms(terms)
    coef = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
    cstride = 0 if coef is None else coef.shape[-1]
    out = np.zeros(len(pb.col))
    lib().cpu_ref_wq(C.c_int64(pb.n), _p(pb.row_ptr), _p(pb.col), _p(pb.supp_ptr), _p(pb.supp), _p(pb.w_ptr),
                     _p(pb.w), C.c_int(nwc), _p(pb.fn_ptr), _p(pb.fns), _p(pb.pt_ptr), _p(pb.tab_ptr), _p(pb.table),
                     C.c_int(nc), C.c_int(nt), _p(wc), _p(tc), _p(cr), _p(sc),
                     _p(coef) if coef is not None else C.c_void_p(0), C.c_int64(cstride), _p(out))
    return out


def gq_assemble(pb, nc, terms, coef=None, kbuf=None):
    """terms: (test table component, trial table component, coefficient row or -1, scale)."""
    nt, scc, tc, cr, sc = _terms(terms)
    coef = None if coef is None else np.ascontiguousarray(coef, dtype=np.float64)
    cstride = 0 if coef is None else coef.shape[-1]
    if kbuf is None:
        kbuf = np.zeros(pb.kb_ptr[-1])
    out = np.zeros(len(pb.col))
    lib().cpu_ref_gq(C.c_int64(pb.n), C.c_int64(pb.E), _p(pb.row_ptr), _p(pb.col), _p(pb.supp_ptr), _p(pb.supp),
                     _p(pb.il), _p(pb.fn_ptr), _p(pb.fns), _p(pb.gp_ptr), _p(pb.gtab_ptr), _p(pb.gtable), _p(pb.gw),
                     C.c_int(nc), C.c_int(nt), _p(scc), _p(tc), _p(cr), _p(sc),
                     _p(coef) if coef is not None else C.c_void_p(0), C.c_int64(cstride), _p(pb.kb_ptr), _p(kbuf),
                     _p(out))
    return out


def threads():
    return int(lib().cpu_ref_threads())


def set_threads(t):
    lib().cpu_ref_set_threads(C.c_int(int(t)))
