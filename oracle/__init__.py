"""FP64 serial CPU oracle for FMG-FAS with segmental refinement.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.  The C source (``srfmg_oracle.c``) restates the paper's
algorithms (Figs. 1-4, Eqs. 4-7, the operators of Sec. 4) step by step; this
module only marshals numpy arrays through ctypes.

Parity pins: every routine is pinned by ``tests/test_oracle_pins.py`` against
closed forms, invariants, brute force on tiny inputs, values printed in the
paper and the paper's qualitative convergence claims.
"""
import ctypes
import os

import numpy as np

from . import build as _build

MAXLEV = 31
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32), ("M0", ctypes.c_int32), ("nRS", ctypes.c_int32),
        ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
        ("smoother", ctypes.c_int32), ("tau_src", ctypes.c_int32),
        ("seg_w", ctypes.c_int32 * (MAXLEV + 1)),
        ("seg_b", ctypes.c_int32 * (MAXLEV + 1)),
    ]


class OracleError(RuntimeError):
    pass


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        i = ctypes.c_int
        sigs = {
            "or_apply_L": [i, dp, dp],
            "or_restrict": [i, dp, dp],
            "or_prolong_lin": [i, dp, dp],
            "or_prolong_fmg": [i, dp, dp],
            "or_thomas": [i, dp, dp],
            "or_tau_rhs": [i, dp, dp, dp],
            "or_smooth": [pp, i, dp, dp, i, dp, dp],
            "or_kaczmarz": [dp, dp, i, i],
            "or_fmg_h": [pp, dp, dp],
            "or_fmg_v": [pp, dp, dp],
            "or_vcycles_h": [pp, dp, dp, i],
        }
        for name, args in sigs.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _arr(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


class Params:
    """Solve parameters; ``seg[l] = (w, b)`` segments level l (w = 0: whole level)."""

    def __init__(self, M, M0=2, nRS=1, nu1=1, nu2=1, smoother="lex", tau_src="assembled", seg=None):
        self.M, self.M0, self.nRS, self.nu1, self.nu2 = M, M0, nRS, nu1, nu2
        self.smoother, self.tau_src = smoother, tau_src
        self.seg = dict(seg or {})

    def c(self):
        p = _Params()
        p.M, p.M0, p.nRS, p.nu1, p.nu2 = self.M, self.M0, self.nRS, self.nu1, self.nu2
        p.smoother = {"lex": 0, "rb": 1}[self.smoother]
        p.tau_src = {"assembled": 0, "segment": 1}[self.tau_src]
        for l, (w, b) in self.seg.items():
            p.seg_w[l] = w
            p.seg_b[l] = b
        return p

    def __repr__(self):
        return (f"Params(M={self.M}, M0={self.M0}, nRS={self.nRS}, nu=({self.nu1},{self.nu2}), "
                f"smoother={self.smoother}, tau_src={self.tau_src}, seg={self.seg})")


def sr_params(M, W, b, nRS=1, nu1=1, nu2=1, M0=2, smoother="lex", tau_src="assembled"):
    """SR levels (the finest nRS) split into segments of W >> (M-l) cells with
    b buffer cells per side; every other level is smoothed as a whole."""
    seg = {}
    for l in range(M - nRS + 1, M + 1):
        w = W >> (M - l)
        if w < 2:
            raise ValueError("segment narrower than 2 cells on an SR level")
        seg[l] = (w, b)
    return Params(M, M0=M0, nRS=nRS, nu1=nu1, nu2=nu2, smoother=smoother, tau_src=tau_src, seg=seg)


def paper_params(M, nRS, halo_type, ns, M0=2):
    """The appendix program's configuration: every non-coarsest level smoothed
    by 2-cell patches with 2 (halo_type 1) or 4 (halo_type 2) buffer cells, or
    as a whole (halo_type 3); lexicographic Gauss-Seidel reversed after every
    sweep; tau from the assembled level; V(ns, ns)."""
    seg = {}
    if halo_type in (1, 2):
        for l in range(M0 + 1, M + 1):
            seg[l] = (2, 2 * halo_type)
    return Params(M, M0=M0, nRS=nRS, nu1=ns, nu2=ns, smoother="lex", tau_src="assembled", seg=seg)


def apply_L(u):
    u = _arr(u)
    out = np.empty_like(u)
    _check(lib().or_apply_L(len(u), _ptr(u), _ptr(out)), "apply_L")
    return out


def restrict(uf):
    uf = _arr(uf)
    uc = np.empty(len(uf) // 2)
    _check(lib().or_restrict(len(uc), _ptr(uf), _ptr(uc)), "restrict")
    return uc


def prolong_lin(uc):
    uc = _arr(uc)
    uf = np.empty(2 * len(uc))
    _check(lib().or_prolong_lin(len(uc), _ptr(uc), _ptr(uf)), "prolong_lin")
    return uf


def prolong_fmg(uc):
    uc = _arr(uc)
    uf = np.empty(2 * len(uc))
    _check(lib().or_prolong_fmg(len(uc), _ptr(uc), _ptr(uf)), "prolong_fmg")
    return uf


def thomas(rhs):
    rhs = _arr(rhs)
    u = np.empty_like(rhs)
    _check(lib().or_thomas(len(rhs), _ptr(rhs), _ptr(u)), "thomas")
    return u


def tau_rhs(ubar, rhs_f):
    ubar, rhs_f = _arr(ubar), _arr(rhs_f)
    out = np.empty(len(ubar) // 2)
    _check(lib().or_tau_rhs(len(ubar), _ptr(ubar), _ptr(rhs_f), _ptr(out)), "tau_rhs")
    return out


def smooth(params, level, u, rhs, nsweeps, uH=None):
    u, rhs = _arr(u), _arr(rhs)
    uH = None if uH is None else _arr(uH)
    out = np.empty_like(u)
    p = params.c()
    _check(lib().or_smooth(ctypes.byref(p), level, _ptr(u), _ptr(rhs), nsweeps, _ptr(uH), _ptr(out)),
           "smooth")
    return out


def kaczmarz(v, uH, e0, e1):
    v = _arr(v).copy()
    uH = _arr(uH)
    _check(lib().or_kaczmarz(_ptr(v), _ptr(uH), e0, e1), "kaczmarz")
    return v


def fmg_h(params, f):
    """One FMG-FAS(-SR) solve with every level stored."""
    f = _arr(f)
    assert len(f) == 1 << params.M
    u = np.empty_like(f)
    p = params.c()
    _check(lib().or_fmg_h(ctypes.byref(p), _ptr(f), _ptr(u)), "fmg_h")
    return u


def fmg_v(params, f):
    """The same solve run serially with segmental refinement (level M never stored)."""
    f = _arr(f)
    assert len(f) == 1 << params.M
    u = np.empty_like(f)
    p = params.c()
    _check(lib().or_fmg_v(ctypes.byref(p), _ptr(f), _ptr(u)), "fmg_v")
    return u


def vcycles_h(params, f, u0, ncycles):
    f = _arr(f)
    u = _arr(u0).copy()
    p = params.c()
    _check(lib().or_vcycles_h(ctypes.byref(p), _ptr(f), _ptr(u), ncycles), "vcycles_h")
    return u
