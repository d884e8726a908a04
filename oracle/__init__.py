"""FP64 serial CPU oracle for FMG-FAS with segmental refinement.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this package.  The C source (``srfmg_oracle.c``) restates the paper's
algorithms (Figs. 1-4, Eqs. 1-7, the operators of Sec. 4, and the Bratu
operator -u'' + lam e^u of the nonlinear FAS of Sec. 2.2) step by step; this
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
        ("op", ctypes.c_int32), ("lam", ctypes.c_double),
        ("coef", ctypes.POINTER(ctypes.c_double)), ("coef_level", ctypes.c_int32),
        ("post", ctypes.c_int32),
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
            "or_apply_N": [i, ctypes.c_double, dp, dp],
            "or_apply_La": [i, dp, dp, dp],
            "or_coef_gradient": [i, dp, dp, dp, dp],
            "or_coarsest": [pp, i, dp, dp],
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

    def __init__(self, M, M0=2, nRS=1, nu1=1, nu2=1, smoother="lex", tau_src="assembled", seg=None,
                 op="laplace", lam=0.0, coef=None, post="full_update"):
        self.M, self.M0, self.nRS, self.nu1, self.nu2 = M, M0, nRS, nu1, nu2
        # post-smoothing leg of the SR levels: "full_update" (Eq. 5 + Fig. 5) or
        # "fas_recompute" (Eq. 4 on the recomputed pre-smoothed level)
        self.post = post
        self.smoother, self.tau_src = smoother, tau_src
        self.seg = dict(seg or {})
        self.op, self.lam = op, lam
        # op "varcoef": the face coefficients a_j, j = 0..2^L, of the finest level L
        self.coef = None if coef is None else _arr(coef)

    def c(self):
        p = _Params()
        p.M, p.M0, p.nRS, p.nu1, p.nu2 = self.M, self.M0, self.nRS, self.nu1, self.nu2
        p.smoother = {"lex": 0, "rb": 1}[self.smoother]
        p.tau_src = {"assembled": 0, "segment": 1}[self.tau_src]
        for l, (w, b) in self.seg.items():
            p.seg_w[l] = w
            p.seg_b[l] = b
        p.op = {"laplace": 0, "bratu": 1, "varcoef": 2}[self.op]
        p.post = {"full_update": 0, "fas_recompute": 1}[self.post]
        p.lam = self.lam
        if self.coef is not None:
            p.coef = _ptr(self.coef)          # self.coef keeps the array alive
            p.coef_level = int(np.log2(len(self.coef) - 1))
        return p

    def __repr__(self):
        return (f"Params(M={self.M}, M0={self.M0}, nRS={self.nRS}, nu=({self.nu1},{self.nu2}), "
                f"smoother={self.smoother}, tau_src={self.tau_src}, seg={self.seg}, op={self.op}, "
                f"lam={self.lam})")


def sr_params(M, W, b, nRS=1, nu1=1, nu2=1, M0=2, smoother="lex", tau_src="assembled", op="laplace",
              lam=0.0, coef=None, post="full_update"):
    """SR levels (the finest nRS) split into segments of W >> (M-l) cells with
    b buffer cells per side; every other level is smoothed as a whole."""
    seg = {}
    for l in range(M - nRS + 1, M + 1):
        w = W >> (M - l)
        if w < 2:
            raise ValueError("segment narrower than 2 cells on an SR level")
        seg[l] = (w, b)
    return Params(M, M0=M0, nRS=nRS, nu1=nu1, nu2=nu2, smoother=smoother, tau_src=tau_src, seg=seg,
                  op=op, lam=lam, coef=coef, post=post)


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


def apply_N(u, lam):
    """N(u) = L u + lam e^u (the Bratu operator; lam = 0: L)."""
    u = _arr(u)
    out = np.empty_like(u)
    _check(lib().or_apply_N(len(u), float(lam), _ptr(u), _ptr(out)), "apply_N")
    return out


def apply_La(u, a):
    """-(a u')' on one level with the face coefficients a (len(u) + 1 values)."""
    u, a = _arr(u), _arr(a)
    assert len(a) == len(u) + 1
    out = np.empty_like(u)
    _check(lib().or_apply_La(len(u), _ptr(a), _ptr(u), _ptr(out)), "apply_La")
    return out


def coef_gradient(a, u, lam):
    """dL/dlog a at the len(u) + 1 faces from the solution u and the adjoint
    state lam = A^{-1} dL/du of -(a u')' = f (face coefficients a)."""
    a, u, lam = _arr(a), _arr(u), _arr(lam)
    assert len(a) == len(u) + 1 and len(lam) == len(u)
    out = np.empty_like(a)
    _check(lib().or_coef_gradient(len(u), _ptr(a), _ptr(u), _ptr(lam), _ptr(out)), "coef_gradient")
    return out


def functionals(u, u_ref=None):
    """The five functionals of a fine-grid solution of N cells (h = 1/N) that
    the SR solve collects while it sweeps the fine grid (Fig. 3 computes a
    functional of the fine grid in the post-smoothing leg):
    [h sum u, h sum u^2, max|u|, h sum (u - u_ref)^2, max|u - u_ref|], the last
    two 0 without a reference.  Plain definitions; sums by math.fsum."""
    import math
    u = _arr(u)
    h = 1.0 / len(u)
    out = [h * math.fsum(u), h * math.fsum(u * u), float(np.max(np.abs(u))), 0.0, 0.0]
    if u_ref is not None:
        d = u - _arr(u_ref)
        out[3] = h * math.fsum(d * d)
        out[4] = float(np.max(np.abs(d)))
    return np.array(out)


def coarsest(params, rhs, u0):
    """The coarsest-level solve of ``params`` (Thomas, or Newton for Bratu)
    from the starting iterate u0."""
    rhs = _arr(rhs)
    u = _arr(u0).copy()
    p = params.c()
    _check(lib().or_coarsest(ctypes.byref(p), len(rhs), _ptr(rhs), _ptr(u)), "coarsest")
    return u


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
