"""The Bratu problem -u'' + lam e^u = f on the GPU (the pointwise Newton
Gauss-Seidel sweep, the nonlinear tau correction and Newton on the coarsest
level) against the FP64 oracle on the same seeded inputs, in both precisions:
FP64, and the mixed precision whose sweeps solve the Newton correction
recurrence in FP32 (residual, tau, interpolation and coarsest solve in FP64).
Tolerance 1e-10 relative max-norm for both: the two sides differ in rounding
order, in the chunked evaluation of the sweep's recurrence and, mixed, in the
FP32 rounding of corrections whose size at the end of the solve is that of
its discretization error.  The host-side argument checks run without a GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


def rel_maxnorm(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def mixed_tol(ref, ue):
    """Tolerance of the mixed precision against the FP64 oracle.  Its sweeps
    round each correction to FP32 (2^-24 of it), and the corrections of a
    solve's last cycles are of the size of the solve's error against the exact
    solution, so the two results may differ by a small multiple of 2^-24 times
    that error: the bound is 2^-20 times the oracle's relative error against
    the exact solution, or 1e-10, whichever is larger (it only exceeds 1e-10
    on the smallest grids, whose discretization error is about 1e-3)."""
    return max(TOL, 2.0 ** -20 * np.max(np.abs(ref - ue)) / np.max(np.abs(ref)))


def _create(**kw):
    lib = srfmg.load()
    p = srfmg.default_params(12)
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    return lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h))


def test_bratu_parameters_are_checked_on_the_host():
    assert _create(op=srfmg.LAPLACE, lambda_=1.0) == srfmg.EINVAL
    assert _create(op=srfmg.BRATU, lambda_=-1.0) == srfmg.EINVAL
    assert _create(op=srfmg.BRATU, lambda_=float("inf")) == srfmg.EINVAL
    assert _create(op=srfmg.BRATU, lambda_=float("nan")) == srfmg.EINVAL
    assert _create(op=3) == srfmg.EINVAL


CASES = [
    # (M, nRS, W, b, nu1, nu2, M0, lam)
    (6, 1, 16, 2, 1, 1, 2, 1.0),
    (10, 1, 256, 4, 1, 1, 2, 1.0),
    (12, 1, 64, 8, 1, 1, 2, 5.0),
    (13, 1, 128, 8, 2, 1, 2, 1.0),
    (14, 1, 4096, 8, 2, 2, 3, 1.0),
    (16, 1, 4096, 64, 1, 1, 6, 0.5),
    (17, 1, 2048, 8, 2, 1, 2, 1.0),
    (8, 0, 0, 0, 1, 1, 2, 1.0),
    (15, 0, 0, 0, 1, 2, 2, 1.0),
]


def oracle_params(M, nRS, W, b, nu1, nu2, M0, lam):
    if nRS == 0:
        return oracle.Params(M, M0=M0, nRS=0, nu1=nu1, nu2=nu2, op="bratu", lam=lam)
    return oracle.sr_params(M, W, b, nRS=1, nu1=nu1, nu2=nu2, M0=M0, op="bratu", lam=lam)


def gpu_solve(M, f, **kw):
    torch = pytest.importorskip("torch")
    s = srfmg.Solver(M, **kw)
    try:
        u = s.solve(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        return u.cpu().numpy()
    finally:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,nRS,W,b,nu1,nu2,M0,lam", CASES)
def test_bratu_parity_gpu(M, nRS, W, b, nu1, nu2, M0, lam, precision):
    f, ue, _ = workloads.bratu_series(M, 16, seed=M, lam=lam)
    kw = dict(op=srfmg.BRATU, lambda_=lam, n_sr_levels=nRS, nu1=nu1, nu2=nu2, log2_n_coarsest=M0,
              precision=precision)
    if nRS:
        kw.update(segment_width=W, buffer_width=b)
    u = gpu_solve(M, f, **kw)
    ref = oracle.fmg_h(oracle_params(M, nRS, W, b, nu1, nu2, M0, lam), f)
    if precision == srfmg.FP64:
        assert rel_maxnorm(u, ref) <= TOL
    else:
        assert rel_maxnorm(u, ref) <= mixed_tol(ref, ue)
        assert np.max(np.abs(u - ue)) <= 1.5 * np.max(np.abs(ref - ue))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_bratu_large_gpu(precision):
    # N = 2^20, 256 segments of 4096 cells, V(2,1): against the serial SR oracle,
    # and at discretization accuracy against the manufactured solution (the
    # mixed-precision bar: error vs exact within 1.5x the FP64 oracle's)
    M, W, b, lam = 20, 4096, 8, 1.0
    f, ue, _ = workloads.bratu_series(M, 16, seed=1, lam=lam)
    u = gpu_solve(M, f, op=srfmg.BRATU, lambda_=lam, segment_width=W, buffer_width=b, nu1=2, nu2=1,
                  precision=precision)
    ref = oracle.fmg_v(oracle.sr_params(M, W, b, nu1=2, nu2=1, op="bratu", lam=lam), f)
    assert rel_maxnorm(u, ref) <= TOL
    assert np.max(np.abs(u - ue)) <= 1.5 * np.max(np.abs(ref - ue))


@pytest.mark.gpu
def test_bratu_has_no_adjoint_gpu():
    torch = pytest.importorskip("torch")
    s = srfmg.Solver(12, op=srfmg.BRATU, lambda_=1.0)
    try:
        x = torch.zeros(1 << 12, dtype=torch.float64, device="cuda")
        with pytest.raises(srfmg.SrfmgError):
            s.adjoint(x)
    finally:
        s.close()


@pytest.mark.gpu
def test_mixed_exponential_matches_exp_gpu():
    # the mixed precision's exponential (Tang's table-driven method, cubic on
    # |r| <= ln2/512) against CUDA's exp: the dropped terms bound it by 1.5e-13
    from paper_1207_6720_gb300 import srfmg
    for lo, hi, n in ((-40.0, 40.0, 1 << 22), (-1e-3, 1e-3, 1 << 16), (-700.0, 700.0, 1 << 22), (0.0, 0.0, 1)):
        assert srfmg.exp_error(lo, hi, n) <= 1.6e-13, (lo, hi)
