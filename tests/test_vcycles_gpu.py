"""Further FAS V-cycles after the FMG cycle (n_vcycles).

Each extra cycle is the V-cycle of Fig. 1 on level M with the SR steps of
Fig. 3 on the SR levels, started from the current fine solution: segmented
smoothing of the fine iterate, restriction and tau, the stored levels, and the
full update with compatible relaxation.  The GPU (K5 from the caller's u, then
the usual launches) is held to the oracle's fmg_h followed by vcycles_h, and
the algebraic error against the exact discrete solution (Thomas) must contract
from cycle to cycle.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


def _create(**kw):
    lib = srfmg.load()
    p = srfmg.default_params(12)
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    return lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h))


def test_n_vcycles_is_checked_on_the_host():
    assert _create(n_vcycles=-1) == srfmg.EINVAL
    assert _create(n_vcycles=17) == srfmg.EINVAL


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    # (M, nRS, W, b, k, op)
    (12, 1, 256, 4, 1, "laplace"),
    (14, 1, 1024, 8, 2, "laplace"),
    (13, 2, 512, 8, 1, "laplace"),
    (17, 1, 4096, 8, 3, "laplace"),
    (13, 1, 512, 8, 1, "bratu"),
    (12, 0, 0, 0, 2, "laplace"),      # without SR: the whole problem below the tail, level M kept stored
    (15, 0, 0, 0, 3, "laplace"),
    (14, 0, 0, 0, 2, "bratu"),
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,nRS,W,b,k,op", CASES)
def test_vcycles_after_fmg_parity_gpu(M, nRS, W, b, k, op, precision):
    pytest.importorskip("torch")
    if op == "bratu":
        f, _, _ = workloads.bratu_series(M, 16, seed=M, lam=1.0)
        kw, okw = dict(op=srfmg.BRATU, lambda_=1.0), dict(op="bratu", lam=1.0)
    else:
        f, _, _ = workloads.sine_series(M, 16, seed=M)
        kw, okw = {}, {}
    s = srfmg.Solver(M, n_sr_levels=nRS, segment_width=W, buffer_width=b, n_vcycles=k, precision=precision, **kw)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    p = oracle.sr_params(M, W, b, nRS=nRS, **okw) if nRS else oracle.Params(M, nRS=0, **okw)
    ref = oracle.vcycles_h(p, f, oracle.fmg_h(p, f), k)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))


def test_sr_vcycles_stop_at_the_full_update_floor():
    # oracle: stored V-cycles converge to the discrete solution; SR V-cycles
    # contract to a floor set by the full update (Eq. 5: the fine level rebuilt
    # from Pi u_{M-1} and nu2 compatible-relaxation sweeps), below the
    # discretization error (1.1e-8 here)
    M = 14
    f, ue, _ = workloads.sine_series(M, 16, seed=1)
    ud = oracle.thomas(f)
    disc = np.max(np.abs(ud - ue))
    for p, floor in ((oracle.Params(M, nRS=0), 1e-11), (oracle.sr_params(M, 1024, 8), 0.5 * disc)):
        u = oracle.fmg_h(p, f)
        errs = [np.max(np.abs(u - ud))]
        for _ in range(4):
            u = oracle.vcycles_h(p, f, u, 1)
            errs.append(np.max(np.abs(u - ud)))
        assert errs[1] < 0.5 * errs[0] and errs[-1] < floor, errs
    # the SR floor is not the discrete solution: it stays put
    assert errs[-1] > 1e-10 and abs(errs[-1] - errs[-2]) < 0.05 * errs[-1]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_vcycles_reduce_the_algebraic_error_gpu(precision):
    pytest.importorskip("torch")
    M, W, b = 14, 1024, 8
    f, _, _ = workloads.sine_series(M, 16, seed=1)
    ud = oracle.thomas(f)
    errs = []
    for k in range(4):
        s = srfmg.Solver(M, segment_width=W, buffer_width=b, n_vcycles=k, precision=precision)
        try:
            u = s.solve(_dev(f)).cpu().numpy()
        finally:
            s.close()
        errs.append(np.max(np.abs(u - ud)))
    # one cycle contracts (7.3e-9 -> 2.2e-9 in the oracle), later ones stay at the SR floor
    assert errs[1] < 0.5 * errs[0], errs
    assert max(errs[2:]) < 1.1 * errs[1], errs


@pytest.mark.gpu
def test_functionals_need_u_with_vcycles_gpu():
    pytest.importorskip("torch")
    M = 12
    f = _dev(workloads.sine_series(M, 8, seed=1)[0])
    s = srfmg.Solver(M, segment_width=256, buffer_width=8, n_vcycles=1)
    try:
        with pytest.raises(srfmg.SrfmgError):
            s.solve_functionals(f)
        u = s.solve(f)
        F = s.solve_functionals(f, u.clone()).cpu().numpy()
        assert abs(F[2] - float(u.abs().max())) <= 1e-10 * F[2]
    finally:
        s.close()
