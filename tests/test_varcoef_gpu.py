"""The variable-coefficient problem -(a u')' = f on the GPU (the
coefficient-weighted sweep, tau and coarsest solve) against the FP64 oracle on
the same seeded inputs, in both precisions: FP64, and the mixed precision
whose sweeps solve the Gauss-Seidel correction recurrence in FP32 (residual,
tau, interpolation and coarsest solve in FP64); tolerance 1e-10 relative
max-norm for both.  The host-side argument checks run without a GPU."""
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


def test_varcoef_parameters_are_checked_on_the_host():
    assert _create(op=srfmg.VARCOEF, lambda_=1.0) == srfmg.EINVAL
    lib = srfmg.load()
    assert lib.srfmg_set_coefficient(None, None, None) == srfmg.EINVAL
    assert lib.srfmg_coef_gradient(None, None, None, None, None) == srfmg.EINVAL


CASES = [
    # (M, nRS, W, b, nu1, nu2, M0)
    (6, 1, 16, 2, 1, 1, 2),
    (10, 1, 256, 4, 1, 1, 2),
    (12, 1, 64, 8, 1, 1, 2),
    (13, 1, 128, 8, 2, 1, 2),
    (14, 1, 4096, 8, 2, 2, 3),
    (16, 1, 4096, 64, 1, 1, 6),
    (17, 1, 2048, 8, 1, 1, 2),
    (8, 0, 0, 0, 1, 1, 2),
    (15, 0, 0, 0, 1, 2, 2),
]


def oracle_params(M, nRS, W, b, nu1, nu2, M0, log_a):
    a = np.exp(log_a)
    if nRS == 0:
        return oracle.Params(M, M0=M0, nRS=0, nu1=nu1, nu2=nu2, op="varcoef", coef=a)
    return oracle.sr_params(M, W, b, nRS=1, nu1=nu1, nu2=nu2, M0=M0, op="varcoef", coef=a)


def _kw(nRS, W, b, nu1, nu2, M0, precision=srfmg.FP64):
    kw = dict(op=srfmg.VARCOEF, n_sr_levels=nRS, nu1=nu1, nu2=nu2, log2_n_coarsest=M0, precision=precision)
    if nRS:
        kw.update(segment_width=W, buffer_width=b)
    return kw


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,nRS,W,b,nu1,nu2,M0", CASES)
def test_varcoef_parity_gpu(M, nRS, W, b, nu1, nu2, M0, precision):
    torch = pytest.importorskip("torch")
    f, ue, log_a = workloads.varcoef_series(M, 16, seed=M)
    s = srfmg.Solver(M, **_kw(nRS, W, b, nu1, nu2, M0, precision))
    try:
        s.set_coefficient(torch.from_numpy(log_a).cuda())
        u = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle_params(M, nRS, W, b, nu1, nu2, M0, log_a), f)
    if precision == srfmg.FP64:
        assert rel_maxnorm(u, ref) <= TOL
    else:
        assert rel_maxnorm(u, ref) <= mixed_tol(ref, ue)
        assert np.max(np.abs(u - ue)) <= 1.5 * np.max(np.abs(ref - ue))


@pytest.mark.gpu
def test_coefficient_can_change_between_replayed_solves_gpu():
    torch = pytest.importorskip("torch")
    M, W, b = 14, 1024, 8
    f, _, la1 = workloads.varcoef_series(M, 16, seed=1)
    _, _, la2 = workloads.varcoef_series(M, 16, seed=2, amp=2.0)
    s = srfmg.Solver(M, **_kw(1, W, b, 1, 1, 2))
    try:
        fd = torch.from_numpy(f).cuda()
        u = torch.empty_like(fd)
        s.solve(fd, u)                                   # a = 1 until set
        u_one = u.cpu().numpy()
        for la in (la1, la2, la1):                       # the same graph replays
            s.set_coefficient(torch.from_numpy(la).cuda())
            s.solve(fd, u)
            ref = oracle.fmg_h(oracle.sr_params(M, W, b, op="varcoef", coef=np.exp(la)), f)
            assert rel_maxnorm(u.cpu().numpy(), ref) <= TOL
    finally:
        s.close()
    ref1 = oracle.fmg_h(oracle.sr_params(M, W, b), f)    # a = 1 is the constant-coefficient solve
    assert rel_maxnorm(u_one, ref1) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_varcoef_batch_gpu(precision):
    torch = pytest.importorskip("torch")
    M, W, b, B = 13, 512, 8, 3
    data = [workloads.varcoef_series(M, 16, seed=10 + k) for k in range(B)]
    s = srfmg.Solver(M, batch=B, **_kw(1, W, b, 1, 1, 2, precision))
    try:
        s.set_coefficient(torch.from_numpy(np.concatenate([d[2] for d in data])).cuda())
        ub = s.solve(torch.from_numpy(np.concatenate([d[0] for d in data])).cuda()).cpu().numpy().reshape(B, -1)
    finally:
        s.close()
    for k, (f, _, la) in enumerate(data):
        ref = oracle.fmg_h(oracle.sr_params(M, W, b, op="varcoef", coef=np.exp(la)), f)
        assert rel_maxnorm(ub[k], ref) <= TOL


@pytest.mark.gpu
def test_set_coefficient_needs_a_varcoef_plan_gpu():
    torch = pytest.importorskip("torch")
    s = srfmg.Solver(12)
    try:
        with pytest.raises(srfmg.SrfmgError):
            s.set_coefficient(torch.zeros((1 << 12) + 1, dtype=torch.float64, device="cuda"))
    finally:
        s.close()


@pytest.mark.gpu
def test_rough_coefficient_is_rejected_and_reset_gpu():
    # the sweep's 99-cell carry is exact for neighbouring faces within a factor
    # 1.5 on every level of 128 or more cells; a rougher coefficient is refused
    # and the plan falls back to a = 1
    torch = pytest.importorskip("torch")
    M, W, b = 12, 512, 8
    n = 1 << M
    f, _, _ = workloads.sine_series(M, 16, seed=3)
    s = srfmg.Solver(M, **_kw(1, W, b, 1, 1, 2))
    fd = torch.from_numpy(f).cuda()
    jump_ok = np.zeros(n + 1)
    jump_ok[n // 2:] = np.log(1.45)                      # one jump by 1.45: accepted
    jump_bad = np.zeros(n + 1)
    jump_bad[n // 2 + 3:] = np.log(1.6)                  # one jump by 1.6 on the finest level
    ramp = np.zeros(n + 1)                               # smooth on the finest level (1.6^(1/32) per face),
    ramp[2048:2081] = np.linspace(0.0, np.log(1.6), 33)  # but faces 2048 and 2080 of level 7 differ by 1.6
    ramp[2081:] = np.log(1.6)
    nan = np.zeros(n + 1)
    nan[17] = np.nan
    big = np.zeros(n + 1)
    big[5] = 800.0
    try:
        s.set_coefficient(torch.from_numpy(jump_ok).cuda())
        u = s.solve(fd).cpu().numpy()
        ref = oracle.fmg_h(oracle.sr_params(M, W, b, op="varcoef", coef=np.exp(jump_ok)), f)
        assert rel_maxnorm(u, ref) <= TOL
        ref1 = oracle.fmg_h(oracle.sr_params(M, W, b), f)
        for la in (jump_bad, ramp, nan, big):
            with pytest.raises(srfmg.SrfmgError):
                s.set_coefficient(torch.from_numpy(la).cuda())
            u = s.solve(fd).cpu().numpy()                # a = 1 after the refusal
            assert rel_maxnorm(u, ref1) <= TOL
    finally:
        s.close()


@pytest.mark.gpu
def test_mixed_refuses_a_contrast_beyond_2_to_the_8_gpu():
    # a smooth ramp of log a from 0 to 6 (contrast e^6 > 2^8): every pair of
    # neighbouring faces is within the sweep's factor 1.5, so FP64 takes it; the
    # fixed-point coefficient refuses it and falls back to a = 1
    torch = pytest.importorskip("torch")
    M, W, b = 12, 512, 8
    n = 1 << M
    ramp = np.linspace(0.0, 6.0, n + 1)
    f, _, _ = workloads.sine_series(M, 16, seed=3)
    fd = torch.from_numpy(f).cuda()
    s64 = srfmg.Solver(M, **_kw(1, W, b, 1, 1, 2))
    smx = srfmg.Solver(M, **_kw(1, W, b, 1, 1, 2, srfmg.MIXED))
    try:
        s64.set_coefficient(torch.from_numpy(ramp).cuda())
        with pytest.raises(srfmg.SrfmgError):
            smx.set_coefficient(torch.from_numpy(ramp).cuda())
        u = smx.solve(fd).cpu().numpy()
        ref1 = oracle.fmg_h(oracle.sr_params(M, W, b), f)
        assert rel_maxnorm(u, ref1) <= TOL
        ok = ramp * (np.log(200.0) / 6.0)               # contrast 200: accepted
        smx.set_coefficient(torch.from_numpy(ok).cuda())
        ue_ref = oracle.fmg_h(oracle.sr_params(M, W, b, op="varcoef", coef=np.exp(ok)), f)
        assert rel_maxnorm(smx.solve(fd).cpu().numpy(), ue_ref) <= 1e-9
    finally:
        s64.close()
        smx.close()
