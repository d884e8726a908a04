"""Parity on the shapes of the workload configurations beyond the headline one
(which test_parity_gpu.py runs at full size): the small plain problem, the
batch of variable-coefficient problems of log-uniform sizes with tuned
segment layouts, the adjoint with the coefficient gradient at N = 2^22, and
the Bratu problem at N = 2^26 with 16384 segments plus a batch of Bratu
problems of log-uniform sizes.  Every case runs in both precisions (FP64, and
the mixed precision that these configurations name: fixed point for the
constant coefficient, FP32 sweep corrections around FP64 residuals, tau and
coarsest solves for the variable coefficient and Bratu); every check is
against the FP64 oracle with the same parameters, tolerance 1e-10 relative
max-norm, and where the truncation error dominates the rounding, the error
against the exact solution is held within 1.5x the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_plain_1024_cells_gpu(precision):
    # N = 1024, coarsest 4 cells (10 levels), 4 segments of 256, buffer 4, V(1,1), 8 modes
    pytest.importorskip("torch")
    M, W, b = 10, 256, 4
    f, ue, _ = workloads.sine_series(M, 8, seed=0)
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b), f)
    assert rel(u, ref) <= TOL
    assert np.max(np.abs(u - ue)) <= 1.5 * np.max(np.abs(ref - ue))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_varcoef_batch_log_uniform_sizes_tuned_gpu(precision):
    # sizes m ~ U{10..20} (seeded), a = exp(g/2) with 16 modes, one batched plan per
    # size with the autotuner's segment layout, every problem against the oracle
    # and within 1.5x the oracle's error against the exact solution
    pytest.importorskip("torch")
    sizes = sorted(set(int(m) for m in workloads.batch_sizes(8, 10, 20, seed=3)))
    for M in sizes:
        best, _ = srfmg.autotune(M, reps=2, op=srfmg.VARCOEF, precision=precision)
        W, b = best.segment_width, best.buffer_width
        data = [workloads.varcoef_series(M, 16, seed=100 * M + k) for k in range(3)]
        s = srfmg.Solver(M, op=srfmg.VARCOEF, segment_width=W, buffer_width=b, batch=3, precision=precision)
        try:
            s.set_coefficient(_dev(np.concatenate([d[2] for d in data])))
            ub = s.solve(_dev(np.concatenate([d[0] for d in data]))).cpu().numpy().reshape(3, -1)
        finally:
            s.close()
        for k, (f, ue, la) in enumerate(data):
            ref = oracle.fmg_v(oracle.sr_params(M, W, b, op="varcoef", coef=np.exp(la)), f)
            assert rel(ub[k], ref) <= TOL, (M, W, b, k)
            assert np.max(np.abs(ub[k] - ue)) <= 1.5 * np.max(np.abs(ref - ue)), (M, k)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_varcoef_adjoint_and_coefficient_gradient_2_22_gpu(precision):
    # N = 2^22: u and lam = dL/df against the oracle's FMG-SR solves of the state
    # and adjoint equations; dL/dlog a by the GPU kernel on the oracle's u and lam;
    # and the face-scaling identity sum_f dL/dlog a_f = -lam^T A u on the GPU's own
    # outputs (A u written out below from the flux definition)
    torch = pytest.importorskip("torch")
    M, W, b = 22, 4096, 8
    f, ue, la = workloads.varcoef_series(M, 16, seed=1)
    rng = np.random.default_rng(11)
    u_obs = ue + rng.normal(0.0, 1e-3, 1 << M)
    a = np.exp(la)
    p = oracle.sr_params(M, W, b, op="varcoef", coef=a)
    s = srfmg.Solver(M, op=srfmg.VARCOEF, segment_width=W, buffer_width=b, precision=precision)
    try:
        s.set_coefficient(_dev(la))
        uo = oracle.fmg_v(p, f)
        lo = oracle.fmg_v(p, uo - u_obs)
        assert rel(s.solve(_dev(f)).cpu().numpy(), uo) <= TOL
        # the adjoint solve on the same right-hand side as the oracle's (dL/du at
        # the oracle's u: lam is tiny against the 1e-3 noise, so a right-hand side
        # formed from the GPU's own u would differ by far more than the solves do).
        # Mixed precision: the fixed-point grid unit is 2^-59 of the a priori bound
        # max|g| / (4 min a) of the solution, which this noise misfit's lam stays
        # 2^15 below; every smoothing pass rounds each cell to a unit, which the
        # scaled discrete operator's Green's function (row sums up to N^2 / 8)
        # amplifies, so the difference is held to four passes' worth, 4 N^2 / 8
        # units (or 1e-10 of max|lam|, whichever is larger; measured 5.8e-10 of
        # max|lam|, far inside it)
        g = uo - u_obs
        la_gpu = s.adjoint(_dev(g)).cpu().numpy()
        if precision == srfmg.FP64:
            assert rel(la_gpu, lo) <= TOL
        else:
            unit = 2.0 ** -59 * np.max(np.abs(g)) / (4.0 * np.min(a))
            n = float(1 << M)
            assert np.max(np.abs(la_gpu - lo)) <= max(TOL * np.max(np.abs(lo)), 4.0 * n * n / 8.0 * unit)
        gk = s.coef_gradient(_dev(uo), _dev(lo)).cpu().numpy()
        go = oracle.coef_gradient(a, uo, lo)
        assert rel(gk, go) <= 1e-13
        # the differentiable solve end to end (its own u, lam and gradient)
        fd = _dev(f).requires_grad_(True)
        lad = _dev(la).requires_grad_(True)
        u = srfmg.solve_autograd(s, fd, log_a=lad)
        L = 0.5 * torch.sum((u - _dev(u_obs)) ** 2)
        g_f, g_la = torch.autograd.grad(L, [fd, lad])
        u_np, lam_np, gla_np = u.detach().cpu().numpy(), g_f.cpu().numpy(), g_la.cpu().numpy()
    finally:
        s.close()
    n = 1 << M
    flux = np.empty(n + 1)                      # a_f (u_f - u_{f-1}), odd ghosts at the walls
    flux[1:n] = a[1:n] * (u_np[1:] - u_np[:-1])
    flux[0] = a[0] * 2.0 * u_np[0]
    flux[n] = a[n] * (-2.0 * u_np[n - 1])
    Au = float(n) * n * (flux[:-1] - flux[1:])
    lhs = gla_np.sum()
    rhs = -(lam_np @ Au)
    assert abs(lhs - rhs) <= 1e-9 * np.sum(np.abs(gla_np))


@pytest.fixture(scope="module")
def bratu_2_26():
    # N = 2^26, 16384 segments of 4096, V(2,1), lam = 1, and the serial SR oracle's
    # solve of it (about 20 s on one host core)
    M, W, b, lam = 26, 4096, 8, 1.0
    f, ue, _ = workloads.bratu_series(M, 16, seed=1, lam=lam)
    ref = oracle.fmg_v(oracle.sr_params(M, W, b, nu1=2, nu2=1, op="bratu", lam=lam), f)
    return M, W, b, lam, f, ref


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_bratu_2_26_gpu(bratu_2_26, precision):
    # the full solve against the oracle (rounding-limited at this size: the O(h^2)
    # truncation error is about 1e-16, so no error-vs-exact criterion applies)
    pytest.importorskip("torch")
    M, W, b, lam, f, ref = bratu_2_26
    s = srfmg.Solver(M, op=srfmg.BRATU, lambda_=lam, segment_width=W, buffer_width=b, nu1=2, nu2=1,
                     precision=precision)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    assert rel(u, ref) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_bratu_batch_log_uniform_sizes_gpu(precision):
    # sizes m ~ U{12..18} (seeded), two problems per size in one batched plan
    pytest.importorskip("torch")
    sizes = sorted(set(int(m) for m in workloads.batch_sizes(8, 12, 18, seed=4)))
    for M in sizes:
        W = min(4096, (1 << M) // 4)
        fs = [workloads.bratu_series(M, 16, seed=10 * M + k, lam=1.0)[0] for k in range(2)]
        s = srfmg.Solver(M, op=srfmg.BRATU, lambda_=1.0, segment_width=W, buffer_width=8, nu1=2, batch=2,
                         precision=precision)
        try:
            ub = s.solve(_dev(np.concatenate(fs))).cpu().numpy().reshape(2, -1)
        finally:
            s.close()
        for k in range(2):
            ref = oracle.fmg_v(oracle.sr_params(M, W, 8, nu1=2, op="bratu", lam=1.0), fs[k])
            assert rel(ub[k], ref) <= TOL, (M, k)
