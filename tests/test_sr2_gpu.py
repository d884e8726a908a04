"""Two SR levels (n_sr_levels = 2) on the GPU against the oracle.

Fig. 3 makes every level above a threshold an SR level: segmented additive
smoothing in the pre-smoothing leg (the top level from Pi of the level below,
the SR levels below it from their assembled restricted iterate), and in the
post-smoothing leg the full update Pi u_{l-1} (Eq. 5) with compatible
relaxation (Fig. 5) on every SR level.  Level M - 1 has segments of W/2 cells
with the same b buffer cells.  The oracle runs the same algorithm (sr_params
with nRS = 2); tolerance 1e-10 relative max-norm.  Host-side argument checks
for two SR levels are in test_abi_host.py.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


def rel_maxnorm(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


CASES = [
    # (M, W, b, nu1, nu2, M0)
    (8, 32, 4, 1, 1, 2),          # the tail reaches level M - 2
    (10, 256, 4, 1, 1, 2),
    (12, 64, 8, 2, 1, 2),
    (14, 4096, 8, 1, 1, 3),
    (16, 1024, 8, 1, 2, 2),       # stored levels 13, 14 between the tail and the SR levels
    (17, 2048, 16, 1, 1, 6),
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,W,b,nu1,nu2,M0", CASES)
def test_two_sr_levels_parity_gpu(M, W, b, nu1, nu2, M0, precision):
    pytest.importorskip("torch")
    f, _, _ = workloads.sine_series(M, 16, seed=M)
    s = srfmg.Solver(M, n_sr_levels=2, segment_width=W, buffer_width=b, nu1=nu1, nu2=nu2, log2_n_coarsest=M0,
                     precision=precision)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=2, nu1=nu1, nu2=nu2, M0=M0), f)
    assert rel_maxnorm(u, ref) <= TOL


@pytest.mark.gpu
def test_two_sr_levels_differ_from_one_gpu():
    # the second SR level changes the answer (segmented smoothing and the full
    # update on level M - 1): the GPU follows the oracle in both, not one for both
    pytest.importorskip("torch")
    M, W, b = 12, 64, 4
    f, _, _ = workloads.sine_series(M, 16, seed=3)
    out = {}
    for nRS in (1, 2):
        s = srfmg.Solver(M, n_sr_levels=nRS, segment_width=W, buffer_width=b)
        try:
            out[nRS] = s.solve(_dev(f)).cpu().numpy()
        finally:
            s.close()
    r1 = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=1), f)
    r2 = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=2), f)
    assert rel_maxnorm(r1, r2) > 1e-8
    assert rel_maxnorm(out[1], r1) <= TOL and rel_maxnorm(out[2], r2) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("op", [srfmg.BRATU, srfmg.VARCOEF])
def test_two_sr_levels_other_operators_gpu(op):
    pytest.importorskip("torch")
    M, W, b = 13, 512, 8
    if op == srfmg.BRATU:
        f, _, _ = workloads.bratu_series(M, 16, seed=4, lam=1.0)
        kw, okw = dict(op=srfmg.BRATU, lambda_=1.0, nu1=2), dict(op="bratu", lam=1.0, nu1=2)
        log_a = None
    else:
        f, _, log_a = workloads.varcoef_series(M, 16, seed=4)
        kw, okw = dict(op=srfmg.VARCOEF), dict(op="varcoef", coef=np.exp(log_a))
    s = srfmg.Solver(M, n_sr_levels=2, segment_width=W, buffer_width=b, **kw)
    try:
        if log_a is not None:
            s.set_coefficient(_dev(log_a))
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=2, **okw), f)
    assert rel_maxnorm(u, ref) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_two_sr_levels_batch_functionals_reconstruct_gpu(precision):
    torch = pytest.importorskip("torch")
    M, W, b, B = 14, 512, 8, 3
    fs = [workloads.sine_series(M, 16, seed=30 + k)[0] for k in range(B)]
    kw = dict(n_sr_levels=2, segment_width=W, buffer_width=b, precision=precision)
    single = srfmg.Solver(M, **kw)
    batched = srfmg.Solver(M, batch=B, **kw)
    try:
        ref = [single.solve(_dev(f)).cpu().numpy() for f in fs]
        fd = _dev(np.concatenate(fs))
        ub = batched.solve(fd).cpu().numpy().reshape(B, -1)
        for k in range(B):
            assert np.array_equal(ub[k], ref[k])
        F = batched.solve_functionals(fd).cpu().numpy().reshape(B, -1)
        part = batched.reconstruct(fd, 5, 4).cpu().numpy().reshape(B, -1)
        assert np.array_equal(part, ub[:, 5 * W:9 * W])
        torch.cuda.synchronize()
    finally:
        single.close()
        batched.close()
    for k in range(B):
        Fo = oracle.functionals(ref[k])
        d = TOL * np.max(np.abs(ref[k]))
        assert abs(F[k, 0] - Fo[0]) <= 2 * d and abs(F[k, 2] - Fo[2]) <= 2 * d
    r = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=2), fs[1])
    assert rel_maxnorm(ub[1], r) <= TOL


@pytest.mark.gpu
def test_two_sr_levels_large_gpu():
    # N = 2^20, 256 segments of 4096 on level 20 and of 2048 on level 19: against
    # the oracle and at discretization accuracy (within 1.5x the oracle's error)
    pytest.importorskip("torch")
    M, W, b = 20, 4096, 8
    f, ue, _ = workloads.sine_series(M, 32, seed=1)
    s = srfmg.Solver(M, n_sr_levels=2, segment_width=W, buffer_width=b, precision=srfmg.MIXED)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=2), f)
    assert rel_maxnorm(u, ref) <= TOL
    assert np.max(np.abs(u - ue)) <= 1.5 * np.max(np.abs(ref - ue))
