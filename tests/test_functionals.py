"""Functionals collected while the fine grid is swept, and PDE decompression.

Fig. 3 computes a functional of the fine grid in the SR post-smoothing leg,
and the paper's section on obtaining the solution names the two ways out of a
solve whose fine grid is never stored: functionals collected on the fly, and a
stored coarse solution expanded locally on demand.  The GPU's post-leg reduces
each segment interior into five functionals (srfmg_solve_functionals, with or
without writing u) and re-runs the post-leg on chosen segments from the kept
coarse solution (srfmg_reconstruct).

Oracle pins (no GPU): the functionals' definitions against closed forms of the
discrete sine series at cell centres.  GPU: functionals against those of the
oracle's solution, with bounds that follow from the 1e-10 parity of u;
the same bits with and without writing u, on every run and for every problem
of a batch; reconstruction bit for bit equal to the solve's own cells.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


# ---------------------------------------------------------------- oracle pins

def test_functionals_of_a_sine_series_have_their_closed_forms():
    # at the cell centres x_i = (i + 1/2) h the sines sin(k pi x) (1 <= k < N) are
    # orthogonal with h sum sin^2 = 1/2, and h sum sin(k pi x_i) is h / sin(k pi h / 2)
    # for odd k and 0 for even k
    for M, K in ((6, 8), (10, 32)):
        N = 1 << M
        rng = np.random.default_rng(M)
        c = rng.normal(size=K) / np.arange(1, K + 1) ** 2
        x = (np.arange(N) + 0.5) / N
        u = sum(c[k - 1] * np.sin(k * np.pi * x) for k in range(1, K + 1))
        F = oracle.functionals(u)
        h = 1.0 / N
        mean = math.fsum(c[k - 1] * h / math.sin(k * math.pi * h / 2) for k in range(1, K + 1, 2))
        assert abs(F[0] - mean) <= 1e-14 * np.sum(np.abs(c)) * 2
        assert abs(F[1] - 0.5 * math.fsum(c * c)) <= 1e-14 * math.fsum(c * c)
        assert F[2] == np.max(np.abs(u)) and F[3] == 0.0 and F[4] == 0.0
        r = u + 1e-3 * np.sin(3 * np.pi * x)          # reference off by one mode
        G = oracle.functionals(u, r)
        assert abs(G[3] - 0.5e-6) <= 1e-18 and abs(G[4] - 1e-3) <= 1e-3 * (1 - math.cos(math.pi * 3 / (2 * N))) + 1e-18
        assert np.array_equal(G[:3], F[:3])


def test_entry_points_check_the_handle_on_the_host():
    lib = srfmg.load()
    assert lib.srfmg_solve_functionals(None, None, None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_reconstruct(None, None, 0, 1, None, None) == srfmg.EINVAL


# ---------------------------------------------------------------- GPU

def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _bounds_hold(Fg, Fo, umax):
    # |u_gpu - u_oracle| <= d = TOL umax gives |dF0| <= d, |dF1| <= d (2 umax + d),
    # |dF2| <= d, |sqrt F3 difference| <= d (triangle inequality of the norm),
    # |dF4| <= d; plus the summation rounding
    d = TOL * umax
    eps = 1e-13 * max(umax, umax * umax)
    assert abs(Fg[0] - Fo[0]) <= d + eps
    assert abs(Fg[1] - Fo[1]) <= d * (2 * umax + d) + eps
    assert abs(Fg[2] - Fo[2]) <= d
    assert abs(math.sqrt(Fg[3]) - math.sqrt(Fo[3])) <= d + eps
    assert abs(Fg[4] - Fo[4]) <= d


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,W,b", [(10, 256, 4), (14, 1024, 8), (17, 4096, 8)])
def test_functionals_parity_gpu(M, W, b, precision):
    torch = pytest.importorskip("torch")
    f, ue, _ = workloads.sine_series(M, 16, seed=M)
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision)
    try:
        fd, ued = _dev(f), _dev(ue)
        u = torch.empty_like(fd)
        Fu = s.solve_functionals(fd, u, ued).cpu().numpy()
        Fn = s.solve_functionals(fd, None, ued).cpu().numpy()      # the fine grid never written
        Fn2 = s.solve_functionals(fd, None, ued).cpu().numpy()
        u_plain = s.solve(fd)
        torch.cuda.synchronize()
        assert np.array_equal(Fu, Fn) and np.array_equal(Fn, Fn2)
        assert torch.equal(u, u_plain)
        F0 = s.solve_functionals(fd).cpu().numpy()                  # no reference
        assert np.array_equal(F0[:3], Fu[:3]) and F0[3] == 0.0 and F0[4] == 0.0
    finally:
        s.close()
    uo = oracle.fmg_h(oracle.sr_params(M, W, b), f)
    Fo = oracle.functionals(uo, ue)
    _bounds_hold(Fu, Fo, np.max(np.abs(uo)))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_functionals_with_a_reference_out_of_range_gpu(precision):
    # the fixed-point path forms u - u_ref on its integer grid and takes FP64 for
    # reference values beyond that grid's range: both kinds in one solve
    pytest.importorskip("torch")
    M, W, b = 12, 512, 8
    f, ue, _ = workloads.sine_series(M, 16, seed=5)
    ref = ue.copy()
    ref[[3, 700, 2049, 4095]] = [1e20, -3e15, 7e100, 2.5]      # squares stay finite
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision)
    try:
        F = s.solve_functionals(_dev(f), None, _dev(ref)).cpu().numpy()
    finally:
        s.close()
    Fo = oracle.functionals(oracle.fmg_h(oracle.sr_params(M, W, b), f), ref)
    assert abs(F[3] - Fo[3]) <= 1e-12 * Fo[3]
    assert abs(F[4] - Fo[4]) <= 1e-12 * Fo[4]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_functionals_of_a_batch_equal_single_solves_gpu(precision):
    torch = pytest.importorskip("torch")
    M, W, b, B = 13, 512, 8, 3
    data = [workloads.sine_series(M, 16, seed=20 + k) for k in range(B)]
    single = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision)
    batched = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision, batch=B)
    try:
        ref = [single.solve_functionals(_dev(f), None, _dev(ue)).cpu().numpy() for f, ue, _ in data]
        Fb = batched.solve_functionals(_dev(np.concatenate([d[0] for d in data])), None,
                                       _dev(np.concatenate([d[1] for d in data]))).cpu().numpy()
    finally:
        single.close()
        batched.close()
    for k in range(B):
        assert np.array_equal(Fb[5 * k:5 * k + 5], ref[k])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("op", [srfmg.LAPLACE, srfmg.BRATU])
def test_reconstruct_equals_the_solve_gpu(precision, op):
    torch = pytest.importorskip("torch")
    M, W, b, B = 14, 512, 8, 2
    kw = dict(op=srfmg.BRATU, lambda_=1.0) if op == srfmg.BRATU else {}
    if op == srfmg.BRATU:
        fs = [workloads.bratu_series(M, 16, seed=k, lam=1.0)[0] for k in range(B)]
    else:
        fs = [workloads.sine_series(M, 16, seed=k)[0] for k in range(B)]
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision, batch=B, **kw)
    nseg = (1 << M) // W
    try:
        fd = _dev(np.concatenate(fs))
        u = s.solve(fd).cpu().numpy().reshape(B, -1)
        for first, count in ((0, 1), (3, 5), (nseg - 2, 2), (0, nseg)):
            part = s.reconstruct(fd, first, count).cpu().numpy().reshape(B, -1)
            for k in range(B):
                assert np.array_equal(part[k], u[k, first * W:(first + count) * W]), (first, count, k)
        # after a functionals-only solve (no fine output) the coarse solution is kept
        s.solve_functionals(fd)
        part = s.reconstruct(fd, 7, 3).cpu().numpy().reshape(B, -1)
        assert np.array_equal(part, u[:, 7 * W:10 * W])
    finally:
        s.close()


@pytest.mark.gpu
def test_functionals_and_reconstruct_argument_checks_gpu():
    torch = pytest.importorskip("torch")
    M = 12
    f = _dev(workloads.sine_series(M, 8, seed=1)[0])
    plain = srfmg.Solver(M, n_sr_levels=0)
    s = srfmg.Solver(M, segment_width=256, buffer_width=8)
    try:
        with pytest.raises(srfmg.SrfmgError):
            plain.solve_functionals(f)
        plain.solve(f)
        with pytest.raises(srfmg.SrfmgError):
            plain.reconstruct(f, 0, 1)
        with pytest.raises(srfmg.SrfmgError):         # nothing solved yet
            s.reconstruct(f, 0, 1)
        s.solve(f)
        for first, count in ((-1, 1), (0, 0), (15, 2), (16, 1)):
            with pytest.raises(srfmg.SrfmgError):
                s.reconstruct(f, first, count)
        with pytest.raises(srfmg.SrfmgError):         # output overlapping the input
            st = s.lib.srfmg_solve_functionals(s.h, ctypes.c_void_p(f.data_ptr()), None, None,
                                               ctypes.c_void_p(f.data_ptr() + 64), None)
            s._check(st, "solve_functionals")
    finally:
        plain.close()
        s.close()
