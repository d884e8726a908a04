"""Edge cases of the solve on the GPU: the zero right-hand side, a point source,
the smallest SR plan, and the largest problem the parameters admit (N = 2^28).

The zero rhs must give exactly zero in both precisions (every operation of the
method maps zero to zero); a point source (rough data that excites every mode)
and the smallest plan with an SR level (one segment of 16 cells) are held to
the oracle; at N = 2^28 the oracle would take minutes, so the solution is held
to the exact continuous one at discretization accuracy, which a wrong index
at that size (2^28 cells, 65536 segments) would break.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

TOL = 1e-10


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


PLANS = [
    (12, dict(segment_width=256, buffer_width=8)),
    (12, dict(n_sr_levels=2, segment_width=256, buffer_width=8)),
    (14, dict(n_sr_levels=0)),
    (9, dict(n_sr_levels=0)),                   # the whole problem in the tail
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,kw", PLANS)
def test_zero_rhs_gives_zero_gpu(M, kw, precision):
    torch = pytest.importorskip("torch")
    s = srfmg.Solver(M, precision=precision, **kw)
    try:
        u = s.solve(torch.zeros(1 << M, dtype=torch.float64, device="cuda"))
        assert torch.count_nonzero(u).item() == 0
        s.check()
    finally:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,kw", PLANS)
def test_point_source_parity_gpu(M, kw, precision):
    pytest.importorskip("torch")
    f = np.zeros(1 << M)
    f[(1 << M) // 3] = float(1 << M)          # a unit point load at one cell
    s = srfmg.Solver(M, precision=precision, **kw)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    nRS = kw.get("n_sr_levels", 1)
    if nRS:
        p = oracle.sr_params(M, kw["segment_width"], kw["buffer_width"], nRS=nRS)
    else:
        p = oracle.Params(M, nRS=0)
    ref = oracle.fmg_h(p, f)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_smallest_sr_plan_gpu(precision):
    pytest.importorskip("torch")
    M, W, b = 4, 16, 2                        # one segment of 16 cells, the tail below
    f, _, _ = workloads.sine_series(M, 4, seed=1)
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, precision=precision)
    try:
        u = s.solve(_dev(f)).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b), f)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_largest_problem_gpu(precision):
    # N = 2^28: 65536 segments of 4096; the input is built on the device, one
    # mode at a time (a 2 GB array per term), from the seeded coefficients
    torch = pytest.importorskip("torch")
    M, K = 28, 8
    n = 1 << M
    c = workloads.sine_coefficients(K, 1)
    x = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n
    f = torch.zeros_like(x)
    ue = torch.zeros_like(x)
    for k in range(1, K + 1):
        sk = torch.sin((k * math.pi) * x)
        f.add_(sk, alpha=float(c[k - 1] * (k * math.pi) ** 2))
        ue.add_(sk, alpha=float(c[k - 1]))
        del sk
    del x
    s = srfmg.Solver(M, segment_width=4096, buffer_width=8, precision=precision)
    try:
        u = s.solve(f)
        err = (u - ue).abs().max().item()
        umax = ue.abs().max().item()
        s.check()
    finally:
        s.close()
    print(f"N = 2^28, precision {precision}: max error vs exact {err:.3e} (max |u| {umax:.3f})")
    # rounding-limited at this size (the O(h^2) truncation error is about 1e-16):
    # measured 1.3e-11 in FP64 and 8.0e-13 in fixed point (exact sums) for max |u| 0.52
    assert err <= (5e-11 if precision == srfmg.FP64 else 5e-12) * umax
