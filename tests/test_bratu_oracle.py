"""Oracle pins for the nonlinear problem -u'' + lam e^u = f (Bratu).

The paper's FAS is written for a nonlinear operator (Sec. 2.2, Eqs. 1-2;
Fig. 1 with a nonlinear smoother); its studies are linear.  The oracle's
nonlinear pieces (pointwise Newton Gauss-Seidel, N(u) in the tau correction,
Newton on the coarsest level) are pinned here against an independent solve of
the same discrete equations (Newton with a banded Jacobian, scipy), against the
FAS fixed-point property, and against the second-order accuracy of one FMG
cycle.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import workloads

scipy_linalg = pytest.importorskip("scipy.linalg")

LAM = 1.0


def discrete_newton(f, lam, tol=1e-15, maxit=50):
    """Solve the cell-centred -u'' + lam e^u = f (odd ghosts) by Newton's method,
    independently of the oracle: banded Jacobian, scipy.linalg.solve_banded."""
    n = len(f)
    h2inv = float(n) * float(n)
    diag = np.full(n, 2.0 * h2inv)
    diag[0] = diag[-1] = 3.0 * h2inv
    u = np.zeros(n)
    for _ in range(maxit):
        Lu = diag * u
        Lu[1:] -= h2inv * u[:-1]
        Lu[:-1] -= h2inv * u[1:]
        r = f - (Lu + lam * np.exp(u))
        ab = np.zeros((3, n))
        ab[0, 1:] = -h2inv
        ab[1] = diag + lam * np.exp(u)
        ab[2, :-1] = -h2inv
        du = scipy_linalg.solve_banded((1, 1), ab, r)
        u = u + du
        if np.max(np.abs(du)) <= tol * max(1.0, np.max(np.abs(u))):
            break
    return u


def bratu(M, nRS=0, W=None, b=8, lam=LAM, nu1=1, nu2=1):
    if nRS:
        return oracle.sr_params(M, W, b, nRS=nRS, nu1=nu1, nu2=nu2, op="bratu", lam=lam)
    return oracle.Params(M, nRS=0, nu1=nu1, nu2=nu2, op="bratu", lam=lam)


def test_lam_zero_is_the_linear_solve_bit_for_bit():
    M = 12
    f, _, _ = workloads.sine_series(M, 16, seed=2)
    a = oracle.fmg_h(oracle.sr_params(M, 256, 8), f)
    b = oracle.fmg_h(oracle.sr_params(M, 256, 8, op="bratu", lam=0.0), f)
    assert np.array_equal(a, b)


def test_operator_adds_the_pointwise_exponential():
    rng = np.random.default_rng(1)
    u = rng.normal(scale=0.3, size=64)
    assert np.allclose(oracle.apply_N(u, 2.5) - oracle.apply_L(u), 2.5 * np.exp(u), rtol=1e-12, atol=0)


@pytest.mark.parametrize("n,lam", [(4, 1.0), (8, 5.0), (64, 0.5), (4, 60.0), (8, 40.0)])
def test_coarsest_newton_matches_an_independent_solve(n, lam):
    # (large lam: the exponential dominates the diagonal, where only Newton's
    # Jacobian, not L alone, converges)
    rng = np.random.default_rng(n)
    rhs = rng.normal(scale=10.0, size=n)
    p = oracle.Params(6, nRS=0, op="bratu", lam=lam)
    u = oracle.coarsest(p, rhs, np.zeros(n))
    ref = discrete_newton(rhs, lam)
    assert np.max(np.abs(u - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))
    # from another starting iterate: the same solution (unique for lam >= 0)
    u2 = oracle.coarsest(p, rhs, ref + 0.5)
    assert np.max(np.abs(u2 - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("M,lam", [(4, LAM), (2, 60.0)])
def test_smoother_fixed_point_is_the_discrete_solution(M, lam):
    # repeated nonlinear Gauss-Seidel sweeps on one small level converge to
    # N(u) = f (at lam = 60 on 4 cells the exponential dominates the diagonal:
    # a smoother that divides by L_ii alone overshoots)
    f, _, _ = workloads.bratu_series(M, 4, seed=3, lam=lam)
    p = bratu(M, lam=lam)
    u = oracle.smooth(p, M, np.zeros(1 << M), f, 2000)   # contraction about 0.96 per sweep at M = 4
    assert np.max(np.abs(u - discrete_newton(f, lam))) <= 1e-12


@pytest.mark.parametrize("M", [6, 9])
def test_discrete_solution_is_a_fixed_point_of_the_fas_vcycle(M):
    # with the exact discrete solution as iterate the coarse correction of
    # Eqs. 1-2 is zero: a wrong nonlinear tau term would move it
    f, _, _ = workloads.bratu_series(M, 16, seed=4, lam=LAM)
    ud = discrete_newton(f, LAM)
    out = oracle.vcycles_h(bratu(M), f, ud, 1)
    assert np.max(np.abs(out - ud)) <= 1e-11 * np.max(np.abs(ud))


def test_vcycles_converge_to_the_discrete_solution():
    M = 10
    f, _, _ = workloads.bratu_series(M, 16, seed=5, lam=LAM)
    ud = discrete_newton(f, LAM)
    u = np.zeros(1 << M)
    errs = []
    for _ in range(8):
        u = oracle.vcycles_h(bratu(M), f, u, 1)
        errs.append(np.max(np.abs(u - ud)))
    rates = [errs[i + 1] / errs[i] for i in range(7)]
    assert max(rates) < 0.2                  # measured 0.05-0.13
    assert errs[-1] < 1e-9 * np.max(np.abs(ud))


@pytest.mark.parametrize("sr", [False, True])
def test_one_fmg_cycle_reaches_discretization_accuracy(sr):
    # error vs the exact continuous solution: second order (ratio ~16 per
    # two halvings of h) and within 1.5x of the exact discrete solution's error
    errs = []
    for M in (8, 10, 12, 14):
        f, ue, _ = workloads.bratu_series(M, 16, seed=6, lam=LAM)
        p = bratu(M, nRS=1, W=(1 << M) // 4) if sr else bratu(M)
        u = oracle.fmg_h(p, f)
        e = np.max(np.abs(u - ue))
        ed = np.max(np.abs(discrete_newton(f, LAM) - ue))
        assert e <= 1.5 * ed
        errs.append(e)
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0


def test_serial_sr_variant_equals_stored_bratu():
    # the serial SR solve (finest level never stored) and the stored one agree
    M = 12
    f, _, _ = workloads.bratu_series(M, 16, seed=7, lam=LAM)
    p = bratu(M, nRS=1, W=512)
    assert np.array_equal(oracle.fmg_h(p, f), oracle.fmg_v(p, f))
