"""Oracle pins for the variable-coefficient problem -(a u')' = f.

Fluxes a_{i+1/2} (u_{i+1} - u_i) with the coefficient at the cell faces of the
finest level; coarse levels take the coefficient of the coinciding fine face
(a reading: the paper's studies have a = 1).  Pinned against properties that
fix the discretisation (symmetry, the constant-coefficient limit, scaling),
against an independent banded solve of the same discrete equations (its
matrix assembled column by column from the oracle's operator), the FAS
fixed-point property, V-cycle convergence and second-order accuracy of one FMG
cycle."""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import workloads

scipy_linalg = pytest.importorskip("scipy.linalg")


def vc(M, log_a, nRS=0, W=None, b=8, nu1=1, nu2=1):
    a = np.exp(log_a)
    if nRS:
        return oracle.sr_params(M, W, b, nRS=nRS, nu1=nu1, nu2=nu2, op="varcoef", coef=a)
    return oracle.Params(M, nRS=0, nu1=nu1, nu2=nu2, op="varcoef", coef=a)


def discrete_solve(f, a):
    """Solve L_a u = f with the banded matrix assembled column by column from
    the oracle's operator applied to unit vectors (scipy.linalg.solve_banded)."""
    n = len(f)
    ab = np.zeros((3, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        col = oracle.apply_La(e, a)
        for i in range(max(0, j - 1), min(n, j + 2)):
            ab[1 + i - j, j] = col[i]
        assert np.all(col[:max(0, j - 1)] == 0) and np.all(col[j + 2:] == 0)
    return scipy_linalg.solve_banded((1, 1), ab, f)


def test_constant_coefficient_limit_is_bitwise():
    rng = np.random.default_rng(0)
    u = rng.normal(size=64)
    assert np.array_equal(oracle.apply_La(u, np.ones(65)), oracle.apply_L(u))
    assert np.allclose(oracle.apply_La(u, np.full(65, 2.5)), 2.5 * oracle.apply_L(u), rtol=1e-14, atol=0)


@pytest.mark.parametrize("M", [3, 6, 9])
def test_operator_is_symmetric_and_positive(M):
    rng = np.random.default_rng(M)
    a = np.exp(rng.normal(scale=0.5, size=(1 << M) + 1))
    x, y = rng.normal(size=1 << M), rng.normal(size=1 << M)
    assert abs(x @ oracle.apply_La(y, a) - oracle.apply_La(x, a) @ y) <= 1e-12 * np.abs(x) @ np.abs(oracle.apply_La(np.abs(y), a))
    assert x @ oracle.apply_La(x, a) > 0


def test_coarsest_thomas_solves_the_level():
    rng = np.random.default_rng(4)
    n = 16
    a = np.exp(rng.normal(scale=0.7, size=n + 1))
    rhs = rng.normal(size=n)
    p = oracle.Params(4, nRS=0, op="varcoef", coef=a)
    u = oracle.coarsest(p, rhs, np.zeros(n))
    assert np.max(np.abs(oracle.apply_La(u, a) - rhs)) <= 1e-12 * np.max(np.abs(rhs))


@pytest.mark.parametrize("M", [6, 9])
def test_discrete_solution_is_a_fixed_point_of_the_fas_vcycle(M):
    f, _, log_a = workloads.varcoef_series(M, 16, seed=2)
    ud = discrete_solve(f, np.exp(log_a))
    out = oracle.vcycles_h(vc(M, log_a), f, ud, 1)
    assert np.max(np.abs(out - ud)) <= 1e-11 * np.max(np.abs(ud))


def test_vcycles_converge_to_the_discrete_solution():
    M = 10
    f, _, log_a = workloads.varcoef_series(M, 16, seed=3)
    ud = discrete_solve(f, np.exp(log_a))
    u = np.zeros(1 << M)
    errs = []
    for _ in range(8):
        u = oracle.vcycles_h(vc(M, log_a), f, u, 1)
        errs.append(np.max(np.abs(u - ud)))
    rates = [errs[i + 1] / errs[i] for i in range(7)]
    assert max(rates) < 0.25
    assert errs[-1] < 1e-8 * np.max(np.abs(ud))


@pytest.mark.parametrize("sr", [False, True])
def test_one_fmg_cycle_reaches_discretization_accuracy(sr):
    errs = []
    for M in (8, 10, 12, 14):
        f, ue, log_a = workloads.varcoef_series(M, 16, seed=6)
        p = vc(M, log_a, nRS=1, W=(1 << M) // 4) if sr else vc(M, log_a)
        u = oracle.fmg_h(p, f)
        e = np.max(np.abs(u - ue))
        ed = np.max(np.abs(discrete_solve(f, np.exp(log_a)) - ue)) if M <= 12 else None
        if ed is not None:
            assert e <= 1.5 * ed
        errs.append(e)
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0          # second order: two halvings of h per step


def test_serial_sr_variant_equals_stored():
    M = 12
    f, _, log_a = workloads.varcoef_series(M, 16, seed=7)
    p = vc(M, log_a, nRS=1, W=512)
    assert np.array_equal(oracle.fmg_h(p, f), oracle.fmg_v(p, f))
