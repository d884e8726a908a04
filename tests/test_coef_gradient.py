"""Gradient of a loss with respect to the variable coefficient: dL/dlog a.

The paper has no gradient; this is the adjoint-state derivative of the
variable-coefficient operator of the Sec. 4 discretisation.  With the adjoint
state lam = A^{-1} dL/du (A symmetric), face f contributes
dL/dlog a_f = -a_f (u_f - u_{f-1}) (lam_f - lam_{f-1}) n^2, the wall faces
-2 a u lam n^2 at their one cell.

Oracle pins (no GPU): central differences of L(log a) through an independent
banded solve of the discrete equations, along random directions and the unit
directions of the wall and interior faces; the identity sum_f dL/dlog a_f =
-lam^T A u (scaling every face by one factor scales A), which holds for any u
and lam; wrong variants (sign, wall factor, dL/da instead of dL/dlog a,
jumps taken one face off) fail both checks.  GPU: the gradient kernel on the
oracle's u and lam, and the whole differentiable solve (forward, adjoint solve,
gradient) against the exact discrete gradient and central differences.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import workloads

scipy_linalg = pytest.importorskip("scipy.linalg")


def banded_solve(rhs, a):
    """A(a) x = rhs with A assembled column by column from the oracle's
    operator applied to unit vectors (scipy.linalg.solve_banded)."""
    n = len(rhs)
    ab = np.zeros((3, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        col = oracle.apply_La(e, a)
        for i in range(max(0, j - 1), min(n, j + 2)):
            ab[1 + i - j, j] = col[i]
    return scipy_linalg.solve_banded((1, 1), ab, rhs)


def problem(M, seed=1, noise=1e-3):
    f, ue, log_a = workloads.varcoef_series(M, 16, seed=seed)
    rng = np.random.default_rng(seed + 100)
    u_obs = ue + rng.normal(0.0, noise, 1 << M)
    return f, u_obs, log_a


def loss(f, u_obs, log_a):
    u = banded_solve(f, np.exp(log_a))
    return 0.5 * np.sum((u - u_obs) ** 2)


def exact_gradient(f, u_obs, log_a):
    a = np.exp(log_a)
    u = banded_solve(f, a)
    lam = banded_solve(u - u_obs, a)
    return u, lam, oracle.coef_gradient(a, u, lam)


def wrong_variants(a, u, lam, g):
    n = len(u)
    n2 = float(n) * n
    shifted = g.copy()
    shifted[1:n - 1] = -(a[1:n - 1] * (u[2:] - u[1:n - 1]) * (lam[2:] - lam[1:n - 1])) * n2
    wall = g.copy()
    wall[0] *= 0.5
    wall[n] *= 0.5
    return {"sign": -g, "wall factor": wall, "dL/da": g / a, "jump one face off": shifted}


M_PIN = 6      # cond(A) eps stays small enough for 1e-6 central differences (N = 256: 8e-6)


@pytest.fixture(scope="module")
def pin_case():
    f, u_obs, log_a = problem(M_PIN)
    u, lam, g = exact_gradient(f, u_obs, log_a)
    return f, u_obs, log_a, u, lam, g


def directions(n_faces, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        d = rng.normal(size=n_faces)
        out.append(d / np.linalg.norm(d))
    for f in (0, 1, n_faces // 2, n_faces - 2, n_faces - 1):
        e = np.zeros(n_faces)
        e[f] = 1.0
        out.append(e)
    return out


def central_difference(f, u_obs, log_a, d, eps=1e-5):
    return (loss(f, u_obs, log_a + eps * d) - loss(f, u_obs, log_a - eps * d)) / (2 * eps)


def test_gradient_matches_central_differences(pin_case):
    f, u_obs, log_a, _, _, g = pin_case
    for d in directions(len(log_a)):
        fd = central_difference(f, u_obs, log_a, d)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-3 * np.max(np.abs(g)))


def test_sum_over_faces_is_minus_lam_A_u():
    # A is linear in a and sum_f a_f dA/da_f = A, so sum_f dL/dlog a_f = -lam^T A u
    # for any u, lam (not only the solution and its adjoint state)
    rng = np.random.default_rng(11)
    for M in (3, 6, 9):
        n = 1 << M
        a = np.exp(rng.normal(scale=0.3, size=n + 1))
        u, lam = rng.normal(size=n), rng.normal(size=n)
        g = oracle.coef_gradient(a, u, lam)
        ref = -(lam @ oracle.apply_La(u, a))
        assert abs(g.sum() - ref) <= 1e-12 * np.sum(np.abs(g))


def test_scaling_identity_at_the_solution(pin_case):
    # at the exact discrete solution: sum_f dL/dlog a_f = dL/dlog c for a -> c a,
    # and u(c a) = u(a) / c, so it equals -(u - u_obs)^T u
    f, u_obs, log_a, u, lam, g = pin_case
    ref = -((u - u_obs) @ u)
    assert abs(g.sum() - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("mistake", ["sign", "wall factor", "dL/da", "jump one face off"])
def test_checks_catch_wrong_gradients(pin_case, mistake):
    f, u_obs, log_a, u, lam, g = pin_case
    a = np.exp(log_a)
    wrong = wrong_variants(a, u, lam, g)[mistake]
    caught_fd = any(
        abs(central_difference(f, u_obs, log_a, d) - wrong @ d)
        > 1e-6 * max(abs(central_difference(f, u_obs, log_a, d)), 1e-3 * np.max(np.abs(g)))
        for d in directions(len(log_a)))
    ref = -(lam @ oracle.apply_La(u, a))
    caught_sum = abs(wrong.sum() - ref) > 1e-10 * np.sum(np.abs(wrong))
    assert caught_fd
    if mistake != "jump one face off":        # an interior shift can keep the sum by chance
        assert caught_sum


# ---------------------------------------------------------------- GPU

def _solver(M, batch=1):
    from paper_1207_6720_gb300 import srfmg
    N = 1 << M
    return srfmg.Solver(M, op=srfmg.VARCOEF, segment_width=min(4096, N // 4), buffer_width=8, batch=batch)


def sr(M, a):
    N = 1 << M
    return oracle.sr_params(M, min(4096, N // 4), 8, op="varcoef", coef=a)


@pytest.mark.gpu
@pytest.mark.parametrize("M,batch", [(6, 1), (11, 1), (13, 3), (16, 1)])
def test_gradient_kernel_parity_gpu(M, batch):
    # the kernel on the oracle's u and lam: the same products on both sides
    torch = pytest.importorskip("torch")
    data = [problem(M, seed=s) for s in range(batch)]
    us, lams, gs = [], [], []
    for f, u_obs, log_a in data:
        a = np.exp(log_a)
        u = oracle.fmg_h(sr(M, a), f)
        lam = oracle.fmg_h(sr(M, a), u - u_obs)
        us.append(u)
        lams.append(lam)
        gs.append(oracle.coef_gradient(a, u, lam))
    s = _solver(M, batch)
    try:
        cat = lambda xs: torch.from_numpy(np.concatenate(xs)).cuda()
        s.set_coefficient(cat([d[2] for d in data]))
        g = s.coef_gradient(cat(us), cat(lams)).cpu().numpy().reshape(batch, -1)
    finally:
        s.close()
    for k in range(batch):
        assert np.max(np.abs(g[k] - gs[k])) <= 1e-13 * np.max(np.abs(gs[k]))


@pytest.mark.gpu
def test_differentiable_solve_gradient_gpu():
    # smooth misfit u_obs = u_exact + 1e-2 sin(3 pi x): one FMG cycle of the state
    # and of the adjoint equation is then at discretization accuracy, and the
    # gradient from them is within 8e-5 of the exact discrete gradient (measured
    # with the oracle's FMG-SR solve; a rough misfit gives about 1e-2).  Central
    # differences through the one-cycle solve are no check of this gradient: the
    # coarse levels take the coefficient by injection, so a face that coincides
    # with a coarse face moves the coarse solutions by O(H), which one cycle
    # does not correct; the exact-solve differences are pinned on the CPU above.
    torch = pytest.importorskip("torch")
    from paper_1207_6720_gb300 import srfmg
    M = 12
    f, ue, log_a = workloads.varcoef_series(M, 16, seed=1)
    x = (np.arange(1 << M) + 0.5) / (1 << M)
    u_obs = ue + 1e-2 * np.sin(3 * np.pi * x)
    s = _solver(M)
    try:
        fd_ = torch.from_numpy(f).cuda().requires_grad_(True)
        la = torch.from_numpy(log_a).cuda().requires_grad_(True)
        uo = torch.from_numpy(u_obs).cuda()
        u = srfmg.solve_autograd(s, fd_, log_a=la)
        L = 0.5 * torch.sum((u - uo) ** 2)
        gf, gla = torch.autograd.grad(L, [fd_, la])
        # the backward pass is the adjoint solve followed by the gradient kernel
        lam = s.adjoint((u.detach() - uo).contiguous())
        assert torch.equal(gf, lam)
        assert torch.equal(gla, s.coef_gradient(u.detach().contiguous(), lam))
        # against the exact discrete gradient
        _, _, gex = exact_gradient(f, u_obs, log_a)
        g_np = gla.cpu().numpy()
        assert np.max(np.abs(g_np - gex)) <= 2e-4 * np.max(np.abs(gex))
        # and the oracle's FMG-SR gradient on the same data
        a = np.exp(log_a)
        uo_ = oracle.fmg_h(sr(M, a), f)
        go = oracle.coef_gradient(a, uo_, oracle.fmg_h(sr(M, a), uo_ - u_obs))
        # (u and lam agree with the oracle to about 3e-13; the jumps amplify that by
        # about N / pi: 1e-12 noise in u and lam moves this gradient by 6e-9)
        assert np.max(np.abs(g_np - go)) <= 2e-8 * np.max(np.abs(go))
    finally:
        s.close()
