"""Adjoint of the solve (dL/df for a loss of the solution).

For the cell-centred operator of Sec. 4 (odd ghosts at the walls) the discrete
operator is symmetric, so the adjoint equation is the forward equation with
dL/du as right-hand side; the GPU computes lambda = dL/df with the same
FMG(-SR) solve.  The oracle side of the checks: the operator's symmetry, the
exact discrete gradient (Thomas) against central finite differences, and the
accuracy of the oracle's FMG-SR solve on a rough adjoint right-hand side.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import workloads


def adjoint_rhs(M, seed=7, noise=1e-3):
    """dL/du = u - u_obs for L = 1/2 sum (u - u_obs)^2, u_obs = exact + noise."""
    f, ue, _ = workloads.sine_series(M, 32, seed=1)
    rng = np.random.default_rng(seed)
    u_obs = ue + rng.normal(0.0, noise, 1 << M)
    return f, u_obs


def sr(M):
    N = 1 << M
    return oracle.sr_params(M, min(4096, N // 4), 8)


# ---------------------------------------------------------------- oracle pins

@pytest.mark.parametrize("M", [4, 7, 10])
def test_operator_is_symmetric(M):
    rng = np.random.default_rng(M)
    a, b = rng.normal(size=1 << M), rng.normal(size=1 << M)
    lhs, rhs = a @ oracle.apply_L(b), oracle.apply_L(a) @ b
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), np.abs(a) @ np.abs(oracle.apply_L(np.abs(b))))


def test_exact_discrete_gradient_matches_central_differences():
    # L(f) = 1/2 |A^-1 f - u_obs|^2 with A^-1 the exact discrete solve: dL/df = A^-1 (u - u_obs)
    M = 9
    f, u_obs = adjoint_rhs(M)
    u = oracle.thomas(f)
    grad = oracle.thomas(u - u_obs)
    loss = lambda ff: 0.5 * np.sum((oracle.thomas(ff) - u_obs) ** 2)
    rng = np.random.default_rng(3)
    eps = 1e-3 * np.max(np.abs(f))
    for _ in range(4):
        d = rng.normal(size=f.size)
        d /= np.linalg.norm(d)
        fd = (loss(f + eps * d) - loss(f - eps * d)) / (2 * eps)
        assert abs(fd - grad @ d) <= 1e-7 * abs(grad @ d)


@pytest.mark.parametrize("mistake", ["no adjoint solve", "scaling", "shifted rhs"])
def test_central_difference_check_catches_wrong_gradients(mistake):
    # the finite-difference check above rejects plausible wrong adjoints
    M = 9
    f, u_obs = adjoint_rhs(M)
    r = oracle.thomas(f) - u_obs
    wrong = {"no adjoint solve": r,
             "scaling": 4.0 * oracle.thomas(r),
             "shifted rhs": oracle.thomas(np.roll(r, 1))}[mistake]
    loss = lambda ff: 0.5 * np.sum((oracle.thomas(ff) - u_obs) ** 2)
    rng = np.random.default_rng(3)
    eps = 1e-3 * np.max(np.abs(f))
    d = rng.normal(size=f.size)
    d /= np.linalg.norm(d)
    fd = (loss(f + eps * d) - loss(f - eps * d)) / (2 * eps)
    assert abs(fd - wrong @ d) > 1e-7 * abs(fd)


@pytest.mark.parametrize("M,bound", [(12, 2e-3), (14, 5e-4)])
def test_fmg_sr_adjoint_accuracy_on_rough_data(M, bound):
    # one FMG-SR cycle on lambda's equation, against the exact discrete adjoint
    f, u_obs = adjoint_rhs(M)
    p = sr(M)
    u = oracle.fmg_h(p, f)
    lam = oracle.fmg_h(p, u - u_obs)
    ex = oracle.thomas(u - u_obs)
    assert np.max(np.abs(lam - ex)) <= bound * np.max(np.abs(ex))


# ---------------------------------------------------------------- GPU

def _solver(M, precision=0, **kw):
    from paper_1207_6720_gb300 import srfmg
    N = 1 << M
    return srfmg.Solver(M, segment_width=min(4096, N // 4), buffer_width=8, precision=precision, **kw)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("M", [10, 14, 17])
def test_adjoint_parity_gpu(M, precision):
    torch = pytest.importorskip("torch")
    f, u_obs = adjoint_rhs(M)
    p = sr(M)
    g = oracle.fmg_h(p, f) - u_obs
    s = _solver(M, precision)
    try:
        lam = s.adjoint(torch.from_numpy(g).cuda())
        torch.cuda.synchronize()
        lam = lam.cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(p, g)
    assert np.max(np.abs(lam - ref)) <= 1e-10 * np.max(np.abs(ref))


@pytest.mark.gpu
def test_autograd_gradient_and_finite_differences_gpu():
    torch = pytest.importorskip("torch")
    from paper_1207_6720_gb300 import srfmg
    M = 14
    f, u_obs = adjoint_rhs(M)
    s = _solver(M)
    try:
        fd_ = torch.from_numpy(f).cuda().requires_grad_(True)
        uo = torch.from_numpy(u_obs).cuda()
        u = srfmg.solve_autograd(s, fd_)
        loss = 0.5 * torch.sum((u - uo) ** 2)
        (grad,) = torch.autograd.grad(loss, fd_)
        # the backward pass is the adjoint call
        direct = s.adjoint((u.detach() - uo).contiguous())
        assert torch.equal(grad, direct)
        # the exact discrete gradient (Thomas) to the solver's algebraic accuracy
        g_np = grad.cpu().numpy()
        ex = oracle.thomas(u.detach().cpu().numpy() - u_obs)
        assert np.max(np.abs(g_np - ex)) <= 5e-4 * np.max(np.abs(ex))
        # central differences through the GPU solve along seeded unit directions
        with torch.no_grad():
            def L(ff):
                return 0.5 * torch.sum((s.solve(ff) - uo) ** 2).item()
            rng = np.random.default_rng(5)
            eps = 1e-3 * float(np.max(np.abs(f)))
            for _ in range(4):
                d = rng.normal(size=f.size)
                d /= np.linalg.norm(d)
                dt = torch.from_numpy(d).cuda()
                fdiff = (L(fd_.detach() + eps * dt) - L(fd_.detach() - eps * dt)) / (2 * eps)
                assert abs(fdiff - float(g_np @ d)) <= 5e-3 * abs(fdiff)
    finally:
        s.close()


@pytest.mark.gpu
def test_solve_and_adjoint_keep_their_graphs_gpu():
    torch = pytest.importorskip("torch")
    M = 13
    f, u_obs = adjoint_rhs(M)
    s = _solver(M, precision=1)
    try:
        fd_ = torch.from_numpy(f).cuda()
        gd = torch.from_numpy(f[::-1].copy()).cuda()
        u, lam = torch.empty_like(fd_), torch.empty_like(fd_)
        s.solve(fd_, u)
        s.adjoint(gd, lam)
        u0, lam0 = u.clone(), lam.clone()
        for _ in range(3):                 # alternate: each pointer pair replays its own graph
            s.solve(fd_, u)
            s.adjoint(gd, lam)
            torch.cuda.synchronize()
            assert torch.equal(u, u0) and torch.equal(lam, lam0)
        # more pointer pairs than graph slots: the least recently used is recaptured
        outs = [s.solve(fd_) for _ in range(6)]
        torch.cuda.synchronize()
        assert all(torch.equal(o, u0) for o in outs)
    finally:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_converged_gradients_match_central_differences_gpu(precision):
    # A plan without SR followed by V-cycles converges to the exact discrete
    # solution, a symmetric linear map of f, so the adjoint solve and the
    # coefficient gradient are the exact gradients of the solve itself:
    # central differences of L = 1/2 |u - u_obs|^2 through the GPU solve, along
    # 64 seeded directions of f and 16 of log a (-(a u')' = f, the adjoint
    # workload's family), agree with them.  L is quadratic in f, so its central
    # difference is exact up to rounding; L(+) - L(-) is formed as
    # 1/2 sum (u+ - u-)(u+ + u- - 2 u_obs), free of the cancellation of two large L.
    torch = pytest.importorskip("torch")
    from paper_1207_6720_gb300 import srfmg
    M = 14
    f, ue, log_a = workloads.varcoef_series(M, 16, seed=1)
    rng = np.random.default_rng(7)
    uo = torch.from_numpy(ue + rng.normal(0.0, 1e-3, 1 << M)).cuda()
    prec = srfmg.FP64 if precision == "fp64" else srfmg.MIXED
    s = srfmg.Solver(M, n_sr_levels=0, op=srfmg.VARCOEF, precision=prec, n_vcycles=16)
    try:
        la = torch.from_numpy(log_a).cuda()
        s.set_coefficient(la)
        fd_ = torch.from_numpy(f).cuda()
        u = torch.zeros_like(fd_)
        s.solve(fd_, u)
        lam = s.adjoint((u - uo).contiguous())
        g_a = s.coef_gradient(u, lam)

        def dL(up, um):
            return float(0.5 * torch.sum((up - um) * (up + um - 2.0 * uo)))

        def solve(ff):
            out = torch.zeros_like(fd_)
            s.solve(ff, out)
            return out
        rng = np.random.default_rng(11)
        eps = float(np.max(np.abs(f)))
        for _ in range(64):
            d = torch.from_numpy(rng.normal(size=f.size)).cuda()
            fdv = dL(solve(fd_ + eps * d), solve(fd_ - eps * d)) / (2.0 * eps)
            assert abs(fdv - float(lam @ d)) <= 1e-6 * abs(fdv)
        eps_a = 1e-5
        for _ in range(16):
            d = torch.from_numpy(rng.normal(size=log_a.size)).cuda()
            s.set_coefficient((la + eps_a * d).contiguous())
            up = solve(fd_)
            s.set_coefficient((la - eps_a * d).contiguous())
            um = solve(fd_)
            fdv = dL(up, um) / (2.0 * eps_a)
            assert abs(fdv - float(g_a @ d)) <= 1e-4 * abs(fdv)
    finally:
        s.close()
