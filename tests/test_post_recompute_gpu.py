"""The post-leg option FAS recompute (SRFMG_POST_FAS_RECOMPUTE: the correction
of Eq. 4 applied to the pre-smoothed fine level, which each segment recomputes
from the kept coarse iterate and the neighbours' kept edge cells, then
smoothing without Kaczmarz) on the GPU against the oracle's solve with the same
option, in both precisions, tolerance 1e-10 relative max-norm; the oracle pins
that option to stored-grid FAS with the same segmented smoother bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10

CASES = [
    # (M, W, b, nu1, nu2, M0, op)
    (8, 32, 4, 1, 1, 2, "laplace"),        # the tail holds every stored level
    (12, 256, 8, 1, 1, 2, "laplace"),
    (14, 1024, 62, 2, 1, 3, "laplace"),
    (15, 4096, 8, 2, 2, 2, "laplace"),
    (13, 512, 8, 2, 1, 2, "bratu"),
    (13, 512, 8, 1, 1, 2, "varcoef"),
]


def _inputs(M, op):
    if op == "bratu":
        f, ue, _ = workloads.bratu_series(M, 16, seed=M, lam=1.0)
        return f, ue, None, dict(op=srfmg.BRATU, lambda_=1.0), dict(op="bratu", lam=1.0)
    if op == "varcoef":
        f, ue, la = workloads.varcoef_series(M, 16, seed=M)
        return f, ue, la, dict(op=srfmg.VARCOEF), dict(op="varcoef", coef=np.exp(la))
    f, ue, _ = workloads.sine_series(M, 16, seed=M)
    return f, ue, None, {}, {}


@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,W,b,nu1,nu2,M0,op", CASES)
def test_post_recompute_parity_gpu(M, W, b, nu1, nu2, M0, op, precision):
    f, ue, la, kw, okw = _inputs(M, op)
    s = srfmg.Solver(M, segment_width=W, buffer_width=b, nu1=nu1, nu2=nu2, log2_n_coarsest=M0,
                     precision=precision, post_leg=srfmg.POST_FAS_RECOMPUTE, **kw)
    try:
        if la is not None:
            s.set_coefficient(torch.from_numpy(la).cuda())
        u = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b, nu1=nu1, nu2=nu2, M0=M0, post="fas_recompute", **okw), f)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))
    # and the stored-grid FAS solve with the same segmented smoother is the same solve
    stored = oracle.fmg_h(oracle.Params(M, M0=M0, nRS=0, nu1=nu1, nu2=nu2, seg={M: (W, b)}, **okw), f)
    assert np.max(np.abs(u - stored)) <= TOL * np.max(np.abs(stored))


@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_post_recompute_batch_functionals_and_replay_gpu(precision):
    # a batch: every problem equals its single solve bit for bit; the functionals
    # solve gives the same u; a replayed graph gives the same bits; reconstruction
    # (which rebuilds segments by the full update) is refused
    M, W, b, B = 13, 512, 8, 3
    fs = [workloads.sine_series(M, 16, seed=20 + k)[0] for k in range(B)]
    kw = dict(segment_width=W, buffer_width=b, precision=precision, post_leg=srfmg.POST_FAS_RECOMPUTE)
    sb = srfmg.Solver(M, batch=B, **kw)
    try:
        fd = torch.from_numpy(np.concatenate(fs)).cuda()
        ub = sb.solve(fd).cpu().numpy().reshape(B, -1)
        ub2 = sb.solve(fd).cpu().numpy().reshape(B, -1)
        assert np.array_equal(ub, ub2)
        u3 = torch.empty_like(fd)
        sb.solve_functionals(fd, u3)
        assert np.array_equal(u3.cpu().numpy().reshape(B, -1), ub)
        with pytest.raises(srfmg.SrfmgError):
            sb.reconstruct(fd, 0, 1)
    finally:
        sb.close()
    for k in range(B):
        s1 = srfmg.Solver(M, **kw)
        try:
            assert np.array_equal(s1.solve(torch.from_numpy(fs[k]).cuda()).cpu().numpy(), ub[k])
        finally:
            s1.close()
