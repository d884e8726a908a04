"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerance: 1e-10 relative max-norm for the FP64 path
(the two sides differ only in rounding order)."""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel_maxnorm(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def gpu_solve(M, f, **kw):
    from paper_1207_6720_gb300 import srfmg
    s = srfmg.Solver(M, **kw)
    try:
        u = s.solve(torch.from_numpy(f).cuda())
        torch.cuda.synchronize()
        return u.cpu().numpy()
    finally:
        s.close()


def oracle_params(M, nRS, W, b, nu1=1, nu2=1, M0=2):
    if nRS == 0:
        return oracle.Params(M, M0=M0, nRS=0, nu1=nu1, nu2=nu2)
    return oracle.sr_params(M, W, b, nRS=1, nu1=nu1, nu2=nu2, M0=M0)


CASES = [
    # (M, nRS, W, b, nu1, nu2, M0)
    (6, 1, 16, 2, 1, 1, 2),       # tail handles level 5, one SR level of 4 segments
    (10, 1, 256, 4, 1, 1, 2),     # the N=1024 workload (4 segments of 256, 4 buffer cells)
    (10, 1, 1024, 8, 1, 1, 2),    # one segment covering the level
    (12, 1, 64, 8, 1, 1, 2),
    (13, 1, 128, 8, 1, 1, 2),     # first stored level above the tail
    (14, 1, 4096, 8, 2, 2, 2),    # V(2,2): alternating sweep directions
    (15, 1, 512, 2, 2, 1, 3),
    (16, 1, 4096, 64, 1, 1, 6),
    (17, 1, 2048, 8, 3, 1, 4),
    (8, 0, 0, 0, 1, 1, 2),        # plain stored FMG, whole problem in the tail
    (12, 0, 0, 0, 1, 1, 2),
    (15, 0, 0, 0, 1, 2, 2),       # plain stored FMG, finest level stored by the level passes
]


PRECISIONS = [0, 1]       # SRFMG_FP64, SRFMG_MIXED (64-bit fixed point)


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("M,nRS,W,b,nu1,nu2,M0", CASES)
def test_parity_small(M, nRS, W, b, nu1, nu2, M0, precision):
    f, _, _ = workloads.sine_series(M, 8 if M <= 10 else 32, seed=M)
    kw = dict(n_sr_levels=nRS, nu1=nu1, nu2=nu2, log2_n_coarsest=M0, precision=precision)
    if nRS:
        kw.update(segment_width=W, buffer_width=b)
    u = gpu_solve(M, f, **kw)
    ref = oracle.fmg_h(oracle_params(M, nRS, W, b, nu1, nu2, M0), f)
    assert rel_maxnorm(u, ref) <= TOL


@pytest.fixture(scope="module")
def full_size_case():
    # the N = 2^24 workload: 4096 segments of 4096 cells, 8 buffer cells, V(1,1)
    M, W, b = 24, 4096, 8
    f, ue, c = workloads.sine_series(M, 32, seed=1)
    ref = oracle.fmg_v(oracle.sr_params(M, W, b, nRS=1), f)
    return M, W, b, f, ue, ref


@pytest.mark.parametrize("precision", PRECISIONS)
def test_parity_full_size(full_size_case, precision):
    M, W, b, f, ue, ref = full_size_case
    u = gpu_solve(M, f, segment_width=W, buffer_width=b, precision=precision)
    assert rel_maxnorm(u, ref) <= TOL
    # discretization accuracy of the GPU result: error vs exact within 1.5x the oracle's
    err_gpu = np.linalg.norm(u - ue)
    err_ref = np.linalg.norm(ref - ue)
    assert err_gpu <= 1.5 * err_ref


def test_deterministic_and_graph_replay():
    from paper_1207_6720_gb300 import srfmg
    M = 16
    f, _, _ = workloads.sine_series(M, 16, seed=3)
    s = srfmg.Solver(M, segment_width=1024, buffer_width=8)
    try:
        fd = torch.from_numpy(f).cuda()
        u1 = s.solve(fd).clone()
        u2 = s.solve(fd).clone()                      # graph replay
        u3 = s.solve(fd.clone(), torch.empty_like(fd))  # new pointers: new capture
        torch.cuda.synchronize()
        assert torch.equal(u1, u2) and torch.equal(u1, u3)
        uh = s.solve_host(f)                          # host buffers, copies inside
        assert np.array_equal(uh, u1.cpu().numpy())
    finally:
        s.close()


def test_launch_count_reported():
    from paper_1207_6720_gb300 import srfmg
    s = srfmg.Solver(24)
    try:
        inf = s.info()
        assert inf.n_segments == 4096 and inf.coarse_tail_level == 12
        assert inf.kernels_per_solve > 20
    finally:
        s.close()


# SRFMG_TAU_SEGMENT: the edge coarse cells' tau from each segment's own buffer
# (Fig. 3 line 4 read literally) against the oracle's tau_src="segment"
SEGMENT_TAU_CASES = [
    # (M, nRS, W, b, op)
    (10, 1, 256, 4, "laplace"),
    (14, 1, 1024, 8, "laplace"),
    (17, 1, 4096, 2, "laplace"),
    (13, 2, 512, 8, "laplace"),
    (13, 1, 512, 8, "bratu"),
    (13, 2, 512, 8, "varcoef"),
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,nRS,W,b,op", SEGMENT_TAU_CASES)
def test_segment_local_tau_parity_gpu(M, nRS, W, b, op, precision):
    torch = pytest.importorskip("torch")
    kw, okw, log_a = {}, {}, None
    if op == "bratu":
        f, _, _ = workloads.bratu_series(M, 16, seed=M, lam=1.0)
        kw, okw = dict(op=srfmg.BRATU, lambda_=1.0), dict(op="bratu", lam=1.0)
    elif op == "varcoef":
        f, _, log_a = workloads.varcoef_series(M, 16, seed=M)
        kw, okw = dict(op=srfmg.VARCOEF), dict(op="varcoef", coef=np.exp(log_a))
    else:
        f, _, _ = workloads.sine_series(M, 16, seed=M)
    s = srfmg.Solver(M, n_sr_levels=nRS, segment_width=W, buffer_width=b, tau_edge=srfmg.TAU_SEGMENT,
                     precision=precision, **kw)
    try:
        if log_a is not None:
            s.set_coefficient(torch.from_numpy(log_a).cuda())
        u = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=nRS, tau_src="segment", **okw), f)
    assert np.max(np.abs(u - ref)) <= TOL * np.max(np.abs(ref))
    # and it is a different reading from the assembled one
    ref_asm = oracle.fmg_h(oracle.sr_params(M, W, b, nRS=nRS, **okw), f)
    assert np.max(np.abs(ref - ref_asm)) > 0.0
