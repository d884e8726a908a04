"""The allocation-free entry point srfmg_solve_small_noalloc against
srfmg_solve and the oracle.

Some callers cannot call cudaMalloc (an open stream capture in global mode,
device memory owned by a caching allocator or pool, loops that must not
allocate after start-up); srfmg_solve_small_noalloc serves them for N <= 4096
with its scratch in a static device array.  This file is collected last so
that a run stopping at its first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _noalloc(lib, M, M0, nu1, nu2, fd, stream):
    u = torch.full_like(fd, float("nan"))
    st = lib.srfmg_solve_small_noalloc(M, M0, nu1, nu2, ctypes.c_void_p(fd.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), stream)
    assert st == srfmg.OK
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_noalloc_matches_solve_on_calls_in_a_row():
    """Two calls in a row with different coarsest levels (each uploads its
    table), the same (M, M0) twice (the cached table, no upload), and a switch
    back to the first coarsest level: each call equals srfmg_solve with
    n_sr_levels = 0 and the same parameters."""
    lib = srfmg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(12, 2, 1, 1, 0), (10, 4, 2, 1, 1), (10, 4, 2, 1, 2), (12, 2, 1, 2, 3), (11, 6, 1, 1, 4)]
    for M, M0, nu1, nu2, seed in cases:
        f, _, _ = workloads.sine_series(M, 8, seed=seed)
        fd = torch.from_numpy(f).cuda()
        ref = srfmg.Solver(M, n_sr_levels=0, log2_n_coarsest=M0, nu1=nu1, nu2=nu2)
        b = ref.solve(fd).cpu().numpy()
        ref.close()
        a = _noalloc(lib, M, M0, nu1, nu2, fd, stream)
        assert np.all(np.isfinite(a))
        assert _rel(a, b) <= TOL, (M, M0, nu1, nu2)


def test_noalloc_matches_the_oracle():
    """The oracle's plain stored FMG-FAS (Fig. 2 with the V-cycle of Fig. 1,
    no SR level) on the same right-hand side, before and after a call with
    another coarsest level."""
    lib = srfmg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    f, _, _ = workloads.sine_series(12, 8, seed=5)
    fd = torch.from_numpy(f).cuda()
    want = oracle.fmg_h(oracle.Params(12, M0=3, nRS=0, nu1=1, nu2=1), f)
    assert _rel(_noalloc(lib, 12, 3, 1, 1, fd, stream), want) <= TOL
    _noalloc(lib, 9, 5, 1, 1, fd[: 1 << 9].clone(), stream)
    assert _rel(_noalloc(lib, 12, 3, 1, 1, fd, stream), want) <= TOL


def test_noalloc_python_wrapper_checks_u():
    f, _, _ = workloads.sine_series(10, 8, seed=6)
    fd = torch.from_numpy(f).cuda()
    u = torch.empty_like(fd)
    out = srfmg.solve_small_noalloc(fd, u)
    assert out.data_ptr() == u.data_ptr()
    for bad in (torch.empty(1 << 9, dtype=torch.float64, device="cuda"),
                torch.empty(1 << 10, dtype=torch.float32, device="cuda"),
                torch.empty(1 << 11, dtype=torch.float64, device="cuda")[::2],
                torch.empty(1 << 10, dtype=torch.float64)):
        with pytest.raises(ValueError):
            srfmg.solve_small_noalloc(fd, bad)


def test_noalloc_rejects_sizes_beyond_its_limit():
    lib = srfmg.load()
    fd = torch.zeros(1 << 13, dtype=torch.float64, device="cuda")
    u = torch.empty_like(fd)
    st = lib.srfmg_solve_small_noalloc(13, 2, 1, 1, ctypes.c_void_p(fd.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), None)
    assert st == srfmg.EINVAL
    st = lib.srfmg_solve_small_noalloc(12, 7, 1, 1, ctypes.c_void_p(fd.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), None)
    assert st == srfmg.EINVAL
