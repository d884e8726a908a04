"""The allocation-free entry point srfmg_solve_small_noalloc against
srfmg_solve.

Some callers cannot call cudaMalloc (an open stream capture in global mode,
device memory owned by a caching allocator or pool, loops that must not
allocate after start-up); srfmg_solve_small_noalloc serves them for N <= 4096
with its scratch in a static device array.  This file is collected last so
that a run stopping at its first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    lib = srfmg.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for M, M0, nu1, nu2, seed in [(12, 2, 1, 1, 0), (10, 4, 2, 1, 1)]:
        f, _, _ = workloads.sine_series(M, 8, seed=seed)
        fd = torch.from_numpy(f).cuda()
        ref = srfmg.Solver(M, n_sr_levels=0, log2_n_coarsest=M0, nu1=nu1, nu2=nu2)
        u_ref = ref.solve(fd)
        u = torch.full_like(fd, float("nan"))
        st = lib.srfmg_solve_small_noalloc(M, M0, nu1, nu2, ctypes.c_void_p(fd.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr()), stream)
        assert st == srfmg.OK
        torch.cuda.synchronize()
        a, b = u.cpu().numpy(), u_ref.cpu().numpy()
        ref.close()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= TOL


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
