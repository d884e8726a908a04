"""Pipelined host solves (srfmg_solve_host_async / srfmg_solve_host_join): a
stream of right-hand sides in host memory, each copied in, solved and copied
back on the plan's staging buffers (two, used in turn) with the copies
overlapping the neighbouring solves.  Every result must equal, bit for bit, the
synchronous srfmg_solve_host of the same right-hand side, whatever the order in
which the calls' copies and solves overlap."""
import numpy as np
import pytest

from paper_1207_6720_gb300 import srfmg, workloads


def _pinned(n, torch):
    t = torch.empty(n, dtype=torch.float64).pin_memory()
    return t, t.numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("M,kw", [
    (14, dict(segment_width=1024, buffer_width=8, precision=srfmg.MIXED)),
    (13, dict(segment_width=512, buffer_width=4, precision=srfmg.FP64)),
    (12, dict(n_sr_levels=0, precision=srfmg.MIXED, batch=3)),
])
def test_pipelined_host_solves_equal_serial_ones_gpu(M, kw):
    torch = pytest.importorskip("torch")
    B = kw.get("batch", 1)
    K = 5
    fs = [np.concatenate([workloads.sine_series(M, 16, seed=10 * k + j)[0] for j in range(B)]) for k in range(K)]
    s = srfmg.Solver(M, **kw)
    try:
        ref = [s.solve_host(f) for f in fs]
        keep = []
        outs = []
        stream = torch.cuda.current_stream()
        for f in fs:
            tf, nf = _pinned(f.size, torch)
            nf[:] = f
            tu, nu = _pinned(f.size, torch)
            nu[:] = np.nan
            keep += [tf, tu]
            s.solve_host_async(nf, nu, stream=stream)
            outs.append(nu)
        s.host_join(stream=stream)
        torch.cuda.synchronize()
        for k in range(K):
            assert np.array_equal(outs[k], ref[k]), k
        # a device solve enqueued between pipelined calls keeps its place in the stream
        fd = torch.from_numpy(fs[1]).cuda()
        tu0, nu0 = _pinned(fs[0].size, torch)
        tf0, nf0 = _pinned(fs[0].size, torch)
        nf0[:] = fs[0]
        s.solve_host_async(nf0, nu0, stream=stream)
        ud = s.solve(fd, stream=stream)
        tu2, nu2 = _pinned(fs[2].size, torch)
        tf2, nf2 = _pinned(fs[2].size, torch)
        nf2[:] = fs[2]
        s.solve_host_async(nf2, nu2, stream=stream)
        s.host_join(stream=stream)
        torch.cuda.synchronize()
        assert np.array_equal(nu0, ref[0]) and np.array_equal(nu2, ref[2])
        assert np.array_equal(ud.cpu().numpy(), ref[1])
        # one host buffer as both f and u, and pageable buffers
        both = fs[3].copy()
        s.solve_host_async(both, both, stream=stream)
        s.host_join(stream=stream)
        torch.cuda.synchronize()
        assert np.array_equal(both, ref[3])
    finally:
        s.close()


@pytest.mark.gpu
def test_join_without_calls_is_a_no_op_gpu():
    torch = pytest.importorskip("torch")
    s = srfmg.Solver(12, precision=srfmg.MIXED)
    try:
        s.host_join()
        torch.cuda.synchronize()
    finally:
        s.close()
