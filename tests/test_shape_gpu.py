"""The CTA shape of a plan (the coarse tail's extent, the cells per block of
the latency-bound stored-level passes and, for the fixed-point -u'' = f, their
chaining into multi-level launches) changes the launch shapes, not the result:
every shape gives the same bits, in both precisions and for every operator;
srfmg_autotune_shape picks one of them."""
import numpy as np
import pytest

from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(0, 0), (9, 128), (10, 512), (11, 64), (12, 2048)]


def _solve(M, f, la=None, **kw):
    s = srfmg.Solver(M, **kw)
    try:
        if la is not None:
            s.set_coefficient(torch.from_numpy(la).cuda())
        return s.solve(torch.from_numpy(f).cuda()).cpu().numpy(), s.info().coarse_tail_level
    finally:
        s.close()


@pytest.mark.parametrize("op", ["laplace", "varcoef", "bratu"])
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
def test_every_shape_gives_the_same_bits_gpu(op, precision):
    M = 16
    la = None
    kw = dict(segment_width=1024, buffer_width=8, precision=precision)
    if op == "varcoef":
        f, _, la = workloads.varcoef_series(M, 16, seed=4)
        kw["op"] = srfmg.VARCOEF
    elif op == "bratu":
        f, _, _ = workloads.bratu_series(M, 16, seed=4, lam=1.0)
        kw.update(op=srfmg.BRATU, lambda_=1.0, nu1=2)
    else:
        f, _, _ = workloads.sine_series(M, 16, seed=4)
    ref, tail = _solve(M, f, la, **kw)
    assert tail == 12
    for t, c in SHAPES[1:]:
        u, tail = _solve(M, f, la, tail_level=t, tile_cells=c, **kw)
        assert tail == t
        assert np.array_equal(u, ref), (t, c)


@pytest.mark.parametrize("M,batch,nu,tail", [(16, 1, (1, 1), 12), (20, 1, (1, 1), 11), (18, 3, (2, 1), 10),
                                              (17, 1, (1, 2), 9)])
def test_chained_passes_give_the_same_bits_gpu(M, batch, nu, tail):
    # chained down and up passes of the latency-bound stored levels (fixed point,
    # -u'' = f): every chain depth and tile gives the bits of the separate passes
    f = np.tile(workloads.sine_series(M, 16, seed=5)[0], batch)
    kw = dict(segment_width=1024, buffer_width=8, precision=srfmg.MIXED, batch=batch, nu1=nu[0], nu2=nu[1],
              tail_level=tail)
    ref, _ = _solve(M, f, **kw)
    for tile, cd, cu in [(256, 2, 0), (256, 0, 3), (512, 2, 4), (128, 3, 2), (1024, 4, 4), (64, 2, 2)]:
        s = srfmg.Solver(M, tile_cells=tile, chain_down=cd, chain_up=cu, **kw)
        try:
            fd = torch.from_numpy(f).cuda()
            chained = s.info().kernels_per_solve
            u = s.solve(fd).cpu().numpy()
            u2 = s.solve(fd).cpu().numpy()
        finally:
            s.close()
        plain = srfmg.Solver(M, tile_cells=tile, **kw)
        unchained = plain.info().kernels_per_solve
        plain.close()
        assert chained < unchained, (tile, cd, cu)
        assert np.array_equal(u, ref) and np.array_equal(u2, ref), (tile, cd, cu)


def test_autotune_shape_picks_a_candidate_gpu():
    M = 20
    p = srfmg.default_params(M, precision=srfmg.MIXED, segment_width=2048, buffer_width=8)
    best, table = srfmg.autotune_shape(p, reps=2)
    assert len(table) == 20 and all(row[-1] > 0 for row in table)
    shape = (best.tail_level, best.tile_cells, best.chain_down, best.chain_up)
    assert shape in [row[:4] for row in table]
    fastest = min(table, key=lambda x: x[-1])
    assert shape == fastest[:4]
    assert (best.segment_width, best.buffer_width, best.log2_n) == (2048, 8, M)
