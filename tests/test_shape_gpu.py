"""The CTA shape of a plan (the coarse tail's extent and the cells per block of
the latency-bound stored-level passes) changes the launch shapes, not the
result: every shape gives the same bits, in both precisions and for every
operator; srfmg_autotune_shape picks one of them."""
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


def test_autotune_shape_picks_a_candidate_gpu():
    M = 20
    p = srfmg.default_params(M, precision=srfmg.MIXED, segment_width=2048, buffer_width=8)
    best, table = srfmg.autotune_shape(p, reps=2)
    assert len(table) == 12 and all(ms > 0 for _, _, ms in table)
    assert (best.tail_level, best.tile_cells) in [(t, c) for t, c, _ in table]
    fastest = min(table, key=lambda x: x[2])
    assert (best.tail_level, best.tile_cells) == fastest[:2]
    assert (best.segment_width, best.buffer_width, best.log2_n) == (2048, 8, M)
