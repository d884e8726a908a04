"""Non-finite detection (SRFMG_ENONFINITE), tested without a GPU fault: a
poisoned input (one NaN or inf in f, or a non-finite reference of the
functionals) goes into a solve, the kernel that reads it records it in the
plan's status word, and srfmg_check reports and clears it."""
import numpy as np
import pytest

from paper_1207_6720_gb300 import srfmg, workloads


def test_check_needs_a_handle():
    assert srfmg.load().srfmg_check(None, None) == srfmg.EINVAL


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


PLANS = [
    (14, dict(segment_width=1024, buffer_width=8)),           # SR: rhs hierarchy reads f
    (14, dict(n_sr_levels=0)),                                # stored levels
    (10, dict(n_sr_levels=0)),                                # the whole problem in the tail
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [srfmg.FP64, srfmg.MIXED])
@pytest.mark.parametrize("M,kw", PLANS)
@pytest.mark.parametrize("poison", [np.nan, np.inf])
def test_poisoned_input_is_reported_gpu(M, kw, precision, poison):
    pytest.importorskip("torch")
    f, _, _ = workloads.sine_series(M, 16, seed=2)
    bad = f.copy()
    bad[(1 << M) // 3] = poison
    s = srfmg.Solver(M, precision=precision, **kw)
    try:
        s.solve(_dev(f))
        s.check()                                  # clean
        s.solve(_dev(bad))
        with pytest.raises(srfmg.SrfmgError) as e:
            s.check()
        assert e.value.status == srfmg.ENONFINITE
        s.check()                                  # the check cleared the word
        s.solve(_dev(f))
        s.check()
    finally:
        s.close()


@pytest.mark.gpu
def test_nonfinite_functional_is_reported_gpu():
    pytest.importorskip("torch")
    M = 12
    f, ue, _ = workloads.sine_series(M, 16, seed=2)
    ref = ue.copy()
    ref[5] = np.inf
    s = srfmg.Solver(M, segment_width=256, buffer_width=8)
    try:
        s.solve_functionals(_dev(f), None, _dev(ue))
        s.check()
        s.solve_functionals(_dev(f), None, _dev(ref))
        with pytest.raises(srfmg.SrfmgError):
            s.check()
    finally:
        s.close()
