"""Batched solves: one plan solves B independent problems of the same size with
the same launches (one grid row per problem).  Each problem of a batch must
give bit for bit the result of its own single solve (the arithmetic is the
same, only the offsets differ), and that result is held to the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads


def _create(**kw):
    lib = srfmg.load()
    p = srfmg.default_params(12)
    for k, v in kw.items():
        setattr(p, k, v)
    h = ctypes.c_void_p()
    return lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h))


def test_batch_count_is_checked_on_the_host():
    assert _create(batch=-1) == srfmg.EINVAL
    assert _create(batch=65536) == srfmg.EINVAL


CASES = [
    # (M, kw)
    (10, dict(segment_width=256, buffer_width=4)),                    # tail + SR level
    (8, dict(n_sr_levels=0)),                                          # whole problem in the tail
    (14, dict(segment_width=1024, buffer_width=8)),                    # stored levels + SR
    (15, dict(n_sr_levels=0, nu2=2)),                                  # stored finest level
    (14, dict(segment_width=1024, buffer_width=8, precision=srfmg.MIXED)),
    (15, dict(n_sr_levels=0, precision=srfmg.MIXED)),
    (12, dict(segment_width=512, buffer_width=8, op=srfmg.BRATU, lambda_=1.0, nu1=2)),
]


@pytest.mark.gpu
@pytest.mark.parametrize("M,kw", CASES)
def test_batch_equals_single_solves_gpu(M, kw):
    torch = pytest.importorskip("torch")
    B = 5
    bratu = kw.get("op") == srfmg.BRATU
    fs = [(workloads.bratu_series(M, 16, seed=s, lam=1.0) if bratu else workloads.sine_series(M, 16, seed=s))[0]
          for s in range(B)]
    single = srfmg.Solver(M, **kw)
    batched = srfmg.Solver(M, batch=B, **kw)
    try:
        ref = [single.solve(torch.from_numpy(f).cuda()).cpu().numpy() for f in fs]
        fb = torch.from_numpy(np.concatenate(fs)).cuda()
        ub = batched.solve(fb).cpu().numpy().reshape(B, -1)
        for k in range(B):
            assert np.array_equal(ub[k], ref[k]), k
        # host buffers, copies inside
        uh = batched.solve_host(np.concatenate(fs)).reshape(B, -1)
        assert np.array_equal(uh, ub)
        if not bratu and kw.get("precision", 0) == 0:
            # the adjoint of a batch is the batch of adjoints
            lb = batched.adjoint(fb).cpu().numpy().reshape(B, -1)
            assert np.array_equal(lb, ub)
    finally:
        single.close()
        batched.close()
    # and the oracle for one problem of the batch
    nRS = kw.get("n_sr_levels", 1)
    if bratu:
        p = oracle.sr_params(M, kw["segment_width"], kw["buffer_width"], nu1=2, op="bratu", lam=1.0)
    elif nRS:
        p = oracle.sr_params(M, kw["segment_width"], kw["buffer_width"])
    else:
        p = oracle.Params(M, nRS=0, nu2=kw.get("nu2", 1))
    r = oracle.fmg_h(p, fs[3])
    assert np.max(np.abs(ub[3] - r)) <= 1e-10 * np.max(np.abs(r))


# ---------------------------------------------------------------- autotuner (row f1)

def test_autotune_checks_arguments_on_the_host():
    lib = srfmg.load()
    p = srfmg.default_params(16)
    best = srfmg.Params()
    assert lib.srfmg_autotune(None, 0, 3, ctypes.byref(best), None, 0, None) == srfmg.EINVAL
    assert lib.srfmg_autotune(ctypes.byref(p), 0, 0, ctypes.byref(best), None, 0, None) == srfmg.EINVAL
    p0 = srfmg.default_params(16, n_sr_levels=0)
    assert lib.srfmg_autotune(ctypes.byref(p0), 0, 3, ctypes.byref(best), None, 0, None) == srfmg.EINVAL
    W, b = ctypes.c_int32(), ctypes.c_int32()
    assert lib.srfmg_autotune_candidate(ctypes.byref(p), 0, ctypes.byref(W), ctypes.byref(b)) == srfmg.OK
    assert (W.value, b.value) == (256, 4)
    assert lib.srfmg_autotune_candidate(ctypes.byref(p), 10, ctypes.byref(W), ctypes.byref(b)) == srfmg.EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_choice_replays_on_the_oracle_gpu(precision):
    torch = pytest.importorskip("torch")
    M = 16
    best, table = srfmg.autotune(M, reps=3, precision=precision)
    assert len(table) == 10 and all(b >= 4 for _, b, _ in table)
    W, b = best.segment_width, best.buffer_width
    assert (W, b) in [(w, bb) for w, bb, _ in table]
    assert min(t for _, _, t in table) == [t for w, bb, t in table if (w, bb) == (W, b)][0]
    f, _, _ = workloads.sine_series(M, 32, seed=9)
    s = srfmg.Solver(M, params=best)
    try:
        u = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        s.close()
    ref = oracle.fmg_h(oracle.sr_params(M, W, b), f)
    assert np.max(np.abs(u - ref)) <= 1e-10 * np.max(np.abs(ref))
