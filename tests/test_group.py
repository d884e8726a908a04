"""Groups: independent problems of uneven sizes, one batched plan per size, all
replayed as one CUDA graph with a branch per plan.  Each problem of a group
must give bit for bit the result of its own single solve with its size's
parameters (same arithmetic, only offsets and launch order differ), and that
result is held to the oracle.  The packed layout and the argument checks need
no GPU."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads


def _create(sizes, tune=0, **kw):
    lib = srfmg.load()
    p = srfmg.default_params(12, **kw)
    arr = (ctypes.c_int32 * max(len(sizes), 1))(*sizes)
    h = ctypes.c_void_p(1)
    st = lib.srfmg_group_create(ctypes.byref(p), len(sizes), arr, tune, 0, ctypes.byref(h))
    return st, h


def test_group_offsets_pack_by_size_then_index():
    sizes = [12, 10, 14, 10, 12, 11]
    offs = srfmg.group_offsets(sizes)
    order = sorted(range(len(sizes)), key=lambda k: (sizes[k], k))   # 1, 3, 5, 0, 4, 2
    at = 0
    for k in order:
        assert offs[k] == at
        at += 1 << sizes[k]
    assert offs[-1] == at == sum(1 << m for m in sizes)
    # a single problem starts at 0
    assert list(srfmg.group_offsets([20])) == [0, 1 << 20]


def test_group_offsets_check_arguments():
    lib = srfmg.load()
    out = (ctypes.c_int64 * 4)()
    sizes = (ctypes.c_int32 * 3)(10, 0, 12)
    assert lib.srfmg_group_offsets(3, sizes, out) == srfmg.EINVAL          # size 0
    sizes = (ctypes.c_int32 * 3)(10, 29, 12)
    assert lib.srfmg_group_offsets(3, sizes, out) == srfmg.EINVAL          # beyond 2^28
    assert lib.srfmg_group_offsets(0, sizes, out) == srfmg.EINVAL
    assert lib.srfmg_group_offsets(3, None, out) == srfmg.EINVAL
    assert lib.srfmg_group_offsets(3, sizes, None) == srfmg.EINVAL


@pytest.mark.parametrize("sizes,tune,kw", [
    ([], 0, {}),                                   # no problems
    ([12, 2], 0, {}),                              # 2^2 is the coarsest level itself
    ([12, 10], -1, {}),                            # negative tune
    ([12, 10], 3, dict(n_sr_levels=0)),            # tuning needs an SR level
    ([12, 10], 0, dict(nu1=0)),                    # a shared parameter is checked per size
])
def test_group_create_checks_arguments_before_cuda(sizes, tune, kw):
    st, h = _create(sizes, tune, **kw)
    assert st == srfmg.EINVAL
    assert h.value is None
    assert srfmg.load().srfmg_group_last_error(None)


def test_group_null_handle_calls():
    lib = srfmg.load()
    assert lib.srfmg_group_solve(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_group_solve_host(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_group_query(None, None, None) == srfmg.EINVAL
    assert lib.srfmg_group_member(None, 0, None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_group_destroy(None) == srfmg.OK


def test_group_without_gpu_is_an_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    st, h = _create([12, 10])
    assert st == srfmg.ECUDA and h.value is None


def _packed(sizes, seeds, bratu=False):
    offs = srfmg.group_offsets(sizes)
    f = np.empty(offs[-1])
    for k, (m, s) in enumerate(zip(sizes, seeds)):
        gen = workloads.bratu_series(m, 16, seed=s, lam=1.0) if bratu else workloads.sine_series(m, 16, seed=s)
        f[offs[k]:offs[k] + (1 << m)] = gen[0]
    return f, offs


GROUPS = [
    # (sizes, kw)
    ([10, 8, 12, 10, 14, 8, 10, 12, 6, 13], dict(precision=srfmg.MIXED)),
    ([10, 8, 12, 10, 14, 8, 10, 12, 6, 13], dict(precision=srfmg.FP64)),
    ([11, 9, 15, 11, 7], dict(precision=srfmg.FP64, n_sr_levels=0)),
    ([12, 10, 12, 16], dict(precision=srfmg.MIXED, segment_width=1024, buffer_width=4, nu1=2)),
    ([12, 9, 13, 12], dict(precision=srfmg.FP64, op=srfmg.BRATU, lambda_=1.0, nu1=2, segment_width=512)),
]


@pytest.mark.gpu
@pytest.mark.parametrize("sizes,kw", GROUPS)
def test_group_equals_single_solves_gpu(sizes, kw):
    torch = pytest.importorskip("torch")
    seeds = [100 + k for k in range(len(sizes))]
    bratu = kw.get("op") == srfmg.BRATU
    f, offs = _packed(sizes, seeds, bratu)
    g = srfmg.Group(sizes, **kw)
    try:
        members = g.members()
        assert [m.n for m in members] == sorted(set(1 << m for m in sizes))
        assert sum(m.batch for m in members) == len(sizes)
        fd = torch.from_numpy(f).cuda()
        ud = g.solve(fd)
        u1 = ud.cpu().numpy()
        ud2 = g.solve(fd)                       # graph replay
        assert np.array_equal(ud2.cpu().numpy(), u1)
        uo = torch.full_like(fd, float("nan"))  # another pointer pair: a new capture
        g.solve(fd, uo)
        assert np.array_equal(uo.cpu().numpy(), u1)
        uh = g.solve_host(f)                    # host buffers, copies inside
        assert np.array_equal(uh, u1)
        info = {mb.n: (mb.params.segment_width, mb.params.buffer_width) for mb in members}
        assert all(mb.params.op == kw.get("op", 0) for mb in members)
    finally:
        g.close()
    nRS = kw.get("n_sr_levels", 1)
    for k, m in enumerate(sizes):
        uk = u1[offs[k]:offs[k] + (1 << m)]
        W, b = info[1 << m]
        over = dict(kw, batch=1)
        if nRS:
            over.update(segment_width=W, buffer_width=b)
        s = srfmg.Solver(m, **over)
        try:
            ref = s.solve(torch.from_numpy(f[offs[k]:offs[k] + (1 << m)]).cuda()).cpu().numpy()
        finally:
            s.close()
        assert np.array_equal(uk, ref), (k, m)
    # and the oracle for the largest problem
    k = int(np.argmax(sizes))
    m = sizes[k]
    W, b = info[1 << m]
    extra = dict(op="bratu", lam=1.0) if bratu else {}
    p = oracle.sr_params(m, W, b, nu1=kw.get("nu1", 1), **extra) if nRS else oracle.Params(m, nRS=0)
    r = oracle.fmg_h(p, f[offs[k]:offs[k] + (1 << m)])
    assert np.max(np.abs(u1[offs[k]:offs[k] + (1 << m)] - r)) <= 1e-10 * np.max(np.abs(r))


@pytest.mark.gpu
def test_group_tuned_layouts_replay_on_the_oracle_gpu():
    torch = pytest.importorskip("torch")
    sizes = [14, 12, 16, 12, 14]
    f, offs = _packed(sizes, range(5))
    g = srfmg.Group(sizes, tune=2, precision=srfmg.MIXED)
    try:
        u = g.solve(torch.from_numpy(f).cuda()).cpu().numpy()
        lay = {mb.n: (mb.params.segment_width, mb.params.buffer_width) for mb in g.members()}
    finally:
        g.close()
    for k, m in enumerate(sizes):
        W, b = lay[1 << m]
        assert b >= 4 and W >= 256
        fk = f[offs[k]:offs[k] + (1 << m)]
        r = oracle.fmg_h(oracle.sr_params(m, W, b), fk)
        assert np.max(np.abs(u[offs[k]:offs[k] + (1 << m)] - r)) <= 1e-10 * np.max(np.abs(r)), (k, m, W, b)


@pytest.mark.gpu
def test_group_member_calls_gpu():
    torch = pytest.importorskip("torch")
    sizes = [10, 12, 10]
    f, offs = _packed(sizes, [1, 2, 3])
    g = srfmg.Group(sizes, precision=srfmg.MIXED)
    try:
        lib = srfmg.load()
        n, tot = ctypes.c_int32(), ctypes.c_int64()
        assert lib.srfmg_group_query(g.h, ctypes.byref(n), ctypes.byref(tot)) == srfmg.OK
        assert (n.value, tot.value) == (2, offs[-1])
        assert lib.srfmg_group_member(g.h, 2, None, None, None, None) == srfmg.EINVAL
        fd = torch.from_numpy(f).cuda()
        ud = g.solve(fd)
        mb = g.members()[0]                     # the two problems of 2^10
        assert (mb.n, mb.batch, mb.offset) == (1 << 10, 2, 0)
        mb.check()                               # no non-finite value seen
        seg = mb.reconstruct(fd[:2 << 10], 0, 1)
        W = mb.params.segment_width
        got = seg.cpu().numpy().reshape(2, W)
        u = ud.cpu().numpy()
        assert np.array_equal(got[0], u[0:W]) and np.array_equal(got[1], u[1 << 10:(1 << 10) + W])
        bad = torch.empty(offs[-1] + 2, dtype=torch.float64, device="cuda")
        assert lib.srfmg_group_solve(g.h, ctypes.c_void_p(bad.data_ptr() + 8), ctypes.c_void_p(ud.data_ptr()),
                                     None) == srfmg.EINVAL     # misaligned
        assert lib.srfmg_group_solve(g.h, ctypes.c_void_p(fd.data_ptr()), ctypes.c_void_p(fd.data_ptr()),
                                     None) == srfmg.EINVAL     # overlap
    finally:
        g.close()


@pytest.mark.gpu
def test_group_variable_coefficient_through_members_gpu():
    """-(a u')' = f in a group: each plan's coefficient is set through its
    member handle (its problems' log a back to back), and every problem equals
    its own single solve with the same coefficient."""
    torch = pytest.importorskip("torch")
    sizes = [11, 13, 11, 12]
    offs = srfmg.group_offsets(sizes)
    data = [workloads.varcoef_series(m, 16, seed=40 + k) for k, m in enumerate(sizes)]
    f = np.empty(offs[-1])
    for k, m in enumerate(sizes):
        f[offs[k]:offs[k] + (1 << m)] = data[k][0]
    kw = dict(op=srfmg.VARCOEF, precision=srfmg.FP64, segment_width=1024)
    g = srfmg.Group(sizes, **kw)
    try:
        lay = {}
        for mb in g.members():
            m = mb.n.bit_length() - 1
            ks = [k for k in sorted(range(len(sizes)), key=lambda k: (sizes[k], k)) if sizes[k] == m]
            assert len(ks) == mb.batch
            mb.set_coefficient(torch.from_numpy(np.concatenate([data[k][2] for k in ks])).cuda())
            lay[m] = (mb.params.segment_width, mb.params.buffer_width)
        u = g.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        g.close()
    for k, m in enumerate(sizes):
        W, b = lay[m]
        s = srfmg.Solver(m, op=srfmg.VARCOEF, precision=srfmg.FP64, segment_width=W, buffer_width=b)
        try:
            s.set_coefficient(torch.from_numpy(data[k][2]).cuda())
            ref = s.solve(torch.from_numpy(data[k][0]).cuda()).cpu().numpy()
        finally:
            s.close()
        assert np.array_equal(u[offs[k]:offs[k] + (1 << m)], ref), (k, m)


def test_group_offsets_property_random_sizes():
    """For random size lists the offsets tile [0, total) without gaps or
    overlaps, in (size, index) order."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 60))
        sizes = [int(m) for m in rng.integers(1, 21, size=n)]
        offs = srfmg.group_offsets(sizes)
        order = sorted(range(n), key=lambda k: (sizes[k], k))
        at = 0
        for k in order:
            assert offs[k] == at
            at += 1 << sizes[k]
        assert offs[n] == at
        spans = sorted((int(offs[k]), int(offs[k]) + (1 << sizes[k])) for k in range(n))
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:])) and spans[0][0] == 0


@pytest.mark.gpu
def test_group_splits_sizes_beyond_one_plan_gpu():
    """More than 65535 problems of one size (the grid-row limit of a plan) are
    split over several plans; every problem still equals its own solve."""
    torch = pytest.importorskip("torch")
    n_small = 65535 + 7
    sizes = [4] * n_small + [8, 4]
    offs = srfmg.group_offsets(sizes)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(int(offs[-1]))
    g = srfmg.Group(sizes, precision=srfmg.MIXED, n_sr_levels=0)
    try:
        members = g.members()
        assert [(mb.n, mb.batch) for mb in members] == [(16, 65535), (16, 8), (256, 1)]
        assert [mb.offset for mb in members] == [0, 65535 * 16, (65535 + 8) * 16]
        u = g.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    finally:
        g.close()
    s4 = srfmg.Solver(4, precision=srfmg.MIXED, n_sr_levels=0, batch=8)
    s8 = srfmg.Solver(8, precision=srfmg.MIXED, n_sr_levels=0)
    try:
        for k in (0, 1, 65534, 65535, 65536, n_small - 1, n_small + 1):
            a, b = int(offs[k]), int(offs[k]) + (1 << sizes[k])
            # the same problem through a plan of its own (the second plan's 8 rows hold it)
            fb = np.zeros(8 << 4) if sizes[k] == 4 else None
            if sizes[k] == 4:
                fb[:16] = f[a:b]
                ref = s4.solve(torch.from_numpy(fb).cuda()).cpu().numpy()[:16]
            else:
                ref = s8.solve(torch.from_numpy(f[a:b].copy()).cuda()).cpu().numpy()
            assert np.array_equal(u[a:b], ref), k
    finally:
        s4.close()
        s8.close()


@pytest.mark.gpu
def test_group_without_graph_equals_graph_gpu(monkeypatch):
    """SRFMG_NO_GRAPH=1 at creation: the group enqueues its branches directly
    (no capture); results are the same bits as the graph's."""
    torch = pytest.importorskip("torch")
    sizes = [10, 12, 10, 13]
    f, offs = _packed(sizes, [7, 8, 9, 10])
    fd = torch.from_numpy(f).cuda()
    g = srfmg.Group(sizes, precision=srfmg.MIXED)
    try:
        u_graph = g.solve(fd).cpu().numpy()
    finally:
        g.close()
    monkeypatch.setenv("SRFMG_NO_GRAPH", "1")
    g = srfmg.Group(sizes, precision=srfmg.MIXED)
    monkeypatch.delenv("SRFMG_NO_GRAPH")
    try:
        u_direct = g.solve(fd).cpu().numpy()
        u_direct2 = g.solve(fd).cpu().numpy()
    finally:
        g.close()
    assert np.array_equal(u_direct, u_graph) and np.array_equal(u_direct2, u_graph)
