"""A seeded sweep over the plan options against the oracle.

Seventy configurations drawn from a fixed seed: the three operators, both
precisions, 0-2 SR levels with random segment and buffer widths, V(1,1) to
V(2,2) (V(2,1) for Bratu), coarsest levels 2^2-2^4, batches of 1-3 problems,
0-2 further V-cycles, and random CTA shapes (coarse tail, tile width, chained
down and up passes for the fixed-point -u'' = f).  Every problem of every plan
is held to the oracle's FMG cycle (and its V-cycles) within 1e-10 relative
max-norm: the shape options must not change the result and the option
combinations must all be the method.
"""
import numpy as np
import pytest

import oracle
from paper_1207_6720_gb300 import srfmg, workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _cases(n, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for it in range(n):
        op = str(rng.choice(["laplace", "laplace", "varcoef", "bratu"]))
        prec = srfmg.MIXED if rng.random() < 0.7 else srfmg.FP64
        M = int(rng.integers(8, 15))
        nRS = int(rng.choice([0, 1, 1, 1, 2]))
        W = int(2 ** rng.integers(max(4, M - 6), min(12, M - 1) + 1)) if nRS else 0
        b = int(rng.choice([2, 4, 8])) if nRS else 0
        if nRS == 2 and (W >> 1) < b:
            b = 2
        nu1, nu2 = (2, 1) if op == "bratu" else (int(rng.integers(1, 3)), int(rng.integers(1, 3)))
        M0 = int(rng.integers(2, 5))
        nv = int(rng.integers(0, 3)) if rng.random() < 0.3 else 0
        batch = int(rng.choice([1, 1, 2, 3]))
        kw = dict(precision=prec, n_sr_levels=nRS, nu1=nu1, nu2=nu2, log2_n_coarsest=M0, batch=batch,
                  n_vcycles=nv)
        if nRS:
            kw.update(segment_width=W, buffer_width=b)
        if rng.random() < 0.6:
            shape = dict(tail_level=int(rng.choice([0, 9, 10, 11, 12])),
                         tile_cells=int(rng.choice([0, 64, 128, 512, 2048])))
            if op == "laplace" and prec == srfmg.MIXED and rng.random() < 0.6:
                shape.update(chain_down=int(rng.integers(0, 5)), chain_up=int(rng.integers(0, 5)))
            kw.update(shape)
        out.append((it, op, M, kw))
    return out


@pytest.mark.parametrize("it,op,M,kw", _cases(70), ids=lambda v: str(v) if isinstance(v, int) else None)
def test_option_sweep_against_the_oracle_gpu(it, op, M, kw):
    okw = {}
    la = None
    if op == "varcoef":
        kw = dict(kw, op=srfmg.VARCOEF)
        f, _, la = workloads.varcoef_series(M, 16, seed=it)
        okw = dict(op="varcoef", coef=np.exp(la))
    elif op == "bratu":
        kw = dict(kw, op=srfmg.BRATU, lambda_=1.0)
        f, _, _ = workloads.bratu_series(M, 16, seed=it, lam=1.0)
        okw = dict(op="bratu", lam=1.0)
    else:
        f, _, _ = workloads.sine_series(M, 16, seed=it)
    batch = kw["batch"]
    s = srfmg.Solver(M, **kw)
    try:
        fd = torch.from_numpy(np.tile(f, batch)).cuda()
        if la is not None:
            s.set_coefficient(torch.from_numpy(np.tile(la, batch)).cuda())
        u = torch.zeros_like(fd)
        s.solve(fd, u)
        u = u.cpu().numpy().reshape(batch, -1)
    finally:
        s.close()
    nRS, nu1, nu2, M0 = kw["n_sr_levels"], kw["nu1"], kw["nu2"], kw["log2_n_coarsest"]
    if nRS:
        p = oracle.sr_params(M, kw["segment_width"], kw["buffer_width"], nRS=nRS, nu1=nu1, nu2=nu2, M0=M0, **okw)
    else:
        p = oracle.Params(M, M0=M0, nRS=0, nu1=nu1, nu2=nu2, **okw)
    ref = oracle.fmg_h(p, f)
    if kw["n_vcycles"]:
        ref = oracle.vcycles_h(p, f, ref, kw["n_vcycles"])
    for k in range(batch):
        assert np.max(np.abs(u[k] - ref)) <= 1e-10 * np.max(np.abs(ref))
