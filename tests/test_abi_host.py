"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/srfmg.h declares, and rejects bad arguments on the host
before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1207_6720_gb300 import srfmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "srfmg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:srfmg_status|const char \*)\s*(srfmg_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("srfmg_create", "srfmg_solve", "srfmg_adjoint", "srfmg_destroy"):
        assert want in names
    assert set(names) == set(srfmg.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = srfmg.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert srfmg.version().startswith("srfmg")


def test_default_params():
    p = srfmg.default_params(24)
    assert (p.log2_n, p.log2_n_coarsest, p.n_sr_levels) == (24, 2, 1)
    assert (p.segment_width, p.buffer_width, p.nu1, p.nu2) == (4096, 8, 1, 1)
    assert srfmg.default_params(10).segment_width == 256
    assert srfmg.load().srfmg_default_params(10, None) == srfmg.EINVAL


@pytest.mark.parametrize("field,value", [
    ("log2_n", 2), ("log2_n", 29), ("log2_n_coarsest", 1), ("log2_n_coarsest", 7),
    ("n_sr_levels", 3), ("n_sr_levels", -1), ("segment_width", 24), ("segment_width", 8),
    ("segment_width", 8192), ("buffer_width", 3), ("buffer_width", 0), ("buffer_width", 66),
    ("nu1", 0), ("nu2", 5), ("op", 3), ("smoother", 1), ("precision", 7),
    ("tail_level", 1), ("tail_level", 13), ("tile_cells", 100), ("tile_cells", 32), ("tile_cells", 4096),
])
def test_create_rejects_bad_params_before_cuda(field, value):
    lib = srfmg.load()
    p = srfmg.default_params(12)
    setattr(p, field, value)
    h = ctypes.c_void_p(1)
    st = lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h))
    assert st == srfmg.EINVAL
    assert h.value is None
    assert lib.srfmg_last_error(None)


@pytest.mark.parametrize("overrides", [
    dict(n_sr_levels=2, log2_n=5, log2_n_coarsest=4),              # no stored level below the SR levels
    dict(n_sr_levels=2, segment_width=16, buffer_width=10),        # buffer wider than level M-1's 8-cell segments
    dict(tau_edge=2),                                               # no such edge-tau reading
    dict(tau_edge=1, n_sr_levels=0),                                # edge tau without SR segments
])
def test_two_sr_levels_are_checked_before_cuda(overrides):
    lib = srfmg.load()
    p = srfmg.default_params(12)
    for k, v in overrides.items():
        setattr(p, k, v)
    h = ctypes.c_void_p(1)
    assert lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h)) == srfmg.EINVAL
    assert h.value is None


def test_create_rejects_bad_post_leg_and_null():
    lib = srfmg.load()
    h = ctypes.c_void_p()
    # an unknown post-leg option, and FAS recompute outside its preconditions
    for kw in (dict(post_leg=7), dict(post_leg=1, n_sr_levels=2), dict(post_leg=1, n_sr_levels=0),
               dict(post_leg=1, tau_edge=1), dict(post_leg=1, n_vcycles=1),
               dict(post_leg=1, segment_width=16, buffer_width=16)):
        p = srfmg.default_params(12)
        for k, v in kw.items():
            setattr(p, k, v)
        assert lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h)) == srfmg.EINVAL, kw
    assert lib.srfmg_create(None, 0, ctypes.byref(h)) == srfmg.EINVAL
    p = srfmg.default_params(12)
    assert lib.srfmg_create(ctypes.byref(p), 0, None) == srfmg.EINVAL


def test_null_handle_calls():
    lib = srfmg.load()
    assert lib.srfmg_solve(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_solve_host(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_solve_host_async(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_solve_host_join(None, None) == srfmg.EINVAL
    assert lib.srfmg_adjoint(None, None, None, None) == srfmg.EINVAL
    assert lib.srfmg_query(None, None) == srfmg.EINVAL
    assert lib.srfmg_destroy(None) == srfmg.OK


def test_noalloc_entry_checks_arguments_on_the_host():
    lib = srfmg.load()
    buf = (ctypes.c_double * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    for args in [(13, 2, 1, 1), (12, 1, 1, 1), (12, 7, 1, 1), (4, 4, 1, 1), (10, 2, 0, 1), (10, 2, 1, 5)]:
        assert lib.srfmg_solve_small_noalloc(*args, p, p, None) == srfmg.EINVAL
    assert lib.srfmg_solve_small_noalloc(10, 2, 1, 1, None, None, None) == srfmg.EINVAL


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(srfmg.SrfmgError) as ei:
        srfmg.Solver(12)
    assert ei.value.status == srfmg.ECUDA


def test_alu_peaks_rejects_null_on_the_host():
    lib = srfmg.load()
    assert lib.srfmg_alu_peaks(0, None) == srfmg.EINVAL


def test_shape_candidates_on_the_host():
    # distinct coarse tails (9..12 clipped to the levels below the SR level) x tiles;
    # for the fixed-point -u'' = f also chained passes on the two finest tails
    lib = srfmg.load()

    def cands(M, **kw):
        p = srfmg.default_params(M, **kw)
        out = []
        for k in range(64):
            c = srfmg.Params()
            if lib.srfmg_autotune_shape_candidate(ctypes.byref(p), k, ctypes.byref(c)) != srfmg.OK:
                break
            assert (c.log2_n, c.precision, c.segment_width) == (p.log2_n, p.precision, p.segment_width)
            out.append((c.tail_level, c.tile_cells, c.chain_down, c.chain_up))
        return out

    plain = [(t, c, 0, 0) for t in (9, 10, 11, 12) for c in (128, 256, 512)]
    assert cands(24) == plain
    assert cands(24, precision=srfmg.MIXED) == plain + [(t, c, 2, u) for t in (11, 12) for c in (256, 512)
                                                         for u in (3, 4)]
    assert cands(24, precision=srfmg.MIXED, op=srfmg.VARCOEF) == plain
    assert cands(11) == [(9, 128, 0, 0), (9, 256, 0, 0), (9, 512, 0, 0), (10, 128, 0, 0), (10, 256, 0, 0),
                         (10, 512, 0, 0)]
    assert cands(11, precision=srfmg.MIXED)[6:] == [(t, c, 2, u) for t in (9, 10) for c in (256, 512)
                                                    for u in (3, 4)]
    assert cands(8) == [(9, 128, 0, 0), (9, 256, 0, 0), (9, 512, 0, 0)]      # one tail: the whole problem


def test_chain_params_are_checked_on_the_host():
    lib = srfmg.load()
    for kw in (dict(chain_down=5), dict(chain_up=-1), dict(chain_up=2),
               dict(chain_down=2, precision=srfmg.MIXED, op=srfmg.VARCOEF),
               dict(chain_up=3, precision=srfmg.MIXED, op=srfmg.BRATU, lambda_=1.0)):
        p = srfmg.default_params(16, **kw)
        h = ctypes.c_void_p()
        assert lib.srfmg_create(ctypes.byref(p), 0, ctypes.byref(h)) == srfmg.EINVAL, kw
        assert "chain" in lib.srfmg_last_error(None).decode()


def test_exp_error_checks_its_arguments_on_the_host():
    lib = srfmg.load()
    out = ctypes.c_double()
    for lo, hi, n in ((1.0, 0.0, 10), (0.0, 1.0, 0), (-800.0, 0.0, 10), (0.0, float("nan"), 10), (0.0, 1.0, 1 << 27)):
        assert lib.srfmg_exp_error(0, lo, hi, n, ctypes.byref(out)) == srfmg.EINVAL
    assert lib.srfmg_exp_error(0, 0.0, 1.0, 10, None) == srfmg.EINVAL
