"""Python binding of the C ABI in include/srfmg.h (argument marshalling only).

Every step of the solve runs in the CUDA kernels of libsrfmg.so; PyTorch is
used only to hold device memory and to supply the current CUDA stream.  There
is no CPU fallback: if the library is missing or no GPU is visible the calls
raise.
"""
import ctypes
import os

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "SRFMG_OK", 1: "SRFMG_EINVAL", 2: "SRFMG_ENOMEM", 3: "SRFMG_ECUDA",
                4: "SRFMG_ETIMEOUT", 5: "SRFMG_ENONFINITE", 6: "SRFMG_EUNSUPPORTED"}
FP64, MIXED = 0, 1
LAPLACE, VARCOEF, BRATU = 0, 1, 2
TAU_ASSEMBLED, TAU_SEGMENT = 0, 1
POST_FULL_UPDATE, POST_FAS_RECOMPUTE = 0, 1
NUM_FUNCTIONALS = 5          # functionals per problem of srfmg_solve_functionals

EXPORTS = ("srfmg_default_params", "srfmg_create", "srfmg_solve", "srfmg_solve_host",
           "srfmg_adjoint", "srfmg_query", "srfmg_profile", "srfmg_launch_name",
           "srfmg_solve_small_noalloc", "srfmg_autotune", "srfmg_autotune_candidate",
           "srfmg_autotune_shape", "srfmg_autotune_shape_candidate",
           "srfmg_set_coefficient", "srfmg_coef_gradient", "srfmg_solve_functionals", "srfmg_reconstruct", "srfmg_check",
           "srfmg_destroy", "srfmg_last_error", "srfmg_version", "srfmg_alu_peaks", "srfmg_exp_error",
           "srfmg_solve_host_async", "srfmg_solve_host_join", "srfmg_group_offsets", "srfmg_group_create", "srfmg_group_solve", "srfmg_group_solve_host",
           "srfmg_group_query", "srfmg_group_member", "srfmg_group_destroy", "srfmg_group_last_error")


class Params(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "op", "precision", "log2_n", "log2_n_coarsest", "n_sr_levels", "segment_width",
        "buffer_width", "nu1", "nu2", "smoother")] + [("lambda_", ctypes.c_double),
                                                      ("batch", ctypes.c_int32),
                                                      ("tau_edge", ctypes.c_int32),
                                                      ("n_vcycles", ctypes.c_int32),
                                                      ("post_leg", ctypes.c_int32),
                                                      ("tail_level", ctypes.c_int32),
                                                      ("tile_cells", ctypes.c_int32),
                                                      ("chain_down", ctypes.c_int32),
                                                      ("chain_up", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_int64), ("kernels_per_solve", ctypes.c_int32),
                ("coarse_tail_level", ctypes.c_int32), ("n_segments", ctypes.c_int32),
                ("segment_width", ctypes.c_int32), ("buffer_width", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


class SrfmgError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libsrfmg.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA extension not built: {path} is missing")
    lib = ctypes.CDLL(path)
    vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    lib.srfmg_default_params.argtypes = [ctypes.c_int32, ctypes.POINTER(Params)]
    lib.srfmg_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(H)]
    lib.srfmg_solve.argtypes = [H, vp, vp, vp]
    lib.srfmg_solve_host.argtypes = [H, dp, dp, vp]
    lib.srfmg_solve_host_async.argtypes = [H, dp, dp, vp]
    lib.srfmg_solve_host_join.argtypes = [H, vp]
    lib.srfmg_adjoint.argtypes = [H, vp, vp, vp]
    lib.srfmg_query.argtypes = [H, ctypes.POINTER(Info)]
    lib.srfmg_destroy.argtypes = [H]
    lib.srfmg_last_error.argtypes = [H]
    lib.srfmg_last_error.restype = ctypes.c_char_p
    lib.srfmg_profile.argtypes = [H, vp, vp, vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float),
                                  ctypes.c_int32]
    lib.srfmg_launch_name.argtypes = [H, ctypes.c_int32]
    lib.srfmg_launch_name.restype = ctypes.c_char_p
    lib.srfmg_solve_small_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, vp, vp, vp]
    lib.srfmg_solve_small_noalloc.restype = ctypes.c_int
    lib.srfmg_autotune.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_int32, ctypes.POINTER(Params),
                                    ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.srfmg_autotune_candidate.argtypes = [ctypes.POINTER(Params), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.srfmg_autotune_shape.argtypes = lib.srfmg_autotune.argtypes
    lib.srfmg_autotune_shape_candidate.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, ctypes.POINTER(Params)]
    lib.srfmg_set_coefficient.argtypes = [H, vp, vp]
    lib.srfmg_coef_gradient.argtypes = [H, vp, vp, vp, vp]
    lib.srfmg_solve_functionals.argtypes = [H, vp, vp, vp, vp, vp]
    lib.srfmg_reconstruct.argtypes = [H, vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
    lib.srfmg_check.argtypes = [H, vp]
    i32p, i64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    lib.srfmg_group_offsets.argtypes = [ctypes.c_int32, i32p, i64p]
    lib.srfmg_group_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int32, i32p, ctypes.c_int32,
                                       ctypes.c_int, ctypes.POINTER(H)]
    lib.srfmg_group_solve.argtypes = [H, vp, vp, vp]
    lib.srfmg_group_solve_host.argtypes = [H, dp, dp, vp]
    lib.srfmg_group_query.argtypes = [H, i32p, i64p]
    lib.srfmg_group_member.argtypes = [H, ctypes.c_int32, ctypes.POINTER(H), i32p, i32p, i64p]
    lib.srfmg_group_destroy.argtypes = [H]
    lib.srfmg_group_last_error.argtypes = [H]
    lib.srfmg_group_last_error.restype = ctypes.c_char_p
    lib.srfmg_version.argtypes = []
    lib.srfmg_version.restype = ctypes.c_char_p
    lib.srfmg_alu_peaks.argtypes = [ctypes.c_int, dp]
    lib.srfmg_exp_error.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int32, dp]
    for name in ("srfmg_default_params", "srfmg_create", "srfmg_solve", "srfmg_solve_host",
                 "srfmg_adjoint", "srfmg_query", "srfmg_profile", "srfmg_destroy", "srfmg_autotune",
                 "srfmg_autotune_candidate", "srfmg_autotune_shape", "srfmg_autotune_shape_candidate",
                 "srfmg_set_coefficient", "srfmg_coef_gradient",
                 "srfmg_solve_functionals", "srfmg_reconstruct", "srfmg_check", "srfmg_solve_host_async",
                 "srfmg_solve_host_join", "srfmg_group_offsets",
                 "srfmg_group_create", "srfmg_group_solve", "srfmg_group_solve_host", "srfmg_group_query",
                 "srfmg_group_member", "srfmg_group_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def default_params(log2_n, **overrides):
    p = Params()
    st = load().srfmg_default_params(log2_n, ctypes.byref(p))
    if st != OK:
        raise SrfmgError(st, "default_params")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, float(v) if k == "lambda_" else int(v))
    return p


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Solver:
    """One plan: ``Solver(log2_n, segment_width=..., buffer_width=..., ...)``.

    ``solve(f)`` takes a CUDA float64 tensor of 2^log2_n right-hand-side values
    at the cell centres and returns the solution tensor (same device).
    """

    def __init__(self, log2_n, device=0, params=None, **overrides):
        self.lib = load()
        self.params = params if params is not None else default_params(log2_n, **overrides)
        self.n = 1 << self.params.log2_n
        self.batch = max(1, self.params.batch)
        self.device = device
        h = ctypes.c_void_p()
        st = self.lib.srfmg_create(ctypes.byref(self.params), device, ctypes.byref(h))
        if st != OK:
            raise SrfmgError(st, self.lib.srfmg_last_error(None).decode())
        self.h = h

    def _check(self, st, what):
        if st != OK:
            raise SrfmgError(st, f"{what}: {self.lib.srfmg_last_error(self.h).decode()}")

    def info(self):
        inf = Info()
        self._check(self.lib.srfmg_query(self.h, ctypes.byref(inf)), "query")
        return inf

    def solve(self, f, u=None, stream=None):
        import torch
        if not (f.is_cuda and f.dtype == torch.float64 and f.is_contiguous()
                and f.numel() == self.n * self.batch):
            raise ValueError("f must be a contiguous CUDA float64 tensor of batch * 2^log2_n values")
        if u is None:
            u = torch.empty_like(f)
        self._check(self.lib.srfmg_solve(self.h, ctypes.c_void_p(f.data_ptr()),
                                          ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream)),
                    "solve")
        return u

    def adjoint(self, dL_du, dL_df=None, stream=None):
        """dL/df for a loss L(u) of the solution, given dL/du (CUDA float64):
        the adjoint solve of the C ABI (the same FMG(-SR) solve applied to the
        adjoint right-hand side; the operator is symmetric)."""
        import torch
        if not (dL_du.is_cuda and dL_du.dtype == torch.float64 and dL_du.is_contiguous()
                and dL_du.numel() == self.n * self.batch):
            raise ValueError("dL_du must be a contiguous CUDA float64 tensor of batch * 2^log2_n values")
        if dL_df is None:
            dL_df = torch.empty_like(dL_du)
        self._check(self.lib.srfmg_adjoint(self.h, ctypes.c_void_p(dL_du.data_ptr()),
                                            ctypes.c_void_p(dL_df.data_ptr()), _stream_ptr(stream)),
                    "adjoint")
        return dL_df

    def set_coefficient(self, log_a, stream=None):
        """SRFMG_OP_VARCOEF: a = exp(log_a) at the 2^log2_n + 1 faces (per problem).
        The library checks the coefficient on the device and synchronises the
        stream; a coefficient the sweeps cannot take exactly (log_a not finite
        or beyond +-700, or neighbouring faces of a level of 128 or more cells
        more than a factor 1.5 apart) raises SrfmgError and resets a to 1."""
        import torch
        if not (log_a.is_cuda and log_a.dtype == torch.float64 and log_a.is_contiguous()
                and log_a.numel() == (self.n + 1) * self.batch):
            raise ValueError("log_a must be a contiguous CUDA float64 tensor of batch * (2^log2_n + 1) values")
        self._check(self.lib.srfmg_set_coefficient(self.h, ctypes.c_void_p(log_a.data_ptr()), _stream_ptr(stream)),
                    "set_coefficient")

    def solve_functionals(self, f, u=None, u_ref=None, out=None, stream=None):
        """SR solve that returns the functionals of the fine solution, NUM_FUNCTIONALS
        per problem: [h sum u, h sum u^2, max|u|, h sum (u - u_ref)^2, max|u - u_ref|]
        (the last two 0 without u_ref).  u: CUDA float64 tensor to receive the
        solution, or None to leave the fine grid unwritten."""
        import torch
        self._check_vec("f", f)
        for name, t in (("u", u), ("u_ref", u_ref)):
            if t is not None:
                self._check_vec(name, t)
        if out is None:
            out = torch.empty(NUM_FUNCTIONALS * self.batch, dtype=torch.float64, device=f.device)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None)
        self._check(self.lib.srfmg_solve_functionals(self.h, ptr(f), ptr(u), ptr(u_ref), ptr(out),
                                                     _stream_ptr(stream)), "solve_functionals")
        return out

    def reconstruct(self, f, seg_begin, seg_count, out=None, stream=None):
        """Fine-grid segments [seg_begin, seg_begin + seg_count) expanded from the
        coarse solution of the last solve (f: that solve's right-hand side);
        returns seg_count * segment_width values per problem."""
        import torch
        self._check_vec("f", f)
        n_out = seg_count * self.params.segment_width * self.batch
        if out is None:
            out = torch.empty(n_out, dtype=torch.float64, device=f.device)
        self._check(self.lib.srfmg_reconstruct(self.h, ctypes.c_void_p(f.data_ptr()), seg_begin, seg_count,
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                    "reconstruct")
        return out

    def check(self, stream=None):
        """Raise SrfmgError (SRFMG_ENONFINITE) if an inf or NaN was seen in f or
        in the functionals since the last check; synchronises the stream."""
        self._check(self.lib.srfmg_check(self.h, _stream_ptr(stream)), "check")

    def _check_vec(self, name, t):
        import torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == self.n * self.batch):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of batch * 2^log2_n values")

    def coef_gradient(self, u, lam, out=None, stream=None):
        """SRFMG_OP_VARCOEF: dL/dlog a at the 2^log2_n + 1 faces (per problem)
        from the solution u and the adjoint state lam = adjoint(dL/du)."""
        import torch
        for name, t in (("u", u), ("lam", lam)):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.numel() == self.n * self.batch):
                raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of batch * 2^log2_n values")
        if out is None:
            out = torch.empty((self.n + 1) * self.batch, dtype=torch.float64, device=u.device)
        self._check(self.lib.srfmg_coef_gradient(self.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)),
                    "coef_gradient")
        return out

    def solve_host(self, f, u=None, stream=None):
        """Solve from and to host numpy arrays (copies inside; synchronises)."""
        import numpy as np
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.size != self.n * self.batch:
            raise ValueError("f must hold batch * 2^log2_n values")
        if u is None:
            u = np.empty_like(f)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.srfmg_solve_host(self.h, f.ctypes.data_as(dp), u.ctypes.data_as(dp),
                                               _stream_ptr(stream)), "solve_host")
        return u

    def solve_host_async(self, f, u, stream=None):
        """Enqueue a solve from and to host numpy arrays (pinned for overlap); the
        copies overlap the neighbouring solves.  Call host_join (and synchronise
        the stream) before reading u or changing f."""
        if f.dtype.name != "float64" or u.dtype.name != "float64" or not (
                f.flags.c_contiguous and u.flags.c_contiguous) or f.size != self.n * self.batch or u.size != f.size:
            raise ValueError("f and u must be contiguous float64 arrays of batch * 2^log2_n values")
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.srfmg_solve_host_async(self.h, f.ctypes.data_as(dp), u.ctypes.data_as(dp),
                                                     _stream_ptr(stream)), "solve_host_async")
        return u

    def host_join(self, stream=None):
        """Make the stream wait for every copy-out of solve_host_async so far."""
        self._check(self.lib.srfmg_solve_host_join(self.h, _stream_ptr(stream)), "solve_host_join")

    def profile(self, f, u=None, nsolves=3, stream=None):
        """Per-launch average durations (ms) of one solve: list of (name, ms)."""
        import torch
        if u is None:
            u = torch.empty_like(f)
        nops = self.info().kernels_per_solve
        buf = (ctypes.c_float * nops)()
        self._check(self.lib.srfmg_profile(self.h, ctypes.c_void_p(f.data_ptr()),
                                            ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream),
                                            nsolves, buf, nops), "profile")
        return [(self.lib.srfmg_launch_name(self.h, i).decode(), float(buf[i])) for i in range(nops)]

    def close(self):
        if getattr(self, "h", None):
            self.lib.srfmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def group_offsets(log2_n):
    """Packed layout of a group (host only): offsets[k] = first cell of problem
    k, offsets[-1] = total cells; problems ordered by size, then by index."""
    import numpy as np
    sizes = np.ascontiguousarray(log2_n, dtype=np.int32)
    offs = np.empty(sizes.size + 1, dtype=np.int64)
    st = load().srfmg_group_offsets(sizes.size, sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if st != OK:
        raise SrfmgError(st, load().srfmg_group_last_error(None).decode())
    return offs


class _Member(Solver):
    """A plan owned by a group (srfmg_group_member): the per-plan calls of
    Solver on its part of the packed arrays; closing it does nothing."""

    def __init__(self, lib, h, log2_n, count, offset, params):
        self.lib, self.h, self.device = lib, h, None
        self.params = params
        self.n, self.batch = 1 << log2_n, count
        self.offset = offset

    def close(self):
        self.h = None


class Group:
    """Independent problems of uneven sizes: ``Group(log2_n_list, **params)``.

    One batched plan per distinct size, all replayed as one CUDA graph.  The
    packed arrays hold the problems ordered by size, then by index
    (``offsets``).  ``tune=k`` autotunes each size's segment layout with k
    timed solves per candidate."""

    def __init__(self, log2_n, device=0, tune=0, **overrides):
        import numpy as np
        self.lib = load()
        self.sizes = np.ascontiguousarray(log2_n, dtype=np.int32)
        self.offsets = group_offsets(self.sizes)
        self.total = int(self.offsets[-1])
        self.params = default_params(int(self.sizes.max()), **overrides)
        h = ctypes.c_void_p()
        st = self.lib.srfmg_group_create(ctypes.byref(self.params), self.sizes.size,
                                         self.sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                         tune, device, ctypes.byref(h))
        if st != OK:
            raise SrfmgError(st, self.lib.srfmg_group_last_error(None).decode())
        self.h = h
        self.device = device

    def _check(self, st, what):
        if st != OK:
            raise SrfmgError(st, f"{what}: {self.lib.srfmg_group_last_error(self.h).decode()}")

    def members(self):
        """The plans, by ascending size (Solver views owned by the group)."""
        n = ctypes.c_int32()
        self._check(self.lib.srfmg_group_query(self.h, ctypes.byref(n), None), "query")
        out = []
        for i in range(n.value):
            hp, m, c, o = ctypes.c_void_p(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
            self._check(self.lib.srfmg_group_member(self.h, i, ctypes.byref(hp), ctypes.byref(m), ctypes.byref(c),
                                                    ctypes.byref(o)), "member")
            inf = Info()
            self._check(self.lib.srfmg_query(hp, ctypes.byref(inf)), "query")
            p = Params()
            ctypes.memmove(ctypes.byref(p), ctypes.byref(self.params), ctypes.sizeof(Params))
            p.log2_n, p.batch = m.value, c.value
            if inf.segment_width:
                p.segment_width, p.buffer_width = inf.segment_width, inf.buffer_width
            out.append(_Member(self.lib, hp, m.value, c.value, o.value, p))
        return out

    def solve(self, f, u=None, stream=None):
        import torch
        if not (f.is_cuda and f.dtype == torch.float64 and f.is_contiguous() and f.numel() == self.total):
            raise ValueError("f must be a contiguous CUDA float64 tensor of the group's total cells")
        if u is None:
            u = torch.empty_like(f)
        self._check(self.lib.srfmg_group_solve(self.h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                               _stream_ptr(stream)), "solve")
        return u

    def solve_host(self, f, u=None, stream=None):
        """Solve from and to host numpy arrays of the packed layout (synchronises)."""
        import numpy as np
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.size != self.total:
            raise ValueError("f must hold the group's total cells")
        if u is None:
            u = np.empty_like(f)
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.srfmg_group_solve_host(self.h, f.ctypes.data_as(dp), u.ctypes.data_as(dp),
                                                    _stream_ptr(stream)), "solve_host")
        return u

    def close(self):
        if getattr(self, "h", None):
            self.lib.srfmg_group_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _solve_functions():
    import torch

    class _Solve(torch.autograd.Function):
        """u = solve(f) with dL/df = adjoint(dL/du) in the backward pass."""

        @staticmethod
        def forward(ctx, f, solver):
            ctx.solver = solver
            return solver.solve(f.contiguous())

        @staticmethod
        def backward(ctx, grad_u):
            return ctx.solver.adjoint(grad_u.contiguous()), None

    class _SolveCoef(torch.autograd.Function):
        """u = solve(f; a = exp(log_a)) with dL/df = lam = adjoint(dL/du) and
        dL/dlog a = coef_gradient(u, lam) in the backward pass."""

        @staticmethod
        def forward(ctx, f, log_a, solver):
            solver.set_coefficient(log_a.detach().contiguous())
            u = solver.solve(f.contiguous())
            ctx.solver = solver
            ctx.save_for_backward(u)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            (u,) = ctx.saved_tensors
            lam = ctx.solver.adjoint(grad_u.contiguous())
            g = ctx.solver.coef_gradient(u, lam) if ctx.needs_input_grad[1] else None
            return lam, g, None

    return _Solve, _SolveCoef


_SOLVE_FNS = None


def solve_autograd(solver, f, log_a=None):
    """Differentiable solve: ``u = solve_autograd(solver, f)``; ``u.backward``
    (or ``torch.autograd.grad``) runs the adjoint solve on the GPU.  For a
    SRFMG_OP_VARCOEF plan, ``log_a`` (the log of the face coefficients) sets the
    coefficient and receives dL/dlog a; the backward pass uses the plan's
    coefficient, so it must run before the plan's coefficient is set again."""
    global _SOLVE_FNS
    if _SOLVE_FNS is None:
        _SOLVE_FNS = _solve_functions()
    if log_a is None:
        return _SOLVE_FNS[0].apply(f, solver)
    return _SOLVE_FNS[1].apply(f, log_a, solver)


def solve_small_noalloc(f, u=None, log2_n_coarsest=2, nu1=1, nu2=1, stream=None):
    """Plain FMG-FAS for N <= 4096 through srfmg_solve_small_noalloc, which
    allocates no device memory (for callers that cannot call cudaMalloc: open
    stream captures, pool-owned device memory, allocation-free loops).  f: CUDA
    float64 tensor of 2^k values; u: a CUDA float64 tensor of the same size on
    the same device, which receives the solution and is returned.  With
    u=None this wrapper allocates u (torch.empty_like), so a caller that must
    not allocate passes u.  The call runs with f's device current (the entry
    point finds its static array on the current device) and on that device's
    current stream unless `stream` is given.  The first call on a device does a
    synchronous set-up and should come before any stream capture."""
    import torch
    n = f.numel()
    log2_n = n.bit_length() - 1
    if not (f.is_cuda and f.dtype == torch.float64 and f.is_contiguous() and n == 1 << log2_n):
        raise ValueError("f must be a contiguous CUDA float64 tensor of 2^k values")
    if u is None:
        u = torch.empty_like(f)
    elif not (u.is_cuda and u.dtype == torch.float64 and u.is_contiguous() and u.numel() == n
              and u.device == f.device):
        raise ValueError("u must be a contiguous CUDA float64 tensor of f's size on f's device")
    with torch.cuda.device(f.device):
        st = load().srfmg_solve_small_noalloc(log2_n, log2_n_coarsest, nu1, nu2,
                                               ctypes.c_void_p(f.data_ptr()),
                                               ctypes.c_void_p(u.data_ptr()), _stream_ptr(stream))
    if st != OK:
        raise SrfmgError(st, "srfmg_solve_small_noalloc (status code only)")
    return u


def autotune(log2_n, device=0, reps=5, **overrides):
    """Time the admissible SR segment layouts (W, b >= 4) for this solve and
    return (best Params, [(W, b, ms per solve), ...])."""
    lib = load()
    base = default_params(log2_n, **overrides)
    best = Params()
    cap = 16
    ms = (ctypes.c_float * cap)()
    n = ctypes.c_int32()
    st = lib.srfmg_autotune(ctypes.byref(base), device, reps, ctypes.byref(best), ms, cap, ctypes.byref(n))
    if st != OK:
        raise SrfmgError(st, lib.srfmg_last_error(None).decode())
    table = []
    for k in range(min(n.value, cap)):
        W, b = ctypes.c_int32(), ctypes.c_int32()
        lib.srfmg_autotune_candidate(ctypes.byref(base), k, ctypes.byref(W), ctypes.byref(b))
        table.append((W.value, b.value, float(ms[k])))
    return best, table


def autotune_shape(params, device=0, reps=5):
    """Time the CTA shapes (coarse tail extent, cells per tile of the latency-bound
    stored levels, chained down and up passes) of the plan `params` and return
    (best Params, [(tail_level, tile_cells, chain_down, chain_up, ms per solve),
    ...]); the shape does not change the result."""
    lib = load()
    base = Params()
    ctypes.memmove(ctypes.byref(base), ctypes.byref(params), ctypes.sizeof(Params))
    best = Params()
    cap = 64
    ms = (ctypes.c_float * cap)()
    n = ctypes.c_int32()
    st = lib.srfmg_autotune_shape(ctypes.byref(base), device, reps, ctypes.byref(best), ms, cap, ctypes.byref(n))
    if st != OK:
        raise SrfmgError(st, lib.srfmg_last_error(None).decode())
    table = []
    for k in range(min(n.value, cap)):
        c = Params()
        lib.srfmg_autotune_shape_candidate(ctypes.byref(base), k, ctypes.byref(c))
        table.append((c.tail_level, c.tile_cells, c.chain_down, c.chain_up, float(ms[k])))
    return best, table


def version():
    return load().srfmg_version().decode()


def exp_error(lo, hi, n, device=0):
    """Largest relative difference between the mixed Bratu exponential and
    CUDA's exp at n evenly spaced points of [lo, hi] (srfmg_exp_error)."""
    lib = load()
    out = ctypes.c_double()
    st = lib.srfmg_exp_error(device, lo, hi, n, ctypes.byref(out))
    if st != OK:
        raise SrfmgError(st, lib.srfmg_last_error(None).decode())
    return out.value


def alu_peaks(device=0):
    """Measured arithmetic throughput of the device (srfmg_alu_peaks): a dict of
    64-bit integer adds/s, 64-bit operations/s in the (x + y + 1) >> 1 step,
    FP64 flops/s and FP32 flops/s."""
    lib = load()
    out = (ctypes.c_double * 4)()
    st = lib.srfmg_alu_peaks(device, out)
    if st != OK:
        raise SrfmgError(st, lib.srfmg_last_error(None).decode())
    return {"i64_add_per_s": out[0], "i64_avg_ops_per_s": out[1], "fp64_flops": out[2], "fp32_flops": out[3]}
