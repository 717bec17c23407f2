"""Thin ctypes binding of libpty (include/pty.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python arguments
(torch tensors on the GPU or the CPU, or numpy arrays) into the raw pointers and sizes
of the C ABI, checks that each array holds the number of elements the call reads or
writes, and turns status codes into exceptions.  There is no fallback: if the library
cannot be built or loaded, importing the functions raises.

Use (one reconstruction on the current CUDA device)::

    ctx = Context(probe, pos, data, H, W)      # probe [P][P] complex64, pos [K][2] int32,
                                               # data [K][P][P] float32 counts
    psi = torch.ones((H, W), dtype=torch.complex64, device="cuda")
    status, report = ctx.cg_solve(psi, 64)     # 64 ML-CG iterations, psi updated in place
    ctx.close()
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

PTY_OK, PTY_ERR_ARG, PTY_ERR_BOUNDS, PTY_ERR_NOMEM, PTY_ERR_CUDA = 0, 1, 2, 3, 4
PTY_ERR_NONFINITE, PTY_STALLED, PTY_ERR_TIMEOUT, PTY_ERR_UNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "PTY_OK", 1: "PTY_ERR_ARG", 2: "PTY_ERR_BOUNDS", 3: "PTY_ERR_NOMEM", 4: "PTY_ERR_CUDA",
                5: "PTY_ERR_NONFINITE", 6: "PTY_STALLED", 7: "PTY_ERR_TIMEOUT", 8: "PTY_ERR_UNSUPPORTED"}

EXPORTED = ["pty_default_opts", "pty_create", "pty_create_subpixel", "pty_destroy", "pty_last_error", "pty_forward", "pty_adjoint",
            "pty_gradient", "pty_cg_solve", "pty_cg_reset", "pty_cg_state_size", "pty_cg_state_save",
            "pty_cg_state_load", "pty_stage_times", "pty_selftest_log1p", "pty_selftest_tc_wait_limit", "pty_gradient_noalloc",
            "pty_get_plan", "pty_selftest_ls_certified", "pty_selftest_cnn_tc",
            "pty_batch_create", "pty_batch_cg_solve", "pty_num_views",
            # learned initial guess (include/pty_cnn.h)
            "pty_default_adam", "pty_cnn_create", "pty_cnn_destroy", "pty_cnn_last_error", "pty_cnn_num_params",
            "pty_cnn_set_params", "pty_cnn_get_params", "pty_cnn_init_params", "pty_cnn_set_loss_weight",
            "pty_cnn_predict", "pty_cnn_loss_grad", "pty_cnn_train_step", "pty_cnn_train", "pty_stitch",
            "pty_learned_init"]


class PtyError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class pty_opts(ctypes.Structure):
    _fields_ = [("gamma0", ctypes.c_double), ("tau", ctypes.c_double), ("t", ctypes.c_double),
                ("max_halvings", ctypes.c_int32), ("eps", ctypes.c_double), ("ls_window", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tile_config", ctypes.c_int32), ("dft", ctypes.c_int32),
                ("estimator", ctypes.c_int32), ("solver", ctypes.c_int32), ("gd_step", ctypes.c_double),
                ("ls_warm", ctypes.c_int32)]


EST_ML, EST_LS = 0, 1  # pty_opts.estimator
SOLVER_CG, SOLVER_GD = 0, 1  # pty_opts.solver


class pty_adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class pty_init_report(ctypes.Structure):
    _fields_ = [("F_learned", ctypes.c_double), ("F_ones", ctypes.c_double), ("used_learned", ctypes.c_int32),
                ("scale", ctypes.c_double), ("ms", ctypes.c_double)]


class pty_cg_report(ctypes.Structure):
    _fields_ = [("F", ctypes.POINTER(ctypes.c_double)), ("gamma", ctypes.POINTER(ctypes.c_double)),
                ("halvings", ctypes.POINTER(ctypes.c_int32)), ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("iters_done", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load libpty (building it first if needed) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libpty not built ({path}); run paper_2106_07575_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    lib.pty_default_opts.argtypes = [ctypes.POINTER(pty_opts)]
    lib.pty_default_opts.restype = None
    lib.pty_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, vp, i32, vp, vp, ctypes.POINTER(pty_opts), vp]
    lib.pty_create_subpixel.argtypes = [ctypes.POINTER(vp), i32, i32, i32, vp, i32, vp, vp, ctypes.POINTER(pty_opts),
                                        vp]
    lib.pty_destroy.argtypes = [vp]
    lib.pty_destroy.restype = None
    lib.pty_last_error.argtypes = [vp]
    lib.pty_last_error.restype = ctypes.c_char_p
    lib.pty_forward.argtypes = [vp, vp, vp]
    lib.pty_adjoint.argtypes = [vp, vp, vp]
    lib.pty_gradient.argtypes = [vp, vp, vp, ctypes.POINTER(dbl)]
    lib.pty_cg_solve.argtypes = [vp, vp, i32, ctypes.POINTER(pty_cg_report)]
    lib.pty_cg_reset.argtypes = [vp]
    lib.pty_cg_state_size.argtypes = [vp]
    lib.pty_cg_state_size.restype = ctypes.c_size_t
    lib.pty_cg_state_save.argtypes = [vp, vp]
    lib.pty_cg_state_load.argtypes = [vp, vp]
    lib.pty_stage_times.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.pty_selftest_log1p.argtypes = [vp, vp, i32]
    lib.pty_selftest_tc_wait_limit.argtypes = [ctypes.c_int64]
    lib.pty_selftest_tc_wait_limit.restype = ctypes.c_int
    lib.pty_selftest_ls_certified.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int32)]
    lib.pty_selftest_cnn_tc.argtypes = [i32]
    lib.pty_selftest_cnn_tc.restype = ctypes.c_int
    lib.pty_gradient_noalloc.argtypes = [i32, i32, i32, vp, i32, vp, vp, dbl, vp, vp, vp, vp]
    lib.pty_get_plan.argtypes = [vp, ctypes.POINTER(i32)]
    lib.pty_batch_create.argtypes = [ctypes.POINTER(vp), i32, vp, vp, vp, i32, vp, vp, vp, ctypes.POINTER(pty_opts),
                                     vp]
    lib.pty_batch_cg_solve.argtypes = [vp, ctypes.POINTER(vp), i32, ctypes.POINTER(pty_cg_report)]
    lib.pty_num_views.argtypes = [vp]
    lib.pty_num_views.restype = i32
    u64, i64 = ctypes.c_uint64, ctypes.c_int64
    lib.pty_default_adam.argtypes = [ctypes.POINTER(pty_adam)]
    lib.pty_default_adam.restype = None
    lib.pty_cnn_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, vp]
    lib.pty_cnn_destroy.argtypes = [vp]
    lib.pty_cnn_destroy.restype = None
    lib.pty_cnn_last_error.argtypes = [vp]
    lib.pty_cnn_last_error.restype = ctypes.c_char_p
    lib.pty_cnn_num_params.argtypes = [vp]
    lib.pty_cnn_num_params.restype = i64
    lib.pty_cnn_set_params.argtypes = [vp, vp]
    lib.pty_cnn_get_params.argtypes = [vp, vp]
    lib.pty_cnn_init_params.argtypes = [vp, u64]
    lib.pty_cnn_set_loss_weight.argtypes = [vp, vp]
    lib.pty_cnn_predict.argtypes = [vp, i32, vp, vp]
    lib.pty_cnn_loss_grad.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(dbl), vp]
    lib.pty_cnn_train_step.argtypes = [vp, i32, vp, vp, vp, ctypes.POINTER(pty_adam), ctypes.POINTER(dbl)]
    lib.pty_cnn_train.argtypes = [vp, i64, vp, vp, i32, i32, u64, ctypes.POINTER(pty_adam), ctypes.POINTER(dbl)]
    lib.pty_stitch.argtypes = [vp, vp, ctypes.c_float, vp]
    lib.pty_learned_init.argtypes = [vp, vp, vp, vp, ctypes.POINTER(pty_init_report)]
    for f in ("pty_create", "pty_create_subpixel", "pty_forward", "pty_adjoint", "pty_gradient", "pty_cg_solve", "pty_cg_reset",
              "pty_cg_state_save", "pty_cg_state_load", "pty_stage_times", "pty_selftest_log1p",
              "pty_gradient_noalloc", "pty_get_plan", "pty_batch_create", "pty_batch_cg_solve", "pty_cnn_create",
              "pty_cnn_set_params", "pty_cnn_get_params", "pty_cnn_init_params", "pty_cnn_set_loss_weight",
              "pty_cnn_predict", "pty_cnn_loss_grad", "pty_cnn_train_step", "pty_cnn_train", "pty_stitch",
              "pty_learned_init"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, dtype_ok):
    """Raw pointer of a contiguous torch tensor or numpy array (no copy)."""
    if a is None:
        return None
    try:
        import torch

        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if str(a.dtype).replace("torch.", "") not in dtype_ok:
                raise TypeError(f"dtype {a.dtype} not in {dtype_ok}")
            return ctypes.c_void_p(a.data_ptr())
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if a.dtype.name not in dtype_ok:
            raise TypeError(f"dtype {a.dtype} not in {dtype_ok}")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported argument type {type(a)}")


_C = ("complex64",)
_F = ("float32",)
_I = ("int32",)


def _need(a, n, what):
    """The library reads or writes exactly n elements behind a's pointer: a must hold n."""
    m = int(a.numel()) if hasattr(a, "numel") else int(np.asarray(a).size)
    if m != n:
        raise ValueError(f"{what}: {m} elements, expected {n}")


def default_opts() -> pty_opts:
    o = pty_opts()
    load().pty_default_opts(ctypes.byref(o))
    return o


def _check(lib, ctx, st, allow=()):
    if st != PTY_OK and st not in allow:
        msg = lib.pty_last_error(ctx)
        raise PtyError(st, msg.decode() if msg else "")
    return st


def pty_create(H, W, P, probe, K, pos, data, opts: pty_opts | None = None, stream=None):
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.pty_create(ctypes.byref(ctx), H, W, P, _ptr(probe, _C), K, _ptr(pos, _I), _ptr(data, _F),
                        ctypes.byref(opts) if opts is not None else None,
                        ctypes.c_void_p(stream) if stream else None)
    _check(lib, None, st)
    return ctx


def pty_create_subpixel(H, W, P, probe, K, pos, data, opts: pty_opts | None = None, stream=None):
    """As pty_create with float32 positions [K][2] that may have a fractional part."""
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.pty_create_subpixel(ctypes.byref(ctx), H, W, P, _ptr(probe, _C), K, _ptr(pos, _F), _ptr(data, _F),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.c_void_p(stream) if stream else None)
    _check(lib, None, st)
    return ctx


def pty_destroy(ctx):
    load().pty_destroy(ctx)


def pty_forward(ctx, psi, out):
    lib = load()
    return _check(lib, ctx, lib.pty_forward(ctx, _ptr(psi, _C), _ptr(out, _C)))


def pty_adjoint(ctx, y, x):
    lib = load()
    return _check(lib, ctx, lib.pty_adjoint(ctx, _ptr(y, _C), _ptr(x, _C)))


def pty_gradient(ctx, psi, grad):
    lib = load()
    F = ctypes.c_double(0.0)
    _check(lib, ctx, lib.pty_gradient(ctx, _ptr(psi, _C), _ptr(grad, _C), ctypes.byref(F)))
    return F.value


def pty_cg_solve(ctx, psi, niter, report=True):
    """Run niter iterations in place; returns (status, dict) with F, gamma, halvings, alpha, iters_done."""
    lib = load()
    rep = None
    arrays = {}
    if report:
        arrays = {"F": np.full(niter + 1, np.nan), "gamma": np.full(max(niter, 1), np.nan),
                  "halvings": np.zeros(max(niter, 1), np.int32), "alpha": np.full(max(niter, 1), np.nan)}
        rep = pty_cg_report(arrays["F"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            arrays["gamma"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            arrays["halvings"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            arrays["alpha"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    st = lib.pty_cg_solve(ctx, _ptr(psi, _C), niter, ctypes.byref(rep) if rep is not None else None)
    _check(lib, ctx, st, allow=(PTY_STALLED,))
    out = {}
    if report:
        n = rep.iters_done
        k = min(niter, n + (st == PTY_STALLED))
        out = {"F": arrays["F"][: n + 1], "gamma": arrays["gamma"][:k], "halvings": arrays["halvings"][:k],
               "alpha": arrays["alpha"][:k], "iters_done": n}
    return st, out


def pty_cg_reset(ctx):
    lib = load()
    return _check(lib, ctx, lib.pty_cg_reset(ctx))


def pty_cg_state_save(ctx) -> bytes:
    lib = load()
    n = lib.pty_cg_state_size(ctx)
    buf = ctypes.create_string_buffer(n)
    _check(lib, ctx, lib.pty_cg_state_save(ctx, buf))
    return buf.raw


def pty_cg_state_load(ctx, blob: bytes):
    lib = load()
    buf = ctypes.create_string_buffer(blob, len(blob))
    return _check(lib, ctx, lib.pty_cg_state_load(ctx, buf))


def pty_stage_times(ctx, reset=False):
    lib = load()
    ms = (ctypes.c_double * 5)()
    n = (ctypes.c_int64 * 5)()
    _check(lib, ctx, lib.pty_stage_times(ctx, ms, n, int(bool(reset))))
    return list(ms), list(n)


def pty_selftest_tc_wait_limit(polls):
    return load().pty_selftest_tc_wait_limit(int(polls))


def pty_selftest_cnn_tc(enable):
    """Switch the tensor-core form of the CNN's hidden convolutions on or off; returns the
    previous setting."""
    return int(load().pty_selftest_cnn_tc(1 if enable else 0))


def pty_selftest_ls_certified(ctx, view=0):
    """Leading line-search trials the certificate rejected in the last iteration of view."""
    lib = load()
    out = ctypes.c_int32(0)
    _check(lib, ctx, lib.pty_selftest_ls_certified(ctx, int(view), ctypes.byref(out)))
    return int(out.value)


def pty_selftest_log1p(t, out):
    lib = load()
    return _check(lib, None, lib.pty_selftest_log1p(_ptr(t, _F), _ptr(out, _F), int(t.numel() if hasattr(t, "numel") else t.size)))


def pty_gradient_noalloc(H, W, P, probe, K, pos, data, eps, psi, grad, F=None, stream=None):
    """Objective and gradient without a context or any allocation; every array on the device.

    Returns the raw status (PTY_OK, PTY_ERR_ARG, PTY_ERR_BOUNDS, PTY_ERR_CUDA).
    """
    lib = load()
    return lib.pty_gradient_noalloc(H, W, P, _ptr(probe, _C), K, _ptr(pos, _I), _ptr(data, _F), float(eps),
                                    _ptr(psi, _C), _ptr(grad, _C), _ptr(F, ("float64",)),
                                    ctypes.c_void_p(stream) if stream else None)


def _reports(niter, n):
    arrays, reps = [], (pty_cg_report * n)()
    for v in range(n):
        a = {"F": np.full(niter + 1, np.nan), "gamma": np.full(max(niter, 1), np.nan),
             "halvings": np.zeros(max(niter, 1), np.int32), "alpha": np.full(max(niter, 1), np.nan)}
        arrays.append(a)
        reps[v] = pty_cg_report(a["F"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                a["gamma"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                a["halvings"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                a["alpha"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0)
    return arrays, reps


def pty_batch_create(Hs, Ws, Ks, P, probe, pos, data, opts: pty_opts | None = None, stream=None):
    lib = load()
    n = len(Hs)
    h = np.ascontiguousarray(Hs, np.int32)
    w = np.ascontiguousarray(Ws, np.int32)
    k = np.ascontiguousarray(Ks, np.int32)
    ctx = ctypes.c_void_p()
    st = lib.pty_batch_create(ctypes.byref(ctx), n, _ptr(h, _I), _ptr(w, _I), _ptr(k, _I), P, _ptr(probe, _C),
                              _ptr(pos, _I), _ptr(data, _F), ctypes.byref(opts) if opts is not None else None,
                              ctypes.c_void_p(stream) if stream else None)
    _check(lib, None, st)
    return ctx


def pty_batch_cg_solve(ctx, psis, niter):
    """psis: list of per-view objects (torch or numpy complex64), updated in place."""
    lib = load()
    n = len(psis)
    ptrs = (ctypes.c_void_p * n)(*[_ptr(p, _C).value for p in psis])
    arrays, reps = _reports(niter, n)
    st = lib.pty_batch_cg_solve(ctx, ptrs, niter, reps)
    _check(lib, ctx, st, allow=(PTY_STALLED,))
    out = []
    for v in range(n):
        d = reps[v].iters_done
        a = arrays[v]
        stalled = st == PTY_STALLED and d < niter and a["halvings"][d] > 0
        k = min(niter, d + (1 if stalled else 0))
        out.append({"F": a["F"][: d + 1], "gamma": a["gamma"][:k], "halvings": a["halvings"][:k],
                    "alpha": a["alpha"][:k], "iters_done": d})
    return st, out


class BatchContext:
    """Owning wrapper of a batch of views reconstructed together."""

    def __init__(self, probe, views, opts: pty_opts | None = None, stream=None):
        """views: list of (H, W, pos [K][2] int32, data [K][P][P] float32) on one device or the host."""
        import torch

        self.P = P = probe.shape[0]
        _need(probe, P * P, "probe")
        Hs = [v[0] for v in views]
        Ws = [v[1] for v in views]
        Ks = [v[2].shape[0] for v in views]
        for i, (_, _, q, d) in enumerate(views):
            _need(q, 2 * q.shape[0], f"view {i} pos")
            _need(d, q.shape[0] * P * P, f"view {i} data")
        self.shapes = list(zip(Hs, Ws))
        pos = torch.cat([torch.as_tensor(v[2]) for v in views]).contiguous()
        data = torch.cat([torch.as_tensor(v[3]) for v in views]).contiguous()
        if data.is_cuda is False and probe.is_cuda:
            pos, data = pos.cuda(), data.cuda()
        self._keep = (probe, pos, data)
        self.ctx = pty_batch_create(Hs, Ws, Ks, self.P, probe, pos, data, opts, stream)

    def close(self):
        if self.ctx:
            pty_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cg_solve(self, psis, niter):
        if len(psis) != len(self.shapes):
            raise ValueError(f"{len(psis)} objects for {len(self.shapes)} views")
        for i, (x, (H, W)) in enumerate(zip(psis, self.shapes)):
            _need(x, H * W, f"view {i} psi")
        return pty_batch_cg_solve(self.ctx, psis, niter)

    def plan(self):
        lib = load()
        out = (ctypes.c_int32 * 4)()
        _check(lib, self.ctx, lib.pty_get_plan(self.ctx, out))
        return {"grad": (out[0], out[1]), "ls": (out[2], out[3])}


@dataclass
class Problem:
    H: int
    W: int
    P: int
    K: int


def _is_float32(a):
    return str(getattr(a, "dtype", "")).replace("torch.", "") == "float32"


class Context:
    """Owning wrapper: one libpty context per reconstruction problem.  Integer positions
    (int32) go to pty_create; float32 positions, which may be fractional, to
    pty_create_subpixel."""

    def __init__(self, probe, pos, data, H, W, opts: pty_opts | None = None, stream=None):
        P = probe.shape[0]
        K = pos.shape[0]
        _need(probe, P * P, "probe")
        _need(pos, 2 * K, "pos")
        _need(data, K * P * P, "data")
        self.shape = (H, W)
        self.P, self.K = P, K
        self._keep = (probe, pos, data)  # borrowed device data must outlive the context
        create = pty_create_subpixel if _is_float32(pos) else pty_create
        self.ctx = create(H, W, P, probe, K, pos, data, opts, stream)

    def close(self):
        if self.ctx:
            pty_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _object(self, a, what):
        _need(a, self.shape[0] * self.shape[1], what)

    def _patterns(self, a, what):
        _need(a, self.K * self.P * self.P, what)

    def forward(self, psi, out):
        self._object(psi, "psi")
        self._patterns(out, "out")
        return pty_forward(self.ctx, psi, out)

    def adjoint(self, y, x):
        self._patterns(y, "y")
        self._object(x, "x")
        return pty_adjoint(self.ctx, y, x)

    def gradient(self, psi, grad):
        self._object(psi, "psi")
        self._object(grad, "grad")
        return pty_gradient(self.ctx, psi, grad)

    def cg_solve(self, psi, niter, report=True):
        self._object(psi, "psi")
        return pty_cg_solve(self.ctx, psi, niter, report)

    def cg_reset(self):
        return pty_cg_reset(self.ctx)

    def state_save(self):
        return pty_cg_state_save(self.ctx)

    def state_load(self, blob):
        return pty_cg_state_load(self.ctx, blob)

    def stage_times(self, reset=False):
        return pty_stage_times(self.ctx, reset)

    def plan(self):
        """(rows, threads) per CTA of the GRAD pass and of the LS pass."""
        lib = load()
        out = (ctypes.c_int32 * 4)()
        _check(lib, self.ctx, lib.pty_get_plan(self.ctx, out))
        return {"grad": (out[0], out[1]), "ls": (out[2], out[3])}


# ---- learned initial guess (include/pty_cnn.h) ----

def default_adam() -> pty_adam:
    a = pty_adam()
    load().pty_default_adam(ctypes.byref(a))
    return a


def _check_cnn(lib, net, st):
    if st != PTY_OK:
        msg = lib.pty_cnn_last_error(net)
        raise PtyError(st, msg.decode() if msg else "")
    return st


def pty_stitch(ctx, patches, floor, psi0):
    lib = load()
    return _check(lib, ctx, lib.pty_stitch(ctx, _ptr(patches, _C), float(floor), _ptr(psi0, _C)))


class Network:
    """Owning wrapper of a pty_cnn network (the learned initial guess)."""

    def __init__(self, P, channels=32, layers=6, max_batch=64, stream=None):
        lib = load()
        net = ctypes.c_void_p()
        _check_cnn(lib, None, lib.pty_cnn_create(ctypes.byref(net), P, channels, layers, max_batch,
                                                 ctypes.c_void_p(stream) if stream else None))
        self.net, self.P, self.channels, self.layers, self.max_batch = net, P, channels, layers, max_batch

    def close(self):
        if self.net:
            load().pty_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        lib = load()
        return _check_cnn(lib, self.net, getattr(lib, name)(self.net, *args))

    @property
    def num_params(self) -> int:
        return int(load().pty_cnn_num_params(self.net))

    def set_params(self, params):
        return self._call("pty_cnn_set_params", _ptr(params, _F))

    def get_params(self, out=None):
        out = np.empty(self.num_params, np.float32) if out is None else out
        self._call("pty_cnn_get_params", _ptr(out, _F))
        return out

    def init_params(self, seed):
        return self._call("pty_cnn_init_params", ctypes.c_uint64(seed))

    def set_loss_weight(self, w):
        return self._call("pty_cnn_set_loss_weight", _ptr(w, _F))

    def predict(self, d, o):
        return self._call("pty_cnn_predict", int(d.shape[0]), _ptr(d, _F), _ptr(o, _C))

    def loss_grad(self, d, t, idx=None, grad=None, B=None):
        B = int(idx.shape[0] if idx is not None else d.shape[0]) if B is None else B
        loss = ctypes.c_double(0.0)
        self._call("pty_cnn_loss_grad", B, _ptr(idx, _I), _ptr(d, _F), _ptr(t, _C), ctypes.byref(loss),
                   _ptr(grad, _F))
        return loss.value

    def train_step(self, d, t, idx=None, adam: pty_adam | None = None, B=None):
        B = int(idx.shape[0] if idx is not None else d.shape[0]) if B is None else B
        loss = ctypes.c_double(0.0)
        self._call("pty_cnn_train_step", B, _ptr(idx, _I), _ptr(d, _F), _ptr(t, _C),
                   ctypes.byref(adam) if adam is not None else None, ctypes.byref(loss))
        return loss.value

    def train(self, d, t, batch, steps, seed=0, adam: pty_adam | None = None):
        losses = np.zeros(max(steps, 1), np.float64)
        self._call("pty_cnn_train", int(d.shape[0]), _ptr(d, _F), _ptr(t, _C), batch, steps, ctypes.c_uint64(seed),
                   ctypes.byref(adam) if adam is not None else None,
                   losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return losses[:steps]

    def learned_init(self, ctx, d, psi0):
        """Write the learned start (or the ones start, whichever has the lower objective) to psi0."""
        lib = load()
        rep = pty_init_report()
        c = ctx.ctx if isinstance(ctx, Context) else ctx
        _check_cnn(lib, self.net, lib.pty_learned_init(c, self.net, _ptr(d, _F), _ptr(psi0, _C), ctypes.byref(rep)))
        return {"F_learned": rep.F_learned, "F_ones": rep.F_ones, "used_learned": bool(rep.used_learned),
                "scale": rep.scale, "ms": rep.ms}
