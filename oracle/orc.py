"""ctypes wrapper of the FP64 oracle (``orc.c``).  TEST INFRASTRUCTURE ONLY.

Every function takes numpy arrays: complex arrays are converted to complex128 (exact
for complex64 inputs), measured intensities stay float32 as the method receives them.
The oracle is a plain CPU restatement of the paper's Eq. 1-3, 5-7 and Algorithm 1; see
the header of ``orc.c`` for the readings it takes where the paper is silent.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass

import numpy as np

ORC_OK, ORC_ERR_ARG, ORC_ERR_BOUNDS, ORC_ERR_NOMEM, ORC_STALLED = 0, 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_lib = None


class _Opts(ctypes.Structure):
    _fields_ = [
        ("gamma0", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("t", ctypes.c_double),
        ("max_halvings", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("est", ctypes.c_int),
        ("solver", ctypes.c_int),
        ("gd_step", ctypes.c_double),
        ("warm", ctypes.c_int),
    ]


EST_ML, EST_LS = 0, 1  # Poisson maximum likelihood (Eq. 2); Gaussian least squares on amplitudes
SOLVER_CG, SOLVER_GD = 0, 1  # Eq. 5-7 with Algorithm 1; Eq. 4 with a constant step


@dataclass
class OrcOpts:
    """Line-search and objective options; defaults follow Algorithm 1 (gamma0=1, tau=0.5, t=0).

    est: EST_ML or EST_LS; solver: SOLVER_CG or SOLVER_GD (step gd_step); warm: start each
    line search after the first at min(gamma0, gamma_prev / tau)."""

    gamma0: float = 1.0
    tau: float = 0.5
    t: float = 0.0
    max_halvings: int = 60
    eps: float = 0.1
    est: int = EST_ML
    solver: int = SOLVER_CG
    gd_step: float = 0.0
    warm: bool = False


def build(force: bool = False) -> str:
    """Compile orc.c into _lib/liborc-<hash>.so with gcc (-O2, OpenMP); return its path.

    Earlier builds (another source hash) are deleted, so _lib/ holds one library."""
    src = open(_SRC, "rb").read()
    tag = hashlib.sha1(src).hexdigest()[:12]
    os.makedirs(_LIBDIR, exist_ok=True)
    out = os.path.join(_LIBDIR, f"liborc-{tag}.so")
    if force or not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        try:
            subprocess.run(cmd, check=True)
            os.replace(tmp, out)
        finally:
            if os.path.exists(tmp):
                os.remove(tmp)
    for name in os.listdir(_LIBDIR):
        path = os.path.join(_LIBDIR, name)
        if name.startswith("liborc-") and name.endswith(".so") and path != out:
            try:
                os.remove(path)
            except OSError:
                pass
    return out


def _get():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i = ctypes.c_int
        d = ctypes.c_double
        lib.orc_fft2.argtypes = [P, i, i]
        lib.orc_shift_probe.argtypes = [i, P, d, d, P]
        lib.orc_Q.argtypes = [i, i, i, P, i, i, P, P, P]
        lib.orc_QH.argtypes = [i, i, i, P, i, i, P, P, P]
        lib.orc_forward.argtypes = [i, i, i, P, i, i, P, P, P, i]
        lib.orc_adjoint.argtypes = [i, i, i, P, i, i, P, P, P, i]
        lib.orc_objective.argtypes = [i, i, i, P, i, i, P, P, d, i, P, P, i]
        lib.orc_gradient.argtypes = [i, i, i, P, i, i, P, P, d, i, P, P, P, i]
        lib.orc_cg_solve.argtypes = [i, i, i, P, i, i, P, P, ctypes.POINTER(_Opts), P, i, P, P, P, P, P, P, i]
        for f in ("orc_fft2", "orc_shift_probe", "orc_Q", "orc_QH", "orc_forward", "orc_adjoint", "orc_objective",
                  "orc_gradient", "orc_cg_solve"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _pos(pos):
    return np.ascontiguousarray(pos, dtype=np.int32).reshape(-1, 2)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _probe(probe, K):
    """(complex128 probe, P, per_pos): one [P][P] probe for every position, or [K][P][P]."""
    probe = _c128(probe)
    if probe.ndim == 3:
        if probe.shape[0] != K or probe.shape[1] != probe.shape[2]:
            raise ValueError(f"per-position probes must be [K={K}][P][P], got {probe.shape}")
        return probe, probe.shape[1], 1
    if probe.ndim != 2 or probe.shape[0] != probe.shape[1]:
        raise ValueError(f"probe must be [P][P] or [K][P][P], got {probe.shape}")
    return probe, probe.shape[0], 0


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st, what):
    if st != ORC_OK:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def fft2(x, inverse=False):
    """Unitary 2-D DFT of a P x P array (Eq. 1's F, or F^H when inverse)."""
    x = _c128(x).copy()
    _check(_get().orc_fft2(_ptr(x), x.shape[0], int(bool(inverse))), "fft2")
    return x


def shift_probe(probe, dy, dx):
    """The probe shifted by (dy, dx) pixels by the Fourier shift theorem (sub-pixel positions);
    see orc_shift_probe in orc.c for the definition, including the Nyquist bins."""
    probe = _c128(probe)
    out = np.empty_like(probe)
    _check(_get().orc_shift_probe(probe.shape[0], _ptr(probe), float(dy), float(dx), _ptr(out)), "shift_probe")
    return out


def subpixel_probes(probe, pos):
    """(integer positions [K][2], per-position probes [K][P][P]) for fractional positions
    (row, col): the window starts at floor(pos), the probe is shifted by pos - floor(pos)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 2)
    base = np.floor(pos)
    frac = pos - base
    probes = np.stack([shift_probe(probe, fy, fx) if (fy or fx) else _c128(probe).copy() for fy, fx in frac])
    return base.astype(np.int32), probes


def Q(psi, probe, pos):
    """Q psi: probe times the P x P patch at every scan position -> [K][P][P].  probe is
    [P][P] (shared) or [K][P][P] (one per position), as for every function below."""
    psi, pos = _c128(psi), _pos(pos)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = psi.shape
    out = np.empty((pos.shape[0], P, P), np.complex128)
    _check(_get().orc_Q(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(psi), _ptr(out)), "Q")
    return out


def QH(y, probe, pos, shape):
    """Q^H y: conj(probe) times each patch, scatter-added into an H x W object."""
    y, pos = _c128(y), _pos(pos)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = shape
    out = np.empty((H, W), np.complex128)
    _check(_get().orc_QH(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(y), _ptr(out)), "QH")
    return out


def forward(psi, probe, pos, nthreads=1):
    """G psi = F Q psi (Eq. 1), unitary F -> [K][P][P] complex128."""
    psi, pos = _c128(psi), _pos(pos)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = psi.shape
    out = np.empty((pos.shape[0], P, P), np.complex128)
    st = _get().orc_forward(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(psi), _ptr(out), nthreads)
    _check(st, "forward")
    return out


def adjoint(y, probe, pos, shape, nthreads=1):
    """G^H y = Q^H F^H y (the operator of Eq. 3) -> [H][W] complex128."""
    y, pos = _c128(y), _pos(pos)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = shape
    out = np.empty((H, W), np.complex128)
    st = _get().orc_adjoint(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(y), _ptr(out), nthreads)
    _check(st, "adjoint")
    return out


def objective(psi, probe, pos, d, eps=0.1, nthreads=1, est=EST_ML):
    """F_eps(psi) = sum |G psi|^2 - d log(|G psi|^2 + eps) (Eq. 2 with the eps guard), or with
    est=EST_LS the amplitude least squares sum |G psi|^2 - 2 sqrt(d) sqrt(|G psi|^2 + eps) + d."""
    psi, pos, d = _c128(psi), _pos(pos), _f32(d)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = psi.shape
    F = ctypes.c_double(0.0)
    st = _get().orc_objective(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(d), eps, est, _ptr(psi),
                              ctypes.byref(F), nthreads)
    _check(st, "objective")
    return F.value


def gradient(psi, probe, pos, d, eps=0.1, nthreads=1, est=EST_ML):
    """(g, F): g = G^H(G psi - d G psi / (|G psi|^2 + eps)) (Eq. 3), F as in objective(); with
    est=EST_LS g = G^H(G psi - sqrt(d) G psi / sqrt(|G psi|^2 + eps))."""
    psi, pos, d = _c128(psi), _pos(pos), _f32(d)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = psi.shape
    g = np.empty((H, W), np.complex128)
    F = ctypes.c_double(0.0)
    st = _get().orc_gradient(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(d), eps, est, _ptr(psi),
                             _ptr(g), ctypes.byref(F), nthreads)
    _check(st, "gradient")
    return g, F.value


def cg_solve(psi0, probe, pos, d, niter, opts: OrcOpts | None = None, nthreads=1):
    """Run niter ML-CG iterations (Eq. 5-7, Algorithm 1 on one device), or Eq. 4's gradient
    descent with opts.solver = SOLVER_GD.

    Returns a dict with psi, F (F_hist[0..iters_done]), gamma, halvings, alpha,
    iters_done, status (ORC_OK or ORC_STALLED) and t (wall seconds from the start of the
    solve to the end of each iteration, for timing only).
    """
    opts = opts or OrcOpts()
    psi = _c128(psi0).copy()
    pos, d = _pos(pos), _f32(d)
    probe, P, pp = _probe(probe, pos.shape[0])
    H, W = psi.shape
    o = _Opts(opts.gamma0, opts.tau, opts.t, opts.max_halvings, opts.eps, int(opts.est), int(opts.solver),
              float(opts.gd_step), int(bool(opts.warm)))
    F = np.full(niter + 1, np.nan)
    gam = np.full(max(niter, 1), np.nan)
    halv = np.zeros(max(niter, 1), np.int32)
    alpha = np.full(max(niter, 1), np.nan)
    tim = np.full(max(niter, 1), np.nan)
    done = ctypes.c_int(0)
    st = _get().orc_cg_solve(H, W, P, _ptr(probe), pp, pos.shape[0], _ptr(pos), _ptr(d), ctypes.byref(o),
                             _ptr(psi), niter, _ptr(F), _ptr(gam), _ptr(halv), _ptr(alpha),
                             ctypes.byref(done), _ptr(tim), nthreads)
    if st not in (ORC_OK, ORC_STALLED):
        _check(st, "cg_solve")
    n = done.value
    return {
        "psi": psi,
        "F": F[: n + 1],
        "gamma": gam[:n],
        "halvings": halv[: min(niter, n + (st == ORC_STALLED))],
        "alpha": alpha[: min(niter, n + (st == ORC_STALLED))],
        "iters_done": n,
        "status": st,
        "t": tim[:n],
    }
