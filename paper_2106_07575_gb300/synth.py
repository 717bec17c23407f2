"""Seeded synthetic inputs for ML-CG ptychography: phantom, probe, scan, detector counts.

This module only MAKES inputs; it holds none of the reconstruction's arithmetic (no
objective, gradient, line search or CG).  Both the FP64 oracle and the CUDA library
receive the arrays it returns and neither calls anything else here.

The workloads stand in for the paper's synthetic siemens-star / coins sets, which are
not available: random-ellipse phantoms (amplitude 0.8-1.0, phase 0-pi/2), a Gaussian
probe with quadratic phase, jittered raster or Fermat-spiral scans, and Poisson counts.
The detector model (``simulate_counts``) is the far-field measurement itself: the
squared modulus of numpy's orthonormal 2-D FFT of probe x object patch, scaled so the
brightest pixel over all patterns holds ``peak`` expected counts, then Poisson-sampled.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ----------------------------------------------------------------------------------
# Object, probe and scan
# ----------------------------------------------------------------------------------
def ellipse_phantom(H: int, W: int, rng: np.random.Generator, n_ellipses: int = 20) -> np.ndarray:
    """Complex transmission: background 1; ellipses with amplitude U[0.8,1], phase U[0,pi/2].

    Each ellipse has a uniform centre in the object, semi-axes U[N/32, N/6] (N = min(H, W)),
    rotation U[0, pi); later ellipses overwrite earlier ones (pixel-centre membership).
    """
    N = min(H, W)
    amp = np.ones((H, W), np.float64)
    ph = np.zeros((H, W), np.float64)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        a, b = rng.uniform(N / 32, N / 6), rng.uniform(N / 32, N / 6)
        th = rng.uniform(0, math.pi)
        A, Ph = rng.uniform(0.8, 1.0), rng.uniform(0, math.pi / 2)
        dy, dx = yy - cy, xx - cx
        u = dx * math.cos(th) + dy * math.sin(th)
        v = -dx * math.sin(th) + dy * math.cos(th)
        m = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        amp[m] = A
        ph[m] = Ph
    return (amp * np.exp(1j * ph)).astype(np.complex64)


def voronoi_phantom(H: int, W: int, rng: np.random.Generator, n_cells: int | None = None) -> np.ndarray:
    """Complex transmission made of Voronoi cells, each with amplitude U[0.8,1], phase U[0,pi/2]."""
    if n_cells is None:
        n_cells = int(rng.integers(50, 301))
    sy, sx = rng.uniform(0, H, n_cells), rng.uniform(0, W, n_cells)
    A, Ph = rng.uniform(0.8, 1.0, n_cells), rng.uniform(0, math.pi / 2, n_cells)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float32)
    best = np.full((H, W), np.inf, np.float32)
    lab = np.zeros((H, W), np.int64)
    for i in range(n_cells):
        dist = (yy - sy[i]) ** 2 + (xx - sx[i]) ** 2
        m = dist < best
        best[m] = dist[m]
        lab[m] = i
    return (A[lab] * np.exp(1j * Ph[lab])).astype(np.complex64)


def gaussian_probe(P: int, sigma: float | None = None, kappa: float = 2.0) -> np.ndarray:
    """P x P probe: amplitude exp(-r^2 / (2 sigma^2)), phase kappa r^2 / sigma^2, centre (P-1)/2.

    sigma defaults to 3P/16 (12 px at P=64, the value the workload names).
    """
    if sigma is None:
        sigma = 3.0 * P / 16.0
    c = (P - 1) / 2.0
    yy, xx = np.mgrid[0:P, 0:P].astype(np.float64)
    r2 = (yy - c) ** 2 + (xx - c) ** 2
    return (np.exp(-r2 / (2 * sigma**2)) * np.exp(1j * kappa * r2 / sigma**2)).astype(np.complex64)


def raster_positions(H: int, W: int, P: int, n: int, step: int, jitter: int,
                     rng: np.random.Generator) -> np.ndarray:
    """n x n raster of top-left corners (row, col), centred, +-jitter uniform integer per axis."""
    ext = (n - 1) * step + P
    oy, ox = (H - ext) // 2, (W - ext) // 2
    gy, gx = np.meshgrid(np.arange(n) * step + oy, np.arange(n) * step + ox, indexing="ij")
    pos = np.stack([gy.ravel(), gx.ravel()], axis=1).astype(np.int64)
    if jitter:
        pos += rng.integers(-jitter, jitter + 1, size=pos.shape)
    pos[:, 0] = np.clip(pos[:, 0], 0, H - P)
    pos[:, 1] = np.clip(pos[:, 1], 0, W - P)
    return pos.astype(np.int32)


def raster_positions_subpixel(H: int, W: int, P: int, n: int, step: int, jitter: float,
                              rng: np.random.Generator) -> np.ndarray:
    """n x n raster of top-left corners (row, col) as float32, centred, with a uniform real
    jitter in [-jitter, jitter] per axis (fractional positions), clipped to [0, H-P] x [0, W-P]."""
    ext = (n - 1) * step + P
    oy, ox = (H - ext) // 2, (W - ext) // 2
    gy, gx = np.meshgrid(np.arange(n) * step + oy, np.arange(n) * step + ox, indexing="ij")
    pos = np.stack([gy.ravel(), gx.ravel()], axis=1).astype(np.float64)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    pos[:, 0] = np.clip(pos[:, 0], 0, H - P)
    pos[:, 1] = np.clip(pos[:, 1], 0, W - P)
    return pos.astype(np.float32)


def spiral_positions(H: int, W: int, P: int, K: int, c: float, jitter: int,
                     rng: np.random.Generator) -> np.ndarray:
    """Vogel (Fermat) spiral r_n = c sqrt(n), theta_n = n * 137.508 deg, rounded, +-jitter."""
    n = np.arange(K, dtype=np.float64)
    r = c * np.sqrt(n)
    th = np.deg2rad(137.508) * n
    cy, cx = (H - P) / 2.0, (W - P) / 2.0
    y = np.floor(cy + r * np.sin(th) + 0.5).astype(np.int64)
    x = np.floor(cx + r * np.cos(th) + 0.5).astype(np.int64)
    pos = np.stack([y, x], axis=1)
    if jitter:
        pos += rng.integers(-jitter, jitter + 1, size=pos.shape)
    pos[:, 0] = np.clip(pos[:, 0], 0, H - P)
    pos[:, 1] = np.clip(pos[:, 1], 0, W - P)
    return pos.astype(np.int32)


# ----------------------------------------------------------------------------------
# Detector
# ----------------------------------------------------------------------------------
def shifted_probes(probe: np.ndarray, frac: np.ndarray) -> np.ndarray:
    """[K][P][P] complex128: the probe moved by frac[k] = (dy, dx) pixels by the Fourier shift
    theorem (numpy FFT): spectrum times exp(-2 pi i (ky dy + kx dx) / P) at the signed
    frequencies, cos(pi d) at the Nyquist index P/2 of each axis."""
    P = probe.shape[0]
    kap = np.fft.fftfreq(P, 1.0 / P)  # 0, 1, .., P/2-1, -P/2, .., -1
    nyq = P // 2
    spec = np.fft.fft2(probe.astype(np.complex128))
    out = np.empty((len(frac), P, P), np.complex128)
    for k, (dy, dx) in enumerate(np.asarray(frac, dtype=np.float64)):
        fy = np.exp(-2j * np.pi * kap * dy / P)
        fx = np.exp(-2j * np.pi * kap * dx / P)
        fy[nyq] = np.cos(np.pi * dy)
        fx[nyq] = np.cos(np.pi * dx)
        out[k] = np.fft.ifft2(spec * fy[:, None] * fx[None, :])
    return out


def _farfield_intensity(psi: np.ndarray, probe: np.ndarray, pos: np.ndarray, batch: int = 256):
    """|orthonormal FFT2(probe * patch_k)|^2 for all k, float64, in batches.  probe is [P][P]
    or one probe per position [K][P][P]."""
    P = probe.shape[-1]
    K = pos.shape[0]
    out = np.empty((K, P, P), np.float64)
    pr = probe.astype(np.complex128)
    iy = np.arange(P)
    for k0 in range(0, K, batch):
        k1 = min(K, k0 + batch)
        rows = pos[k0:k1, 0][:, None, None] + iy[None, :, None]
        cols = pos[k0:k1, 1][:, None, None] + iy[None, None, :]
        patches = psi[rows, cols].astype(np.complex128)
        pk = pr[k0:k1] if pr.ndim == 3 else pr[None]
        f = np.fft.fft2(pk * patches, norm="ortho")
        out[k0:k1] = f.real**2 + f.imag**2
    return out


def simulate_counts(psi_true: np.ndarray, probe_unit: np.ndarray, pos: np.ndarray, peak: float,
                    rng: np.random.Generator | None, noise: bool = True):
    """Return (probe, d): the probe scaled to counts and the measured intensities [K][P][P] f32.

    scale s = peak / max_k,j |FFT(probe_unit * patch_k)|^2; probe = sqrt(s) * probe_unit;
    d = Poisson(s |FFT(probe_unit * patch_k)|^2) (or its mean when noise is False).
    """
    I0 = _farfield_intensity(psi_true, probe_unit, pos)
    s = peak / I0.max()
    probe = (np.sqrt(s) * probe_unit.astype(np.complex128)).astype(np.complex64)
    lam = I0 * s
    if noise:
        d = rng.poisson(lam).astype(np.float32)
    else:
        d = lam.astype(np.float32)
    return probe, d


# ----------------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    psi_true: np.ndarray  # [H][W] complex64
    probe: np.ndarray  # [P][P] complex64, scaled to counts
    pos: np.ndarray  # [K][2] int32 (row, col)
    d: np.ndarray  # [K][P][P] float32
    niter: int
    meta: dict = field(default_factory=dict)

    @property
    def H(self):
        return self.psi_true.shape[0]

    @property
    def W(self):
        return self.psi_true.shape[1]

    @property
    def P(self):
        return self.probe.shape[0]

    @property
    def K(self):
        return self.pos.shape[0]

    def psi0(self):
        """Uniform-ones start."""
        return np.ones((self.H, self.W), np.complex64)


def small_problem(H=256, W=256, P=64, n=15, step=8, jitter=1, peak=1e4, seed=0, noise=True,
                  niter=10, name="ml-cg 256x256 object, 64x64 probe, 225 positions"):
    """Raster workload; defaults: 256^2 ellipse phantom, 64^2 probe, 15x15 raster, peak 1e4."""
    rng = np.random.default_rng(seed)
    psi = ellipse_phantom(H, W, rng)
    pos = raster_positions(H, W, P, n, step, jitter, rng)
    probe, d = simulate_counts(psi, gaussian_probe(P), pos, peak, rng, noise)
    return Problem(name, psi, probe, pos, d, niter, {"seed": seed, "peak": peak, "step": step,
                                                      "jitter": jitter})


def production_problem(seed=1, noise=True):
    """1024^2 ellipse phantom, 128^2 probe, 60x60 raster (step 14, +-2), peak 1e5, 64 iterations."""
    return small_problem(H=1024, W=1024, P=128, n=60, step=14, jitter=2, peak=1e5, seed=seed,
                         noise=noise, niter=64,
                         name="ml-cg 1024x1024 object, 128x128 probe, 3600 positions")


def subpixel_problem(H=256, W=256, P=64, n=15, step=8, jitter=1.0, peak=1e4, seed=0, noise=True,
                     niter=10, name=None):
    """Raster with fractional positions (uniform real jitter +-jitter): Problem.pos is float32
    [K][2] (row, col); the data come from the probe shifted by each position's fraction
    within the window that starts at floor(pos).  meta["pos_int"] and meta["frac"] hold the
    split.  Defaults: the 256^2 / 64^2 / 15x15 workload."""
    rng = np.random.default_rng(seed)
    psi = ellipse_phantom(H, W, rng)
    pos = raster_positions_subpixel(H, W, P, n, step, jitter, rng)
    base = np.floor(pos.astype(np.float64))
    frac = pos.astype(np.float64) - base
    unit = gaussian_probe(P)
    I0 = _farfield_intensity(psi, shifted_probes(unit, frac), base.astype(np.int64))
    s = peak / I0.max()
    probe = (np.sqrt(s) * unit.astype(np.complex128)).astype(np.complex64)
    lam = I0 * s
    d = (rng.poisson(lam) if noise else lam).astype(np.float32)
    name = name or f"ml-cg {H}x{W} object, {P}x{P} probe, {n * n} sub-pixel positions"
    return Problem(name, psi, probe, pos, d, niter, {"seed": seed, "peak": peak, "step": step, "jitter": jitter,
                                                      "pos_int": base.astype(np.int32), "frac": frac})


def spiral_problem(seed=2, noise=True, K=10000, H=2048, P=256, c=8.94, peak=1e6):
    """2048^2 ellipse phantom, 256^2 probe, 10,000-point jittered Fermat spiral, peak 1e6."""
    rng = np.random.default_rng(seed)
    psi = ellipse_phantom(H, H, rng)
    pos = spiral_positions(H, H, P, K, c, 2, rng)
    probe, d = simulate_counts(psi, gaussian_probe(P), pos, peak, rng, noise)
    return Problem(f"ml-cg {H}x{H} object, {P}x{P} probe, {K} spiral positions", psi, probe, pos, d, 0,
                   {"seed": seed, "peak": peak})


def view_sizes(n_views=64, seed=3, lo=512, hi=2048, step=128):
    """Object sizes of a multi-view series: uniform over {lo, lo + step, ..., hi}."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.choice(np.arange(lo, hi + 1, step), size=n_views)]


def measure(psi: np.ndarray, probe: np.ndarray, pos: np.ndarray, rng: np.random.Generator, noise: bool = True):
    """Counts for an already scaled probe: Poisson(|orthonormal FFT2(probe * patch_k)|^2)."""
    lam = _farfield_intensity(psi, probe, pos)
    return (rng.poisson(lam) if noise else lam).astype(np.float32)


def _measure_torch(psi, probe, pos, seed, batch=512):
    """Same detector model on the GPU (torch.fft in float64, torch.poisson), for large series."""
    import torch

    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    P = probe.shape[0]
    K = pos.shape[0]
    out = torch.empty((K, P, P), dtype=torch.float32, device=dev)
    ps = torch.from_numpy(psi.astype(np.complex128)).to(dev)
    pr = torch.from_numpy(probe.astype(np.complex128)).to(dev)
    iy = torch.arange(P, device=dev)
    pt = torch.from_numpy(pos.astype(np.int64)).to(dev)
    for k0 in range(0, K, batch):
        k1 = min(K, k0 + batch)
        rows = pt[k0:k1, 0][:, None, None] + iy[None, :, None]
        cols = pt[k0:k1, 1][:, None, None] + iy[None, None, :]
        f = torch.fft.fft2(pr[None] * ps[rows, cols], norm="ortho")
        lam = f.real**2 + f.imag**2
        out[k0:k1] = torch.poisson(lam, generator=g).to(torch.float32)
    return out


def view_batch(n_views=64, seed=3, sizes=None, P=128, step=16, jitter=2, peak=1e5, backend="numpy"):
    """A series of views sharing one probe (scaled so view 0's brightest pixel has `peak`).

    View v: N_v x N_v ellipse phantom (seed seed + v), raster filling the view at `step`
    (k = (N - P - 4) // step + 1 per side), +-jitter.  Returns (probe, views) with
    views = [(psi_true, pos, d)]; d is a numpy array, or a CUDA tensor with backend="torch".
    """
    if sizes is None:
        sizes = view_sizes(n_views, seed)
    views = []
    probe = None
    for v, N in enumerate(sizes):
        rng = np.random.default_rng(seed + v)
        k = (N - P - 4) // step + 1
        psi = ellipse_phantom(N, N, rng)
        pos = raster_positions(N, N, P, k, step, jitter, rng)
        if probe is None:
            I0 = _farfield_intensity(psi, gaussian_probe(P), pos[: min(len(pos), 64)])
            probe = (np.sqrt(peak / I0.max()) * gaussian_probe(P).astype(np.complex128)).astype(np.complex64)
        if backend == "torch":
            d = _measure_torch(psi, probe, pos, seed * 1000 + v)
        else:
            d = measure(psi, probe, pos, rng)
        views.append((psi, pos, d))
    return probe, views
