"""Training pairs and the training/evaluation driver of the learned initial guess.

Pairs (diffraction pattern, object patch) come from the library's own forward model:
phantom objects (random ellipses and Voronoi cells, alternating, amplitude 0.8-1, phase
0-pi/2) are scanned at uniformly random positions, ``pty_forward`` gives u = F(p * patch)
with the test's probe (already scaled to counts), and the counts are Poisson(|u|^2).  The
target is the object patch itself.  Everything stays on the GPU.
"""
from __future__ import annotations

import time

import numpy as np

from . import pty, synth


def training_pairs(probe, n_pairs: int, N: int = 1024, per_phantom: int = 8192, seed: int = 100,
                   phantoms=("ellipse", "voronoi")):
    """(d [n][P][P] float32, t [n][P][P] complex64) CUDA tensors from the forward model.

    Phantom i (N x N, generator seed + i) is of kind phantoms[i % len(phantoms)]."""
    import torch

    dev = torch.device("cuda")
    pr = torch.as_tensor(np.ascontiguousarray(probe, np.complex64)).to(dev)
    P = pr.shape[0]
    d = torch.empty((n_pairs, P, P), dtype=torch.float32, device=dev)
    t = torch.empty((n_pairs, P, P), dtype=torch.complex64, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    opts = pty.default_opts()
    opts.tile_config = 0  # one fixed configuration: no autotuning of throw-away contexts
    iy = torch.arange(P, device=dev)
    k, i = 0, 0
    while k < n_pairs:
        rng = np.random.default_rng(seed + i)
        kind = phantoms[i % len(phantoms)]
        psi = synth.ellipse_phantom(N, N, rng) if kind == "ellipse" else synth.voronoi_phantom(N, N, rng)
        m = min(per_phantom, n_pairs - k)
        pos = rng.integers(0, N - P + 1, size=(m, 2)).astype(np.int32)
        psi_d = torch.from_numpy(psi).to(dev)
        pos_d = torch.from_numpy(pos).to(dev)
        zeros = torch.zeros((m, P, P), dtype=torch.float32, device=dev)
        ctx = pty.Context(pr, pos_d, zeros, N, N, opts)
        u = torch.empty((m, P, P), dtype=torch.complex64, device=dev)
        ctx.forward(psi_d, u)
        ctx.close()
        del zeros
        d[k:k + m] = torch.poisson((u.real**2 + u.imag**2).to(torch.float32), generator=gen)
        pl = pos_d.to(torch.int64)
        rows = pl[:, 0][:, None, None] + iy[None, :, None]
        cols = pl[:, 1][:, None, None] + iy[None, None, :]
        t[k:k + m] = psi_d[rows, cols]
        k += m
        i += 1
    torch.cuda.synchronize()
    return d, t


def relative_gap(F, F_star, F0_ones):
    """(F_m - F*) / (F_0^ones - F*): the objective gap normalised by the ones start."""
    return (np.asarray(F, np.float64) - F_star) / (F0_ones - F_star)


def iterations_to_gap(F, F_star, F0_ones, target=1e-3):
    """First iteration m with gap(F_m) <= target (F[0] is the start), or None."""
    g = relative_gap(F, F_star, F0_ones)
    hit = np.nonzero(g <= target)[0]
    return int(hit[0]) if hit.size else None


def solve_to_gap(ctx, psi, F_star, F0_ones, max_iter, target=1e-3, chunk=8):
    """Run CG from psi (in place) until the gap reaches target; returns (iterations, ms, F history)."""
    import torch

    F_hist = []
    done = 0
    t0 = time.perf_counter()
    while done < max_iter:
        n = min(chunk, max_iter - done)
        st, rep = ctx.cg_solve(psi, n)
        F = list(rep["F"])
        F_hist = F if not F_hist else F_hist + F[1:]
        done += rep["iters_done"]
        m = iterations_to_gap(F_hist, F_star, F0_ones, target)
        if m is not None or st != pty.PTY_OK or rep["iters_done"] < n:
            break
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    return iterations_to_gap(F_hist, F_star, F0_ones, target), ms, F_hist
