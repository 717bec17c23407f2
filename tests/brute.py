"""Brute-force restatement of ML-CG for tiny inputs, used to pin the oracle.

Written independently of the oracle's C code and in a different style: explicit DFT
matrices instead of an FFT, dense operator matrices for Q, and a literal reading of
Eq. 2, 3, 6, 7 and Algorithm 1 of the paper.  Only for H*W and K*P^2 up to a few hundred.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(P):
    """Unitary DFT matrix, entries exp(-2 pi i j k / P) / sqrt(P)."""
    j = np.arange(P)
    return np.exp(-2j * np.pi * np.outer(j, j) / P) / np.sqrt(P)


def g_matrix(H, W, P, probe, pos):
    """Dense matrix of G = F Q acting on vec(psi) (row-major), shape (K*P*P, H*W).

    probe is [P][P] (one for every position) or [K][P][P] (one per position)."""
    K = len(pos)
    Fm = dft_matrix(P)
    F2 = np.kron(Fm, Fm)  # acts on row-major vec of a P x P array: vec(F X F^T)
    G = np.zeros((K * P * P, H * W), np.complex128)
    for k, (r, c) in enumerate(pos):
        pk = probe[k] if probe.ndim == 3 else probe
        Qk = np.zeros((P * P, H * W), np.complex128)
        for y in range(P):
            for x in range(P):
                Qk[y * P + x, (r + y) * W + (c + x)] = pk[y, x]
        G[k * P * P:(k + 1) * P * P] = F2 @ Qk
    return G


class Brute:
    """Dense restatement.  est "ml": Eq. 2 / Eq. 3 with the eps guard; est "ls": the
    amplitude least-squares estimator (|u| - sqrt d)^2 with |u| -> sqrt(|u|^2 + eps)."""

    def __init__(self, H, W, P, probe, pos, d, eps, est="ml"):
        self.G = g_matrix(H, W, P, np.asarray(probe, np.complex128), np.asarray(pos))
        self.d = np.asarray(d, np.float64).ravel()
        self.eps = eps
        self.est = est
        self.shape = (H, W)

    def objective(self, psi):
        u = self.G @ psi.ravel()
        a = np.abs(u) ** 2
        has = self.d > 0
        if self.est == "ls":
            # (s - sqrt d)^2 expanded, s = sqrt(|u|^2 + eps); |u|^2 where nothing was counted
            s = np.sqrt(a + self.eps)
            return float(np.sum(np.where(has, a - 2.0 * np.sqrt(self.d) * s + self.d, a)))
        logterm = np.where(has, self.d * np.log(np.where(has, a + self.eps, 1.0)), 0.0)
        return float(np.sum(a - logterm))

    def gradient(self, psi):
        u = self.G @ psi.ravel()
        a = np.abs(u) ** 2
        has = self.d > 0
        if self.est == "ls":
            # d/d conj(u) of (s - sqrt d)^2 = (s - sqrt d) u / s
            s = np.sqrt(a + self.eps)
            resid = np.where(has, (s - np.sqrt(self.d)) / s, 1.0) * u
        else:
            resid = u - np.where(has, self.d / np.where(has, a + self.eps, 1.0), 0.0) * u
        return (self.G.conj().T @ resid).reshape(self.shape)

    def gd(self, psi0, niter, step):
        """Eq. 4 with a constant step: psi <- psi - step * grad F(psi)."""
        psi = np.array(psi0, np.complex128)
        F = []
        for _ in range(niter):
            F.append(self.objective(psi))
            psi = psi - step * self.gradient(psi)
        F.append(self.objective(psi))
        return {"F": F, "psi": psi}

    def cg(self, psi0, niter, gamma0=1.0, tau=0.5, t=0.0, max_halvings=60, warm=False):
        psi = np.array(psi0, np.complex128)
        out = {"F": [], "gamma": [], "halvings": [], "alpha": []}
        g_prev = eta = None
        last = None  # accepted step of the previous iteration (warm start)
        for m in range(niter):
            g = self.gradient(psi)
            Fm = self.objective(psi)
            out["F"].append(Fm)
            if m == 0:
                alpha = 0.0
            else:
                den = float(np.real(np.vdot(eta, g - g_prev)))
                num = float(np.real(np.vdot(g, g)))
                alpha = num / den if den > 0 and np.isfinite(den) else 0.0
            eta = -g if m == 0 else -g + alpha * eta
            out["alpha"].append(alpha)
            gam = gamma0 if (not warm or last is None) else min(gamma0, last / tau)
            for k in range(1, max_halvings + 1):
                gam *= tau
                Ft = self.objective(psi + gam * eta)
                if Ft <= Fm + gam * t:
                    break
            else:
                raise RuntimeError("stalled")
            out["gamma"].append(gam)
            out["halvings"].append(k)
            psi = psi + gam * eta
            g_prev = g
            last = gam
        out["F"].append(self.objective(psi))
        out["psi"] = psi
        return out
