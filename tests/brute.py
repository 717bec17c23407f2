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
    """Dense matrix of G = F Q acting on vec(psi) (row-major), shape (K*P*P, H*W)."""
    K = len(pos)
    Fm = dft_matrix(P)
    F2 = np.kron(Fm, Fm)  # acts on row-major vec of a P x P array: vec(F X F^T)
    G = np.zeros((K * P * P, H * W), np.complex128)
    for k, (r, c) in enumerate(pos):
        Qk = np.zeros((P * P, H * W), np.complex128)
        for y in range(P):
            for x in range(P):
                Qk[y * P + x, (r + y) * W + (c + x)] = probe[y, x]
        G[k * P * P:(k + 1) * P * P] = F2 @ Qk
    return G


class Brute:
    def __init__(self, H, W, P, probe, pos, d, eps):
        self.G = g_matrix(H, W, P, np.asarray(probe, np.complex128), np.asarray(pos))
        self.d = np.asarray(d, np.float64).ravel()
        self.eps = eps
        self.shape = (H, W)

    def objective(self, psi):
        u = self.G @ psi.ravel()
        a = np.abs(u) ** 2
        logterm = np.where(self.d > 0, self.d * np.log(np.where(self.d > 0, a + self.eps, 1.0)), 0.0)
        return float(np.sum(a - logterm))

    def gradient(self, psi):
        u = self.G @ psi.ravel()
        a = np.abs(u) ** 2
        resid = u - np.where(self.d > 0, self.d / np.where(self.d > 0, a + self.eps, 1.0), 0.0) * u
        return (self.G.conj().T @ resid).reshape(self.shape)

    def cg(self, psi0, niter, gamma0=1.0, tau=0.5, t=0.0, max_halvings=60):
        psi = np.array(psi0, np.complex128)
        out = {"F": [], "gamma": [], "halvings": [], "alpha": []}
        g_prev = eta = None
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
            gam = gamma0
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
        out["F"].append(self.objective(psi))
        out["psi"] = psi
        return out
