"""The line-search certificate's inequality on oracle data (CPU): with t = q / (|u|^2 + eps)
and weights d / D per pattern, Jensen's inequality on the concave log1p gives
    sum_e d log1p(t_e) <= D log1p(sum_e d t_e / D),
so the per-pattern bound LB(gamma) = sum_all q - sum_k D_k log1p(T_k / D_k) never exceeds the
exact objective change F(psi + gamma eta) - F(psi) of Eq. 2.  Checked in FP64 on the oracle's
u = G psi and v = G eta for a small problem, at the trials gamma0 tau^(j+1) the GPU
certifies, and at a steepest-descent direction where the bound is tight enough to reject the
leading trials."""
import numpy as np
import pytest

from oracle import orc
from paper_2106_07575_gb300 import synth


@pytest.fixture(scope="module")
def case():
    p = synth.small_problem(seed=0)
    eps = 0.1
    psi = np.ones((p.H, p.W), np.complex128)
    g, F0 = orc.gradient(psi, p.probe, p.pos, p.d, eps)
    eta = -g
    u = orc.forward(psi, p.probe, p.pos)
    v = orc.forward(eta, p.probe, p.pos)
    return p, eps, psi, eta, u, v, F0


def exact_change(p, eps, psi, eta, gamma, F0):
    return orc.objective(psi + gamma * eta, p.probe, p.pos, p.d, eps) - F0


def jensen_bound(d, u, v, eps, gamma):
    a = np.abs(u) ** 2
    b = 2 * np.real(np.conj(u) * v)
    c = np.abs(v) ** 2
    q = gamma * (b + gamma * c)
    m = d > 0
    w = np.where(m, d / (a + eps), 0.0)
    T = (w * q).sum(axis=(1, 2))  # sum_e d t_e per pattern
    D = d.sum(axis=(1, 2))
    safe = D > 0
    logs = np.zeros_like(D)
    logs[safe] = D[safe] * np.log1p(T[safe] / D[safe])
    return q.sum() - logs.sum()


def test_bound_never_exceeds_the_exact_change(case):
    p, eps, psi, eta, u, v, F0 = case
    d = p.d.astype(np.float64)
    for j in range(24):
        gamma = 0.5 ** (j + 1)
        lb = jensen_bound(d, u, v, eps, gamma)
        ex = exact_change(p, eps, psi, eta, gamma, F0)
        assert lb <= ex + 1e-9 * abs(ex) + 1e-6, (j, lb, ex)


def test_bound_rejects_leading_trials_and_not_the_accepted_one(case):
    """The first accepted trial (plain backtracking, t = 0) has a bound <= 0, and the
    bound already exceeds 0 at the first trial."""
    p, eps, psi, eta, u, v, F0 = case
    d = p.d.astype(np.float64)
    accepted = next(j for j in range(60) if exact_change(p, eps, psi, eta, 0.5 ** (j + 1), F0) <= 0)
    assert jensen_bound(d, u, v, eps, 0.5 ** (accepted + 1)) <= 0
    assert jensen_bound(d, u, v, eps, 0.5) > 0
