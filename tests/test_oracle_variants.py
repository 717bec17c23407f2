"""Pins of the oracle's variants of the method (CPU only): the least-squares estimator named
beside Eq. 2, the gradient-descent solver of Eq. 4 and the warm-started line search of
Eq. 7.  Each is checked against hand derivations (tests/golden/), a dense restatement
(tests/brute.py), finite differences or closed forms -- never against the oracle itself.
"""
import json
import math
import os

import numpy as np
import pytest

from tests.brute import Brute
from paper_2106_07575_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        gd = json.load(f)
    ev = lambda s: eval(s, {"log": math.log})  # expressions in the fixtures are arithmetic only
    inp = gd["inputs"]
    probe = np.array([[complex(*inp["probe"])]])
    psi0 = np.array([[complex(*inp["psi0"])]])
    d = np.array(inp["d"], np.float32).reshape(1, 1, 1)
    return gd, ev, inp, probe, psi0, d


def tiny(seed, H=12, W=12, P=4, K=9):
    rng = np.random.default_rng(seed)
    psi_true = (0.8 + 0.2 * rng.random((H, W))) * np.exp(1j * rng.uniform(0, np.pi / 2, (H, W)))
    pos = np.stack([rng.integers(0, H - P + 1, K), rng.integers(0, W - P + 1, K)], 1).astype(np.int32)
    probe = 3.0 * crand(rng, P, P)
    b0 = Brute(H, W, P, probe, pos, np.ones(K * P * P), 0)
    d = rng.poisson(np.abs(b0.G @ psi_true.ravel()) ** 2).astype(np.float32)
    d[:7] = 0.0  # pixels without counts
    return rng, psi_true, probe, pos, d


# ---------------------------------------------------------------- LS estimator
def test_ls_objective_and_gradient_against_bruteforce(orc):
    """LS objective and its Wirtinger gradient equal the dense restatement (incl. d = 0)."""
    rng, psi_true, probe, pos, d = tiny(21)
    psi = psi_true * (1 + 0.2 * crand(rng, 12, 12))
    b = Brute(12, 12, 4, probe, pos, d, 1e-3, est="ls")
    g, F = orc.gradient(psi, probe, pos, d.reshape(9, 4, 4), eps=1e-3, est=orc.EST_LS)
    assert F == pytest.approx(b.objective(psi), rel=1e-13)
    assert F == pytest.approx(orc.objective(psi, probe, pos, d.reshape(9, 4, 4), eps=1e-3, est=orc.EST_LS),
                              rel=1e-14)
    assert rel(g, b.gradient(psi)) <= 1e-12


def test_ls_at_eps_zero_is_the_amplitude_misfit(orc):
    """At eps = 0 the LS objective is sum (|G psi| - sqrt d)^2, written here from numpy's FFT."""
    p = synth.small_problem(H=40, W=40, P=16, n=3, step=8, jitter=1, peak=1e3, seed=4)
    rng = np.random.default_rng(5)
    psi = p.psi_true * (1 + 0.1 * crand(rng, p.H, p.W))
    tot = 0.0
    for (r, c), dk in zip(p.pos, p.d):
        u = np.fft.fft2(p.probe * psi[r:r + p.P, c:c + p.P], norm="ortho")
        tot += np.sum((np.abs(u) - np.sqrt(dk.astype(np.float64))) ** 2)
    assert orc.objective(psi, p.probe, p.pos, p.d, eps=0.0, est=orc.EST_LS) == pytest.approx(tot, rel=1e-12)


@pytest.mark.parametrize("direction", ["real", "imag", "random"])
def test_ls_gradient_finite_differences(orc, direction):
    """dF/dt (psi + t delta)|_0 = 2 Re <g, delta> for the LS objective's gradient."""
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=6)
    rng = np.random.default_rng(17)
    psi = p.psi_true.astype(np.complex128) * (1 + 0.1 * crand(rng, p.H, p.W))
    delta = {"real": rng.standard_normal((p.H, p.W)), "imag": 1j * rng.standard_normal((p.H, p.W)),
             "random": crand(rng, p.H, p.W)}[direction]
    eps = 1e-3
    g, _ = orc.gradient(psi, p.probe, p.pos, p.d, eps=eps, est=orc.EST_LS)

    def central(h):
        Fp = orc.objective(psi + h * delta, p.probe, p.pos, p.d, eps=eps, est=orc.EST_LS)
        Fm = orc.objective(psi - h * delta, p.probe, p.pos, p.d, eps=eps, est=orc.EST_LS)
        return (Fp - Fm) / (2 * h)

    h = 1e-5
    fd = (4 * central(h) - central(2 * h)) / 3
    an = 2 * np.real(np.vdot(g, delta))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_ls_noise_free_truth_is_zero_and_stationary(orc):
    """Noise-free d = |G psi_true|^2, eps = 0: F_LS(psi_true) = 0 and grad F_LS = 0."""
    p = synth.small_problem(H=64, W=64, P=16, n=5, step=8, jitter=1, peak=1e4, seed=3, noise=False)
    u = orc.forward(p.psi_true, p.probe, p.pos)
    d_exact = (np.abs(u) ** 2).astype(np.float32)
    g, F = orc.gradient(p.psi_true, p.probe, p.pos, d_exact, eps=0.0, est=orc.EST_LS)
    scale = float(np.sum(d_exact.astype(np.float64)))
    assert abs(F) <= 1e-12 * scale  # float32 rounding of d only
    gscale = np.linalg.norm(orc.adjoint(u, p.probe, p.pos, (p.H, p.W)))
    assert np.linalg.norm(g) <= 1e-6 * gscale


def test_ls_hand_derived_scalar_cg(orc):
    """Two CG iterations of the LS estimator on the P=1 instance of golden/scalar_p1_ls_cg.json."""
    gd, ev, inp, probe, psi0, d = golden("scalar_p1_ls_cg.json")
    opts = orc.OrcOpts(eps=inp["eps"], est=orc.EST_LS)
    out = orc.cg_solve(psi0, probe, inp["pos"], d, 2, opts)
    ex = gd["expected"]
    assert out["status"] == orc.ORC_OK
    np.testing.assert_allclose(out["F"], [ev(s) for s in ex["F"]], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(out["gamma"], [ev(s) for s in ex["gamma"]], rtol=0)
    assert list(out["halvings"]) == ex["halvings"]
    np.testing.assert_allclose(out["alpha"], [ev(s) for s in ex["alpha"]], rtol=1e-14)
    assert out["psi"][0, 0] == pytest.approx(ev(ex["psi_final"]), rel=1e-14)
    g, _ = orc.gradient(psi0, probe, inp["pos"], d, eps=0.0, est=orc.EST_LS)
    assert g[0, 0] == pytest.approx(ev(ex["g0"]), rel=1e-14)


def test_ls_cg_against_bruteforce(orc):
    """Five LS-estimator CG iterations equal the dense restatement."""
    rng, psi_true, probe, pos, d = tiny(22)
    b = Brute(12, 12, 4, probe, pos, d, 0.1, est="ls")
    psi0 = np.ones((12, 12), complex)
    want = b.cg(psi0, 5)
    got = orc.cg_solve(psi0, probe, pos, d.reshape(9, 4, 4), 5, orc.OrcOpts(eps=0.1, est=orc.EST_LS))
    assert got["status"] == orc.ORC_OK
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-11)
    np.testing.assert_array_equal(got["gamma"], want["gamma"])
    np.testing.assert_array_equal(got["halvings"], want["halvings"])
    assert rel(got["psi"], want["psi"]) <= 1e-10


def test_ls_global_phase_invariance(orc):
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=9)
    F0 = orc.objective(p.psi_true, p.probe, p.pos, p.d, est=orc.EST_LS)
    F1 = orc.objective(p.psi_true * np.exp(-1.3j), p.probe, p.pos, p.d, est=orc.EST_LS)
    assert F1 == pytest.approx(F0, rel=1e-13)


def test_bad_estimator_and_solver_rejected(orc):
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=9)
    with pytest.raises(RuntimeError, match="status 1"):
        orc.objective(p.psi_true, p.probe, p.pos, p.d, est=7)
    with pytest.raises(RuntimeError, match="status 1"):
        orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 1, orc.OrcOpts(solver=5))


# ---------------------------------------------------------------- GD solver (Eq. 4)
def test_gd_hand_derived_scalar(orc):
    """Two constant-step GD iterations of golden/scalar_p1_gd.json."""
    gd, ev, inp, probe, psi0, d = golden("scalar_p1_gd.json")
    opts = orc.OrcOpts(eps=inp["eps"], solver=orc.SOLVER_GD, gd_step=inp["step"])
    ex = gd["expected"]
    out = orc.cg_solve(psi0, probe, inp["pos"], d, 2, opts)
    assert out["status"] == orc.ORC_OK and out["iters_done"] == 2
    np.testing.assert_allclose(out["F"], [ev(s) for s in ex["F"]], rtol=1e-14)
    assert out["psi"][0, 0] == pytest.approx(ev(ex["psi"][1]), rel=1e-14)
    one = orc.cg_solve(psi0, probe, inp["pos"], d, 1, opts)
    assert one["psi"][0, 0] == pytest.approx(ev(ex["psi"][0]), rel=1e-14)
    assert list(out["halvings"]) == [0, 0] and list(out["gamma"]) == [inp["step"]] * 2


@pytest.mark.parametrize("est", ["ml", "ls"])
def test_gd_against_bruteforce(orc, est):
    """Six GD iterations equal the dense restatement, for both estimators."""
    rng, psi_true, probe, pos, d = tiny(23)
    b = Brute(12, 12, 4, probe, pos, d, 0.1, est=est)
    psi0 = np.ones((12, 12), complex)
    step = 2e-4
    want = b.gd(psi0, 6, step)
    opts = orc.OrcOpts(eps=0.1, est=orc.EST_LS if est == "ls" else orc.EST_ML, solver=orc.SOLVER_GD, gd_step=step)
    got = orc.cg_solve(psi0, probe, pos, d.reshape(9, 4, 4), 6, opts)
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-12)
    assert rel(got["psi"], want["psi"]) <= 1e-12


def test_gd_small_step_decreases(orc):
    """A small enough constant step decreases F every iteration (descent direction -g)."""
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=12)
    g, _ = orc.gradient(p.psi0(), p.probe, p.pos, p.d)
    out = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 5, orc.OrcOpts(solver=orc.SOLVER_GD, gd_step=1e-6))
    assert np.all(np.diff(out["F"]) < 0)


# ---------------------------------------------------------------- warm-started line search
def test_warm_hand_derived_scalar_cg(orc):
    """Two warm-started CG iterations of golden/scalar_p1_warm_cg.json."""
    gd, ev, inp, probe, psi0, d = golden("scalar_p1_warm_cg.json")
    out = orc.cg_solve(psi0, probe, inp["pos"], d, 2, orc.OrcOpts(eps=inp["eps"], warm=True))
    ex = gd["expected"]
    assert out["status"] == orc.ORC_OK
    np.testing.assert_allclose(out["F"], [ev(s) for s in ex["F"]], rtol=1e-14)
    np.testing.assert_allclose(out["gamma"], [ev(s) for s in ex["gamma"]], rtol=0)
    assert list(out["halvings"]) == ex["halvings"]
    np.testing.assert_allclose(out["alpha"], [ev(s) for s in ex["alpha"]], rtol=1e-14)
    assert out["psi"][0, 0] == pytest.approx(ev(ex["psi_final"]), rel=1e-14)


def test_warm_cg_against_bruteforce(orc):
    rng, psi_true, probe, pos, d = tiny(24)
    b = Brute(12, 12, 4, probe, pos, d, 0.1)
    psi0 = np.ones((12, 12), complex)
    want = b.cg(psi0, 6, warm=True)
    got = orc.cg_solve(psi0, probe, pos, d.reshape(9, 4, 4), 6, orc.OrcOpts(eps=0.1, warm=True))
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-11)
    np.testing.assert_array_equal(got["gamma"], want["gamma"])
    np.testing.assert_array_equal(got["halvings"], want["halvings"])
    assert rel(got["psi"], want["psi"]) <= 1e-10


def test_warm_invariants(orc):
    """Warm start: same first iteration as Algorithm 1's search; every step gamma0 tau^k;
    steps never grow; F never increases; fewer trials in total over the solve."""
    p = synth.small_problem(H=96, W=96, P=32, n=6, step=10, jitter=1, peak=1e4, seed=31)
    plain = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 8)
    warm = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 8, orc.OrcOpts(warm=True))
    assert warm["status"] == orc.ORC_OK
    assert warm["gamma"][0] == plain["gamma"][0] and warm["halvings"][0] == plain["halvings"][0]
    for gam in warm["gamma"]:
        k = -math.log2(gam)
        assert k == int(k)
    assert np.all(np.diff(warm["gamma"]) <= 0)
    assert np.all(np.diff(warm["F"]) <= 0)
    assert warm["halvings"][1:].sum() < plain["halvings"][1:].sum()


def test_timestamps_are_per_iteration(orc):
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=12)
    out = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 3)
    assert len(out["t"]) == 3 and np.all(np.diff(out["t"]) >= 0)
