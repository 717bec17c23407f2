"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test names the equation it pins and the class of mistake it would catch.
"""
import json
import math
import os

import numpy as np
import pytest

from tests.brute import Brute, dft_matrix
from paper_2106_07575_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def tiny_problem(seed=0, H=12, W=10, P=4, K=6, eps=1e-6, noise=True):
    rng = np.random.default_rng(seed)
    psi_true = (0.8 + 0.2 * rng.random((H, W))) * np.exp(1j * rng.uniform(0, np.pi / 2, (H, W)))
    pos = np.stack([rng.integers(0, H - P + 1, K), rng.integers(0, W - P + 1, K)], 1).astype(np.int32)
    probe = 3.0 * crand(rng, P, P)
    return rng, psi_true, probe, pos


# ---------------------------------------------------------------- F (Eq. 1's Fourier operator)
@pytest.mark.parametrize("P", [1, 2, 4, 8])
def test_fft_matches_bruteforce_dft(orc, P):
    """Unitary 2-D DFT = explicit O(N^2) sum (catches sign, normalisation, index order)."""
    rng = np.random.default_rng(P)
    x = crand(rng, P, P)
    Fm = dft_matrix(P)
    want = Fm @ x @ Fm.T
    assert rel(orc.fft2(x), want) <= 1e-13
    assert rel(orc.fft2(x, inverse=True), Fm.conj() @ x @ Fm.conj().T) <= 1e-13


@pytest.mark.parametrize("P", [64, 128, 256])
def test_fft_matches_numpy(orc, P):
    """Library special case: numpy.fft.fft2 with norm='ortho' (FP64)."""
    rng = np.random.default_rng(P)
    x = crand(rng, P, P)
    assert rel(orc.fft2(x), np.fft.fft2(x, norm="ortho")) <= 1e-13
    assert rel(orc.fft2(x, inverse=True), np.fft.ifft2(x, norm="ortho")) <= 1e-13


def test_fft_closed_forms(orc):
    """Delta -> constant phase ramp; plane wave -> delta (closed forms of the DFT)."""
    P = 16
    x = np.zeros((P, P), complex)
    x[3, 5] = 1.0
    k = np.arange(P)
    want = np.exp(-2j * np.pi * (k[:, None] * 3 + k[None, :] * 5) / P) / P
    assert rel(orc.fft2(x), want) <= 1e-14
    wave = np.exp(2j * np.pi * (k[:, None] * 2 + k[None, :] * 7) / P)
    y = orc.fft2(wave)
    expect = np.zeros((P, P), complex)
    expect[2, 7] = P
    assert np.max(np.abs(y - expect)) <= 1e-12


def test_parseval_and_inverse(orc):
    rng = np.random.default_rng(7)
    x = crand(rng, 128, 128)
    y = orc.fft2(x)
    assert abs(np.linalg.norm(y) / np.linalg.norm(x) - 1) <= 1e-14
    assert rel(orc.fft2(y, inverse=True), x) <= 1e-14


# ---------------------------------------------------------------- Q, G and their adjoints
def test_adjoint_dot_tests(orc):
    """<Q x, y> = <x, Q^H y>, <G x, y> = <x, G^H y> (catches a missing conj or wrong scatter)."""
    rng, _, probe, pos = tiny_problem(1, H=40, W=36, P=8, K=13)
    x = crand(rng, 40, 36)
    y = crand(rng, len(pos), 8, 8)
    lhs = np.vdot(orc.Q(x, probe, pos), y)
    rhs = np.vdot(x, orc.QH(y, probe, pos, (40, 36)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    lhs = np.vdot(orc.forward(x, probe, pos), y)
    rhs = np.vdot(x, orc.adjoint(y, probe, pos, (40, 36)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forward_adjoint_against_dense_matrix(orc):
    """G and G^H equal the dense operator built from Q's definition and the DFT matrix."""
    rng, _, probe, pos = tiny_problem(2)
    G = Brute(12, 10, 4, probe, pos, np.ones(len(pos) * 16), 0.0).G
    x = crand(rng, 12, 10)
    y = crand(rng, len(pos), 4, 4)
    assert rel(orc.forward(x, probe, pos).ravel(), G @ x.ravel()) <= 1e-13
    assert rel(orc.adjoint(y, probe, pos, (12, 10)).ravel(), G.conj().T @ y.ravel()) <= 1e-13


def test_illumination_map_by_counting(orc):
    """Q^H Q 1 = sum over positions of |p|^2 placed at each position (counted by loops)."""
    rng, _, probe, pos = tiny_problem(3, H=30, W=30, P=8, K=20)
    pos[3] = pos[4]  # a duplicate position counts twice
    pos[5] = (0, 0)
    pos[6] = (22, 22)
    ones = np.ones((30, 30), complex)
    got = orc.QH(orc.Q(ones, probe, pos), probe, pos, (30, 30))
    want = np.zeros((30, 30))
    for r, c in pos:
        for y in range(8):
            for x in range(8):
                want[r + y, c + x] += abs(probe[y, x]) ** 2
    assert np.max(np.abs(got - want)) <= 1e-12 * want.max()


def test_forward_linearity(orc):
    """G(psi + gamma eta) = G psi + gamma G eta (Eq. 1 is linear in psi)."""
    rng, psi, probe, pos = tiny_problem(4, H=64, W=64, P=16, K=9)
    eta = crand(rng, 64, 64)
    gam = 0.37
    lhs = orc.forward(psi + gam * eta, probe, pos)
    rhs = orc.forward(psi, probe, pos) + gam * orc.forward(eta, probe, pos)
    assert rel(lhs, rhs) <= 1e-13


def test_forward_multithreaded_equals_single(orc):
    rng, psi, probe, pos = tiny_problem(5, H=64, W=64, P=16, K=17)
    assert np.array_equal(orc.forward(psi, probe, pos, 1), orc.forward(psi, probe, pos, 4))


# ---------------------------------------------------------------- Objective (Eq. 2) and gradient (Eq. 3)
def _noisy_case(seed=6):
    p = synth.small_problem(H=48, W=40, P=16, n=4, step=6, jitter=1, peak=1e3, seed=seed)
    return p


@pytest.mark.parametrize("direction", ["real", "imag", "random"])
def test_gradient_finite_differences(orc, direction):
    """dF/dt (psi + t delta)|_0 = 2 Re <g, delta> for the Wirtinger gradient g of Eq. 3.

    Real, imaginary and random complex directions: a dropped conj, sign or factor fails one.
    """
    p = _noisy_case()
    rng = np.random.default_rng(11)
    psi = p.psi_true.astype(np.complex128) * (1 + 0.1 * crand(rng, p.H, p.W))
    delta = {"real": rng.standard_normal((p.H, p.W)),
             "imag": 1j * rng.standard_normal((p.H, p.W)),
             "random": crand(rng, p.H, p.W)}[direction]
    g, F0 = orc.gradient(psi, p.probe, p.pos, p.d, eps=1e-6)
    assert F0 == pytest.approx(orc.objective(psi, p.probe, p.pos, p.d, eps=1e-6), rel=1e-14)
    def central(h):
        Fp = orc.objective(psi + h * delta, p.probe, p.pos, p.d, eps=1e-6)
        Fm = orc.objective(psi - h * delta, p.probe, p.pos, p.d, eps=1e-6)
        return (Fp - Fm) / (2 * h)

    h = 1e-5  # Richardson extrapolation removes the O(h^2) truncation term
    fd = (4 * central(h) - central(2 * h)) / 3
    an = 2 * np.real(np.vdot(g, delta))
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_objective_and_gradient_against_bruteforce(orc):
    """Objective and gradient equal the dense-matrix restatement (incl. d = 0 pixels)."""
    rng, psi, probe, pos = tiny_problem(8)
    u = Brute(12, 10, 4, probe, pos, np.ones(len(pos) * 16), 0).G @ psi.ravel()
    d = rng.poisson(np.abs(u) ** 2).astype(np.float32)
    d[:5] = 0.0
    b = Brute(12, 10, 4, probe, pos, d, 1e-6)
    g, F = orc.gradient(psi, probe, pos, d.reshape(len(pos), 4, 4), eps=1e-6)
    assert F == pytest.approx(b.objective(psi), rel=1e-13)
    assert rel(g, b.gradient(psi)) <= 1e-12


def test_noise_free_truth_is_stationary(orc):
    """Noise-free d at psi_true, eps = 0: grad F = 0 and F = F_min = sum(d - d log d)."""
    p = synth.small_problem(H=64, W=64, P=16, n=5, step=8, jitter=1, peak=1e4, seed=3, noise=False)
    d = p.d.astype(np.float64)
    # the stored d is float32; rebuild the exact model intensities to stay at the true minimum
    u = orc.forward(p.psi_true, p.probe, p.pos)
    d_exact = (np.abs(u) ** 2).astype(np.float32)
    g, F = orc.gradient(p.psi_true, p.probe, p.pos, d_exact, eps=0.0)
    gscale = np.linalg.norm(orc.adjoint(u, p.probe, p.pos, (p.H, p.W)))
    assert np.linalg.norm(g) <= 1e-6 * gscale  # float32 rounding of d only
    dd = d_exact.astype(np.float64)
    Fmin = float(np.sum(np.where(dd > 0, dd - dd * np.log(np.where(dd > 0, dd, 1)), 0.0)))
    assert F == pytest.approx(Fmin, rel=1e-7)
    # the synthetic generator's intensities agree with the oracle's forward model
    assert rel(d, np.abs(u) ** 2) <= 1e-6


def test_global_phase_invariance(orc):
    """F(psi e^{i phi}) = F(psi) (phase retrieval's global-phase ambiguity)."""
    p = _noisy_case(9)
    F0 = orc.objective(p.psi_true, p.probe, p.pos, p.d)
    F1 = orc.objective(p.psi_true * np.exp(0.7j), p.probe, p.pos, p.d)
    assert F1 == pytest.approx(F0, rel=1e-13)


# ---------------------------------------------------------------- CG (Eq. 5-7, Algorithm 1)
def _golden_scalar():
    with open(os.path.join(GOLDEN, "scalar_p1_cg.json")) as f:
        gd = json.load(f)
    ev = lambda s: eval(s, {"log": math.log})  # expressions in the fixture are arithmetic only
    return gd, ev


def test_cg_hand_derived_scalar_case(orc):
    """Two iterations of the P=1 scalar instance against the hand derivation in golden/."""
    gd, ev = _golden_scalar()
    inp = gd["inputs"]
    probe = np.array([[complex(*inp["probe"])]])
    psi0 = np.array([[complex(*inp["psi0"])]])
    d = np.array(inp["d"], np.float32).reshape(1, 1, 1)
    out = orc.cg_solve(psi0, probe, inp["pos"], d, 2, orc.OrcOpts(eps=inp["eps"]))
    ex = gd["expected"]
    assert out["status"] == orc.ORC_OK
    np.testing.assert_allclose(out["F"], [ev(s) for s in ex["F"]], rtol=1e-14)
    np.testing.assert_allclose(out["gamma"], [ev(s) for s in ex["gamma"]], rtol=0)
    assert list(out["halvings"]) == ex["halvings"]
    np.testing.assert_allclose(out["alpha"], [ev(s) for s in ex["alpha"]], rtol=1e-14)
    assert out["psi"][0, 0] == pytest.approx(ev(ex["psi_final"]), rel=1e-14)
    g, _ = orc.gradient(psi0, probe, inp["pos"], d, eps=0.0)
    assert g[0, 0] == pytest.approx(ev(ex["g0"]), rel=1e-14)


def test_cg_against_bruteforce(orc):
    """Five CG iterations equal the dense restatement: F_m, gamma_m, trials, alpha_m, psi."""
    rng, psi_true, probe, pos = tiny_problem(10, H=12, W=12, P=4, K=9)
    b0 = Brute(12, 12, 4, probe, pos, np.ones(9 * 16), 0)
    d = rng.poisson(np.abs(b0.G @ psi_true.ravel()) ** 2).astype(np.float32)
    b = Brute(12, 12, 4, probe, pos, d, 0.1)
    psi0 = np.ones((12, 12), complex)
    want = b.cg(psi0, 5)
    got = orc.cg_solve(psi0, probe, pos, d.reshape(9, 4, 4), 5, orc.OrcOpts(eps=0.1))
    assert got["status"] == orc.ORC_OK
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-11)
    np.testing.assert_array_equal(got["gamma"], want["gamma"])
    np.testing.assert_array_equal(got["halvings"], want["halvings"])
    np.testing.assert_allclose(got["alpha"], want["alpha"], rtol=1e-9, atol=1e-12)
    assert rel(got["psi"], want["psi"]) <= 1e-10


@pytest.mark.parametrize("t", [3e4, -5e3])
def test_cg_termination_parameter_against_bruteforce(orc, t):
    """Eq. 7 with t != 0: a trial is accepted when F(psi + gamma eta) <= F(psi) + gamma t, so
    t > 0 accepts some increases and t < 0 asks for a decrease of at least gamma |t|.  Both
    change the trial counts of the t = 0 solve here (a dropped or sign-flipped t fails)."""
    rng, psi_true, probe, pos = tiny_problem(10, H=12, W=12, P=4, K=9)
    b0 = Brute(12, 12, 4, probe, pos, np.ones(9 * 16), 0)
    d = rng.poisson(np.abs(b0.G @ psi_true.ravel()) ** 2).astype(np.float32)
    b = Brute(12, 12, 4, probe, pos, d, 0.1)
    psi0 = np.ones((12, 12), complex)
    want = b.cg(psi0, 5, t=t)
    assert want["halvings"] != b.cg(psi0, 5)["halvings"]
    got = orc.cg_solve(psi0, probe, pos, d.reshape(9, 4, 4), 5, orc.OrcOpts(eps=0.1, t=t))
    assert got["status"] == orc.ORC_OK
    np.testing.assert_array_equal(got["halvings"], want["halvings"])
    np.testing.assert_array_equal(got["gamma"], want["gamma"])
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-11)
    assert rel(got["psi"], want["psi"]) <= 1e-10


def test_cg_invariants(orc):
    """F_{m+1} <= F_m (Eq. 7, t=0); gamma_m in {2^-k}; eta_0 = -g_0 (first step is steepest descent)."""
    p = _noisy_case(12)
    psi0 = p.psi0()
    out = orc.cg_solve(psi0, p.probe, p.pos, p.d, 6)
    assert out["status"] == orc.ORC_OK and out["iters_done"] == 6
    assert np.all(np.diff(out["F"]) <= 0)
    for gam, k in zip(out["gamma"], out["halvings"]):
        assert gam == 2.0 ** -k
    # first iterate: psi_1 = psi_0 - gamma_0 g_0 exactly
    g0, _ = orc.gradient(psi0, p.probe, p.pos, p.d)
    one = orc.cg_solve(psi0, p.probe, p.pos, p.d, 1)
    assert rel(one["psi"], psi0 - one["gamma"][0] * g0) <= 1e-15
    assert one["alpha"][0] == 0.0


def test_cg_stall_leaves_psi(orc):
    """No step accepted within max_halvings -> status STALLED, psi keeps the last iterate."""
    p = _noisy_case(13)
    psi0 = p.psi0()
    out = orc.cg_solve(psi0, p.probe, p.pos, p.d, 3, orc.OrcOpts(gamma0=1e12, max_halvings=2))
    assert out["status"] == orc.ORC_STALLED and out["iters_done"] == 0
    assert np.array_equal(out["psi"], psi0.astype(np.complex128))


def test_bad_arguments(orc):
    p = _noisy_case(14)
    bad = p.pos.copy()
    bad[0] = (p.H - p.P + 1, 0)
    with pytest.raises(RuntimeError, match="status 2"):
        orc.forward(p.psi_true, p.probe, bad)
    with pytest.raises(RuntimeError, match="status 1"):
        orc.forward(p.psi_true, np.ones((6, 6), complex), p.pos)


# ---------------------------------------------------------------- shapes swept against the dense restatement
@pytest.mark.parametrize("H,W,P,K,seed", [
    (1, 1, 1, 1, 30),    # one pixel
    (3, 5, 1, 7, 31),    # P = 1: every position a single pixel, duplicates likely
    (6, 3, 2, 5, 32),    # tall object, P = 2
    (5, 9, 4, 4, 33),    # wide object, the window spans every row
    (8, 8, 8, 2, 34),    # P equal to the object
    (11, 7, 4, 12, 35),  # odd sizes, more positions than rows
])
@pytest.mark.parametrize("est", ["ml", "ls"])
def test_operators_objective_gradient_swept_against_bruteforce(orc, H, W, P, K, seed, est):
    """G, G^H, F and grad F at assorted shapes (P = 1 .. 8, square and rectangular objects,
    corner, edge and repeated positions) equal the dense restatement: catches an index or
    stride that only square, power-of-two-sized objects hide."""
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.integers(0, H - P + 1, K), rng.integers(0, W - P + 1, K)], 1).astype(np.int32)
    pos[0] = (H - P, W - P)  # the last window that fits
    probe = crand(rng, P, P)
    psi = crand(rng, H, W)
    b0 = Brute(H, W, P, probe, pos, np.ones(K * P * P), 0)
    y = crand(rng, K, P, P)
    assert rel(orc.forward(psi, probe, pos).ravel(), b0.G @ psi.ravel()) <= 1e-13
    assert rel(orc.adjoint(y, probe, pos, (H, W)).ravel(), b0.G.conj().T @ y.ravel()) <= 1e-13
    d = rng.poisson(2.0 * np.abs(b0.G @ psi.ravel()) ** 2).astype(np.float32)
    d[::3] = 0.0
    b = Brute(H, W, P, probe, pos, d, 0.05, est=est)
    e = orc.EST_ML if est == "ml" else orc.EST_LS
    g, F = orc.gradient(psi, probe, pos, d.reshape(K, P, P), eps=0.05, est=e)
    assert F == pytest.approx(b.objective(psi), rel=1e-12, abs=1e-12)
    assert rel(g, b.gradient(psi)) <= 1e-12


@pytest.mark.parametrize("nthreads", [2, 3, 7])
def test_threaded_paths_against_bruteforce(orc, nthreads):
    """The per-thread scatter buffers and the per-pattern objective partials (the paths the
    parity tests take with every host core) equal the dense restatement, for thread counts
    that split 7 patterns evenly, unevenly and one per thread."""
    rng, psi, probe, pos = tiny_problem(36, H=12, W=10, P=4, K=7)
    b0 = Brute(12, 10, 4, probe, pos, np.ones(7 * 16), 0)
    y = crand(rng, 7, 4, 4)
    assert rel(orc.adjoint(y, probe, pos, (12, 10), nthreads).ravel(), b0.G.conj().T @ y.ravel()) <= 1e-13
    d = rng.poisson(np.abs(b0.G @ psi.ravel()) ** 2).astype(np.float32)
    b = Brute(12, 10, 4, probe, pos, d, 0.1)
    g, F = orc.gradient(psi, probe, pos, d.reshape(7, 4, 4), eps=0.1, nthreads=nthreads)
    assert F == pytest.approx(b.objective(psi), rel=1e-13)
    assert orc.objective(psi, probe, pos, d.reshape(7, 4, 4), eps=0.1, nthreads=nthreads) == pytest.approx(
        b.objective(psi), rel=1e-13)
    assert rel(g, b.gradient(psi)) <= 1e-12
