"""Pins of the oracle's sub-pixel positions: the probe shift by the Fourier shift theorem
(orc_shift_probe) and the forward model, gradient and CG with one probe per position.

The paper's scan positions are float32 inputs of Algorithm 1; how a fraction enters Q is
not stated.  The reading: the window starts at floor(s) and the probe is moved by the
fraction with the Fourier shift theorem, Nyquist bins multiplied by cos(pi delta).  Each
pin below is fixed by mathematics, not by re-running the oracle's own formula:
integer shifts are circular rolls, plane waves shift by a closed-form phase, real probes
stay real, shifts of band-limited probes compose, the numpy generator's independent
implementation agrees, and the per-position forward model keeps the adjoint identity,
the finite-difference gradient and the noise-free minimum."""
import numpy as np
import pytest

import oracle
from paper_2106_07575_gb300 import synth


def _rand_probe(P, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P))


def test_zero_shift_is_identity():
    p = _rand_probe(16, 0)
    assert np.max(np.abs(oracle.shift_probe(p, 0.0, 0.0) - p)) < 1e-13


@pytest.mark.parametrize("dy,dx", [(1, 0), (0, 1), (3, -2), (-5, 7), (16, 16)])
def test_integer_shift_is_circular_roll(dy, dx):
    p = _rand_probe(16, 1)
    want = np.roll(np.roll(p, dy, axis=0), dx, axis=1)
    assert np.max(np.abs(oracle.shift_probe(p, dy, dx) - want)) < 1e-12


@pytest.mark.parametrize("a,b", [(1, 0), (0, 3), (-5, 2), (7, -7)])
def test_plane_wave_shifts_by_its_phase(a, b):
    # p(y, x) = exp(2 pi i (a y + b x) / P), |a|, |b| < P/2: p(r - delta) in closed form
    P, dy, dx = 16, 0.37, -0.81
    y, x = np.mgrid[0:P, 0:P]
    p = np.exp(2j * np.pi * (a * y + b * x) / P)
    want = np.exp(2j * np.pi * (a * (y - dy) + b * (x - dx)) / P)
    assert np.max(np.abs(oracle.shift_probe(p, dy, dx) - want)) < 1e-12


def test_band_limited_function_is_evaluated_between_samples():
    # a trigonometric polynomial below Nyquist is reproduced exactly at shifted points
    P, dy, dx = 32, 0.25, 0.6
    rng = np.random.default_rng(2)
    freqs = rng.integers(-15, 16, size=(6, 2))
    coef = rng.standard_normal(6) + 1j * rng.standard_normal(6)

    def f(y, x):
        return sum(c * np.exp(2j * np.pi * (a * y + b * x) / P) for c, (a, b) in zip(coef, freqs))

    y, x = np.mgrid[0:P, 0:P].astype(np.float64)
    assert np.max(np.abs(oracle.shift_probe(f(y, x), dy, dx) - f(y - dy, x - dx))) < 1e-11


def test_nyquist_rows_take_cos_pi_delta():
    # content only at the Nyquist row: (-1)^y -> cos(pi dy) (-1)^y
    P, dy = 8, 0.3
    y, _ = np.mgrid[0:P, 0:P]
    p = (-1.0) ** y + 0j
    assert np.max(np.abs(oracle.shift_probe(p, dy, 0.0) - np.cos(np.pi * dy) * p)) < 1e-13


def test_real_probe_stays_real():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((32, 32)) + 0j
    assert np.max(np.abs(oracle.shift_probe(p, 0.43, 0.91).imag)) < 1e-13


def test_shifts_of_a_band_limited_probe_compose():
    P = 32
    spec = np.fft.fft2(_rand_probe(P, 4))
    spec[P // 2, :] = 0
    spec[:, P // 2] = 0
    p = np.fft.ifft2(spec)
    two = oracle.shift_probe(oracle.shift_probe(p, 0.3, 0.45), 0.55, 0.2)
    assert np.max(np.abs(two - oracle.shift_probe(p, 0.85, 0.65))) < 1e-12


def test_agrees_with_the_generator_numpy_implementation():
    P = 64
    p = synth.gaussian_probe(P).astype(np.complex128)
    frac = np.array([[0.1, 0.7], [0.5, 0.5], [0.93, 0.02]])
    ref = synth.shifted_probes(p, frac)
    for k, (dy, dx) in enumerate(frac):
        assert np.max(np.abs(oracle.shift_probe(p, dy, dx) - ref[k])) < 1e-12


def test_integer_positions_give_the_shared_probe_path():
    prob = synth.small_problem(H=96, W=96, P=32, n=4, step=14, jitter=1, peak=1e3, seed=5)
    pos_i, probes = oracle.subpixel_probes(prob.probe, prob.pos.astype(np.float32))
    assert np.array_equal(pos_i, prob.pos)
    psi = prob.psi_true
    assert np.array_equal(oracle.forward(psi, probes, pos_i), oracle.forward(psi, prob.probe, prob.pos))


def _subpx(seed=6, noise=True):
    return synth.subpixel_problem(H=96, W=96, P=32, n=4, step=14, jitter=1.5, peak=1e3, seed=seed, noise=noise)


def test_subpixel_adjoint_dot():
    prob = _subpx()
    pos_i, probes = oracle.subpixel_probes(prob.probe, prob.pos)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((prob.H, prob.W)) + 1j * rng.standard_normal((prob.H, prob.W))
    y = rng.standard_normal((prob.K, prob.P, prob.P)) + 1j * rng.standard_normal((prob.K, prob.P, prob.P))
    lhs = np.vdot(oracle.forward(x, probes, pos_i), y)
    rhs = np.vdot(x, oracle.adjoint(y, probes, pos_i, x.shape))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_subpixel_gradient_finite_difference():
    prob = _subpx()
    pos_i, probes = oracle.subpixel_probes(prob.probe, prob.pos)
    rng = np.random.default_rng(8)
    psi = prob.psi0().astype(np.complex128) * (1 + 0.05 * rng.standard_normal((prob.H, prob.W)))
    g, F = oracle.gradient(psi, probes, pos_i, prob.d)
    delta = rng.standard_normal(psi.shape) + 1j * rng.standard_normal(psi.shape)

    def central(h):
        Fp = oracle.objective(psi + h * delta, probes, pos_i, prob.d)
        Fm = oracle.objective(psi - h * delta, probes, pos_i, prob.d)
        return (Fp - Fm) / (2 * h)

    h = 1e-5  # Richardson extrapolation removes the O(h^2) truncation term
    fd = (4 * central(h) - central(2 * h)) / 3
    assert abs(fd - 2 * np.real(np.vdot(g, delta))) <= 1e-6 * abs(fd)


def test_subpixel_noise_free_truth_is_the_minimum():
    # the generator's intensities (its own numpy shift) equal the oracle's per-position model;
    # at psi_true with eps = 0 the gradient vanishes and F = F_min = sum(d - d log d)
    prob = _subpx(noise=False)
    pos_i, probes = oracle.subpixel_probes(prob.probe, prob.pos)
    u = oracle.forward(prob.psi_true, probes, pos_i)
    a = np.abs(u) ** 2
    assert np.linalg.norm(prob.d - a) <= 1e-6 * np.linalg.norm(a)
    d_exact = a.astype(np.float32)
    g, F = oracle.gradient(prob.psi_true, probes, pos_i, d_exact, eps=0.0)
    gscale = np.linalg.norm(oracle.adjoint(u, probes, pos_i, (prob.H, prob.W)))
    assert np.linalg.norm(g) <= 1e-6 * gscale  # float32 rounding of d only
    dd = d_exact.astype(np.float64)
    Fmin = float(np.sum(np.where(dd > 0, dd - dd * np.log(np.where(dd > 0, dd, 1)), 0.0)))
    assert F == pytest.approx(Fmin, rel=1e-7)


def test_subpixel_cg_decreases_monotonically():
    prob = _subpx()
    pos_i, probes = oracle.subpixel_probes(prob.probe, prob.pos)
    out = oracle.cg_solve(prob.psi0(), probes, pos_i, prob.d, 6)
    F = out["F"]
    assert out["iters_done"] == 6
    assert np.all(np.diff(F) <= 0)
    g = out["gamma"]
    k = np.log2(g)
    assert np.allclose(k, np.round(k))  # gamma = 2^-k


def test_per_position_probes_against_the_dense_restatement():
    """One probe per position ([K][P][P], the sub-pixel path): G, G^H and grad F equal the
    dense restatement whose k-th block uses the k-th probe (catches a probe stride that
    stays at the first position or advances by the wrong amount)."""
    from tests.brute import Brute

    rng = np.random.default_rng(40)
    H, W, P, K = 10, 9, 4, 6
    pos = np.stack([rng.integers(0, H - P + 1, K), rng.integers(0, W - P + 1, K)], 1).astype(np.int32)
    pos[1] = pos[0]  # two positions on one window, with different probes
    probes = rng.standard_normal((K, P, P)) + 1j * rng.standard_normal((K, P, P))
    psi = rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))
    y = rng.standard_normal((K, P, P)) + 1j * rng.standard_normal((K, P, P))
    b0 = Brute(H, W, P, probes, pos, np.ones(K * P * P), 0)

    def rel(a, b):
        return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))

    assert rel(oracle.forward(psi, probes, pos), b0.G @ psi.ravel()) <= 1e-13
    assert rel(oracle.adjoint(y, probes, pos, (H, W)), b0.G.conj().T @ y.ravel()) <= 1e-13
    d = rng.poisson(np.abs(b0.G @ psi.ravel()) ** 2).astype(np.float32)
    b = Brute(H, W, P, probes, pos, d, 0.1)
    g, F = oracle.gradient(psi, probes, pos, d.reshape(K, P, P), eps=0.1)
    assert F == pytest.approx(b.objective(psi), rel=1e-12)
    assert rel(g, b.gradient(psi)) <= 1e-12


def test_per_position_probes_cg_against_the_dense_restatement():
    """Four CG iterations with one probe per position (fractional positions turned into
    windows and shifted probes by the oracle) equal the dense restatement's: F, steps,
    trials, Dai-Yuan coefficients and the iterate."""
    from tests.brute import Brute

    rng = np.random.default_rng(41)
    H, W, P, K = 12, 11, 4, 8
    fpos = np.stack([rng.uniform(0, H - P, K), rng.uniform(0, W - P, K)], 1)
    pos_i, probes = oracle.subpixel_probes(3.0 * (rng.standard_normal((P, P)) + 1j * rng.standard_normal((P, P))),
                                           fpos)
    psi_true = (0.8 + 0.2 * rng.random((H, W))) * np.exp(1j * rng.uniform(0, np.pi / 2, (H, W)))
    b0 = Brute(H, W, P, probes, pos_i, np.ones(K * P * P), 0)
    d = rng.poisson(np.abs(b0.G @ psi_true.ravel()) ** 2).astype(np.float32)
    b = Brute(H, W, P, probes, pos_i, d, 0.1)
    psi0 = np.ones((H, W), complex)
    want = b.cg(psi0, 4)
    got = oracle.cg_solve(psi0, probes, pos_i, d.reshape(K, P, P), 4, oracle.OrcOpts(eps=0.1))
    assert got["status"] == oracle.ORC_OK
    np.testing.assert_allclose(got["F"], want["F"], rtol=1e-11)
    np.testing.assert_array_equal(got["gamma"], want["gamma"])
    np.testing.assert_array_equal(got["halvings"], want["halvings"])
    np.testing.assert_allclose(got["alpha"], want["alpha"], rtol=1e-9, atol=1e-12)
    assert np.linalg.norm(got["psi"] - want["psi"]) <= 1e-10 * np.linalg.norm(want["psi"])
