"""The seeded input generators against the workload recipe (CPU).

Phantom value ranges, probe shape, raster and spiral geometry, the count scaling of the
detector model, view sizes and seeding: the properties the parity tests and the bench rely
on when they stand in for the paper's measured data."""
import math

import numpy as np
import pytest

from paper_2106_07575_gb300 import synth


def test_same_seed_same_inputs_other_seed_other_inputs():
    a, b, c = synth.small_problem(seed=0), synth.small_problem(seed=0), synth.small_problem(seed=1)
    for x, y in ((a.psi_true, b.psi_true), (a.pos, b.pos), (a.d, b.d), (a.probe, b.probe)):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.psi_true, c.psi_true)
    assert not np.array_equal(a.d, c.d)


def test_ellipse_phantom_ranges():
    psi = synth.ellipse_phantom(256, 256, np.random.default_rng(0))
    amp, ph = np.abs(psi).astype(np.float64), np.angle(psi).astype(np.float64)
    bg = np.isclose(amp, 1.0, atol=1e-6) & np.isclose(ph, 0.0, atol=1e-6)
    assert 0.05 < bg.mean() < 0.95  # background and ellipses both present
    assert np.all((amp >= 0.8 - 1e-6) & (amp <= 1.0 + 1e-6))
    assert np.all((ph >= -1e-6) & (ph <= math.pi / 2 + 1e-6))
    assert psi.dtype == np.complex64


def test_voronoi_phantom_ranges():
    psi = synth.voronoi_phantom(128, 128, np.random.default_rng(3), n_cells=40)
    amp, ph = np.abs(psi), np.angle(psi)
    assert np.all((amp >= 0.8 - 1e-6) & (amp <= 1.0 + 1e-6))
    assert np.all((ph >= -1e-6) & (ph <= math.pi / 2 + 1e-6))
    assert len(np.unique(psi)) <= 40


@pytest.mark.parametrize("P", [64, 128, 256])
def test_probe_gaussian_amplitude_quadratic_phase(P):
    p = synth.gaussian_probe(P).astype(np.complex128)
    sigma, c = 3.0 * P / 16.0, (P - 1) / 2.0
    for y, x in ((0, 0), (P // 2, P // 2), (P // 4, 3 * P // 4), (P - 1, 5)):
        r2 = (y - c) ** 2 + (x - c) ** 2
        assert abs(abs(p[y, x]) - math.exp(-r2 / (2 * sigma**2))) < 1e-6
        want = 2.0 * r2 / sigma**2  # kappa = 2 rad
        assert abs(np.angle(p[y, x] * np.exp(-1j * want))) < 1e-5
    # symmetric about the centre (P-1)/2 in both axes
    assert np.allclose(p, p[::-1, :], atol=1e-6) and np.allclose(p, p[:, ::-1], atol=1e-6)


def test_raster_geometry():
    H, P, n, step, j = 1024, 128, 60, 14, 2
    pos = synth.raster_positions(H, H, P, n, step, j, np.random.default_rng(0))
    assert pos.shape == (n * n, 2) and pos.dtype == np.int32
    assert pos.min() >= 0 and pos.max() <= H - P
    ext = (n - 1) * step + P
    o = (H - ext) // 2
    grid = np.stack(np.meshgrid(np.arange(n) * step + o, np.arange(n) * step + o, indexing="ij"), -1).reshape(-1, 2)
    dev = pos - grid
    assert np.abs(dev).max() <= j and len(np.unique(dev)) == 2 * j + 1  # uniform integer jitter
    # centred: the extent's margins differ by at most one pixel
    assert abs((H - ext) - 2 * o) <= 1


def test_spiral_geometry():
    from scipy.spatial import cKDTree

    H, P, K = 2048, 256, 10000
    pos = synth.spiral_positions(H, H, P, K, 8.94, 2, np.random.default_rng(2))
    assert pos.shape == (K, 2)
    assert pos.min() >= 0 and pos.max() <= H - P
    # r_max + jitter within the half-extent: no position was clipped
    raw = synth.spiral_positions(H, H, P, K, 8.94, 0, np.random.default_rng(2))
    c = (H - P) / 2.0
    assert np.hypot(raw[:, 0] - c, raw[:, 1] - c).max() + 2 <= c + 1
    # mean nearest-neighbour spacing: 14.8 px without the jitter, 13.6 px with it (the
    # 20 px of the paper's spiral do not fit 10,000 points into the 2048^2 object)
    for q, lo, hi in ((raw, 14.5, 15.2), (pos, 13.3, 13.9)):
        nn = cKDTree(q.astype(np.float64)).query(q.astype(np.float64), k=2)[0][:, 1]
        assert lo < nn.mean() < hi


def test_counts_scaled_to_peak_and_poisson():
    rng = np.random.default_rng(0)
    psi = synth.ellipse_phantom(128, 128, rng)
    pos = synth.raster_positions(128, 128, 64, 5, 12, 1, rng)
    probe, lam = synth.simulate_counts(psi, synth.gaussian_probe(64), pos, 1e4, None, noise=False)
    assert abs(lam.max() - 1e4) <= 1e4 * 1e-6
    # the scaled probe predicts the counts: |orthonormal FFT(probe * patch)|^2 = lam
    k = 3
    r, c = pos[k]
    f = np.fft.fft2(probe.astype(np.complex128) * psi[r:r + 64, c:c + 64], norm="ortho")
    assert np.allclose(np.abs(f) ** 2, lam[k], rtol=1e-5, atol=1e-3)
    _, d = synth.simulate_counts(psi, synth.gaussian_probe(64), pos, 1e4, np.random.default_rng(1))
    assert np.all(d >= 0) and np.array_equal(d, np.round(d))
    # Poisson: mean and variance of (d - lam) / sqrt(lam) over bright pixels near 0 and 1
    m = lam > 50
    z = (d[m] - lam[m]) / np.sqrt(lam[m])
    assert abs(z.mean()) < 0.05 and abs(z.var() - 1) < 0.1


def test_small_workload_recipe():
    p = synth.small_problem(seed=0)
    assert (p.H, p.W, p.P, p.K) == (256, 256, 64, 225)
    assert p.d.shape == (225, 64, 64) and p.d.dtype == np.float32
    assert 0.01 < np.count_nonzero(p.d) / p.d.size < 0.9


def test_view_sizes_and_rasters():
    sizes = synth.view_sizes(64, seed=3)
    assert len(sizes) == 64 and set(sizes) <= set(range(512, 2049, 128))
    assert sizes == synth.view_sizes(64, seed=3)
    probe, views = synth.view_batch(n_views=2, seed=40, sizes=[256, 320], P=64, step=12, jitter=1, peak=1e4)
    for N, (psi, pos, d) in zip((256, 320), views):
        k = (N - 64 - 4) // 12 + 1
        assert psi.shape == (N, N) and pos.shape == (k * k, 2) and d.shape == (k * k, 64, 64)
        assert pos.min() >= 0 and pos.max() <= N - 64


def test_production_workload_recipe():
    """1024^2 object, 128^2 probe, 60 x 60 raster: 12.2 % of the detector pixels hold counts
    and the brightest holds about the 1e5 counts of the scaling (Poisson)."""
    p = synth.production_problem()
    assert (p.H, p.W, p.P, p.K) == (1024, 1024, 128, 3600)
    frac = np.count_nonzero(p.d) / p.d.size
    assert 0.120 < frac < 0.125
    assert abs(p.d.max() - 1e5) < 6 * math.sqrt(1e5)
