"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same inputs.

Tolerances (from the workload statement): forward and gradient relative L2 <= 1e-5,
objective per iteration relative <= 1e-4 over the first 10 CG iterations.  Integer
decisions (line-search trial counts) must agree exactly.  Each test prints the error
against FP64 so the log states it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty, synth  # noqa: E402

FWD_TOL = 1e-5
GRAD_TOL = 1e-5
OBJ_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_ctx(p, opts=None, host_data=False):
    data = p.d if host_data else dev(p.d)
    ctx = pty.Context(dev(p.probe), dev(p.pos), data, p.H, p.W, opts,
                      stream=torch.cuda.current_stream().cuda_stream)
    return ctx


@pytest.fixture(scope="module")
def small():
    return synth.small_problem()


@pytest.fixture(scope="module")
def production():
    return synth.production_problem()


def random_object(p, seed):
    rng = np.random.default_rng(seed)
    return (p.psi_true * (1 + 0.05 * (rng.standard_normal((p.H, p.W)) + 1j * rng.standard_normal((p.H, p.W))))
            ).astype(np.complex64)


# ------------------------------------------------------------------------------- forward
def test_forward_parity_small(orc, small):
    p = small
    ctx = make_ctx(p)
    psi = random_object(p, 1)
    out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    want = orc.forward(psi, p.probe, p.pos, nthreads=0)
    e = rel(out.cpu().numpy(), want)
    print(f"forward rel L2 vs FP64: {e:.3e}")
    assert e <= FWD_TOL


def test_forward_host_pointers_match_device(small):
    p = small
    ctx = make_ctx(p, host_data=True)
    psi = random_object(p, 2)
    out_h = np.empty((p.K, p.P, p.P), np.complex64)
    ctx.forward(psi, out_h)
    out_d = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out_d)
    assert np.array_equal(out_h, out_d.cpu().numpy())


# ------------------------------------------------------------------------------- adjoint
def test_adjoint_parity_and_dot_test(orc, small):
    p = small
    ctx = make_ctx(p)
    rng = np.random.default_rng(3)
    y = (rng.standard_normal((p.K, p.P, p.P)) + 1j * rng.standard_normal((p.K, p.P, p.P))).astype(np.complex64)
    x = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    ctx.adjoint(dev(y), x)
    xg = x.cpu().numpy()
    want = orc.adjoint(y, p.probe, p.pos, (p.H, p.W), nthreads=0)
    e = rel(xg, want)
    print(f"adjoint rel L2 vs FP64: {e:.3e}")
    assert e <= GRAD_TOL
    # <G x, y> = <x, G^H y> with both operators on the GPU
    xx = random_object(p, 4)
    gx = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(xx), gx)
    lhs = np.vdot(gx.cpu().numpy().astype(np.complex128), y.astype(np.complex128))
    rhs = np.vdot(xx.astype(np.complex128), xg.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


# ------------------------------------------------------------------------------- gradient
def test_gradient_parity_small(orc, small):
    p = small
    ctx = make_ctx(p)
    psi = random_object(p, 5)
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0)
    e = rel(g.cpu().numpy(), gw)
    print(f"gradient rel L2 vs FP64: {e:.3e}; objective rel {abs(F - Fw) / abs(Fw):.3e}")
    assert e <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)
    # bitwise reproducible (fixed-order scatter and reductions)
    g2 = torch.empty_like(g)
    F2 = ctx.gradient(dev(psi), g2)
    assert F2 == F and torch.equal(g, g2)


def test_gradient_at_uniform_start(orc, small):
    """The CG start point (uniform ones), far from the data: large residuals."""
    p = small
    ctx = make_ctx(p)
    psi = p.psi0()
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0)
    assert rel(g.cpu().numpy(), gw) <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)


# ------------------------------------------------------------------------------- CG
def _cg_compare(orc, p, niter, opts=None, gpu_opts=None):
    ctx = make_ctx(p, gpu_opts)
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, niter)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, niter, opts, nthreads=0)
    return ctx, st, rep, want, psi


def test_cg_ten_iterations_small(orc, small):
    p = small
    ctx, st, rep, want, psi = _cg_compare(orc, p, 10)
    assert st == pty.PTY_OK and rep["iters_done"] == 10
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print("per-iteration objective rel err vs FP64:", " ".join(f"{x:.2e}" for x in relF))
    print("trials gpu", list(rep["halvings"]), "oracle", list(want["halvings"]))
    assert np.all(relF <= OBJ_TOL)
    assert list(rep["halvings"]) == list(want["halvings"])
    np.testing.assert_array_equal(rep["gamma"], want["gamma"])
    np.testing.assert_allclose(rep["alpha"], want["alpha"], rtol=1e-3, atol=1e-9)
    e = rel(psi.cpu().numpy(), want["psi"])
    print(f"psi_10 rel L2 vs FP64: {e:.3e}")
    assert e <= 1e-3  # iterate error after 10 FP32 iterations (reported; no stated tolerance)


def test_cg_window_size_does_not_change_the_step(small):
    p = small
    reps = {}
    for L in (4, 32, 0):
        o = pty.default_opts()
        o.ls_window = L
        ctx = make_ctx(p, o)
        psi = dev(p.psi0())
        st, rep = ctx.cg_solve(psi, 4)
        reps[L] = (rep, psi.cpu().numpy())
    for L in (32, 0):
        assert list(reps[4][0]["halvings"]) == list(reps[L][0]["halvings"])
        np.testing.assert_array_equal(reps[4][0]["gamma"], reps[L][0]["gamma"])
        assert np.array_equal(reps[4][1], reps[L][1])


def test_cg_deterministic_and_resumable(small):
    """Two runs are bit-identical; 3 + checkpoint + 3 equals 6 iterations bit for bit."""
    p = small
    ctx = make_ctx(p)
    a = dev(p.psi0())
    ctx.cg_solve(a, 6)
    ctx.cg_reset()
    b = dev(p.psi0())
    ctx.cg_solve(b, 3)
    blob = ctx.state_save()
    ctx2 = make_ctx(p)
    ctx2.state_load(blob)
    ctx2.cg_solve(b, 3)
    assert torch.equal(a, b)
    ctx.cg_reset()
    c = dev(p.psi0())
    ctx.cg_solve(c, 6)
    assert torch.equal(a, c)


def test_cg_host_psi(small):
    p = small
    ctx = make_ctx(p)
    h = p.psi0()
    ctx.cg_solve(h, 2)
    ctx.cg_reset()
    d = dev(p.psi0())
    ctx.cg_solve(d, 2)
    assert np.array_equal(h, d.cpu().numpy())


def test_cg_stall_is_reported(small):
    p = small
    o = pty.default_opts()
    o.gamma0 = 1e12
    o.max_halvings = 4
    o.ls_window = 4
    ctx = make_ctx(p, o)
    psi = dev(p.psi0())
    before = psi.clone()
    st, rep = ctx.cg_solve(psi, 3)
    assert st == pty.PTY_STALLED and rep["iters_done"] == 0
    assert torch.equal(psi, before)
    assert rep["halvings"][0] == 4


# ------------------------------------------------------------------------------- edge cases
def test_edge_positions_duplicates_and_ragged_object(orc):
    """Ragged object (not a multiple of the scatter tile), corners, duplicates, K=1-like sparse scan."""
    rng = np.random.default_rng(7)
    H, W, P = 200, 131, 64
    psi_true = synth.ellipse_phantom(H, W, rng)
    pos = np.array([[0, 0], [H - P, W - P], [0, W - P], [H - P, 0], [37, 41], [37, 41], [100, 3]], np.int32)
    probe, d = synth.simulate_counts(psi_true, synth.gaussian_probe(P), pos, 1e4, rng)
    d[2] = 0.0  # a pattern with no counts at all
    p = synth.Problem("edge", psi_true, probe, pos, d, 3)
    ctx = make_ctx(p)
    psi = random_object(p, 8)
    g = torch.empty((H, W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, probe, pos, d)
    assert rel(g.cpu().numpy(), gw) <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)
    out = torch.empty((len(pos), P, P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    assert rel(out.cpu().numpy(), orc.forward(psi, probe, pos)) <= FWD_TOL
    st, rep = ctx.cg_solve(dev(p.psi0()), 3)
    want = orc.cg_solve(p.psi0(), probe, pos, d, 3)
    assert list(rep["halvings"]) == list(want["halvings"])
    assert np.all(np.abs(rep["F"] - want["F"]) <= OBJ_TOL * np.abs(want["F"]))


def test_single_position(orc):
    rng = np.random.default_rng(9)
    psi_true = synth.ellipse_phantom(192, 160, rng)
    pos = np.array([[32, 17]], np.int32)
    probe, d = synth.simulate_counts(psi_true, synth.gaussian_probe(128), pos, 1e5, rng)
    p = synth.Problem("one", psi_true, probe, pos, d, 2)
    ctx = make_ctx(p)
    g = torch.empty((192, 160), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(p.psi0()), g)
    gw, Fw = orc.gradient(p.psi0(), probe, pos, d)
    assert rel(g.cpu().numpy(), gw) <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)


def test_nonfinite_data_rejected(small):
    p = small
    d = p.d.copy()
    d[3, 5, 7] = np.nan
    with pytest.raises(pty.PtyError) as e:
        pty.Context(dev(p.probe), dev(p.pos), dev(d), p.H, p.W)
    assert e.value.status == pty.PTY_ERR_NONFINITE
    d[3, 5, 7] = -1.0
    with pytest.raises(pty.PtyError) as e:
        pty.Context(dev(p.probe), dev(p.pos), dev(d), p.H, p.W)
    assert e.value.status == pty.PTY_ERR_NONFINITE


# ------------------------------------------------------------------------------- production size
def test_production_forward_sampled(orc, production):
    """1024^2 object, 128^2 probe, 3600 positions: forward checked on sampled patterns."""
    p = production
    ctx = make_ctx(p)
    psi = random_object(p, 10)
    out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    idx = np.random.default_rng(0).choice(p.K, 64, replace=False)
    want = orc.forward(psi, p.probe, p.pos[idx], nthreads=0)
    e = rel(out[torch.from_numpy(idx).cuda()].cpu().numpy(), want)
    print(f"production forward rel L2 (64 sampled patterns): {e:.3e}")
    assert e <= FWD_TOL


def test_production_gradient(orc, production):
    p = production
    ctx = make_ctx(p)
    psi = p.psi0()
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0)
    e = rel(g.cpu().numpy(), gw)
    print(f"production gradient rel L2: {e:.3e}, objective rel {abs(F - Fw) / abs(Fw):.3e}")
    assert e <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)


def test_production_cg_ten_iterations(orc, production):
    """Production size (1024^2, P = 128, K = 3600), the first 10 CG iterations of Algorithm 1:
    objective per iteration within 1e-4 of the FP64 oracle and identical trial counts."""
    p = production
    ctx, st, rep, want, psi = _cg_compare(orc, p, 10)
    assert st == pty.PTY_OK and rep["iters_done"] == 10
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print("production 10 iterations: objective rel", " ".join(f"{x:.1e}" for x in relF))
    print("trials gpu", list(rep["halvings"]), "oracle", list(want["halvings"]))
    assert np.all(relF <= OBJ_TOL)
    assert list(rep["halvings"]) == list(want["halvings"])
    np.testing.assert_array_equal(rep["gamma"], want["gamma"])
    e = rel(psi.cpu().numpy(), want["psi"])
    print(f"production psi_10 rel L2 vs FP64: {e:.3e}")
    assert e <= 1e-2  # reported: CG amplifies the FP32 rounding of the iterates (no stated tolerance)


def test_objective_sum_matches_fp64_sum_of_the_same_terms(production):
    """The objective's float-float reduction against an FP64 sum of the same per-pixel terms.

    u = G psi comes from the library's own forward pass (the DFT the gradient pass runs, same
    bits); the terms |u|^2 - d log(|u|^2 + eps) are formed from those FP32 values in FP64 and
    summed in FP64.  What remains is each term's FP32 rounding on the GPU and the reduction's
    error: bounded by 1e-6 of sum |terms|."""
    p = production
    ctx = make_ctx(p)
    psi = random_object(p, 12)
    out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    u = out.to(torch.complex128)
    d = torch.from_numpy(p.d).cuda().to(torch.float64)
    a = u.real ** 2 + u.imag ** 2
    terms = a - torch.where(d > 0, d * torch.log(a + 0.1), torch.zeros_like(a))
    F64 = float(terms.sum())
    mag = float(terms.abs().sum())
    F32 = float(terms.to(torch.float32).view(-1).cumsum(0, dtype=torch.float32)[-1])  # plain FP32 running sum
    print(f"objective: float-float {F:.10e}, FP64 sum of the same terms {F64:.10e}, |diff|/sum|terms| "
          f"{abs(F - F64) / mag:.2e} (plain FP32 running sum: {abs(F32 - F64) / mag:.2e})")
    assert abs(F - F64) <= 1e-6 * mag


def test_dai_yuan_sums_match_fp64_sums_of_the_same_vectors(production):
    """alpha of Eq. 6 from the float-float tile sums against FP64 sums of the same g vectors.

    With the linear form off every GRAD pass is the full one, so the g of the CG iteration is
    bit for bit pty_gradient's; alpha_1 = ||g_1||^2 / Re <eta_0, g_1 - g_0>, eta_0 = -g_0, is
    recomputed in FP64 from those FP32 vectors."""
    p = production
    o = pty.default_opts()
    o.flags = 2  # no linear form
    ctx = make_ctx(p, o)
    psi = dev(p.psi0())
    g0 = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    ctx.gradient(psi, g0)
    ctx.cg_solve(psi, 1)
    g1 = torch.empty_like(g0)
    ctx.gradient(psi, g1)
    st, rep = ctx.cg_solve(psi, 1)  # continues the CG state: its alpha is alpha_1
    a, b = g0.to(torch.complex128), g1.to(torch.complex128)
    num = float((b.real ** 2 + b.imag ** 2).sum())
    den = float(((-a).real * (b - a).real + (-a).imag * (b - a).imag).sum())
    alpha64 = num / den
    e = abs(rep["alpha"][0] - alpha64) / abs(alpha64)
    print(f"alpha_1: GPU {rep['alpha'][0]:.10e}, FP64 sums of the same vectors {alpha64:.10e}, rel {e:.2e}")
    assert e <= 1e-5


def test_production_cg_two_iterations(orc, production):
    p = production
    ctx, st, rep, want, psi = _cg_compare(orc, p, 2)
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print("production objective rel err:", relF, "trials", list(rep["halvings"]), list(want["halvings"]))
    assert np.all(relF <= OBJ_TOL)
    assert list(rep["halvings"]) == list(want["halvings"])


# ------------------------------------------------------------------------------- configurations
def _cfg_opts(idx):
    o = pty.default_opts()
    o.tile_config = idx
    return o


@pytest.fixture(scope="module")
def mid128():
    """A 128^2-probe problem small enough for the oracle: 384^2 object, 10 x 10 raster."""
    return synth.small_problem(H=384, W=352, P=128, n=10, step=22, jitter=2, peak=1e5, seed=21, niter=3,
                               name="mid")


@pytest.mark.parametrize("cfg", [0, 1, 2, 3])
def test_p128_configurations(orc, mid128, cfg):
    """One CTA per pattern (512 or 1024 threads) and clusters of 2 and 4 CTAs give oracle parity."""
    p = mid128
    ctx = make_ctx(p, _cfg_opts(cfg))
    psi = random_object(p, 30)
    out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    e_f = rel(out.cpu().numpy(), orc.forward(psi, p.probe, p.pos, nthreads=0))
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0)
    e_g = rel(g.cpu().numpy(), gw)
    print(f"P=128 config {cfg}: forward {e_f:.2e}, gradient {e_g:.2e}, objective {abs(F - Fw) / abs(Fw):.2e}")
    assert e_f <= FWD_TOL and e_g <= GRAD_TOL and abs(F - Fw) <= OBJ_TOL * abs(Fw)
    st, rep = ctx.cg_solve(dev(p.psi0()), 3)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 3, nthreads=0)
    assert list(rep["halvings"]) == list(want["halvings"])
    assert np.all(np.abs(rep["F"] - want["F"]) <= OBJ_TOL * np.abs(want["F"]))


@pytest.fixture(scope="module")
def small256():
    """256^2 probe: 640^2 object, 5 x 5 raster (step 80), peak 1e6."""
    return synth.small_problem(H=640, W=640, P=256, n=5, step=80, jitter=2, peak=1e6, seed=22, niter=2,
                               name="p256")


@pytest.mark.parametrize("cfg", [0, 1])
def test_p256_parity(orc, small256, cfg):
    """P = 256: the exit wave is shared by a cluster of 8 (or 4) CTAs."""
    p = small256
    ctx = make_ctx(p, _cfg_opts(cfg))
    psi = random_object(p, 31)
    out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
    ctx.forward(dev(psi), out)
    e_f = rel(out.cpu().numpy(), orc.forward(psi, p.probe, p.pos, nthreads=0))
    rng = np.random.default_rng(4)
    y = (rng.standard_normal((p.K, p.P, p.P)) + 1j * rng.standard_normal((p.K, p.P, p.P))).astype(np.complex64)
    x = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    ctx.adjoint(dev(y), x)
    e_a = rel(x.cpu().numpy(), orc.adjoint(y, p.probe, p.pos, (p.H, p.W), nthreads=0))
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0)
    e_g = rel(g.cpu().numpy(), gw)
    print(f"P=256 config {cfg}: forward {e_f:.2e}, adjoint {e_a:.2e}, gradient {e_g:.2e}, "
          f"objective {abs(F - Fw) / abs(Fw):.2e}")
    assert e_f <= FWD_TOL and e_a <= GRAD_TOL and e_g <= GRAD_TOL and abs(F - Fw) <= OBJ_TOL * abs(Fw)
    st, rep = ctx.cg_solve(dev(p.psi0()), 2)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 2, nthreads=0)
    print("P=256 trials", list(rep["halvings"]), list(want["halvings"]))
    assert list(rep["halvings"]) == list(want["halvings"])
    assert np.all(np.abs(rep["F"] - want["F"]) <= OBJ_TOL * np.abs(want["F"]))
