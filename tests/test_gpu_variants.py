"""GPU parity of the method's options against the FP64 oracle, through the C ABI:
the least-squares estimator on amplitudes, gradient descent with a constant step (Eq. 4)
and the warm-started line search (Eq. 7 with the previous accepted step as the first
trial).  Tolerances as for the plain method: gradient relative L2 <= 1e-5, objective per
iteration relative <= 1e-4, trial counts exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty, synth  # noqa: E402

GRAD_TOL = 1e-5
OBJ_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def opts(**kw):
    o = pty.default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def make_ctx(p, o=None):
    return pty.Context(dev(p.probe), dev(p.pos), dev(p.d), p.H, p.W, o,
                       stream=torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module")
def small():
    return synth.small_problem()


@pytest.fixture(scope="module")
def mid128():
    return synth.small_problem(H=384, W=352, P=128, n=10, step=22, jitter=2, peak=1e5, seed=21, niter=3,
                               name="mid")


@pytest.fixture(scope="module")
def p256():
    """P = 256 (the cluster form of the pattern passes): 640^2 object, 5 x 5 raster, peak 1e6."""
    return synth.small_problem(H=640, W=640, P=256, n=5, step=80, jitter=2, peak=1e6, seed=23, niter=2,
                               name="p256")


def random_object(p, seed):
    rng = np.random.default_rng(seed)
    return (p.psi_true * (1 + 0.05 * (rng.standard_normal((p.H, p.W)) + 1j * rng.standard_normal((p.H, p.W))))
            ).astype(np.complex64)


# ------------------------------------------------------------------------------- LS estimator
@pytest.mark.parametrize("which", ["small", "mid128", "p256"])
def test_ls_estimator_gradient_parity(orc, request, which):
    p = request.getfixturevalue(which)
    ctx = make_ctx(p, opts(estimator=pty.EST_LS))
    for seed in (1, 2):
        psi = random_object(p, seed) if seed == 1 else p.psi0()
        g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
        F = ctx.gradient(dev(psi), g)
        gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, nthreads=0, est=orc.EST_LS)
        e = rel(g.cpu().numpy(), gw)
        print(f"LS estimator ({which}, {'perturbed truth' if seed == 1 else 'ones'}): gradient rel L2 {e:.2e}, "
              f"objective rel {abs(F - Fw) / abs(Fw):.2e}")
        assert e <= GRAD_TOL
        assert abs(F - Fw) <= OBJ_TOL * abs(Fw)


@pytest.mark.parametrize("which", ["small", "mid128", "p256"])
def test_ls_estimator_cg_parity(orc, request, which):
    p = request.getfixturevalue(which)
    n = {"small": 10, "mid128": 4, "p256": 3}[which]
    ctx = make_ctx(p, opts(estimator=pty.EST_LS))
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, n)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, n, orc.OrcOpts(est=orc.EST_LS), nthreads=0)
    assert st == pty.PTY_OK and want["status"] == orc.ORC_OK
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print(f"LS estimator CG ({which}): objective rel", " ".join(f"{x:.1e}" for x in relF),
          "trials", list(rep["halvings"]), list(want["halvings"]))
    assert np.all(relF <= OBJ_TOL)
    assert list(rep["halvings"]) == list(want["halvings"])
    np.testing.assert_array_equal(rep["gamma"], want["gamma"])
    assert rel(psi.cpu().numpy(), want["psi"]) <= 1e-3


def test_ls_estimator_batched_views_equal_single(small):
    """Two views in one batched context give the single-view results of the LS estimator."""
    p = small
    q = synth.small_problem(H=224, W=192, P=64, n=12, step=10, jitter=1, peak=1e4, seed=44)
    o = opts(estimator=pty.EST_LS)
    stream = torch.cuda.current_stream().cuda_stream
    b = pty.BatchContext(dev(p.probe), [(p.H, p.W, dev(p.pos), p.d), (q.H, q.W, dev(q.pos), q.d)], o, stream=stream)
    xs = [dev(p.psi0()), dev(q.psi0())]
    st, reps = b.cg_solve(xs, 3)
    for prob, x, r in zip((p, q), xs, reps):
        # the batch shares the first view's probe: the single-view solve uses it too
        c = pty.Context(dev(p.probe), dev(prob.pos), dev(prob.d), prob.H, prob.W, o, stream=stream)
        y = dev(prob.psi0())
        _, r1 = c.cg_solve(y, 3)
        assert list(r["halvings"]) == list(r1["halvings"])
        assert np.all(np.abs(r["F"] - r1["F"]) <= 1e-6 * np.abs(r1["F"]))


# ------------------------------------------------------------------------------- GD (Eq. 4)
@pytest.mark.parametrize("est", ["ml", "ls"])
def test_gd_parity(orc, small, est):
    p = small
    e = orc.EST_LS if est == "ls" else orc.EST_ML
    # a constant step half the first accepted CG step: a descent step for this problem
    step = 0.5 * orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 1, orc.OrcOpts(est=e), nthreads=0)["gamma"][0]
    ctx = make_ctx(p, opts(estimator=e, solver=pty.SOLVER_GD, gd_step=step))
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, 10)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, 10, orc.OrcOpts(est=e, solver=orc.SOLVER_GD, gd_step=step),
                        nthreads=0)
    assert st == pty.PTY_OK and rep["iters_done"] == 10
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print(f"GD ({est}, step {step:.3g}): objective rel", " ".join(f"{x:.1e}" for x in relF))
    assert len(rep["F"]) == 11 and np.all(relF <= OBJ_TOL)
    assert np.all(rep["gamma"] == step) and np.all(rep["halvings"] == 0) and np.all(rep["alpha"] == 0)
    assert np.all(np.diff(rep["F"]) < 0)
    e_psi = rel(psi.cpu().numpy(), want["psi"])
    print(f"GD ({est}) psi_10 rel L2 vs FP64: {e_psi:.2e}")
    assert e_psi <= 1e-3  # iterate error after 10 FP32 iterations (reported; no stated tolerance)


def test_gd_continues_across_calls(small):
    """5 + 5 iterations equal 10 (the constant step has no state to restart)."""
    p = small
    o = opts(solver=pty.SOLVER_GD, gd_step=1e-4)
    a = dev(p.psi0())
    make_ctx(p, o).cg_solve(a, 10)
    c = make_ctx(p, o)
    b = dev(p.psi0())
    c.cg_solve(b, 5)
    c.cg_solve(b, 5)
    assert torch.equal(a, b)


# ------------------------------------------------------------------------------- warm start
@pytest.mark.parametrize("which", ["small", "mid128", "p256"])
def test_warm_start_parity(orc, request, which):
    p = request.getfixturevalue(which)
    n = {"small": 10, "mid128": 5, "p256": 3}[which]
    ctx = make_ctx(p, opts(ls_warm=1))
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, n)
    want = orc.cg_solve(p.psi0(), p.probe, p.pos, p.d, n, orc.OrcOpts(warm=True), nthreads=0)
    relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
    print(f"warm start ({which}): objective rel", " ".join(f"{x:.1e}" for x in relF),
          "trials", list(rep["halvings"]), list(want["halvings"]))
    assert st == pty.PTY_OK
    assert list(rep["halvings"]) == list(want["halvings"])
    np.testing.assert_array_equal(rep["gamma"], want["gamma"])
    assert np.all(relF <= OBJ_TOL)
    # the iterate has no stated tolerance: its error is reported plain and weighted by the
    # illumination map D = sum_k |p|^2 (where the data fix psi).  At P = 256, peak 1e6 the FP32
    # iterate departs from FP64 by about 6x per iteration with or without the warm start
    # (2.6e-6, 1.7e-4, 1.1e-3 after 1, 2, 3 iterations, same steps and trials): the start's
    # gradient differs by 1.3e-5 and the CG directions amplify it.  The bounds only catch a
    # broken update.
    D = np.real(orc.QH(np.ascontiguousarray(np.broadcast_to(p.probe, (p.K, p.P, p.P))), p.probe, p.pos, (p.H, p.W)))
    x = psi.cpu().numpy()
    e_plain = rel(x, want["psi"])
    e_w = rel(np.sqrt(D) * x, np.sqrt(D) * want["psi"])
    print(f"warm start ({which}): iterate rel L2 {e_plain:.2e}, illumination-weighted {e_w:.2e}")
    bound = 1e-2 if which == "p256" else 1e-3
    assert e_w <= bound and e_plain <= bound


@pytest.mark.parametrize("L", [0, 8])
def test_warm_start_window_does_not_change_the_step(small, L):
    p = small
    base = make_ctx(p, opts(ls_warm=1, ls_window=4))
    a = dev(p.psi0())
    _, ra = base.cg_solve(a, 6)
    c = make_ctx(p, opts(ls_warm=1, ls_window=L))
    b = dev(p.psi0())
    _, rb = c.cg_solve(b, 6)
    assert list(ra["halvings"]) == list(rb["halvings"]) and torch.equal(a, b)


def test_warm_start_stall_counts_its_own_trials(small):
    p = small
    ctx = make_ctx(p, opts(ls_warm=1, max_halvings=3, gamma0=1e12, ls_window=4))
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, 2)
    assert st == pty.PTY_STALLED and rep["halvings"][0] == 3


# ------------------------------------------------------------------------------- options
def test_option_combinations_rejected(small):
    p = small
    for o, code in ((opts(estimator=pty.EST_LS, dft=1), pty.PTY_ERR_UNSUPPORTED),
                    (opts(solver=pty.SOLVER_GD, gd_step=1e-3, dft=1), pty.PTY_ERR_UNSUPPORTED),
                    (opts(ls_warm=1, dft=1), pty.PTY_ERR_UNSUPPORTED),
                    (opts(solver=pty.SOLVER_GD, gd_step=0.0), pty.PTY_ERR_ARG),
                    (opts(solver=pty.SOLVER_GD, gd_step=1e-3, ls_warm=1), pty.PTY_ERR_ARG),
                    (opts(estimator=2), pty.PTY_ERR_ARG)):
        with pytest.raises(pty.PtyError) as e:
            make_ctx(p, o)
        assert e.value.status == code
