"""GPU parity of sub-pixel scan positions (pty_create_subpixel) against the FP64 oracle,
through the C ABI.  The oracle takes the same positions as integer windows plus one probe
per position moved by the Fourier shift theorem (oracle.subpixel_probes); the library
builds its own shifted probes on the device.  Tolerances as for the plain method: forward
and gradient relative L2 <= 1e-5, objective per iteration relative <= 1e-4 over 10 CG
iterations, trial counts exact.
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


def make_ctx(p, pos=None, o=None):
    pos = p.pos if pos is None else pos
    return pty.Context(dev(p.probe), dev(pos), dev(p.d), p.H, p.W, o, stream=torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module")
def small():
    return synth.subpixel_problem()


@pytest.fixture(scope="module")
def mid128():
    # several P = 128 tiles, ragged object edge, fractional positions up to the far edge
    return synth.subpixel_problem(H=384, W=352, P=128, n=10, step=22, jitter=2.0, peak=1e5, seed=31, niter=4)


@pytest.fixture(scope="module")
def p256():
    return synth.subpixel_problem(H=640, W=576, P=256, n=4, step=96, jitter=2.0, peak=1e6, seed=32, niter=2)


def oracle_probes(orc, p):
    return orc.subpixel_probes(p.probe, p.pos)


def random_object(p, seed):
    rng = np.random.default_rng(seed)
    return (p.psi_true * (1 + 0.05 * (rng.standard_normal((p.H, p.W)) + 1j * rng.standard_normal((p.H, p.W))))
            ).astype(np.complex64)


@pytest.mark.parametrize("which", ["small", "mid128", "p256"])
def test_subpixel_forward_parity(orc, request, which):
    p = request.getfixturevalue(which)
    pos_i, probes = oracle_probes(orc, p)
    ctx = make_ctx(p)
    for psi in (p.psi0(), random_object(p, 1)):
        out = torch.empty((p.K, p.P, p.P), dtype=torch.complex64, device="cuda")
        ctx.forward(dev(psi), out)
        want = orc.forward(psi, probes, pos_i, nthreads=0)
        e = rel(out.cpu().numpy(), want)
        print(f"sub-pixel forward ({which}): rel L2 {e:.2e}")
        assert e <= FWD_TOL
    ctx.close()


@pytest.mark.parametrize("which", ["small", "mid128", "p256"])
def test_subpixel_gradient_and_adjoint_parity(orc, request, which):
    p = request.getfixturevalue(which)
    pos_i, probes = oracle_probes(orc, p)
    ctx = make_ctx(p)
    psi = random_object(p, 2)
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    F = ctx.gradient(dev(psi), g)
    gw, Fw = orc.gradient(psi, probes, pos_i, p.d, nthreads=0)
    e = rel(g.cpu().numpy(), gw)
    print(f"sub-pixel gradient ({which}): rel L2 {e:.2e}, objective rel {abs(F - Fw) / abs(Fw):.2e}")
    assert e <= GRAD_TOL
    assert abs(F - Fw) <= OBJ_TOL * abs(Fw)
    rng = np.random.default_rng(3)
    y = (rng.standard_normal((p.K, p.P, p.P)) + 1j * rng.standard_normal((p.K, p.P, p.P))).astype(np.complex64)
    x = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    ctx.adjoint(dev(y), x)
    xw = orc.adjoint(y, probes, pos_i, (p.H, p.W), nthreads=0)
    assert rel(x.cpu().numpy(), xw) <= GRAD_TOL
    ctx.close()


@pytest.mark.parametrize("which,n", [("small", 10), ("mid128", 4), ("p256", 2)])
def test_subpixel_cg_parity(orc, request, which, n):
    p = request.getfixturevalue(which)
    pos_i, probes = oracle_probes(orc, p)
    ctx = make_ctx(p)
    psi = dev(p.psi0())
    st, rep = ctx.cg_solve(psi, n)
    want = orc.cg_solve(p.psi0(), probes, pos_i, p.d, n, nthreads=0)
    eF = np.max(np.abs(rep["F"] - want["F"]) / np.abs(want["F"]))
    print(f"sub-pixel CG ({which}, {n} iterations): objective max rel {eF:.2e}, trials {list(rep['halvings'])}")
    assert st == pty.PTY_OK and rep["iters_done"] == n
    assert list(rep["halvings"]) == list(want["halvings"])
    assert eF <= OBJ_TOL
    # the iterate has no stated tolerance: its error against FP64 is reported (plain and
    # weighted by the illumination map D = sum_k |p_k|^2, where the data fix psi), with a
    # coarse bound that only catches a broken update
    D = np.real(orc.QH(probes, probes, pos_i, (p.H, p.W)))
    x = psi.cpu().numpy()
    e_plain = rel(x, want["psi"])
    e_w = rel(np.sqrt(D) * x, np.sqrt(D) * want["psi"])
    print(f"sub-pixel CG ({which}): iterate rel L2 {e_plain:.2e}, illumination-weighted {e_w:.2e}")
    assert e_plain <= 1e-2
    ctx.close()


def test_integer_float_positions_match_pty_create(small):
    # positions with no fraction: the same probe, so the same results bit for bit
    p = small
    ipos = np.floor(p.pos).astype(np.int32)
    fctx = make_ctx(p, pos=ipos.astype(np.float32))
    ictx = make_ctx(p, pos=ipos)
    psi = p.psi0()
    g1 = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    g2 = torch.empty_like(g1)
    F1 = fctx.gradient(dev(psi), g1)
    F2 = ictx.gradient(dev(psi), g2)
    assert F1 == F2 and torch.equal(g1, g2)
    x1, x2 = dev(psi), dev(psi)
    _, r1 = fctx.cg_solve(x1, 3)
    _, r2 = ictx.cg_solve(x2, 3)
    assert np.array_equal(r1["F"], r2["F"]) and torch.equal(x1, x2)
    fctx.close()
    ictx.close()


def test_subpixel_argument_errors(small):
    p = small
    bad = p.pos.copy()
    bad[3, 0] = np.nan
    with pytest.raises(pty.PtyError) as e:
        make_ctx(p, pos=bad)
    assert e.value.status == pty.PTY_ERR_BOUNDS
    bad = p.pos.copy()
    bad[0, 1] = p.W - p.P + 0.5  # floor = W - P: the window still fits
    make_ctx(p, pos=bad).close()
    bad[0, 1] = p.W - p.P + 1.0
    with pytest.raises(pty.PtyError) as e:
        make_ctx(p, pos=bad)
    assert e.value.status == pty.PTY_ERR_BOUNDS
    bad[0, 1] = -0.25  # floor = -1
    with pytest.raises(pty.PtyError) as e:
        make_ctx(p, pos=bad)
    assert e.value.status == pty.PTY_ERR_BOUNDS
    o = pty.default_opts()
    o.dft = 1
    with pytest.raises(pty.PtyError) as e:
        make_ctx(p, o=o)
    assert e.value.status == pty.PTY_ERR_UNSUPPORTED
