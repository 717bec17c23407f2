"""Scatter-add with the per-pattern results fetched by tensor copies against the per-thread
load form: the same values added in the same order (the copies add exact zeros outside a
pattern), so gradients, objectives and CG steps agree bit for bit."""
import numpy as np
import pytest

from paper_2106_07575_gb300 import pty, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def ctx_for(p, tma):
    o = pty.default_opts()
    if not tma:
        o.flags |= 16
    return pty.Context(dev(p.probe), dev(p.pos), dev(p.d), p.H, p.W, o)


PROBLEMS = {
    "small": lambda: synth.small_problem(seed=0),
    "mid": lambda: synth.small_problem(H=512, W=512, P=128, n=27, step=14, jitter=2, peak=1e5, seed=4),
    "p256": lambda: synth.small_problem(H=640, W=640, P=256, n=5, step=80, jitter=2, peak=1e6, seed=24),
}


@pytest.mark.parametrize("name", ["small", "mid", "p256"])
def test_gradient_and_steps_equal_per_thread_form(name):
    p = PROBLEMS[name]()
    rng = np.random.default_rng(7)
    psi = dev((p.psi0() * (1 + 0.01 * rng.standard_normal(p.psi0().shape))).astype(np.complex64))
    out = {}
    for tma in (True, False):
        ctx = ctx_for(p, tma)
        g = torch.empty_like(psi)
        F = ctx.gradient(psi, g)
        x = dev(p.psi0())
        st, rep = ctx.cg_solve(x, 6)
        assert st == pty.PTY_OK
        out[tma] = (g.cpu().numpy(), F, rep, x.cpu().numpy())
        ctx.close()
    (g1, F1, r1, x1), (g0, F0, r0, x0) = out[True], out[False]
    assert np.array_equal(g1, g0)
    assert F1 == F0
    assert list(r1["halvings"]) == list(r0["halvings"])
    assert np.array_equal(r1["F"], r0["F"])
    assert np.array_equal(x1, x0)


def test_adjoint_equal_per_thread_form():
    p = PROBLEMS["small"]()
    rng = np.random.default_rng(8)
    y = (rng.standard_normal((p.pos.shape[0], p.P, p.P)) + 1j * rng.standard_normal((p.pos.shape[0], p.P, p.P)))
    y = dev(y.astype(np.complex64))
    res = []
    for tma in (True, False):
        ctx = ctx_for(p, tma)
        x = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
        ctx.adjoint(y, x)
        res.append(x.cpu().numpy())
        ctx.close()
    assert np.array_equal(res[0], res[1])
