"""Certified skip of leading line-search trials (adaptive search): the lower bound of the
objective change (Jensen's inequality on the concave log, per pattern) may only reject
trials that the plain backtracking search rejects too, so the accepted steps, trial counts
and objective histories equal those of the search without the certificate, bit for bit."""
import numpy as np
import pytest

from paper_2106_07575_gb300 import pty, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(p, niter, cert, linear=True):
    o = pty.default_opts()
    if not cert:
        o.flags |= 4
    if not linear:
        o.flags |= 2
    ctx = pty.Context(dev(p.probe), dev(p.pos), dev(p.d), p.H, p.W, o)
    x = dev(p.psi0())
    certified = []
    reps = []
    for _ in range(niter):  # one iteration per call: read the certificate of each
        st, rep = ctx.cg_solve(x, 1)
        assert st == pty.PTY_OK
        reps.append(rep)
        certified.append(pty.pty_selftest_ls_certified(ctx.ctx, 0))
    ctx.close()
    F = np.array([reps[0]["F"][0]] + [r["F"][1] for r in reps])
    gam = np.array([r["gamma"][0] for r in reps])
    halv = [int(r["halvings"][0]) for r in reps]
    return F, gam, halv, certified, x.cpu().numpy()


@pytest.mark.parametrize("name", ["small", "mid"])
def test_certificate_keeps_every_decision(name):
    if name == "small":
        p = synth.small_problem(seed=0)
    else:  # 512^2 object, 128^2 probe, 27 x 27 raster: many trials per search, as in production
        p = synth.small_problem(H=512, W=512, P=128, n=27, step=14, jitter=2, peak=1e5, seed=4)
    n = 12
    Fc, gc, hc, kc, xc = run(p, n, True)
    Fn, gn, hn, kn, xn = run(p, n, False)
    print(f"{name}: trials {hc}, certified {kc}")
    assert kn == [0] * n
    assert hc == hn
    assert np.array_equal(gc, gn)
    assert np.array_equal(Fc, Fn)
    assert np.array_equal(xc, xn)
    # the certificate never rejects the accepted trial, and it does engage
    assert all(k < h for k, h in zip(kc, hc))
    assert sum(kc) > 0


def test_certificate_with_full_form_grad():
    """Every GRAD pass in the full form (no kept model values): same decisions."""
    p = synth.small_problem(seed=1)
    Fc, gc, hc, kc, _ = run(p, 6, True, linear=False)
    Fn, gn, hn, _, _ = run(p, 6, False, linear=False)
    assert hc == hn and np.array_equal(gc, gn) and np.array_equal(Fc, Fn)
