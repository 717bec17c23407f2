"""The guard eps of the implemented objective F_eps = sum |u|^2 - d log(|u|^2 + eps): the
GPU's single-precision gradient and objective against the FP64 oracle at the library's
default eps = 0.1 counts and at eps = 1e-6, on the 256^2 / P = 64 and the 1024^2 / P = 128
workloads.  The paper's Eq. 2 and 3 carry no guard; with a small one the gradient at dark
detector pixels holding counts has sensitivity d / eps, which single precision cannot
follow.  The errors are printed (they are the figures the design notes state); the default
is held to the method's 1e-5 gradient tolerance, the small guard only to a coarse bound."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty, synth  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("which", ["small", "production"])
def test_eps_reading_errors(orc, which):
    p = synth.small_problem() if which == "small" else synth.production_problem()
    rng = np.random.default_rng(11)
    pert = (p.psi_true * (1 + 0.05 * (rng.standard_normal((p.H, p.W)) + 1j * rng.standard_normal((p.H, p.W))))
            ).astype(np.complex64)
    res = {}
    for eps in (0.1, 1e-6):
        o = pty.default_opts()
        o.eps = eps
        ctx = pty.Context(dev(p.probe), dev(p.pos), dev(p.d), p.H, p.W, o,
                          stream=torch.cuda.current_stream().cuda_stream)
        for name, psi in (("ones", p.psi0()), ("perturbed truth", pert)):
            g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
            F = ctx.gradient(dev(psi), g)
            gw, Fw = orc.gradient(psi, p.probe, p.pos, p.d, eps=eps, nthreads=0)
            res[(eps, name)] = (rel(g.cpu().numpy(), gw), abs(F - Fw) / abs(Fw))
            print(f"eps {eps:g} ({which}, {name}): gradient rel L2 {res[(eps, name)][0]:.2e}, "
                  f"objective rel {res[(eps, name)][1]:.2e}")
        ctx.close()
    for name in ("ones", "perturbed truth"):
        assert res[(0.1, name)][0] <= 1e-5 and res[(0.1, name)][1] <= 1e-4
        eg, eF = res[(1e-6, name)]
        assert np.isfinite(eg) and eg <= 1e-1 and eF <= 1e-4
