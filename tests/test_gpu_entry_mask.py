"""The linear GRAD pass with the entry masks (the first inverse pass reads only the spectrum
slots that hold entries; the tile is not zeroed) against the same pass that zeroes the tile
(opts.flags bit 5): a masked slot is read as the zero it would have held, so the
transforms, the CG steps, the objective histories and the iterates agree bit for bit."""
import numpy as np
import pytest

from paper_2106_07575_gb300 import pty, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


PROBLEMS = {
    # one CTA per pattern in every case: P = 64 (256 threads), P = 128 (512 or 1024 threads)
    "p64": (lambda: synth.small_problem(seed=0), -1),
    "p128_512": (lambda: synth.small_problem(H=512, W=512, P=128, n=27, step=14, jitter=2, peak=1e5, seed=4), 0),
    "p128_1024": (lambda: synth.small_problem(H=512, W=512, P=128, n=27, step=14, jitter=2, peak=1e5, seed=4), 3),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_masked_linear_grad_equals_zeroed(name):
    make, tile = PROBLEMS[name]
    p = make()
    out = {}
    for masked in (True, False):
        o = pty.default_opts()
        o.tile_config = tile
        if not masked:
            o.flags |= 32
        ctx = pty.Context(dev(p.probe), dev(p.pos), dev(p.d), p.H, p.W, o)
        x = dev(p.psi0())
        st, rep = ctx.cg_solve(x, 8)  # iterations 2..8 of the call run the linear form
        assert st == pty.PTY_OK
        out[masked] = (rep, x.cpu().numpy())
        ctx.close()
    (r1, x1), (r0, x0) = out[True], out[False]
    assert list(r1["halvings"]) == list(r0["halvings"])
    assert np.array_equal(r1["F"], r0["F"])
    assert np.array_equal(x1, x0)
