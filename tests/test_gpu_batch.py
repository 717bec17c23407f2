"""Batched form: several views of uneven size reconstructed by one context, every stage one
launch over all views, the iteration replayed as a CUDA graph.  Each view must follow the
iteration the oracle computes for it alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty, synth  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def series():
    return synth.view_batch(n_views=4, seed=40, sizes=[256, 320, 192, 384], P=64, step=12, jitter=1, peak=1e4)


def test_batch_matches_oracle_per_view(orc, series):
    probe, views = series
    stream = torch.cuda.current_stream().cuda_stream
    bctx = pty.BatchContext(dev(probe), [(psi.shape[0], psi.shape[1], dev(pos), dev(d)) for psi, pos, d in views],
                            stream=stream)
    psis = [dev(np.ones_like(psi)) for psi, _, _ in views]
    st, reps = bctx.cg_solve(psis, 4)
    assert st == pty.PTY_OK
    for v, ((psi, pos, d), rep) in enumerate(zip(views, reps)):
        want = orc.cg_solve(np.ones_like(psi), probe, pos, d, 4, nthreads=0)
        relF = np.abs(rep["F"] - want["F"]) / np.abs(want["F"])
        print(f"view {v} {psi.shape}: K={len(pos)} trials {list(rep['halvings'])} vs {list(want['halvings'])}, "
              f"max objective rel err {relF.max():.2e}")
        assert list(rep["halvings"]) == list(want["halvings"])
        assert np.all(relF <= 1e-4)
        e = np.linalg.norm(psis[v].cpu().numpy() - want["psi"]) / np.linalg.norm(want["psi"])
        assert e <= 1e-3


def test_batch_equals_single_view_solves(series):
    """Each view of the batch takes the same steps as a context made for that view alone."""
    probe, views = series
    stream = torch.cuda.current_stream().cuda_stream
    bctx = pty.BatchContext(dev(probe), [(psi.shape[0], psi.shape[1], dev(pos), dev(d)) for psi, pos, d in views],
                            stream=stream)
    psis = [dev(np.ones_like(psi)) for psi, _, _ in views]
    st, reps = bctx.cg_solve(psis, 5)
    for v, (psi, pos, d) in enumerate(views):
        ctx = pty.Context(dev(probe), dev(pos), dev(d), psi.shape[0], psi.shape[1], stream=stream)
        one = dev(np.ones_like(psi))
        st1, rep1 = ctx.cg_solve(one, 5)
        assert list(rep1["halvings"]) == list(reps[v]["halvings"])
        np.testing.assert_array_equal(rep1["gamma"], reps[v]["gamma"])
        np.testing.assert_allclose(rep1["F"], reps[v]["F"], rtol=1e-9)
        e = (torch.linalg.norm(one - psis[v]) / torch.linalg.norm(one)).item()
        assert e <= 1e-6


def test_batch_graph_replay_is_deterministic(series):
    probe, views = series
    stream = torch.cuda.current_stream().cuda_stream
    mk = lambda: pty.BatchContext(dev(probe), [(p.shape[0], p.shape[1], dev(q), dev(d)) for p, q, d in views],
                                  stream=stream)
    a, b = mk(), mk()
    pa = [dev(np.ones_like(p)) for p, _, _ in views]
    pb = [dev(np.ones_like(p)) for p, _, _ in views]
    a.cg_solve(pa, 3)
    b.cg_solve(pb, 3)
    for x, y in zip(pa, pb):
        assert torch.equal(x, y)
