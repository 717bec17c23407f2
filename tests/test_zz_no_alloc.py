"""pty_gradient_noalloc: the gradient entry point that allocates nothing.

Some callers cannot allocate device memory (a fixed memory budget owned by another
framework, a plug-in that must not grow the device footprint, a path that must not take
cudaMalloc's implicit synchronisation).  This test calls the entry point through the C ABI
twice in a row -- the shared scratch array keeps the first call's contents -- and checks
both results against pty_gradient on the same inputs.  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty, synth  # noqa: E402

TOL = 1e-5  # the gradient tolerance of the parity tests (relative L2)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_gradient_matches_pty_gradient_twice():
    p = synth.small_problem()
    stream = torch.cuda.current_stream().cuda_stream
    probe, pos, d = dev(p.probe), dev(p.pos), dev(p.d)
    opts = pty.default_opts()
    ctx = pty.Context(probe, pos, d, p.H, p.W, opts, stream=stream)
    rng = np.random.default_rng(0)
    objects = [p.psi0(), (p.psi_true * (1 + 0.05 * rng.standard_normal((p.H, p.W)))).astype(np.complex64)]
    want = []
    for psi in objects:
        g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
        F = ctx.gradient(dev(psi), g)
        want.append((g.cpu().numpy(), F))
    ctx.close()
    for (g_ref, F_ref), psi in zip(want, objects):  # two calls in a row on the shared scratch
        g = torch.full((p.H, p.W), float("nan"), dtype=torch.complex64, device="cuda")
        F = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = pty.pty_gradient_noalloc(p.H, p.W, p.P, probe, p.K, pos, d, opts.eps, dev(psi), g, F, stream)
        assert st == pty.PTY_OK
        e = rel(g.cpu().numpy(), g_ref)
        print(f"noalloc vs pty_gradient: gradient rel L2 {e:.2e}, objective rel {abs(F.item() - F_ref) / abs(F_ref):.2e}")
        assert e <= TOL
        assert abs(F.item() - F_ref) <= TOL * abs(F_ref)


def test_noalloc_rejects_oversize_and_bad_positions():
    p = synth.production_problem()  # 3600 x 128 x 128 values: beyond the scratch limit
    stream = torch.cuda.current_stream().cuda_stream
    probe, pos, d = dev(p.probe), dev(p.pos), dev(p.d)
    g = torch.empty((p.H, p.W), dtype=torch.complex64, device="cuda")
    st = pty.pty_gradient_noalloc(p.H, p.W, p.P, probe, p.K, pos, d, 0.1, dev(p.psi0()), g, None, stream)
    assert st == pty.PTY_ERR_ARG
    q = synth.small_problem()
    bad = q.pos.copy()
    bad[5] = (q.H - q.P + 1, 0)
    g = torch.empty((q.H, q.W), dtype=torch.complex64, device="cuda")
    st = pty.pty_gradient_noalloc(q.H, q.W, q.P, dev(q.probe), q.K, dev(bad), dev(q.d), 0.1, dev(q.psi0()), g,
                                  None, stream)
    assert st == pty.PTY_ERR_BOUNDS
    # misaligned device pointers (4 mod 8) are rejected before anything launches
    pos_flat = torch.zeros(2 * q.K + 1, dtype=torch.int32, device="cuda")
    pos_off = pos_flat[1:]
    assert pos_off.data_ptr() % 8 == 4
    st = pty.pty_gradient_noalloc(q.H, q.W, q.P, dev(q.probe), q.K, pos_off, dev(q.d), 0.1, dev(q.psi0()), g,
                                  None, stream)
    assert st == pty.PTY_ERR_ARG
    F_flat = torch.zeros(2, dtype=torch.float32, device="cuda")
    F_off = F_flat[1:].view(torch.float32)
    assert F_off.data_ptr() % 8 == 4
    lib = pty.load()
    import ctypes
    st = lib.pty_gradient_noalloc(q.H, q.W, q.P, ctypes.c_void_p(dev(q.probe).data_ptr()), q.K,
                                  ctypes.c_void_p(dev(q.pos).data_ptr()), ctypes.c_void_p(dev(q.d).data_ptr()), 0.1,
                                  ctypes.c_void_p(dev(q.psi0()).data_ptr()), ctypes.c_void_p(g.data_ptr()),
                                  ctypes.c_void_p(F_off.data_ptr()), ctypes.c_void_p(stream))
    assert st == pty.PTY_ERR_ARG
