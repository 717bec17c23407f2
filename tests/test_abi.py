"""The C-ABI library builds for sm_103a, loads, and exports every entry point of include/pty.h."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    import glob

    src = "".join(open(f).read() for f in glob.glob(os.path.join(ROOT, "include", "*.h")))
    return sorted(set(re.findall(r"PTY_API\s+[\w\s\*]*?\b(pty_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("pty_create", "pty_forward", "pty_gradient", "pty_cg_solve", "pty_destroy", "pty_adjoint"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2106_07575_gb300 import build, pty

    path = build.build()
    lib = ctypes.CDLL(path)  # loading needs no GPU; no compute call is made
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(pty.EXPORTED) == declared_symbols()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pty_\w+)", out))
    assert exported == set(declared_symbols())


def test_default_options_match_algorithm_1():
    from paper_2106_07575_gb300 import pty

    o = pty.default_opts()  # pure host function
    assert (o.gamma0, o.tau, o.t, o.max_halvings) == (1.0, 0.5, 0.0, 60)
    assert o.ls_window in (0, 4, 8, 16, 32) and o.tile_config == -1


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    """Argument checks run on the host before any CUDA call."""
    import numpy as np
    from paper_2106_07575_gb300 import pty

    probe = np.ones((64, 64), np.complex64)
    pos = np.zeros((1, 2), np.int32)
    data = np.ones((1, 64, 64), np.float32)
    with pytest.raises(pty.PtyError) as e:
        pty.pty_create(256, 256, 48, probe, 1, pos, data)
    assert e.value.status == pty.PTY_ERR_ARG
    with pytest.raises(pty.PtyError) as e:
        pty.pty_create(32, 256, 64, probe, 1, pos, data)
    assert e.value.status == pty.PTY_ERR_ARG
    bad = np.array([[0, 200]], np.int32)
    with pytest.raises(pty.PtyError) as e:
        pty.pty_create(256, 256, 64, probe, 1, bad, data)
    assert e.value.status == pty.PTY_ERR_BOUNDS
    for field, value in (("tau", 1.5), ("gamma0", float("inf")), ("gamma0", 0.0), ("eps", float("inf")),
                         ("eps", float("nan")), ("t", float("nan")), ("max_halvings", 0)):
        o = pty.default_opts()
        setattr(o, field, value)
        with pytest.raises(pty.PtyError) as e:
            pty.pty_create(256, 256, 64, probe, 1, pos, data, o)
        assert e.value.status == pty.PTY_ERR_ARG, (field, value)


def test_valid_options_pass_the_checks():
    """Boundary values of the options (a huge finite gamma0, eps = 0, a negative t) pass the
    host checks: without a GPU the call gets as far as its first CUDA call."""
    import numpy as np
    from paper_2106_07575_gb300 import pty

    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the host path only where no GPU answers")
    probe = np.ones((64, 64), np.complex64)
    pos = np.zeros((1, 2), np.int32)
    data = np.ones((1, 64, 64), np.float32)
    for field, value in ((None, None), ("gamma0", 1e12), ("eps", 0.0), ("t", -3.0), ("max_halvings", 1000)):
        o = pty.default_opts()
        if field:
            setattr(o, field, value)
        with pytest.raises(pty.PtyError) as e:
            pty.pty_create(256, 256, 64, probe, 1, pos, data, o)
        assert e.value.status == pty.PTY_ERR_CUDA, (field, value)


def test_binding_checks_array_sizes_before_the_library():
    """The wrappers know the problem's shapes: an array of the wrong size raises ValueError on
    the host; an array of the right size reaches the library (here a NULL context, which the
    library rejects before any CUDA call)."""
    import numpy as np
    from paper_2106_07575_gb300 import pty

    probe = np.ones((64, 64), np.complex64)
    pos = np.zeros((2, 2), np.int32)
    with pytest.raises(ValueError):
        pty.Context(probe, pos, np.ones((1, 64, 64), np.float32), 256, 256)
    with pytest.raises(ValueError):
        pty.Context(probe, np.zeros((2, 3), np.int32), np.ones((2, 64, 64), np.float32), 256, 256)
    with pytest.raises(ValueError):
        pty.Context(np.ones((64, 32), np.complex64), pos, np.ones((2, 64, 64), np.float32), 256, 256)
    with pytest.raises(ValueError):
        pty.BatchContext(probe, [(256, 256, pos, np.ones((3, 64, 64), np.float32))])

    c = pty.Context.__new__(pty.Context)
    c.shape, c.P, c.K, c.ctx = (256, 200), 64, 2, None
    obj, pats = np.ones((256, 200), np.complex64), np.ones((2, 64, 64), np.complex64)
    for call in (lambda: c.forward(obj[:100], pats), lambda: c.forward(obj, pats[:1]),
                 lambda: c.adjoint(pats, obj.T[:10]), lambda: c.gradient(obj, obj[:, :199]),
                 lambda: c.cg_solve(np.ones((200, 256, 2), np.complex64), 1)):
        with pytest.raises(ValueError):
            call()
    for call in (lambda: c.forward(obj, pats), lambda: c.adjoint(pats, obj), lambda: c.gradient(obj, obj.copy()),
                 lambda: c.cg_solve(obj, 1)):
        with pytest.raises(pty.PtyError) as e:
            call()
        assert e.value.status == pty.PTY_ERR_ARG


def test_create_error_message_is_per_thread():
    """The message of a failed pty_create belongs to the calling thread."""
    import threading

    import numpy as np
    from paper_2106_07575_gb300 import pty

    lib = pty.load()
    probe = np.ones((64, 64), np.complex64)
    pos = np.zeros((1, 2), np.int32)
    data = np.ones((1, 64, 64), np.float32)
    with pytest.raises(pty.PtyError):
        pty.pty_create(256, 256, 48, probe, 1, pos, data)
    mine = lib.pty_last_error(None).decode()
    assert "P=48" in mine
    other = {}

    def worker():
        o = pty.default_opts()
        o.tau = 1.5
        try:
            pty.pty_create(256, 256, 64, probe, 1, pos, data, o)
        except pty.PtyError:
            other["msg"] = lib.pty_last_error(None).decode()

    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert "invalid options" in other["msg"]
    assert lib.pty_last_error(None).decode() == mine
