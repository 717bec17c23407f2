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
    o = pty.default_opts()
    o.tau = 1.5
    with pytest.raises(pty.PtyError) as e:
        pty.pty_create(256, 256, 64, probe, 1, pos, data, o)
    assert e.value.status == pty.PTY_ERR_ARG
