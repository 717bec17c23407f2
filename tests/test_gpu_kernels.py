"""GPU checks of the library's device building blocks against higher-precision references."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2106_07575_gb300 import pty  # noqa: E402


def test_line_search_log1p_within_5_ulp():
    """The single-precision log(1 + t) of the line-search kernels vs FP64, t in (-1, 1e7]."""
    rng = np.random.default_rng(0)
    t = np.concatenate([-1 + np.logspace(-7, 0, 20000)[:-1], -np.logspace(-30, -0.31, 20000),
                        np.logspace(-30, 7, 40000), rng.uniform(-0.5, 2.0, 40000), [0.0]]).astype(np.float32)
    t = t[t > -1]
    out = np.empty_like(t)
    pty.pty_selftest_log1p(t, out)
    ref = np.log1p(t.astype(np.float64))
    nz = ref != 0
    ulp = np.spacing(np.abs(ref[nz]).astype(np.float32)).astype(np.float64)
    err = np.abs(out[nz].astype(np.float64) - ref[nz]) / ulp
    print(f"log1p max error {err.max():.2f} ulp at t={t[nz][np.argmax(err)]!r}")
    assert err.max() <= 5.0
    assert np.all(out[~nz] == 0.0)
    # device pointers take the same path
    td = torch.from_numpy(t).cuda()
    od = torch.empty_like(td)
    pty.pty_selftest_log1p(td, od)
    assert np.array_equal(od.cpu().numpy(), out)
