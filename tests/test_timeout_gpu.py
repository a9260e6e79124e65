"""The failure path of the bounded device waits, exercised without a fault:
a warp waits, with the library's bounded wait, on a barrier nothing signals
(lbm_nphase_selftest_wait_timeout). The host must report LBM_ETIMEOUT at the
next diagnostics call, refuse to step (LBM_ESTATE) until re-initialised, and
then run exactly as a fresh handle does."""
import numpy as np
import pytest

from paper_1904_12553_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

LBM_ETIMEOUT, LBM_ESTATE = 4, 6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12553_gb300 import build
    build.build()


def test_wait_timeout_is_reported_and_recoverable():
    from paper_1904_12553_gb300 import LbmError, Solver, binding
    w = W.random_smooth(8, 3, 64, 40, precision="fp32", amp_u=0.01)
    s = Solver(w.params)
    assert s.pipelined
    s.init(w.c0, w.u0)
    s.step(3)
    binding.lbm_nphase_selftest_wait_timeout(s.handle)
    with pytest.raises(LbmError) as e:
        s.diagnostics()
    assert e.value.status == LBM_ETIMEOUT
    with pytest.raises(LbmError) as e:
        s.step(1)
    assert e.value.status == LBM_ESTATE
    # re-initialised, the handle steps like a fresh one, bit for bit
    s.init(w.c0, w.u0)
    s.step(6)
    a = s.moments()
    s.close()
    f = Solver(w.params)
    f.init(w.c0, w.u0)
    f.step(6)
    b = f.moments()
    f.close()
    for k in ("phi", "u", "p"):
        np.testing.assert_array_equal(a[k], b[k])
