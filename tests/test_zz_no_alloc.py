"""The allocation-free diagnostics entry point, through the C ABI.

lbm_nphase_diagnostics_static serves callers that cannot allocate device
memory when they ask for diagnostics: it uses a static device array inside
the library instead of workspace scratch. Its results must equal those of
lbm_nphase_diagnostics, call after call (the array is reused and keeps the
previous call's contents). This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12553_gb300 import build
    build.build()


def _sigma(seed, N, rho=None):
    """Seeded sigma whose lambda the library accepts."""
    from paper_1904_12553_gb300 import LbmError, lbm_nphase_derive, workloads as W

    def ok(sig):
        try:
            lbm_nphase_derive(W.base_params(N, 4, 4, sig, rho=rho))
            return True
        except LbmError:
            return False
    return W.sample_sigma(np.random.default_rng(seed), N, accept=ok)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_static_diagnostics_match_workspace_diagnostics(prec):
    from paper_1904_12553_gb300 import Solver, binding, workloads as W
    rho = [1.0, 2.0, 3.0, 4.0]
    w = W.random_smooth(21, 4, 70, 45, rho=rho, amp_u=0.02, precision=prec,
                        sigma=_sigma(21, 4, rho))
    s = Solver(w.params)
    s.init(w.c0, w.u0)
    for _ in range(2):          # two calls in a row, state changing between
        s.step(7)
        ref = binding.lbm_nphase_diagnostics(s.handle, s.N)
        got = binding.lbm_nphase_diagnostics_static(s.handle, s.N)
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        assert abs(got[1] - ref[1]) <= 1e-12 * abs(ref[1])
        assert abs(got[2] - ref[2]) <= 1e-12 * abs(ref[2])
    # a second, smaller grid afterwards: the array keeps the larger grid's
    # partials, which must not leak into this result
    w2 = W.random_smooth(22, 3, 33, 17, amp_u=0.01, precision=prec,
                         sigma=_sigma(22, 3))
    s2 = Solver(w2.params)
    s2.init(w2.c0, w2.u0)
    s2.step(3)
    ref = binding.lbm_nphase_diagnostics(s2.handle, s2.N)
    got = binding.lbm_nphase_diagnostics_static(s2.handle, s2.N)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
    assert abs(got[1] - ref[1]) <= 1e-12 * abs(ref[1])
    s.close()
    s2.close()


def test_static_diagnostics_d3q15_handle():
    """A D3Q15 handle: one partial per 32 x 4 x 2 tile in the same array."""
    from paper_1904_12553_gb300 import Solver, binding, workloads as W
    w = W.random_smooth3(23, 3, 34, 9, 6, amp_u=0.02, precision="fp32")
    s = Solver(w.params)
    s.init(w.c0, w.u0)
    for _ in range(2):
        s.step(4)
        ref = binding.lbm_nphase_diagnostics(s.handle, s.N)
        got = binding.lbm_nphase_diagnostics_static(s.handle, s.N)
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        assert abs(got[1] - ref[1]) <= 1e-12 * abs(ref[1])
        assert abs(got[2] - ref[2]) <= 1e-12 * abs(ref[2])
    s.close()


def test_static_diagnostics_reports_a_wait_that_gave_up():
    """After a bounded device wait gave up (the library's self-test waits on
    a barrier nothing signals; no fault), the static entry point reports
    LBM_ETIMEOUT like the workspace one, and the handle refuses to step."""
    from paper_1904_12553_gb300 import LbmError, Solver, binding, workloads as W
    w = W.random_smooth(24, 3, 64, 40, precision="fp32", amp_u=0.01)
    s = Solver(w.params)
    s.init(w.c0, w.u0)
    s.step(2)
    binding.lbm_nphase_selftest_wait_timeout(s.handle)
    with pytest.raises(LbmError) as e:
        binding.lbm_nphase_diagnostics_static(s.handle, s.N)
    assert e.value.status == 4          # LBM_ETIMEOUT
    with pytest.raises(LbmError) as e:
        s.step(1)
    assert e.value.status == 6          # LBM_ESTATE
    s.init(w.c0, w.u0)
    s.step(2)
    ref = binding.lbm_nphase_diagnostics(s.handle, s.N)
    got = binding.lbm_nphase_diagnostics_static(s.handle, s.N)
    np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
    s.close()


def test_static_diagnostics_rejects_grids_beyond_limit():
    from paper_1904_12553_gb300 import LbmError, Solver, binding, workloads as W
    # 8192 x 520 nodes = 256 x 65 tiles > 16384 partial slots
    w = W.quiescent(2, 8192, 520, precision="fp16")
    s = Solver(w.params)
    s.init(w.c0)
    with pytest.raises(LbmError) as e:
        binding.lbm_nphase_diagnostics_static(s.handle, s.N)
    assert e.value.status == 1
    mass, ke, _ = binding.lbm_nphase_diagnostics(s.handle, s.N)
    assert np.isfinite(mass).all()
    s.close()
