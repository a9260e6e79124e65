"""Checkpoint / resume and graph-replayed stepping, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1904_12553_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12553_gb300 import build
    build.build()


def _ok(sig):
    ev = np.linalg.eigvalsh(oracle.lam(W.base_params(sig.shape[0], 4, 4, sig)))
    return ev[0] > 1e-3 * ev[-1]


def _work(prec):
    return W.random_smooth(31, 4, 64, 40, amp_u=0.02, precision=prec,
                           sigma=W.sample_sigma(np.random.default_rng(31), 4,
                                                accept=_ok))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("on_device", [False, True])
def test_resume_is_bit_exact(prec, on_device):
    from paper_1904_12553_gb300 import Solver
    w = _work(prec)
    a = Solver(w.params)
    a.init(w.c0, w.u0)
    a.step(23)
    blob = a.get_state(device=on_device)
    a.step(17)
    ref = a.moments()
    b = Solver(w.params)
    b.set_state(blob)
    assert b.steps_taken == 23
    b.step(17)
    got = b.moments()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    a.close()
    b.close()


def test_set_state_rejects_other_grids():
    from paper_1904_12553_gb300 import LbmError, Solver
    w = _work("fp32")
    a = Solver(w.params)
    a.init(w.c0, w.u0)
    blob = a.get_state()
    other = Solver({**w.params, "nx": 72})
    with pytest.raises(LbmError):
        other.set_state(blob)
    bad = blob.clone()
    bad[0] = 0
    with pytest.raises(LbmError):
        a.set_state(bad)
    a.close()
    other.close()


@pytest.mark.parametrize("field,value", [("wall_y", 1), ("grad_scheme", 1)])
def test_set_state_rejects_other_boundaries_and_schemes(field, value):
    """A blob saved with periodic y and the central scheme does not resume
    into a handle with walls or with the Eq. N40 gradient (LBM_EINVAL)."""
    from paper_1904_12553_gb300 import LbmError, Solver
    w = _work("fp64")
    a = Solver(w.params)
    a.init(w.c0, w.u0)
    blob = a.get_state()
    other = Solver({**w.params, field: value})
    with pytest.raises(LbmError) as e:
        other.set_state(blob)
    assert e.value.status == 1
    a.close()
    other.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_graph_stepping_matches_direct_launches(prec):
    from paper_1904_12553_gb300 import Solver
    w = _work(prec)
    a = Solver(w.params)
    a.init(w.c0, w.u0)
    for _ in range(41):
        a.step(1)              # below the graph threshold: direct launches
    b = Solver(w.params)
    b.init(w.c0, w.u0)
    b.step(41)                 # one direct step, then graph pairs
    ra, rb = a.moments(), b.moments()
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k
    assert a.steps_taken == b.steps_taken == 41
    a.close()
    b.close()


def _parts(blob, N, V, wide, q=8, uplanes=2):
    """Split a state blob: rest slots, moving h, g, phi(t-1), u(t-1)."""
    dt = np.float64 if wide else np.float32
    a = blob.numpy()[64:].view(dt)
    n = N - 1
    sizes = [n * V, n * q * V, q * V, n * V, uplanes * V]
    out, o = [], 0
    for sz in sizes:
        out.append(a[o:o + sz].astype(np.float64))
        o += sz
    assert o == a.size
    return out


@pytest.mark.parametrize("lattice", ["d2q9", "d3q15"])
@pytest.mark.parametrize("rho", [None, [1.0, 2.0, 3.0, 4.0]])
@pytest.mark.parametrize("wall", [0, 1])
def test_fp32_start_is_the_fp64_start_rounded(lattice, rho, wall):
    """The equilibrium start is computed in FP64 for every storage form:
    the FP32 form's moving populations, phi(t-1) and u(t-1) are the FP64
    form's rounded once, and its node mass phi(t-1) + d_0 + sum_k h_k is
    the FP64 phi up to the rounding of d_0."""
    from paper_1904_12553_gb300 import Solver
    sig = W.sample_sigma(np.random.default_rng(43), 4, accept=_ok)
    if lattice == "d2q9":
        w = W.random_smooth(43, 4, 40, 24, rho=rho, sigma=sig, wall_y=wall,
                            amp_u=0.02, precision="fp64")
        q, D = 8, 2
    else:
        w = W.random_smooth3(43, 4, 12, 10, 8, rho=rho, sigma=sig,
                             wall_y=wall, amp_u=0.02, precision="fp64")
        q, D = 14, 3
    V = w.c0[0].size
    blobs = {}
    for prec in ("fp64", "fp32"):
        s = Solver({**w.params, "precision": prec})
        s.init(w.c0, w.u0)
        blobs[prec] = s.get_state()
        s.close()
    r64, hm64, gm64, pp64, u64 = _parts(blobs["fp64"], 4, V, True, q, D)
    d0, hm32, gm32, pp32, u32 = _parts(blobs["fp32"], 4, V, False, q, D)
    f32 = lambda v: v.astype(np.float32).astype(np.float64)  # noqa: E731
    np.testing.assert_array_equal(hm32, f32(hm64))
    np.testing.assert_array_equal(gm32, f32(gm64))
    np.testing.assert_array_equal(pp32, f32(pp64))
    np.testing.assert_array_equal(u32, f32(u64))
    n = 3
    phi64 = pp64.reshape(n, V)
    mass32 = (pp32.reshape(n, V) + d0.reshape(n, V) +
              hm32.reshape(n, q, V).sum(1))
    # d_0 is rounded to nearest: within half an FP32 ulp of its value
    bound = 2.0 ** -24 * np.abs(d0.reshape(n, V)) + 1e-15
    assert (np.abs(mass32 - phi64) <= bound).all()
    # the FP64 form's own start: h_0 + sum_k h_k = phi
    mass64 = r64.reshape(n, V) + hm64.reshape(n, q, V).sum(1)
    assert np.abs(mass64 - phi64).max() < 1e-14
