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
