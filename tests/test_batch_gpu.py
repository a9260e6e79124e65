"""Batched ensemble against the same cases run one by one.

The batch kernel applies the single-grid per-node arithmetic to (case, tile)
work items; every schedule and tile height must reproduce the single-grid
results, and the single-grid path is itself checked against the oracle.
"""
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


def _accept(sig):
    p = W.base_params(sig.shape[0], 4, 4, sig)
    ev = np.linalg.eigvalsh(oracle.lam(p))
    return ev[0] > 1e-3 * ev[-1]


@pytest.fixture(scope="module")
def cases():
    cs = W.ensemble(seed=9, ncases=10, sides=(64, 96, 40), accept=_accept)
    # plus a ragged grid and a two-phase case
    cs.append(W.random_smooth(3, 2, 72, 37, precision="fp32", amp_u=0.02,
                              sigma=W.sample_sigma(np.random.default_rng(3), 2)))
    cs.append(W.random_smooth(4, 5, 48, 29, precision="fp32", amp_u=0.02,
                              wall_y=1, sigma=W.sample_sigma(
                                  np.random.default_rng(4), 5, accept=_accept)))
    for w in cs:
        w.params["precision"] = "fp32"
    return cs


def _single(w, steps):
    from paper_1904_12553_gb300 import Solver
    s = Solver(w.params)
    s.init(w.c0, w.u0)
    s.step(steps)
    m = s.moments()
    s.close()
    return m


@pytest.fixture(scope="module")
def singles(cases):
    return [_single(w, 13) for w in cases]


def _close(a, b):
    for k in ("phi", "u", "p"):
        scale = np.abs(b[k]).max() + 1e-30
        assert np.abs(a[k] - b[k]).max() <= 1e-6 * scale, k


@pytest.mark.parametrize("tby", [4, 8])
@pytest.mark.parametrize("sched", [0, 1, 2])
def test_batch_matches_single_grids(cases, singles, tby, sched):
    from paper_1904_12553_gb300 import Batch
    b = Batch([w.params for w in cases])
    b.set_schedule(tby, sched)
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.step(6)
    b.step(7)          # odd count: graph pairs plus one direct launch
    assert b.schedule()["tile_height"] == tby
    for i in range(len(cases)):
        _close(b.moments(i), singles[i])
    b.close()


@pytest.mark.parametrize("sched", [0, 1, 2])
def test_pipelined_batch_matches_single_grids(cases, singles, sched):
    """TMA-pipelined tile body: items of different cases and N in flight in
    the same CTA's stages."""
    from paper_1904_12553_gb300 import Batch
    b = Batch([w.params for w in cases])
    b.set_schedule(8, sched, pipelined=True)
    s = b.schedule()
    assert s["pipelined"] == 1 and s["tile_height"] == 8
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.step(6)
    b.step(7)
    for i in range(len(cases)):
        _close(b.moments(i), singles[i])
    b.close()


@pytest.mark.parametrize("pipelined", [False, True])
@pytest.mark.parametrize("chunk", [4, 16])
def test_dynamic_chunks(cases, singles, pipelined, chunk):
    """Dynamic schedule taking several consecutive items per atomic grab
    (chunks that straddle cases and the end of the item list)."""
    from paper_1904_12553_gb300 import Batch
    b = Batch([w.params for w in cases])
    b.set_schedule(8, 2, pipelined=pipelined, chunk=chunk)
    assert b.schedule()["chunk"] == chunk
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.step(13)
    for i in range(len(cases)):
        _close(b.moments(i), singles[i])
    b.close()


@pytest.mark.parametrize("ctas", [1, 3])
def test_pipelined_batch_few_ctas(cases, singles, ctas):
    """One or three persistent CTAs walk every item: many case switches per
    CTA, both stages refilled across case boundaries."""
    from paper_1904_12553_gb300 import Batch
    b = Batch([w.params for w in cases])
    b.set_schedule(8, 0, ctas=ctas, pipelined=True)
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    b.step(13)
    for i in range(len(cases)):
        _close(b.moments(i), singles[i])
    b.close()


def test_pipelined_batch_needs_tensor_maps():
    """A case whose nx is not a multiple of 8 has no tensor maps: the
    pipelined schedule is refused and the generic one still runs."""
    from paper_1904_12553_gb300 import Batch, LbmError
    w = W.random_smooth(6, 3, 36, 20, precision="fp32", amp_u=0.02,
                        sigma=W.sample_sigma(np.random.default_rng(6), 3,
                                             accept=_accept))
    b = Batch([w.params])
    with pytest.raises(LbmError):
        b.set_schedule(8, 0, pipelined=True)
    assert b.schedule()["pipelined"] == 0
    b.close()


def test_autotune_and_reinit(cases, singles):
    from paper_1904_12553_gb300 import Batch
    b = Batch([w.params for w in cases])
    for i, w in enumerate(cases):
        b.init(i, w.c0, w.u0)
    ms = b.autotune(2)
    assert ms > 0
    s = b.schedule()
    assert s["tile_height"] in (4, 8) and s["schedule"] in (0, 1, 2)
    assert s["pipelined"] in (0, 1)
    for i, w in enumerate(cases):     # the trials advanced the state
        b.init(i, w.c0, w.u0)
    b.step(13)
    for i in range(len(cases)):
        _close(b.moments(i), singles[i])
        mass, ke, _ = b.diagnostics(i)
        assert np.isfinite(mass).all()
    b.close()


def test_batch_moments_and_diagnostics_entry_points(cases):
    """lbm_nphase_batch_moments / _diagnostics give what the single-grid
    calls give on the case's handle, and reject a case index outside the
    batch."""
    from paper_1904_12553_gb300 import Batch, LbmError, binding
    b = Batch([w.params for w in cases[:3]])
    for i, w in enumerate(cases[:3]):
        b.init(i, w.c0, w.u0)
    b.step(5)
    for i, w in enumerate(cases[:3]):
        N = int(w.params["N"])
        m1 = b.moments(i)
        d1 = b.diagnostics(i)
        d2 = binding.lbm_nphase_diagnostics(b.case_handle(i), N)
        np.testing.assert_array_equal(d1[0], d2[0])
        assert d1[1:] == d2[1:]
        assert np.isfinite(m1["phi"]).all()
    with pytest.raises(LbmError):
        binding.lbm_nphase_batch_diagnostics(b.handle, 3, 3)
    with pytest.raises(LbmError):
        binding.lbm_nphase_batch_moments(b.handle, -1)
    b.close()


def test_batch_rejects_unsupported(cases):
    from paper_1904_12553_gb300 import binding
    p = dict(cases[0].params, precision="fp64")
    assert binding.lbm_nphase_batch_workspace_bytes([p]) == 0
    p = dict(cases[0].params, rho=[1.0, 2.0] + [1.0] * (cases[0].params["N"] - 2))
    assert binding.lbm_nphase_batch_workspace_bytes([p]) == 0
