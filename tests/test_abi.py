"""C-ABI library checks that need no GPU: it loads, exports every function
declared in include/lbm_nphase.h, and its host-side parameter logic (checks,
lambda from Eqs. N14-N16, beta from Eq. N36, a_i from Eq. N30) agrees with
the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_1904_12553_gb300 as P
from paper_1904_12553_gb300 import binding, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_12553_gb300 import build
    build.build()
    return P.load_library()


def _declared():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names += re.findall(r"\b(lbm_nphase_\w+)\s*\(", txt)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "lbm_nphase_step" in names and len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    so = ctypes.CDLL(binding.library_path())
    for n in names:
        ctypes.cast(getattr(so, n), ctypes.c_void_p)


def test_no_cpu_fallback(monkeypatch):
    """Without the built library every call fails loudly."""
    from paper_1904_12553_gb300 import build
    monkeypatch.setattr(build, "LIB", "/nonexistent/liblbm_nphase.so")
    monkeypatch.setattr(binding, "_LIB", None)
    with pytest.raises(RuntimeError, match="missing"):
        binding.lbm_nphase_workspace_bytes(W.static_drops().params)


@pytest.mark.parametrize("N", [2, 3, 4, 5])
@pytest.mark.parametrize("seed", range(4))
def test_derive_matches_oracle(lib, N, seed):
    rng = np.random.default_rng(100 * N + seed)
    rho = rng.uniform(0.5, 20, N) if seed % 2 else np.ones(N)

    def spd(sig):
        p = W.base_params(N, 4, 4, sig, rho=rho)
        return np.linalg.eigvalsh(oracle.lam(p)).min() > 0

    sig = W.sample_sigma(rng, N, accept=spd)
    p = W.base_params(N, 16, 9, sig, rho=rho,
                      tau=list(rng.uniform(0.6, 1.4, N - 1)),
                      mobility=list(rng.uniform(0.01, 0.3, N - 1)))
    d = P.lbm_nphase_derive(p)
    s = oracle.OracleSim(p)
    ref = s.constants()
    s.close()
    np.testing.assert_allclose(d["lambda"], ref["lam"], rtol=1e-11,
                               atol=1e-13 * np.abs(ref["lam"]).max())
    assert abs(d["beta"] - ref["beta"]) < 1e-15
    np.testing.assert_allclose(d["a"], ref["a"], rtol=1e-15)
    assert abs(d["Gamma"] - ref["Gamma"]) < 1e-13
    ev = np.linalg.eigvalsh(ref["lam"])
    assert abs(d["lambda_eig_min"] - ev[0]) < 1e-12 * ev[-1]
    assert abs(d["lambda_eig_max"] - ev[-1]) < 1e-12 * ev[-1]
    assert d["uniform_density"] == bool(np.all(rho == rho[0]))
    assert abs(d["nu"] - (p["tau_g"] - 0.5) / 3) < 1e-16


def _bad(**kw):
    p = W.static_drops().params
    p = {**p, **kw}
    return p


@pytest.mark.parametrize("bad", [
    dict(N=1), dict(N=6), dict(nx=0), dict(ny=-3), dict(tau_g=0.5),
    dict(tau=[0.8, 0.4]), dict(mobility=[0.1, 0.0]), dict(eta=0.0),
    dict(rho=[1.0, -1.0, 1.0]), dict(precision=7), dict(wall_y=2),
    dict(grad_scheme=2),
    dict(sigma=[[0, 1e-3, 1e-3], [2e-3, 0, 1e-3], [1e-3, 1e-3, 0]]),
    dict(sigma=[[0, 1e-3, 0], [1e-3, 0, 1e-3], [0, 1e-3, 0]]),
])
def test_invalid_parameters_rejected(lib, bad):
    p = _bad(**bad)
    if p["N"] in (1, 6):
        p["rho"] = [1.0] * 5
        p["tau"] = [0.8] * 4
        p["mobility"] = [0.1] * 4
        p["sigma"] = (np.full((5, 5), 1e-3)).tolist()
    with pytest.raises(P.LbmError) as e:
        P.lbm_nphase_derive(p)
    assert e.value.status == 1
    assert P.lbm_nphase_workspace_bytes(p) == 0


@pytest.mark.parametrize("bad", [
    dict(lattice=2), dict(lattice=1, nz=0), dict(lattice=0, nz=3),
    dict(lattice=1, nz=4, grad_scheme=1), dict(gravity=[0.0, 0.0, 1e-5]),
])
def test_invalid_lattice_parameters_rejected(lib, bad):
    p = {**W.static_drops().params, **bad}
    with pytest.raises(P.LbmError) as e:
        P.lbm_nphase_derive(p)
    assert e.value.status == 1


@pytest.mark.parametrize("shape,ok", [
    (dict(nx=8, ny=524280), True), (dict(nx=8, ny=524281), False),
    (dict(nx=1 << 20, ny=4), True), (dict(nx=(1 << 20) + 1, ny=4), False),
    (dict(lattice=1, nx=8, ny=262140, nz=2), True),
    (dict(lattice=1, nx=8, ny=262141, nz=2), False),
    (dict(lattice=1, nx=8, ny=8, nz=131070), True),
    (dict(lattice=1, nx=8, ny=8, nz=131071), False),
])
def test_grid_extent_limits(lib, shape, ok):
    """The largest extents the launch grids allow are accepted, one more
    node is rejected."""
    base = W.random_smooth3(0, 3, 8, 8, 8) if shape.get("lattice") else \
        W.static_drops()
    p = {**base.params, **shape}
    if ok:
        P.lbm_nphase_derive(p)
        assert P.lbm_nphase_workspace_bytes(p) > 0
    else:
        with pytest.raises(P.LbmError) as e:
            P.lbm_nphase_derive(p)
        assert e.value.status == 1


def test_d3q15_workspace(lib):
    p3 = W.base_params3(3, 16, 12, 10, 1e-3, precision="fp32")
    b = P.lbm_nphase_workspace_bytes(p3)
    V = 16 * 12 * 10
    # 2 x (2 rest + 2 x 14 moving + 14 NS + 2 phi_prev) + 3 u_prev floats
    assert b >= (2 * (2 + 28 + 14 + 2) + 3) * V * 4


def test_indefinite_lambda_rejected(lib):
    """N = 4 with sigma_13 = 2e-3 and the other pairs 1e-3 gives a lambda of
    Eq. N14 with a negative eigenvalue: the gradient energy of Eq. N11 is
    not positive, so the parameter set is refused."""
    sig = np.full((4, 4), 1e-3)
    sig[0, 2] = sig[2, 0] = 2e-3
    p = W.base_params(4, 8, 8, sig)
    assert np.linalg.eigvalsh(oracle.lam(p)).min() < 0
    with pytest.raises(P.LbmError) as e:
        P.lbm_nphase_derive(p)
    assert e.value.status == 1


def test_workspace_bytes_scale(lib):
    p = W.static_drops().params
    b1 = P.lbm_nphase_workspace_bytes(p)
    b2 = P.lbm_nphase_workspace_bytes({**p, "nx": 256, "ny": 256})
    assert 3.5 < b2 / b1 < 4.5
    # FP64 stores (10N - ...) doubles per node, twice for the populations
    V = 128 * 128
    assert b1 > 2 * (9 * 2 + 8) * V * 8
    pm = {**p, "precision": "fp16"}
    assert P.lbm_nphase_workspace_bytes(pm) < P.lbm_nphase_workspace_bytes(
        {**p, "precision": "fp32"})


@pytest.mark.parametrize("lattice", [0, 1])
def test_16bit_workspace_holds_p_prev(lib, lattice):
    """The 16-bit forms keep p(t-1) as one more plane of the u(t-1)
    ping-pong buffers (their g storage is relative to it). On a grid whose
    sections need no alignment padding, FP32 minus BF16 workspace is exactly
    the halved moving populations less that plane:
    2 x (Q-1)(N-1+1) x V x 2 bytes - 2 x V x 4 bytes."""
    N, nx, ny, nz = 3, 64, 64, 8
    if lattice == 0:
        p = W.base_params(N, nx, ny, 1e-3)
        V, QM = nx * ny, 8
    else:
        p = W.base_params3(N, nx, ny, nz, 1e-3)
        V, QM = nx * ny * nz, 14
    b32 = P.lbm_nphase_workspace_bytes({**p, "precision": "fp32"})
    b16 = P.lbm_nphase_workspace_bytes({**p, "precision": "bf16"})
    bh = P.lbm_nphase_workspace_bytes({**p, "precision": "fp16"})
    assert b16 == bh
    moving = QM * (N - 1) + QM
    assert b32 - b16 == 2 * moving * V * 2 - 2 * V * 4


def test_create_rejects_bad_workspace(lib):
    p = W.static_drops().params
    with pytest.raises(P.LbmError) as e:
        P.lbm_nphase_create(p, 0, 1 << 20, 0)
    assert e.value.status == 1
    with pytest.raises(P.LbmError) as e:
        P.lbm_nphase_create(p, 256, 16, 0)
    assert e.value.status == 2


def test_strerror(lib):
    for s in range(7):
        assert len(P.strerror(s)) > 3
