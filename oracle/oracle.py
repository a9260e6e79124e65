"""ctypes wrapper of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this module. It imports nothing from
the CUDA package; the two sides share only the seeded input generators.

The oracle follows the phase-field lattice Boltzmann model of Yuan, Liang,
Chai and Shi (arXiv:1904.12553): local algebra Eqs. N12, N17, N18, N29;
stencils Eq. N31 (and Eq. N40); NS collision Eq. 24 with Eq. 25, Eq. N20_1,
Eq. N22_1, Eq. N23; CH collision Eq. N24 with Eqs. N25-N28; lambda from
Eqs. N14-N16; beta from Eq. N36; a_i from Eq. N30.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRC3 = os.path.join(_HERE, "lbm_oracle3d.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

MAXN = 5


class OrcParams(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("wall_y", C.c_int32), ("grad_scheme", C.c_int32), ("pad_", C.c_int32),
        ("rho_t", C.c_double * MAXN),
        ("sigma", (C.c_double * MAXN) * MAXN),
        ("eta", C.c_double), ("beta", C.c_double), ("tau_g", C.c_double),
        ("tau", C.c_double * (MAXN - 1)), ("mob", C.c_double * (MAXN - 1)),
        ("grav", C.c_double * 2), ("rho0", C.c_double),
    ]


class O3Params(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("nz", C.c_int32), ("wall_y", C.c_int32), ("pad_", C.c_int32),
        ("rho_t", C.c_double * MAXN),
        ("sigma", (C.c_double * MAXN) * MAXN),
        ("eta", C.c_double), ("beta", C.c_double), ("tau_g", C.c_double),
        ("tau", C.c_double * (MAXN - 1)), ("mob", C.c_double * (MAXN - 1)),
        ("grav", C.c_double * 3), ("rho0", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FP contraction, OpenMP rows)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC3))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, _SRC3, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB_PATH)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(OrcParams)
        lib.orc_create.argtypes = [pp]
        lib.orc_create.restype = C.c_void_p
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_init.argtypes = [C.c_void_p, dp, dp, C.c_double]
        lib.orc_init.restype = C.c_int
        lib.orc_step.argtypes = [C.c_void_p, C.c_long]
        lib.orc_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.orc_chemical_potential.argtypes = [C.c_void_p, dp]
        lib.orc_fluxes.argtypes = [C.c_void_p, dp, dp]
        lib.orc_diagnostics.argtypes = [C.c_void_p, dp, dp, dp]
        lib.orc_constants.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc_stencils.argtypes = [C.c_void_p, dp, dp, dp]
        lib.orc_local_fractions.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc_local_phi_from_c.argtypes = [pp, dp, dp]
        lib.orc_lambda.argtypes = [pp, dp]
        lib.orc_lambda.restype = C.c_int
        lib.orc_beta.argtypes = [pp]
        lib.orc_beta.restype = C.c_double
        lib.orc_geq.argtypes = [pp, C.c_double, C.c_double, C.c_double,
                                C.c_double, dp]
        lib.orc_force_dist.argtypes = [C.c_double] * 9 + [dp]
        lib.orc_heq.argtypes = [C.c_double] * 5 + [dp]
        lib.orc_source.argtypes = [C.c_double] * 7 + [dp]
        lib.orc_sizeof_params.restype = C.c_int
        assert lib.orc_sizeof_params() == C.sizeof(OrcParams)
        p3 = C.POINTER(O3Params)
        lib.o3_create.argtypes = [p3]
        lib.o3_create.restype = C.c_void_p
        lib.o3_destroy.argtypes = [C.c_void_p]
        lib.o3_init.argtypes = [C.c_void_p, dp, dp, C.c_double]
        lib.o3_step.argtypes = [C.c_void_p, C.c_long]
        lib.o3_moments.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.o3_stencils.argtypes = [C.c_void_p, dp, dp, dp]
        lib.o3_fluxes.argtypes = [C.c_void_p, dp, dp, dp]
        lib.o3_populations.argtypes = [C.c_void_p, dp, dp]
        lib.o3_geq.argtypes = [C.c_double] * 3 + [dp, dp]
        lib.o3_force_dist.argtypes = [C.c_double, dp, dp, dp, dp, dp]
        lib.o3_heq.argtypes = [C.c_double] * 3 + [dp, dp]
        lib.o3_source.argtypes = [C.c_double, C.c_double, dp, C.c_double, dp, dp]
        lib.o3_sizeof_params.restype = C.c_int
        assert lib.o3_sizeof_params() == C.sizeof(O3Params)
        _lib = lib
        return lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(p: dict) -> OrcParams:
    """Fill the oracle's parameter struct from a workload parameter dict."""
    N = int(p["N"])
    o = OrcParams()
    o.N, o.nx, o.ny = N, int(p["nx"]), int(p["ny"])
    o.wall_y = int(p.get("wall_y", 0))
    o.grad_scheme = int(p.get("grad_scheme", 0))
    for k in range(N):
        o.rho_t[k] = float(p["rho"][k])
        for l in range(N):
            o.sigma[k][l] = float(p["sigma"][k][l])
    o.eta = float(p["eta"])
    o.beta = float(p.get("beta", 0.0))
    o.tau_g = float(p["tau_g"])
    for i in range(N - 1):
        o.tau[i] = float(p["tau"][i])
        o.mob[i] = float(p["mobility"][i])
    g = p.get("gravity", (0.0, 0.0))
    o.grav[0], o.grav[1] = float(g[0]), float(g[1])
    o.rho0 = float(p.get("rho0", 1.0))
    return o


def lam(p: dict) -> np.ndarray:
    """lambda_ij of Eq. N14 as an (N-1)x(N-1) array."""
    lib = _load()
    n = int(p["N"]) - 1
    out = np.zeros(n * n)
    if lib.orc_lambda(C.byref(make_params(p)), _dp(out)) != 0:
        raise ValueError("singular lambda system")
    return out.reshape(n, n)


def beta(p: dict) -> float:
    return _load().orc_beta(C.byref(make_params(p)))


def geq(p: dict, pr, rho, ux, uy) -> np.ndarray:
    """g_k^eq of Eq. 25, k = 0..8."""
    out = np.zeros(9)
    _load().orc_geq(C.byref(make_params(p)), pr, rho, ux, uy, _dp(out))
    return out


def force_dist(tau_g, u, F, grad_rho, J) -> np.ndarray:
    """G_k of Eq. N20_1, k = 0..8."""
    out = np.zeros(9)
    _load().orc_force_dist(tau_g, u[0], u[1], F[0], F[1], grad_rho[0],
                           grad_rho[1], J[0], J[1], _dp(out))
    return out


def heq(a_i, phi, Ci, u) -> np.ndarray:
    """h_k^{i,eq} of Eq. N25, k = 0..8."""
    out = np.zeros(9)
    _load().orc_heq(a_i, phi, Ci, u[0], u[1], _dp(out))
    return out


def source(tau_i, phi, u, phi_prev, u_prev) -> np.ndarray:
    """R_k of Eq. N26 with Eq. N27, k = 0..8."""
    out = np.zeros(9)
    _load().orc_source(tau_i, phi, u[0], u[1], phi_prev, u_prev[0],
                       u_prev[1], _dp(out))
    return out


def phi_from_c(p: dict, c) -> np.ndarray:
    out = np.zeros(int(p["N"]) - 1)
    cc = np.ascontiguousarray(c, dtype=np.float64)
    _load().orc_local_phi_from_c(C.byref(make_params(p)), _dp(cc), _dp(out))
    return out


class OracleSim:
    """One oracle simulation; arrays are numpy float64 [field][y][x]."""

    def __init__(self, params: dict):
        self.lib = _load()
        self.params = dict(params)
        self._p = make_params(params)
        self.N, self.nx, self.ny = self._p.N, self._p.nx, self._p.ny
        self.V = self.nx * self.ny
        self.h = self.lib.orc_create(C.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self.h:
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, c0, u0=None, p0: float = 0.0):
        c0 = np.ascontiguousarray(c0, dtype=np.float64)
        assert c0.shape == (self.N, self.ny, self.nx)
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
            assert u0.shape == (2, self.ny, self.nx)
        self.lib.orc_init(self.h, _dp(c0), _dp(u0), float(p0))

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    def moments(self) -> dict:
        n, N, sh = self.N - 1, self.N, (self.ny, self.nx)
        phi = np.zeros((n,) + sh)
        c = np.zeros((N,) + sh)
        u = np.zeros((2,) + sh)
        p = np.zeros(sh)
        rho = np.zeros(sh)
        self.lib.orc_moments(self.h, _dp(phi), _dp(c), _dp(u), _dp(p), _dp(rho))
        return {"phi": phi, "c": c, "u": u, "p": p, "rho": rho}

    def chemical_potential(self) -> np.ndarray:
        C_ = np.zeros((self.N - 1, self.ny, self.nx))
        self.lib.orc_chemical_potential(self.h, _dp(C_))
        return C_

    def fluxes(self):
        """J~ and grad(rho) of Eq. N18 at the current state, [2][y][x] each."""
        J = np.zeros((2, self.ny, self.nx))
        grho = np.zeros((2, self.ny, self.nx))
        self.lib.orc_fluxes(self.h, _dp(J), _dp(grho))
        return J, grho

    def diagnostics(self):
        mass = np.zeros(self.N)
        ke = C.c_double()
        um = C.c_double()
        self.lib.orc_diagnostics(self.h, _dp(mass), C.byref(ke), C.byref(um))
        return mass, ke.value, um.value

    def constants(self) -> dict:
        n = self.N - 1
        lam_ = np.zeros(n * n)
        a = np.zeros(n)
        b = C.c_double()
        G = C.c_double()
        self.lib.orc_constants(self.h, _dp(lam_), _dp(a), C.byref(b), C.byref(G))
        return {"lam": lam_.reshape(n, n), "a": a, "beta": b.value,
                "Gamma": G.value}

    def get_state(self) -> dict:
        n, sh = self.N - 1, (self.ny, self.nx)
        h = np.zeros((n, 9) + sh)
        g = np.zeros((9,) + sh)
        pp = np.zeros((n,) + sh)
        up = np.zeros((2,) + sh)
        self.lib.orc_get_state(self.h, _dp(h), _dp(g), _dp(pp), _dp(up))
        return {"h": h, "g": g, "phi_prev": pp, "u_prev": up}

    def set_state(self, st: dict):
        arrs = [np.ascontiguousarray(st[k], dtype=np.float64)
                for k in ("h", "g", "phi_prev", "u_prev")]
        self.lib.orc_set_state(self.h, *[_dp(a) for a in arrs])

    def stencils(self, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        assert z.shape == (self.ny, self.nx)
        grad = np.zeros((2, self.ny, self.nx))
        lap = np.zeros((self.ny, self.nx))
        self.lib.orc_stencils(self.h, _dp(z), _dp(grad), _dp(lap))
        return grad, lap

    def local_fractions(self, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        c = np.zeros(self.N)
        hf = np.zeros(self.N - 1)
        rho = C.c_double()
        self.lib.orc_local_fractions(self.h, _dp(phi), _dp(c), C.byref(rho),
                                     _dp(hf))
        return c, rho.value, hf


def run(params: dict, c0, u0=None, p0: float = 0.0, steps: int = 0) -> dict:
    """Convenience: init, advance ``steps`` and return the moments."""
    s = OracleSim(params)
    s.init(c0, u0, p0)
    s.step(steps)
    m = s.moments()
    s.close()
    return m


# ---------------------------------------------------------------------------
# D3Q15 (three dimensions)
# ---------------------------------------------------------------------------

def make_params3(p: dict) -> O3Params:
    N = int(p["N"])
    o = O3Params()
    o.N, o.nx, o.ny, o.nz = N, int(p["nx"]), int(p["ny"]), int(p["nz"])
    o.wall_y = int(p.get("wall_y", 0))
    for k in range(N):
        o.rho_t[k] = float(p["rho"][k])
        for l in range(N):
            o.sigma[k][l] = float(p["sigma"][k][l])
    o.eta, o.beta, o.tau_g = float(p["eta"]), float(p.get("beta", 0.0)), float(p["tau_g"])
    for i in range(N - 1):
        o.tau[i] = float(p["tau"][i])
        o.mob[i] = float(p["mobility"][i])
    g = list(p.get("gravity", (0.0, 0.0))) + [0.0] * 3
    o.grav[0], o.grav[1], o.grav[2] = float(g[0]), float(g[1]), float(g[2])
    o.rho0 = float(p.get("rho0", 1.0))
    return o


def _v3(v):
    a = np.ascontiguousarray(v, dtype=np.float64)
    assert a.shape == (3,)
    return a


def geq3(rho0, pr, rho, u) -> np.ndarray:
    out = np.zeros(15)
    _load().o3_geq(rho0, pr, rho, _dp(_v3(u)), _dp(out))
    return out


def force_dist3(tau_g, u, F, grad_rho, J) -> np.ndarray:
    out = np.zeros(15)
    _load().o3_force_dist(tau_g, _dp(_v3(u)), _dp(_v3(F)), _dp(_v3(grad_rho)),
                          _dp(_v3(J)), _dp(out))
    return out


def heq3(a_i, phi, Ci, u) -> np.ndarray:
    out = np.zeros(15)
    _load().o3_heq(a_i, phi, Ci, _dp(_v3(u)), _dp(out))
    return out


def source3(tau_i, phi, u, phi_prev, u_prev) -> np.ndarray:
    out = np.zeros(15)
    _load().o3_source(tau_i, phi, _dp(_v3(u)), phi_prev, _dp(_v3(u_prev)),
                      _dp(out))
    return out


class OracleSim3D:
    """D3Q15 oracle simulation; arrays are [field][z][y][x], u has 3 parts."""

    def __init__(self, params: dict):
        self.lib = _load()
        self._p = make_params3(params)
        self.N = self._p.N
        self.shape = (self._p.nz, self._p.ny, self._p.nx)
        self.h = self.lib.o3_create(C.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self.h:
            self.lib.o3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, c0, u0=None, p0: float = 0.0):
        c0 = np.ascontiguousarray(c0, dtype=np.float64)
        assert c0.shape == (self.N,) + self.shape
        if u0 is not None:
            u0 = np.ascontiguousarray(u0, dtype=np.float64)
            assert u0.shape == (3,) + self.shape
        self.lib.o3_init(self.h, _dp(c0), _dp(u0), float(p0))

    def step(self, n: int = 1):
        self.lib.o3_step(self.h, int(n))

    def moments(self) -> dict:
        sh = self.shape
        out = {"phi": np.zeros((self.N - 1,) + sh), "c": np.zeros((self.N,) + sh),
               "u": np.zeros((3,) + sh), "p": np.zeros(sh), "rho": np.zeros(sh)}
        self.lib.o3_moments(self.h, *[_dp(out[k]) for k in ("phi", "c", "u", "p", "rho")])
        return out

    def populations(self):
        """h[N-1][15] and g[15] of the current state."""
        sh = self.shape
        h = np.zeros((self.N - 1, 15) + sh)
        g = np.zeros((15,) + sh)
        self.lib.o3_populations(self.h, _dp(h), _dp(g))
        return h, g

    def fluxes(self):
        """C_i, J~ and grad(rho) (Eq. N18) at the current state."""
        sh = self.shape
        C_ = np.zeros((self.N - 1,) + sh)
        J = np.zeros((3,) + sh)
        grho = np.zeros((3,) + sh)
        self.lib.o3_fluxes(self.h, _dp(C_), _dp(J), _dp(grho))
        return C_, J, grho

    def stencils(self, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        grad = np.zeros((3,) + self.shape)
        lap = np.zeros(self.shape)
        self.lib.o3_stencils(self.h, _dp(z), _dp(grad), _dp(lap))
        return grad, lap


def run3(params: dict, c0, u0=None, p0: float = 0.0, steps: int = 0) -> dict:
    s = OracleSim3D(params)
    s.init(c0, u0, p0)
    s.step(steps)
    m = s.moments()
    s.close()
    return m
