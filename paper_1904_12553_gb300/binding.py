"""Python binding of the C ABI declared in ``include/lbm_nphase.h``.

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/liblbm_nphase.so``. The functions keep the C names; each raises
:class:`LbmError` when the library returns a status other than ``LBM_OK``.
PyTorch provides the device workspace and the CUDA stream.

If the library has not been built, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MAXN = 5
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
STATUS = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA",
          4: "LBM_ETIMEOUT", 5: "LBM_EUNSTABLE", 6: "LBM_ESTATE"}


class LbmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} "
                         f"({strerror(status) if _LIB else ''})")


class LbmParams(C.Structure):
    _fields_ = [
        ("N", C.c_int32), ("nx", C.c_int32), ("ny", C.c_int32),
        ("nz", C.c_int32), ("lattice", C.c_int32),
        ("wall_y", C.c_int32), ("precision", C.c_int32),
        ("grad_scheme", C.c_int32),
        ("rho", C.c_double * MAXN),
        ("sigma", (C.c_double * MAXN) * MAXN),
        ("eta", C.c_double), ("beta", C.c_double), ("tau_g", C.c_double),
        ("tau", C.c_double * (MAXN - 1)),
        ("mobility", C.c_double * (MAXN - 1)),
        ("gravity", C.c_double * 3), ("rho0", C.c_double),
    ]


class LbmModel(C.Structure):
    _fields_ = [
        ("lambda_", (C.c_double * (MAXN - 1)) * (MAXN - 1)),
        ("lambda_eig_min", C.c_double), ("lambda_eig_max", C.c_double),
        ("beta", C.c_double), ("a", C.c_double * (MAXN - 1)),
        ("Gamma", C.c_double), ("nu", C.c_double),
        ("uniform_density", C.c_int32), ("pad_", C.c_int32),
    ]


class LbmSchedule(C.Structure):
    _fields_ = [("tile_height", C.c_int32), ("schedule", C.c_int32),
                ("ctas", C.c_int32), ("pipelined", C.c_int32),
                ("chunk", C.c_int32)]


_LIB = None
_LOCK = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load_library():
    """Load the CUDA library; raise if it is missing (no CPU fallback)."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is missing: build it with "
                "`python -m paper_1904_12553_gb300.build`")
        lib = C.CDLL(path)
        vp, pp = C.c_void_p, C.POINTER(LbmParams)
        dp = C.c_void_p  # double* (host or device address)
        lib.lbm_nphase_derive.argtypes = [pp, C.POINTER(LbmModel)]
        lib.lbm_nphase_workspace_bytes.argtypes = [pp]
        lib.lbm_nphase_workspace_bytes.restype = C.c_size_t
        lib.lbm_nphase_create.argtypes = [pp, vp, C.c_size_t, vp,
                                          C.POINTER(vp)]
        lib.lbm_nphase_init.argtypes = [vp, dp, dp, C.c_double]
        lib.lbm_nphase_step.argtypes = [vp, C.c_int64]
        lib.lbm_nphase_moments.argtypes = [vp, dp, dp, dp, dp, dp]
        lib.lbm_nphase_diagnostics.argtypes = [vp, dp, dp, dp]
        lib.lbm_nphase_diagnostics_static.argtypes = [vp, dp, dp, dp]
        lib.lbm_nphase_steps_taken.argtypes = [vp]
        lib.lbm_nphase_steps_taken.restype = C.c_int64
        lib.lbm_nphase_cuda_error.argtypes = [vp]
        lib.lbm_nphase_batch_workspace_bytes.argtypes = [pp, C.c_int]
        lib.lbm_nphase_batch_workspace_bytes.restype = C.c_size_t
        lib.lbm_nphase_batch_create.argtypes = [pp, C.c_int, vp, C.c_size_t,
                                                vp, C.POINTER(vp)]
        lib.lbm_nphase_batch_init.argtypes = [vp, C.c_int, dp, dp, C.c_double]
        lib.lbm_nphase_batch_step.argtypes = [vp, C.c_int64]
        lib.lbm_nphase_selftest_wait_timeout.argtypes = [vp]
        lib.lbm_nphase_batch_case.argtypes = [vp, C.c_int]
        lib.lbm_nphase_batch_case.restype = vp
        lib.lbm_nphase_batch_moments.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp]
        lib.lbm_nphase_batch_diagnostics.argtypes = [vp, C.c_int, dp, dp, dp]
        lib.lbm_nphase_batch_autotune.argtypes = [vp, C.c_int,
                                                  C.POINTER(C.c_double)]
        lib.lbm_nphase_batch_set_schedule.argtypes = [vp, C.POINTER(LbmSchedule)]
        lib.lbm_nphase_batch_get_schedule.argtypes = [vp, C.POINTER(LbmSchedule)]
        lib.lbm_nphase_batch_size.argtypes = [vp]
        lib.lbm_nphase_batch_destroy.argtypes = [vp]
        for name in ("create", "init", "step", "autotune", "set_schedule",
                     "get_schedule", "destroy"):
            getattr(lib, "lbm_nphase_batch_" + name).restype = C.c_int
        lib.lbm_nphase_state_bytes.argtypes = [vp]
        lib.lbm_nphase_state_bytes.restype = C.c_size_t
        lib.lbm_nphase_get_state.argtypes = [vp, vp, C.c_size_t]
        lib.lbm_nphase_get_state.restype = C.c_int
        lib.lbm_nphase_set_state.argtypes = [vp, vp, C.c_size_t]
        lib.lbm_nphase_set_state.restype = C.c_int
        lib.lbm_nphase_uses_pipelined_kernel.argtypes = [vp]
        lib.lbm_nphase_uses_pipelined_kernel.restype = C.c_int
        lib.lbm_nphase_destroy.argtypes = [vp]
        lib.lbm_nphase_strerror.argtypes = [C.c_int]
        lib.lbm_nphase_strerror.restype = C.c_char_p
        for name in ("derive", "create", "init", "step", "moments",
                     "diagnostics", "diagnostics_static", "destroy"):
            getattr(lib, "lbm_nphase_" + name).restype = C.c_int
        _LIB = lib
        return lib


def _check(st: int, where: str):
    if st != 0:
        raise LbmError(st, where)


def make_params(p: dict) -> LbmParams:
    """Fill the C parameter struct from a workload parameter dict."""
    N = int(p["N"])
    s = LbmParams()
    s.N, s.nx, s.ny = N, int(p["nx"]), int(p["ny"])
    s.lattice = int(p.get("lattice", 0))
    s.nz = int(p.get("nz", 1 if s.lattice == 1 else 0))
    s.wall_y = int(p.get("wall_y", 0))
    prec = p.get("precision", "fp64")
    s.precision = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    s.grad_scheme = int(p.get("grad_scheme", 0))
    n = max(0, min(N, MAXN))  # out-of-range N is rejected by the library
    for k in range(n):
        s.rho[k] = float(p["rho"][k])
        for l in range(n):
            s.sigma[k][l] = float(p["sigma"][k][l])
    s.eta = float(p["eta"])
    s.beta = float(p.get("beta", 0.0))
    s.tau_g = float(p["tau_g"])
    for i in range(max(0, n - 1)):
        s.tau[i] = float(p["tau"][i])
        s.mobility[i] = float(p["mobility"][i])
    g = list(p.get("gravity", (0.0, 0.0))) + [0.0, 0.0]
    s.gravity[0], s.gravity[1], s.gravity[2] = float(g[0]), float(g[1]), float(g[2])
    s.rho0 = float(p.get("rho0", 1.0))
    return s


# ---------------------------------------------------------------------------
# C functions, same names
# ---------------------------------------------------------------------------

def strerror(status: int) -> str:
    return load_library().lbm_nphase_strerror(int(status)).decode()


def lbm_nphase_derive(params: dict) -> dict:
    lib = load_library()
    m = LbmModel()
    _check(lib.lbm_nphase_derive(C.byref(make_params(params)), C.byref(m)),
           "lbm_nphase_derive")
    n = int(params["N"]) - 1
    lam = np.array([[m.lambda_[i][j] for j in range(n)] for i in range(n)])
    return {"lambda": lam, "lambda_eig_min": m.lambda_eig_min,
            "lambda_eig_max": m.lambda_eig_max, "beta": m.beta,
            "a": np.array([m.a[i] for i in range(n)]), "Gamma": m.Gamma,
            "nu": m.nu, "uniform_density": bool(m.uniform_density)}


def lbm_nphase_workspace_bytes(params: dict) -> int:
    return int(load_library().lbm_nphase_workspace_bytes(
        C.byref(make_params(params))))


def lbm_nphase_create(params: dict, workspace_ptr: int, nbytes: int,
                      stream_ptr: int) -> int:
    lib = load_library()
    h = C.c_void_p()
    _check(lib.lbm_nphase_create(C.byref(make_params(params)),
                                 C.c_void_p(workspace_ptr), nbytes,
                                 C.c_void_p(stream_ptr), C.byref(h)),
           "lbm_nphase_create")
    return h.value


def lbm_nphase_init(handle: int, c_ptr: int, u_ptr, p0: float = 0.0):
    _check(load_library().lbm_nphase_init(C.c_void_p(handle), c_ptr,
                                          u_ptr or None, float(p0)),
           "lbm_nphase_init")


def lbm_nphase_step(handle: int, nsteps: int):
    _check(load_library().lbm_nphase_step(C.c_void_p(handle), int(nsteps)),
           "lbm_nphase_step")


def lbm_nphase_moments(handle: int, phi=None, c=None, u=None, p=None,
                       rho=None):
    _check(load_library().lbm_nphase_moments(
        C.c_void_p(handle), phi or None, c or None, u or None, p or None,
        rho or None), "lbm_nphase_moments")


def lbm_nphase_diagnostics(handle: int, N: int):
    mass = np.zeros(N)
    ke = np.zeros(1)
    um = np.zeros(1)
    _check(load_library().lbm_nphase_diagnostics(
        C.c_void_p(handle), mass.ctypes.data, ke.ctypes.data, um.ctypes.data),
        "lbm_nphase_diagnostics")
    return mass, float(ke[0]), float(um[0])


def lbm_nphase_diagnostics_static(handle: int, N: int):
    """Diagnostics whose scratch is the library's static device array (for
    callers that cannot allocate device memory); same results as
    lbm_nphase_diagnostics."""
    mass = np.zeros(N)
    ke = np.zeros(1)
    um = np.zeros(1)
    _check(load_library().lbm_nphase_diagnostics_static(
        C.c_void_p(handle), mass.ctypes.data, ke.ctypes.data, um.ctypes.data),
        "lbm_nphase_diagnostics_static")
    return mass, float(ke[0]), float(um[0])


def lbm_nphase_steps_taken(handle: int) -> int:
    return int(load_library().lbm_nphase_steps_taken(C.c_void_p(handle)))


def lbm_nphase_state_bytes(handle: int) -> int:
    return int(load_library().lbm_nphase_state_bytes(C.c_void_p(handle)))


def lbm_nphase_get_state(handle: int, dst_ptr: int, nbytes: int):
    _check(load_library().lbm_nphase_get_state(C.c_void_p(handle),
                                               C.c_void_p(dst_ptr), nbytes),
           "lbm_nphase_get_state")


def lbm_nphase_set_state(handle: int, src_ptr: int, nbytes: int):
    _check(load_library().lbm_nphase_set_state(C.c_void_p(handle),
                                               C.c_void_p(src_ptr), nbytes),
           "lbm_nphase_set_state")


def lbm_nphase_uses_pipelined_kernel(handle: int) -> int:
    return int(load_library().lbm_nphase_uses_pipelined_kernel(
        C.c_void_p(handle)))


def lbm_nphase_destroy(handle: int):
    load_library().lbm_nphase_destroy(C.c_void_p(handle))


# ---------------------------------------------------------------------------
# Convenience wrapper: workspace and stream from PyTorch
# ---------------------------------------------------------------------------

class Solver:
    """One simulation on the current CUDA device.

    The workspace is a torch uint8 tensor owned by this object; the stream is
    torch's current stream unless one is given.
    """

    def __init__(self, params: dict, stream=None, device=None):
        import torch

        self.torch = torch
        self.params = dict(params)
        self.N = int(params["N"])
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        self.three_d = int(params.get("lattice", 0)) == 1
        self.nz = int(params.get("nz", 1)) if self.three_d else 1
        self.D = 3 if self.three_d else 2
        self.grid = ((self.nz,) if self.three_d else ()) + (self.ny, self.nx)
        self.V = self.nx * self.ny * self.nz
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        nbytes = lbm_nphase_workspace_bytes(params)
        if nbytes == 0:
            raise LbmError(1, "lbm_nphase_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8,
                                     device=self.device)
        self.handle = lbm_nphase_create(params, self.workspace.data_ptr(),
                                        nbytes, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_nphase_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, a, shape):
        t = self.torch
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
        a = a.to(device=self.device, dtype=t.float64).contiguous()
        assert tuple(a.shape) == shape, (a.shape, shape)
        return a

    def init(self, c0, u0=None, p0: float = 0.0):
        """c0[N][(nz)][ny][nx], u0[D][(nz)][ny][nx] (numpy or torch, host or
        device)."""
        c = self._dev(c0, (self.N,) + self.grid)
        u = None if u0 is None else self._dev(u0, (self.D,) + self.grid)
        lbm_nphase_init(self.handle, c.data_ptr(),
                        None if u is None else u.data_ptr(), p0)

    def step(self, n: int = 1):
        lbm_nphase_step(self.handle, n)

    def moments(self, numpy: bool = True) -> dict:
        t = self.torch
        sh = self.grid
        out = {"phi": t.empty((self.N - 1,) + sh, dtype=t.float64, device=self.device),
               "c": t.empty((self.N,) + sh, dtype=t.float64, device=self.device),
               "u": t.empty((self.D,) + sh, dtype=t.float64, device=self.device),
               "p": t.empty(sh, dtype=t.float64, device=self.device),
               "rho": t.empty(sh, dtype=t.float64, device=self.device)}
        lbm_nphase_moments(self.handle, out["phi"].data_ptr(),
                           out["c"].data_ptr(), out["u"].data_ptr(),
                           out["p"].data_ptr(), out["rho"].data_ptr())
        if numpy:
            return {k: v.cpu().numpy() for k, v in out.items()}
        return out

    def diagnostics(self):
        return lbm_nphase_diagnostics(self.handle, self.N)

    def get_state(self, device: bool = False):
        """The current state as a uint8 tensor (host, or device)."""
        t = self.torch
        n = lbm_nphase_state_bytes(self.handle)
        buf = t.empty(n, dtype=t.uint8,
                      device=self.device if device else "cpu")
        lbm_nphase_get_state(self.handle, buf.data_ptr(), n)
        return buf

    def set_state(self, blob):
        lbm_nphase_set_state(self.handle, blob.data_ptr(), blob.numel())

    @property
    def pipelined(self) -> bool:
        """True if steps run the TMA-pipelined D2Q9 kernel."""
        return lbm_nphase_uses_pipelined_kernel(self.handle) == 1

    @property
    def step_kernel(self) -> str:
        return {1: "pipelined (TMA)", 2: "z-marching 3-D",
                3: "z-marching 3-D (TMA)"}.get(
            lbm_nphase_uses_pipelined_kernel(self.handle), "generic tile")

    @property
    def steps_taken(self) -> int:
        return lbm_nphase_steps_taken(self.handle)


# ---------------------------------------------------------------------------
# Batched ensemble
# ---------------------------------------------------------------------------

def _param_array(params_list):
    arr = (LbmParams * len(params_list))()
    for i, p in enumerate(params_list):
        arr[i] = make_params(p)
    return arr


def lbm_nphase_batch_workspace_bytes(params_list) -> int:
    return int(load_library().lbm_nphase_batch_workspace_bytes(
        _param_array(params_list), len(params_list)))


def lbm_nphase_batch_create(params_list, workspace_ptr: int, nbytes: int,
                            stream_ptr: int) -> int:
    b = C.c_void_p()
    _check(load_library().lbm_nphase_batch_create(
        _param_array(params_list), len(params_list), C.c_void_p(workspace_ptr),
        nbytes, C.c_void_p(stream_ptr), C.byref(b)), "lbm_nphase_batch_create")
    return b.value


def lbm_nphase_batch_init(batch: int, case: int, c_ptr: int, u_ptr,
                          p0: float = 0.0):
    _check(load_library().lbm_nphase_batch_init(
        C.c_void_p(batch), int(case), c_ptr, u_ptr or None, float(p0)),
        "lbm_nphase_batch_init")


def lbm_nphase_batch_step(batch: int, nsteps: int):
    _check(load_library().lbm_nphase_batch_step(C.c_void_p(batch),
                                                int(nsteps)),
           "lbm_nphase_batch_step")


def lbm_nphase_selftest_wait_timeout(handle: int):
    _check(load_library().lbm_nphase_selftest_wait_timeout(C.c_void_p(handle)),
           "lbm_nphase_selftest_wait_timeout")


def lbm_nphase_batch_case(batch: int, case: int) -> int:
    return load_library().lbm_nphase_batch_case(C.c_void_p(batch), int(case))


def lbm_nphase_batch_moments(batch: int, case: int, phi=None, c=None, u=None,
                             p=None, rho=None):
    _check(load_library().lbm_nphase_batch_moments(
        C.c_void_p(batch), int(case), phi or None, c or None, u or None,
        p or None, rho or None), "lbm_nphase_batch_moments")


def lbm_nphase_batch_diagnostics(batch: int, case: int, N: int):
    mass = np.zeros(N)
    ke = np.zeros(1)
    um = np.zeros(1)
    _check(load_library().lbm_nphase_batch_diagnostics(
        C.c_void_p(batch), int(case), mass.ctypes.data, ke.ctypes.data,
        um.ctypes.data), "lbm_nphase_batch_diagnostics")
    return mass, float(ke[0]), float(um[0])


def lbm_nphase_batch_autotune(batch: int, trial_steps: int) -> float:
    ms = C.c_double()
    _check(load_library().lbm_nphase_batch_autotune(
        C.c_void_p(batch), int(trial_steps), C.byref(ms)),
        "lbm_nphase_batch_autotune")
    return ms.value


def lbm_nphase_batch_set_schedule(batch: int, tile_height: int, schedule: int,
                                  ctas: int = 0, pipelined: int = 0,
                                  chunk: int = 1):
    s = LbmSchedule(tile_height, schedule, ctas, pipelined, chunk)
    _check(load_library().lbm_nphase_batch_set_schedule(C.c_void_p(batch),
                                                        C.byref(s)),
           "lbm_nphase_batch_set_schedule")


def lbm_nphase_batch_get_schedule(batch: int) -> dict:
    s = LbmSchedule()
    _check(load_library().lbm_nphase_batch_get_schedule(C.c_void_p(batch),
                                                        C.byref(s)),
           "lbm_nphase_batch_get_schedule")
    return {"tile_height": s.tile_height, "schedule": s.schedule,
            "ctas": s.ctas, "pipelined": s.pipelined, "chunk": s.chunk}


def lbm_nphase_batch_destroy(batch: int):
    load_library().lbm_nphase_batch_destroy(C.c_void_p(batch))


class Batch:
    """Many independent grids advanced together (FP32, equal densities)."""

    SCHEDULES = {0: "strided", 1: "cost-balanced lists", 2: "dynamic"}

    def __init__(self, params_list, stream=None, device=None):
        import torch

        self.torch = torch
        self.params = [dict(p) for p in params_list]
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        nbytes = lbm_nphase_batch_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(1, "lbm_nphase_batch_workspace_bytes")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8,
                                     device=self.device)
        self.handle = lbm_nphase_batch_create(
            self.params, self.workspace.data_ptr(), nbytes,
            self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            lbm_nphase_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.params)

    def init(self, case: int, c0, u0=None, p0: float = 0.0):
        t = self.torch
        p = self.params[case]
        N, ny, nx = int(p["N"]), int(p["ny"]), int(p["nx"])
        c = t.as_tensor(np.ascontiguousarray(c0, dtype=np.float64)).to(self.device)
        assert tuple(c.shape) == (N, ny, nx)
        u = None
        if u0 is not None:
            u = t.as_tensor(np.ascontiguousarray(u0, dtype=np.float64)).to(self.device)
        lbm_nphase_batch_init(self.handle, case, c.data_ptr(),
                              None if u is None else u.data_ptr(), p0)

    def step(self, n: int = 1):
        lbm_nphase_batch_step(self.handle, n)

    def autotune(self, trial_steps: int = 3) -> float:
        return lbm_nphase_batch_autotune(self.handle, trial_steps)

    def set_schedule(self, tile_height: int, schedule: int, ctas: int = 0,
                     pipelined: bool = False, chunk: int = 1):
        lbm_nphase_batch_set_schedule(self.handle, tile_height, schedule, ctas,
                                      int(pipelined), chunk)

    def schedule(self) -> dict:
        return lbm_nphase_batch_get_schedule(self.handle)

    def case_handle(self, case: int) -> int:
        return lbm_nphase_batch_case(self.handle, case)

    def moments(self, case: int) -> dict:
        t = self.torch
        p = self.params[case]
        N, sh = int(p["N"]), (int(p["ny"]), int(p["nx"]))
        out = {"phi": t.empty((N - 1,) + sh, dtype=t.float64, device=self.device),
               "c": t.empty((N,) + sh, dtype=t.float64, device=self.device),
               "u": t.empty((2,) + sh, dtype=t.float64, device=self.device),
               "p": t.empty(sh, dtype=t.float64, device=self.device),
               "rho": t.empty(sh, dtype=t.float64, device=self.device)}
        lbm_nphase_batch_moments(self.handle, case, out["phi"].data_ptr(),
                                 out["c"].data_ptr(), out["u"].data_ptr(),
                                 out["p"].data_ptr(), out["rho"].data_ptr())
        return {k: v.cpu().numpy() for k, v in out.items()}

    def diagnostics(self, case: int):
        return lbm_nphase_batch_diagnostics(self.handle, case,
                                            int(self.params[case]["N"]))
