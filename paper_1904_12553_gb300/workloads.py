"""Seeded synthetic workloads: initial volume fractions and model parameters.

This module holds the initial conditions only (interface profiles, drop
placement, parameter draws). It contains none of the lattice Boltzmann
arithmetic, so both the CUDA path and the CPU oracle can be fed from it.

The drop and interface profiles are the tanh forms the paper uses for its
initial conditions (Eqs. N31_a, N31_b, N35, N38, N39):
``c = 1/2 + 1/2 tanh(d / (sqrt(2) eta))`` with d the signed distance to the
interface. An interface width W = 4 lattice units is read as eta = sqrt(2).

Each generator returns a :class:`Workload`: a parameter dict whose keys match
the C-ABI parameter struct, the initial fractions ``c0[N][ny][nx]``, an
optional initial velocity ``u0[2][ny][nx]``, the initial pressure and the step
count of the workload.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

ETA_W4 = math.sqrt(2.0)  # W = 4  <=>  tanh(2 d / W) = tanh(d / (sqrt(2) eta))


@dataclasses.dataclass
class Workload:
    name: str
    params: dict
    c0: np.ndarray
    u0: Optional[np.ndarray] = None
    p0: float = 0.0
    steps: int = 0
    seed: Optional[int] = None

    @property
    def V(self) -> int:
        return (int(self.params["nx"]) * int(self.params["ny"])
                * int(self.params.get("nz", 1)))


def base_params(N: int, nx: int, ny: int, sigma, *, rho=None, tau=0.8,
                tau_g=None, mobility=0.1, eta=ETA_W4, wall_y=0,
                precision="fp64", gravity=(0.0, 0.0), beta=0.0,
                grad_scheme=0) -> dict:
    """Parameter dict. ``sigma`` is a scalar (all pairs) or an NxN array."""
    if np.isscalar(sigma):
        sig = np.full((N, N), float(sigma))
        np.fill_diagonal(sig, 0.0)
    else:
        sig = np.array(sigma, dtype=np.float64)
    taus = [float(tau)] * (N - 1) if np.isscalar(tau) else [float(t) for t in tau]
    mobs = ([float(mobility)] * (N - 1) if np.isscalar(mobility)
            else [float(m) for m in mobility])
    return {
        "N": N, "nx": nx, "ny": ny, "wall_y": int(wall_y),
        "precision": precision, "grad_scheme": int(grad_scheme),
        "rho": [1.0] * N if rho is None else [float(r) for r in rho],
        "sigma": sig.tolist(), "eta": float(eta), "beta": float(beta),
        "tau_g": float(taus[0] if tau_g is None else tau_g),
        "tau": taus, "mobility": mobs,
        "gravity": [float(gravity[0]), float(gravity[1])], "rho0": 1.0,
    }


# --------------------------------------------------------------------------
# Profiles
# --------------------------------------------------------------------------

def _step(d, eta):
    """Smooth step 1/2 + 1/2 tanh(d / (sqrt 2 eta))."""
    return 0.5 + 0.5 * np.tanh(d / (math.sqrt(2.0) * eta))


def _grid(nx, ny):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y


def _dist(x, y, xc, yc, nx, ny, px=True, py=True):
    dx = x - xc
    dy = y - yc
    if px:
        dx = dx - nx * np.round(dx / nx)
    if py:
        dy = dy - ny * np.round(dy / ny)
    return np.sqrt(dx * dx + dy * dy)


def drop(nx, ny, xc, yc, R, eta=ETA_W4, px=True, py=True):
    """Circular drop fraction 1/2 + 1/2 tanh((R - r) / (sqrt 2 eta))."""
    x, y = _grid(nx, ny)
    return _step(R - _dist(x, y, xc, yc, nx, ny, px, py), eta)


def _layer(ny, nx, lo, hi, eta):
    """Periodic-in-y smooth indicator of the band lo <= y < hi (images -1..1)."""
    _, y = _grid(nx, ny)
    out = np.zeros((ny, nx))
    for m in (-1, 0, 1):
        out += _step(y + m * ny - lo, eta) - _step(y + m * ny - hi, eta)
    return out


# --------------------------------------------------------------------------
# Surface tensions
# --------------------------------------------------------------------------

def triangle_ok(sig: np.ndarray, margin: float = 1e-4) -> bool:
    """Strict triangle inequality on every triple of phases."""
    N = sig.shape[0]
    for a in range(N):
        for b in range(N):
            for c in range(N):
                if len({a, b, c}) < 3:
                    continue
                if not sig[a, b] < sig[a, c] + sig[b, c] - margin:
                    return False
    return True


def sample_sigma(rng: np.random.Generator, N: int, lo=5e-4, hi=2e-3,
                 accept: Optional[Callable[[np.ndarray], bool]] = None,
                 max_tries: int = 10000) -> np.ndarray:
    """Seeded sigma_kl ~ U[lo, hi] with strict triangle inequalities.

    ``accept`` is an extra test supplied by the caller (for instance that the
    mixing-energy matrix derived from sigma is well conditioned); draws are
    repeated from the same stream until it passes.
    """
    for _ in range(max_tries):
        sig = np.zeros((N, N))
        for k in range(N):
            for l in range(k + 1, N):
                sig[k, l] = sig[l, k] = rng.uniform(lo, hi)
        if triangle_ok(sig) and (accept is None or accept(sig)):
            return sig
    raise RuntimeError("no admissible sigma drawn")


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def static_drops(nx=128, ny=128, R=20.0, centres=((40, 64), (88, 64)), N=3,
                 sigma=1e-3, tau=0.8, mobility=0.1, rho=None,
                 precision="fp64", steps=1000, eta=ETA_W4) -> Workload:
    """Static drops (Section 4.1): phase 1 background, phases 2..N drops.

    The default is the N=3, 128x128 periodic FP64 case: drops of radius 20
    at (40, 64) and (88, 64), sigma = 1e-3, tau = 0.8, M = 0.1.
    """
    assert len(centres) == N - 1
    c = np.zeros((N, ny, nx))
    for j, (xc, yc) in enumerate(centres):
        c[j + 1] = drop(nx, ny, xc, yc, R, eta)
    c[0] = 1.0 - c[1:].sum(0)
    p = base_params(N, nx, ny, sigma, rho=rho, tau=tau, mobility=mobility,
                    precision=precision, eta=eta)
    return Workload(f"static_drops_N{N}_{nx}x{ny}", p, c, None, 0.0, steps)


def paper_static_drops(N=3, absent=None, nx=300, ny=100, R=20.0,
                       precision="fp64", eta=ETA_W4, steps=20000) -> Workload:
    """The paper's static drops (Section 4.1, Eqs. N31_a, N31_b): drops of
    phases 1..N-1 (R = 20) at (50, 50), (150, 50), (250, 50) in phase N, a
    300 x 100 periodic box; densities 20:1:5 (N = 3) or 20:1:10:5 (N = 4),
    all sigma = 0.01, tau = 0.8, m = 0.001, eta = sqrt(2), beta = sqrt(0.06).

    ``absent`` (a 0-based phase index) sets that phase's fraction to zero
    everywhere and leaves its drop out: the paper's reduction-consistency
    case is N = 4 with the third phase absent, against N = 3."""
    rho = {3: [20.0, 1.0, 5.0], 4: [20.0, 1.0, 10.0, 5.0]}[N]
    centres = ((50.0, 50.0), (150.0, 50.0), (250.0, 50.0))
    c = np.zeros((N, ny, nx))
    for j in range(N - 1):
        if j != absent:
            c[j] = drop(nx, ny, centres[j][0], centres[j][1], R, eta)
    c[N - 1] = 1.0 - c[:N - 1].sum(0)
    p = base_params(N, nx, ny, 0.01, rho=rho, tau=0.8, mobility=0.001,
                    precision=precision, eta=eta, beta=math.sqrt(0.06))
    tag = "" if absent is None else f"_absent{absent + 1}"
    return Workload(f"paper_static_drops_N{N}{tag}", p, c, None, 0.0, steps)


def lens(nx=256, ny=256, R=40.0, s13=0.8e-3, s12=1e-3, s23=None,
         tau=0.8, mobility=0.1, rho=None, precision="fp32", steps=20000,
         eta=ETA_W4, wall_y=1, N=3, beta=0.0) -> Workload:
    """Liquid lens (Section 4.2, Eq. N35 with the drop as phase 3).

    Phases 1 | 2 meet at a horizontal interface at y = ny/2; a drop of phase
    3 of radius R sits on it. Periodic in x, bounce-back walls in y.

    ``beta=0.0`` takes Eq. N36 (sigma_min), so the narrowest interface has
    the width of W = 4; ``beta="flat"`` fixes beta^2 = 3 sqrt(2) sigma_12 eta
    from the flat 1|2 interface (the paper's lens runs keep one beta for all
    tension ratios); a number sets it.
    """
    s23 = s13 if s23 is None else s23
    yc, xc = ny / 2.0, nx / 2.0
    c = np.zeros((N, ny, nx))
    c[2] = drop(nx, ny, xc, yc, R, eta, px=True, py=not wall_y)
    _, y = _grid(nx, ny)
    c[1] = np.maximum(_step(y - yc, eta) - c[2], 0.0)
    c[0] = 1.0 - c[1] - c[2]
    sig = np.zeros((N, N))
    sig[0, 1] = sig[1, 0] = s12
    sig[0, 2] = sig[2, 0] = s13
    sig[1, 2] = sig[2, 1] = s23
    if beta == "flat":
        beta = math.sqrt(3.0 * math.sqrt(2.0) * s12 * eta)
    p = base_params(N, nx, ny, sig, rho=rho, tau=tau, mobility=mobility,
                    precision=precision, eta=eta, wall_y=wall_y, beta=beta)
    return Workload(f"lens_{nx}x{ny}_s13_{s13:g}", p, c, None, 0.0, steps)


# Tension ratios sigma_12 : sigma_13 : sigma_23 of the paper's lens runs
# (Section 4.2, Tables 1 and 2).
PAPER_LENS_RATIOS = {
    "1:4/3:1": (1.0, 4.0 / 3.0, 1.0),
    "1:1:1": (1.0, 1.0, 1.0),
    "0.6:0.6:1": (0.6, 0.6, 1.0),
}


def paper_lens(ratio="1:1:1", scale="min", n=150, R=30.0,
               rho=(10.0, 1.0, 5.0), precision="fp64", eta=ETA_W4,
               beta=math.sqrt(0.06), steps=200000) -> Workload:
    """The paper's own liquid lens (Section 4.2, Eq. N35): a drop of phase 1
    (R = 30) centred on the flat interface between phase 2 above and phase 3
    below, in a 150 x 150 box periodic in x with halfway bounce-back walls in
    y; densities 10:1:5, tau_g = tau_i = 0.8, m_i = 0.1, eta = sqrt(2),
    beta = sqrt(0.06).

    The paper gives the tensions only as ratios. ``scale="min"`` makes the
    smallest tension 0.01, the value for which Eq. N36 gives the stated
    beta = sqrt(0.06) at eta = sqrt(2) (as in the static-drop runs of
    Section 4.1); ``scale="unit"`` takes the ratio's 1 as 0.01 (for 0.6:0.6:1
    this puts sigma_min at 0.006, where Eq. N36 would give beta^2 = 0.036).
    A number sets the scale itself.
    """
    r12, r13, r23 = PAPER_LENS_RATIOS[ratio]
    if scale == "min":
        unit = 0.01 / min(r12, r13, r23)
    elif scale == "unit":
        unit = 0.01
    else:
        unit = float(scale)
    N = 3
    xc, yc = (n - 1) / 2.0, (n - 1) / 2.0
    c = np.zeros((N, n, n))
    c[0] = drop(n, n, xc, yc, R, eta, px=True, py=False)
    _, y = _grid(n, n)
    c[1] = np.maximum(_step(y - yc, eta) - c[0], 0.0)
    c[2] = 1.0 - c[0] - c[1]
    sig = np.zeros((N, N))
    sig[0, 1] = sig[1, 0] = r12 * unit
    sig[0, 2] = sig[2, 0] = r13 * unit
    sig[1, 2] = sig[2, 1] = r23 * unit
    p = base_params(N, n, n, sig, rho=list(rho), tau=0.8, mobility=0.1,
                    precision=precision, eta=eta, wall_y=1,
                    beta=0.0 if beta is None else beta)
    return Workload(f"paper_lens_{ratio}_{n}", p, c, None, 0.0, steps)


def puddle(g, nx=400, ny=200, R=30.0, sigma=0.01, rho=(3.0, 1.0, 6.0),
           tau=0.8, mobility=0.1, precision="fp32", steps=200000,
           eta=ETA_W4) -> Workload:
    """Lens under gravity (Section 4.2, Eq. N37): a drop of phase 1
    (density 3) on the interface between phase 2 above (density 1) and phase
    3 below (density 6), body force G = (0, -rho g), walls in y, periodic in
    x, equal sigma. For large g the drop flattens into a puddle whose
    thickness the paper compares with de Gennes' asymptote (Eq. N37)."""
    N = 3
    yc, xc = ny / 2.0, nx / 2.0
    c = np.zeros((N, ny, nx))
    c[0] = drop(nx, ny, xc, yc, R, eta, px=True, py=False)
    _, y = _grid(nx, ny)
    c[1] = np.maximum(_step(y - yc, eta) - c[0], 0.0)
    c[2] = 1.0 - c[0] - c[1]
    p = base_params(N, nx, ny, sigma, rho=list(rho), tau=tau,
                    mobility=mobility, precision=precision, eta=eta, wall_y=1,
                    gravity=(0.0, -g))
    return Workload(f"puddle_g{g:g}_{nx}x{ny}", p, c, None, 0.0, steps)


def paper_four_phase(s13=0.01, precision="fp64", g=1e-5, eta=ETA_W4):
    """Droplet and bubble under gravity, four phases (Section 5.1):
    NY x NX = 320 x 200, walls in y; phase 1 drop (D = 60) at (160, 280) in
    phase 3 (upper half), phase 2 bubble at (160, 40) in phase 4 (lower
    half); densities 6:1:3:2; sigma_13 = s13, the other pairs 0.01;
    tau = 0.8, m = 0.1, beta = sqrt(0.06); G = (0, -rho g)."""
    N, nx, ny, R = 4, 200, 320, 30.0
    c = np.zeros((N, ny, nx))
    c[0] = drop(nx, ny, 160.0, 280.0, R, eta, px=True, py=False)
    c[1] = drop(nx, ny, 160.0, 40.0, R, eta, px=True, py=False)
    _, y = _grid(nx, ny)
    c[2] = _step(y - ny / 2.0, eta) * (1.0 - c[0])
    c[3] = 1.0 - c[0] - c[1] - c[2]
    sig = np.full((N, N), 0.01)
    np.fill_diagonal(sig, 0.0)
    sig[0, 2] = sig[2, 0] = s13
    p = base_params(N, nx, ny, sig, rho=[6.0, 1.0, 3.0, 2.0], tau=0.8,
                    mobility=0.1, precision=precision, eta=eta, wall_y=1,
                    gravity=(0.0, -g), beta=math.sqrt(0.06))
    return Workload(f"paper_four_phase_s13_{s13:g}", p, c, None, 0.0, 30000)


def paper_five_phase(rho=(6.0, 4.0, 1.0, 2.0, 3.0), precision="fp64", g=1e-5,
                     eta=ETA_W4, grad_scheme=1):
    """Droplets and interfaces, five phases (Section 5.2): 320 x 200, walls
    in y; drops of phases 1, 2 (R = 30) at (60, 280), (140, 280) in phase 4
    (upper), bubble of phase 3 at (100, 40) in phase 5 (lower); equal sigma
    = 0.01, tau = 0.8, m = 0.1, beta = sqrt(0.06), G = (0, -rho g), the
    mixed gradient scheme of Eq. N40."""
    N, nx, ny, R = 5, 200, 320, 30.0
    c = np.zeros((N, ny, nx))
    c[0] = drop(nx, ny, 60.0, 280.0, R, eta, px=True, py=False)
    c[1] = drop(nx, ny, 140.0, 280.0, R, eta, px=True, py=False)
    c[2] = drop(nx, ny, 100.0, 40.0, R, eta, px=True, py=False)
    _, y = _grid(nx, ny)
    c[4] = (1.0 - _step(y - ny / 2.0, eta)) * (1.0 - c[2])
    c[3] = 1.0 - c[0] - c[1] - c[2] - c[4]
    p = base_params(N, nx, ny, 0.01, rho=list(rho), tau=0.8, mobility=0.1,
                    precision=precision, eta=eta, wall_y=1,
                    gravity=(0.0, -g), beta=math.sqrt(0.06),
                    grad_scheme=grad_scheme)
    return Workload("paper_five_phase", p, c, None, 0.0, 30000)


def _place(rng, nx, ny, radii, gap, tries=20000):
    """Seeded non-overlapping centres with min-image spacing r_a+r_b+gap."""
    cs = []
    for r in radii:
        for _ in range(tries):
            xc, yc = rng.uniform(0, nx), rng.uniform(0, ny)
            ok = True
            for (xa, ya, ra) in cs:
                dx = (xc - xa) - nx * round((xc - xa) / nx)
                dy = (yc - ya) - ny * round((yc - ya) / ny)
                if math.hypot(dx, dy) < r + ra + gap:
                    ok = False
                    break
            if ok:
                cs.append((xc, yc, r))
                break
        else:
            raise RuntimeError("could not place drops")
    return cs


def collision(seed=3, n=512, N=4, R=50.0, spacing=120.0, speed=0.01,
              precision="fp32", steps=2000, accept=None,
              mobility=0.1) -> Workload:
    """N=4 drop collision: three radius-50 drops (phases 2-4) in phase 1.

    Centres are seeded with >= ``spacing`` min-image distance; each drop
    moves at ``speed`` toward the domain centre; sigma ~ U[5e-4, 2e-3]
    (strict triangle inequality, plus ``accept``); tau_g and tau_i ~
    U[0.6, 0.9]; M = 0.1; unit densities.
    """
    rng = np.random.default_rng(seed)
    sig = sample_sigma(rng, N, accept=accept)
    taus = rng.uniform(0.6, 0.9, size=N)  # tau_g, tau_1..tau_{N-1}
    scale = n / 512.0
    Rs = R * scale
    cs = _place(rng, n, n, [Rs] * (N - 1), spacing * scale - 2 * Rs)
    c = np.zeros((N, n, n))
    u = np.zeros((2, n, n))
    for j, (xc, yc, r) in enumerate(cs):
        cd = drop(n, n, xc, yc, r)
        c[j + 1] = cd
        vx, vy = n / 2.0 - xc, n / 2.0 - yc
        nrm = math.hypot(vx, vy) or 1.0
        u[0] += cd * speed * vx / nrm
        u[1] += cd * speed * vy / nrm
    c[0] = 1.0 - c[1:].sum(0)
    p = base_params(N, n, n, sig, tau=list(taus[1:]), tau_g=taus[0],
                    mobility=mobility, precision=precision)
    return Workload(f"collision_N{N}_{n}x{n}", p, c, u, 0.0, steps, seed)


def droplets_interfaces(seed=4, n=2048, N=5, ndrops=16, rmin=30.0, rmax=120.0,
                        tau=0.7, mobility=0.05, precision="fp32",
                        steps=10000, accept=None) -> Workload:
    """N=5 droplets and interfaces (Section 5.2 analogue, periodic).

    Phases 1 | 2 | 3 are stacked in y (interfaces at ny/3 and 2ny/3 and, by
    periodicity, one between 3 and 1); ``ndrops`` seeded drops of radius
    U[rmin, rmax] (scaled with n/2048) of phases 4 and 5 (alternating) do
    not overlap; the layer fractions are multiplied by 1 - sum(drops) as in
    Eqs. N38/N39. sigma ~ U[5e-4, 2e-3]; M = 0.05; tau = 0.7.
    """
    rng = np.random.default_rng(seed)
    sig = sample_sigma(rng, N, accept=accept)
    scale = n / 2048.0
    radii = sorted(rng.uniform(rmin * scale, rmax * scale, size=ndrops),
                   reverse=True)
    cs = _place(rng, n, n, radii, 8.0)
    c = np.zeros((N, n, n))
    for j, (xc, yc, r) in enumerate(cs):
        c[3 + (j % 2)] += drop(n, n, xc, yc, r)
    dsum = c[3] + c[4]
    y1, y2 = n / 3.0, 2.0 * n / 3.0
    l2 = _layer(n, n, y1, y2, ETA_W4)
    l3 = _layer(n, n, y2, n - 0.5, ETA_W4)
    l1 = 1.0 - l2 - l3
    c[0], c[1], c[2] = l1 * (1 - dsum), l2 * (1 - dsum), l3 * (1 - dsum)
    p = base_params(N, n, n, sig, tau=tau, mobility=mobility,
                    precision=precision)
    return Workload(f"droplets_interfaces_N{N}_{n}x{n}", p, c, None, 0.0,
                    steps, seed)


SIDES = (64, 96, 128, 192, 256, 384, 512)


def ensemble(seed=5, ncases=256, sides=SIDES, steps=2000, precision="fp32",
             accept=None):
    """Batched ensemble: independent static-drop or lens cases.

    Each case draws its grid side from ``sides``, N from {3, 4, 5}, sigma
    from U[5e-4, 2e-3] and its kind. A static-drop case puts N-1 drops
    (phases 2..N) in phase 1, periodic. A lens case puts a phase-3 drop on a
    1 | 2 interface with walls in y, plus N-3 small drops of the remaining
    phases.
    """
    rng = np.random.default_rng(seed)
    cases = []
    for ci in range(ncases):
        side = int(rng.choice(sides))
        N = int(rng.integers(3, 6))
        kind = "lens" if rng.random() < 0.5 else "static"
        sig = sample_sigma(rng, N, accept=accept)
        if kind == "static":
            R = side / 8.0
            cs = _place(rng, side, side, [R] * (N - 1), 6.0)
            c = np.zeros((N, side, side))
            for j, (xc, yc, r) in enumerate(cs):
                c[j + 1] = drop(side, side, xc, yc, r)
            c[0] = 1.0 - c[1:].sum(0)
            wall = 0
        else:
            R = side / 6.0
            c = np.zeros((N, side, side))
            c[2] = drop(side, side, side / 2.0, side / 2.0, R, py=False)
            others = np.zeros((side, side))
            for j in range(3, N):
                xc = side * (0.15 + 0.7 * (j - 3) / max(1, N - 3))
                c[j] = drop(side, side, xc, side * 0.25, side / 16.0,
                            py=False)
                others += c[j]
            _, y = _grid(side, side)
            c[1] = np.maximum(_step(y - side / 2.0, ETA_W4) - c[2], 0.0)
            c[1] *= (1.0 - others)
            c[0] = 1.0 - c[1:].sum(0)
            wall = 1
        p = base_params(N, side, side, sig, tau=0.8, mobility=0.1,
                        precision=precision, wall_y=wall)
        cases.append(Workload(f"case{ci}_{kind}_N{N}_{side}", p, c, None, 0.0,
                              steps, seed))
    return cases


def flat_interface(N=3, nx=8, ny=64, sigma=1e-3, tau=0.8, mobility=0.1,
                   precision="fp64", steps=5000, eta=ETA_W4) -> Workload:
    """Two flat tanh interfaces between phases 1 and 2 (periodic in y).

    Phase 2 occupies ny/4 <= y < 3ny/4. Other phases are absent.
    """
    c = np.zeros((N, ny, nx))
    c[1] = _layer(ny, nx, ny / 4.0, 3.0 * ny / 4.0, eta)
    c[0] = 1.0 - c[1]
    p = base_params(N, nx, ny, sigma, tau=tau, mobility=mobility,
                    precision=precision, eta=eta)
    return Workload(f"flat_N{N}_{nx}x{ny}", p, c, None, 0.0, steps)


def pair_band(sigma, k, l, rho=None, nx=4, ny=64, beta=0.0, eta=ETA_W4,
              tau=0.8, mobility=0.1, precision="fp64",
              steps=10000) -> Workload:
    """A band of phase k (ny/4 <= y < 3ny/4) in phase l, periodic in y, the
    other phases absent: two flat k|l interfaces. ``sigma`` is the NxN
    tension matrix of the whole system (0-based k, l)."""
    sig = np.array(sigma, dtype=np.float64)
    N = sig.shape[0]
    c = np.zeros((N, ny, nx))
    c[k] = _layer(ny, nx, ny / 4.0, 3.0 * ny / 4.0, eta)
    c[l] = 1.0 - c[k]
    p = base_params(N, nx, ny, sig, rho=rho, tau=tau, mobility=mobility,
                    precision=precision, eta=eta, beta=beta)
    return Workload(f"pair_band_{k + 1}{l + 1}_N{N}", p, c, None, 0.0, steps)


def quiescent(N=3, nx=16, ny=12, frac=None, precision="fp64", steps=1000,
              sigma=1e-3, rho=None, wall_y=0) -> Workload:
    """Spatially uniform mixture at rest."""
    frac = np.full(N, 1.0 / N) if frac is None else np.asarray(frac, float)
    c = np.broadcast_to(frac[:, None, None], (N, ny, nx)).copy()
    p = base_params(N, nx, ny, sigma, rho=rho, precision=precision,
                    wall_y=wall_y)
    return Workload(f"quiescent_N{N}_{nx}x{ny}", p, c, None, 0.0, steps)


def random_smooth(seed, N, nx, ny, rho=None, sigma=None, wall_y=0,
                  precision="fp64", amp_u=0.0, tau=None, mobility=None,
                  gravity=(0.0, 0.0), grad_scheme=0, nblobs=6) -> Workload:
    """Seeded random smooth mixture for parity tests (tiles, ragged tails).

    Sums of seeded drops of every phase, normalised to sum 1, with optional
    smooth random velocity of amplitude ``amp_u``.
    """
    rng = np.random.default_rng(seed)
    if sigma is None:
        sigma = sample_sigma(rng, N)
    c = np.full((N, ny, nx), 1e-3)
    for j in range(N):
        for _ in range(nblobs):
            xc, yc = rng.uniform(0, nx), rng.uniform(0, ny)
            R = rng.uniform(1.5, max(2.0, min(nx, ny) / 4.0))
            c[j] += rng.uniform(0.5, 1.0) * drop(nx, ny, xc, yc, R,
                                                  py=not wall_y)
    c /= c.sum(0, keepdims=True)
    u = None
    if amp_u:
        x, y = _grid(nx, ny)
        ph = rng.uniform(0, 2 * math.pi, size=4)
        u = np.stack([
            amp_u * np.sin(2 * math.pi * y / ny + ph[0]) * np.cos(2 * math.pi * x / nx + ph[1]),
            amp_u * np.cos(2 * math.pi * x / nx + ph[2]) * np.sin(2 * math.pi * y / ny + ph[3]),
        ])
    taus = rng.uniform(0.6, 1.2, size=N) if tau is None else np.full(N, tau)
    mobs = rng.uniform(0.02, 0.2, size=N - 1) if mobility is None else mobility
    p = base_params(N, nx, ny, sigma, rho=rho, tau=list(taus[1:]),
                    tau_g=taus[0], mobility=mobs, precision=precision,
                    wall_y=wall_y, gravity=gravity, grad_scheme=grad_scheme)
    return Workload(f"random_N{N}_{nx}x{ny}_s{seed}", p, c, u, 0.0, 0, seed)


# --------------------------------------------------------------------------
# Three dimensions (D3Q15)
# --------------------------------------------------------------------------

def _grid3(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def sphere(nx, ny, nz, xc, yc, zc, R, eta=ETA_W4, py=True):
    """Sphere fraction 1/2 + 1/2 tanh((R - r) / (sqrt 2 eta)), min-image
    distances in x and z (and y when periodic)."""
    x, y, z = _grid3(nx, ny, nz)
    dx = x - xc
    dx -= nx * np.round(dx / nx)
    dz = z - zc
    dz -= nz * np.round(dz / nz)
    dy = y - yc
    if py:
        dy -= ny * np.round(dy / ny)
    return _step(R - np.sqrt(dx * dx + dy * dy + dz * dz), eta)


def base_params3(N, nx, ny, nz, sigma, **kw) -> dict:
    """Parameter dict of a D3Q15 grid (keys of base_params plus nz and
    lattice = 1); gravity has three components."""
    g = kw.pop("gravity", (0.0, 0.0, 0.0))
    p = base_params(N, nx, ny, sigma, **kw)
    p.update(nz=int(nz), lattice=1, gravity=[float(v) for v in g])
    return p


def random_smooth3(seed, N, nx, ny, nz, rho=None, sigma=None, wall_y=0,
                   precision="fp64", amp_u=0.0, nblobs=4,
                   gravity=(0.0, 0.0, 0.0)) -> Workload:
    """Seeded random smooth 3-D mixture (spheres of every phase normalised
    to sum 1) with an optional smooth velocity, for parity tests."""
    rng = np.random.default_rng(seed)
    if sigma is None:
        sigma = sample_sigma(rng, N)
    c = np.full((N, nz, ny, nx), 1e-3)
    for j in range(N):
        for _ in range(nblobs):
            xc, yc, zc = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(0, nz)
            R = rng.uniform(1.5, max(2.0, min(nx, ny, nz) / 3.0))
            c[j] += rng.uniform(0.5, 1.0) * sphere(nx, ny, nz, xc, yc, zc, R,
                                                   py=not wall_y)
    c /= c.sum(0, keepdims=True)
    u = None
    if amp_u:
        x, y, z = _grid3(nx, ny, nz)
        ph = rng.uniform(0, 2 * math.pi, size=3)
        u = np.stack([
            amp_u * np.sin(2 * math.pi * y / ny + ph[0]) * np.cos(2 * math.pi * z / nz),
            amp_u * np.sin(2 * math.pi * z / nz + ph[1]) * np.cos(2 * math.pi * x / nx),
            amp_u * np.sin(2 * math.pi * x / nx + ph[2]) * np.cos(2 * math.pi * y / ny),
        ])
    taus = rng.uniform(0.6, 1.2, size=N)
    mobs = rng.uniform(0.02, 0.2, size=N - 1)
    p = base_params3(N, nx, ny, nz, sigma, rho=rho, tau=list(taus[1:]),
                     tau_g=taus[0], mobility=mobs, precision=precision,
                     wall_y=wall_y, gravity=gravity)
    return Workload(f"random3_N{N}_{nx}x{ny}x{nz}_s{seed}", p, c, u, 0.0, 0, seed)


def sphere_drops3(n=96, N=3, R=16.0, sigma=1e-3, precision="fp32", tau=0.8,
                  mobility=0.1, steps=2000) -> Workload:
    """N-1 sphere drops (phases 2..N) in phase 1 on an n^3 periodic D3Q15
    grid, spaced along x (the 3-D analogue of the static-drop case)."""
    c = np.zeros((N, n, n, n))
    for j in range(1, N):
        c[j] = sphere(n, n, n, n * j / N, n / 2.0, n / 2.0, R)
    c[0] = 1.0 - c[1:].sum(0)
    p = base_params3(N, n, n, n, sigma, tau=tau, mobility=mobility,
                     precision=precision)
    return Workload(f"sphere_drops3_N{N}_{n}", p, c, None, 0.0, steps)
