"""Physics of the GPU path on the paper's validation problems.

- Static drop (Section 4.1): the pressure jump of the FP32 and 16-bit storage
  forms agrees with the FP64 oracle's within 1%, and with sigma / R within 5%.
- Liquid lens (Section 4.2): contact angles theta = 2 arctan(2 h / d) of the
  equilibrated lens against the Neumann triangle, Eq. N32.
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1904_12553_gb300 import workloads as W

sys.path.insert(0, os.path.dirname(__file__))
import lens_measure as LM  # noqa: E402

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_12553_gb300 import build
    build.build()


def _drop(n=64, R=12.0, sig=1e-3):
    w = W.static_drops(nx=n, ny=n, R=R, centres=((n / 2, n / 2), (0, 0)),
                       N=3, sigma=sig)
    w.c0[2] = 0.0
    w.c0[0] = 1.0 - w.c0[1]
    return w


def _dp(m, n, R):
    y, x = np.mgrid[0:n, 0:n]
    r = np.hypot(x - n / 2, y - n / 2)
    return (m["p"][r < R / 2].mean()
            - m["p"][(m["c"][0] > 0.999) & (r > R + 12)].mean())


@pytest.fixture(scope="module")
def laplace_oracle():
    n, R, steps = 64, 12.0, 8000
    w = _drop(n, R)
    s = oracle.OracleSim(w.params)
    s.init(w.c0)
    s.step(steps)
    dp = _dp(s.moments(), n, R)
    s.close()
    return dp


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp16"])
def test_laplace_jump_of_each_form(prec, laplace_oracle):
    from paper_1904_12553_gb300 import Solver
    n, R, steps, sig = 64, 12.0, 8000, 1e-3
    w = _drop(n, R, sig)
    s = Solver({**w.params, "precision": prec})
    s.init(w.c0)
    s.step(steps)
    dp = _dp(s.moments(), n, R)
    s.close()
    rel = abs(dp / laplace_oracle - 1)
    print(f"\nLaplace {prec}: dp={dp:.6e} oracle={laplace_oracle:.6e} "
          f"rel={rel:.2e} sigma/R={sig / R:.6e}")
    assert rel <= (1e-9 if prec == "fp64" else 1e-2), rel
    assert abs(dp / (sig / R) - 1) <= 0.05


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_lens_precision_forms_2e4_steps(prec):
    """The lens (N=3, 256x256, walls, sigma_13 = 0.8e-3) after 2e4 steps in
    each reduced-precision form against FP64 on the GPU: max |dphi| <= 1e-3
    (measured 0.8-1.1e-4) and both contact angles within 0.05 degree."""
    from paper_1904_12553_gb300 import Solver
    w = W.lens(nx=256, ny=256, R=40, s13=0.8e-3, precision="fp64")
    out = {}
    for p in ("fp64", prec):
        s = Solver({**w.params, "precision": p})
        s.init(w.c0)
        s.step(20000)
        out[p] = s.moments()
        s.close()
    ref, g = out["fp64"], out[prec]
    assert np.abs(g["phi"] - ref["phi"]).max() <= 1e-3
    ang = []
    for m in (g, ref):
        d, hu, hd, _ = LM.measure(m["c"][0], m["c"][2])
        ang.append(LM.angles(d, hu, hd))
    assert max(abs(ang[0][0] - ang[1][0]), abs(ang[0][1] - ang[1][1])) <= 0.05


def _lens_angles(s13, beta=0.0):
    """Equilibrated lens (N=3, 256x256, walls in y, FP32, sigma_12 = 1e-3,
    sigma_13 = sigma_23 = s13): stepped in chunks of 2e4 until both angles
    move less than 0.05 degree per chunk (at most 1e6 steps)."""
    from paper_1904_12553_gb300 import Solver
    w = W.lens(nx=256, ny=256, R=40, s13=s13, precision="fp32", beta=beta)
    s = Solver(w.params)
    s.init(w.c0)
    prev, steps, drift = None, 0, None
    while steps < 1_000_000:
        s.step(20000)
        steps += 20000
        c = s.moments()["c"]
        d, hu, hd, _ = LM.measure(c[0], c[2])
        cur = LM.angles(d, hu, hd)
        if prev is not None:
            drift = max(abs(cur[0] - prev[0]), abs(cur[1] - prev[1]))
            if drift < 0.05:
                break
        prev = cur
    s.close()
    want = LM.neumann_symmetric(1e-3, s13)
    print(f"\nlens s13={s13:g} beta={beta}: steps={steps} d={d:.1f} "
          f"h=({hu:.1f}, {hd:.1f}) theta=({cur[0]:.2f}, {cur[1]:.2f}) "
          f"neumann={want:.2f} rel=({cur[0] / want - 1:+.3f}, "
          f"{cur[1] / want - 1:+.3f}) drift per 2e4 steps={drift:.3f} deg")
    return cur, want


@pytest.fixture(scope="module")
def lens_results():
    return {s13: _lens_angles(s13) for s13 in (0.6e-3, 0.8e-3, 1.0e-3)}


@pytest.mark.parametrize("s13", [0.8e-3, 1.0e-3])
def test_lens_neumann_angles(lens_results, s13):
    """Resolved lenses (theta = 51.3 and 60 degrees): within 3% of Eq. N32
    (1.0-2.0% measured when this test was written)."""
    (t1, t2), want = lens_results[s13]
    assert abs(t1 / want - 1) <= 0.03 and abs(t2 / want - 1) <= 0.03


def test_thin_lens_and_ordering(lens_results):
    """The thin lens (sigma_13 = 0.6e-3, theta = 33.6 degrees, ~22 nodes
    high) carries the finite-interface error of W = 4: -13% measured when
    this test was written. Angles must still rise with sigma_13 as Eq. N32
    says."""
    (t1, t2), want = lens_results[0.6e-3]
    assert abs(t1 / want - 1) <= 0.15 and abs(t2 / want - 1) <= 0.15
    th = [sum(lens_results[s][0]) / 2 for s in (0.6e-3, 0.8e-3, 1.0e-3)]
    assert th[0] < th[1] < th[2]


def _thickness(c_drop):
    """Largest vertical extent of the c_drop > 1/2 region (linear
    interpolation of the contour at both ends) over the columns."""
    ny, nx = c_drop.shape
    best = 0.0
    for x in range(nx):
        col = c_drop[:, x]
        idx = np.where(col > 0.5)[0]
        if len(idx) == 0 or idx.min() == 0 or idx.max() == ny - 1:
            continue
        lo, hi = idx.min(), idx.max()
        y0 = lo - 1 + (0.5 - col[lo - 1]) / (col[lo] - col[lo - 1])
        y1 = hi + (0.5 - col[hi]) / (col[hi + 1] - col[hi])
        best = max(best, y1 - y0)
    return best


@pytest.fixture(scope="module")
def puddles():
    """Equilibrated drops under gravity (densities 3:1:6, equal sigma =
    0.01, R = 30, 400x200, FP32), run in chunks of 2e4 steps until the
    thickness moves less than 0.02 per chunk (at most 4e5 steps)."""
    from paper_1904_12553_gb300 import Solver
    out = {}
    for g in (2e-5, 5e-5, 1e-4):
        w = W.puddle(g)
        s = Solver(w.params)
        s.init(w.c0)
        prev, steps = None, 0
        while steps < 400_000:
            s.step(20000)
            steps += 20000
            H = _thickness(s.moments()["c"][0])
            if prev is not None and abs(H - prev) < 0.02:
                break
            prev = H
        mass, ke, umax = s.diagnostics()
        s.close()
        Hd = LM.de_gennes_thickness(g, 0.01, 3.0, 1.0, 6.0)
        Hp = LM.de_gennes_thickness(g, 0.01, 3.0, 1.0, 6.0, upper=False)
        print(f"\npuddle g={g:g}: steps={steps} H={H:.2f} balance={Hd:.2f} "
              f"rel={H / Hd - 1:+.3f} (Eq. N37 as printed {Hp:.2f}, "
              f"rel={H / Hp - 1:+.3f}) umax={umax:.2e}")
        out[g] = (H, Hd)
    return out


def test_puddle_thickness_de_gennes(puddles):
    """Puddle thickness against de Gennes' balance including the upper
    fluid's density (densities 3:1:6): within 10% for g = 2e-5 .. 1e-4
    (-2.2%, +1.1%, +7.4% measured when written; the thinnest puddle, 13
    nodes, carries the interface-width error), falling with g."""
    hs = [puddles[g][0] for g in (2e-5, 5e-5, 1e-4)]
    assert hs[0] > hs[1] > hs[2]
    for g in (2e-5, 5e-5, 1e-4):
        H, Hd = puddles[g]
        assert abs(H / Hd - 1) <= 0.10, (g, H, Hd)


def test_puddle_geometry_parity_fp64():
    """Gravity, unequal densities (J~, grad rho) and walls on the puddle
    geometry, reduced to 100x50 with R = 10: FP64 GPU against the oracle
    after 1000 steps."""
    from paper_1904_12553_gb300 import Solver
    w = W.puddle(1e-4, nx=100, ny=50, R=10.0, precision="fp64")
    s = Solver(w.params)
    s.init(w.c0)
    s.step(1000)
    g = s.moments()
    s.close()
    o = oracle.run(w.params, w.c0, steps=1000)
    assert np.abs(g["phi"] - o["phi"]).max() <= 1e-10
    assert np.abs(g["u"] - o["u"]).max() <= 1e-12


def _centroid_y(c):
    y = np.arange(c.shape[0])[:, None]
    return float((c * y).sum() / c.sum())


@pytest.mark.parametrize("case", ["four", "five"])
def test_paper_applications_parity_fp64(case):
    """The paper's 320 x 200 application cases (Sections 5.1, 5.2), full
    size, FP64 GPU against the oracle after 300 steps."""
    from paper_1904_12553_gb300 import Solver
    w = W.paper_four_phase() if case == "four" else W.paper_five_phase()
    s = Solver(w.params)
    s.init(w.c0)
    s.step(300)
    g = s.moments()
    s.close()
    o = oracle.run(w.params, w.c0, steps=300)
    assert np.abs(g["phi"] - o["phi"]).max() <= 1e-11
    assert np.abs(g["u"] - o["u"]).max() <= 1e-13


def test_paper_four_phase_motion():
    """Section 5.1 to t = 12.25 (t = t_l / sqrt(D / g), D = 60): the drop of
    phase 1 (density 6 in phase 3 of density 3) falls, the bubble of phase 2
    (1 in 2) rises; per-phase mass is conserved."""
    from paper_1904_12553_gb300 import Solver
    w = W.paper_four_phase(precision="fp64")
    steps = int(12.25 * math.sqrt(60 / 1e-5))
    s = Solver(w.params)
    s.init(w.c0)
    m0, _, _ = s.diagnostics()
    s.step(steps)
    m1, ke, umax = s.diagnostics()
    c = s.moments()["c"]
    s.close()
    y1, y2 = _centroid_y(c[0]), _centroid_y(c[1])
    print(f"\nfour phases, {steps} steps: drop y 280 -> {y1:.1f}, bubble y 40 "
          f"-> {y2:.1f}, umax={umax:.3e}, mass drift "
          f"{np.abs(m1 / m0 - 1).max():.1e}")
    assert np.abs(m1 / m0 - 1).max() <= 1e-10
    assert y1 < 280 - 20 and y2 > 40 + 20
    assert math.isfinite(ke)


def test_paper_five_phase_motion():
    """Section 5.2 (Eq. N40) to t = 6: the drops of phases 1 and 2 (densities
    6, 4 in phase 4 of density 2) fall, phase 1 faster; the bubble of phase
    3 (1 in 3) rises; per-phase mass is conserved."""
    from paper_1904_12553_gb300 import Solver
    w = W.paper_five_phase(precision="fp64")
    steps = int(6.0 * math.sqrt(60 / 1e-5))
    s = Solver(w.params)
    s.init(w.c0)
    m0, _, _ = s.diagnostics()
    s.step(steps)
    m1, ke, umax = s.diagnostics()
    c = s.moments()["c"]
    s.close()
    y1, y2, y3 = (_centroid_y(c[k]) for k in range(3))
    print(f"\nfive phases, {steps} steps: drops y 280 -> {y1:.1f}, {y2:.1f}; "
          f"bubble y 40 -> {y3:.1f}; umax={umax:.3e}, mass drift "
          f"{np.abs(m1 / m0 - 1).max():.1e}")
    assert np.abs(m1 / m0 - 1).max() <= 1e-10
    assert y1 < y2 < 280 and y3 > 40
    assert math.isfinite(ke)
