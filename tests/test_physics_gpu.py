"""Physics of the GPU path on the paper's validation problems.

- Static drop (Section 4.1): the pressure jump of the FP32 and 16-bit storage
  forms agrees with the FP64 oracle's within 1%, and with sigma / R within 5%.
- Liquid lens (Section 4.2): contact angles theta = 2 arctan(2 h / d) of the
  equilibrated lens against the Neumann triangle (Eq. N32), length and cap
  heights against Eqs. N33/N34, for the paper's own case and the 256 x 256
  set; with unequal tensions against the model's own pair tensions.
- Reduction consistency (Section 4.1).
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


def _equilibrate(w, below, drop, chunk, tol, max_steps, prec=None):
    """Step a lens in chunks until both angles move less than `tol` degrees
    per chunk; returns (theta_1, theta_2, d, h_1, h_2, area, steps) from
    circles fitted to the caps (lens_measure.measure_fit)."""
    from paper_1904_12553_gb300 import Solver
    s = Solver({**w.params, **({"precision": prec} if prec else {})})
    s.init(w.c0)
    prev, steps = None, 0
    while steps < max_steps:
        s.step(chunk)
        steps += chunk
        c = s.moments()["c"]
        try:
            d, hu, hd, _ = LM.measure_fit(c[below], c[drop])
        except (ValueError, np.linalg.LinAlgError):  # no lens shape yet
            prev = None
            continue
        cur = LM.angles(d, hu, hd)
        if prev is not None and max(abs(cur[0] - prev[0]),
                                    abs(cur[1] - prev[1])) < tol:
            break
        prev = cur
    s.close()
    return cur[0], cur[1], d, hu, hd, LM.contour_area(c[drop]), steps


def _effective_neumann(params, drop, up, low, ny=64, steps=30000):
    """Eq. N32 with the model's own pair tensions: each pair's flat
    interfaces relaxed on the GPU (FP64, a band of one phase in the other,
    the third phase free to enter), tension = excess of the discrete free
    energy (lens_measure.band_tension). Returns the (upper, lower) angles."""
    import paper_1904_12553_gb300 as P
    from paper_1904_12553_gb300 import Solver
    sig = np.array(params["sigma"])
    d = P.lbm_nphase_derive(params)
    T = {}
    for k, l in ((drop, up), (drop, low), (up, low)):
        w = W.pair_band(sig, k, l, rho=params["rho"], ny=ny,
                        beta=params["beta"], eta=params["eta"])
        s = Solver(w.params)
        s.init(w.c0)
        s.step(steps)
        m = s.moments()
        s.close()
        T[(k, l)] = LM.band_tension(m["phi"][:, :, 0], m["c"][:, :, 0],
                                    d["lambda"], d["beta"], params["eta"])
    return LM.neumann(T[(drop, up)], T[(drop, low)], T[(up, low)])


@pytest.fixture(scope="module")
def paper_lens_results():
    """The paper's lens (Section 4.2: 150 x 150, R = 30, densities 10:1:5,
    tau = 0.8, m = 0.1, eta = sqrt(2), beta = sqrt(0.06), walls in y,
    sigma_min = 0.01), FP64, run to equilibrium (chunks of 2e4 steps, less
    than 0.01 degree per chunk, at most 1.6e6 steps)."""
    out = {}
    for ratio in ("1:1:1", "1:4/3:1", "0.6:0.6:1"):
        w = W.paper_lens(ratio)
        sig = np.array(w.params["sigma"])
        res = _equilibrate(w, 2, 0, 20000, 0.01, 1_600_000)
        nom = LM.neumann(sig[0, 1], sig[0, 2], sig[1, 2])
        eff = _effective_neumann(w.params, 0, 1, 2)
        print(f"\npaper lens {ratio}: steps={res[6]} theta=({res[0]:.2f}, "
              f"{res[1]:.2f}) d={res[2]:.2f} h=({res[3]:.2f}, {res[4]:.2f}) "
              f"A={res[5]:.1f}; Eq. N32 nominal ({nom[0]:.2f}, {nom[1]:.2f}),"
              f" with the model's pair tensions ({eff[0]:.2f}, {eff[1]:.2f})")
        out[ratio] = (res, nom, eff)
    return out


def test_paper_lens_equal_tensions_matches_eqs_n32_n34(paper_lens_results):
    """1:1:1: angles within 1% of Eq. N32 (60 degrees; 0.2% measured), and
    d, h_1, h_2 within 2% of Eqs. N33/N34 at the drop's area (0.2%)."""
    (t1, t2, d, h1, h2, A, _), nom, _ = paper_lens_results["1:1:1"]
    assert abs(t1 / nom[0] - 1) <= 0.01 and abs(t2 / nom[1] - 1) <= 0.01
    dd, g1, g2 = LM.lens_from_area(A, *nom)
    assert abs(d / dd - 1) <= 0.02
    assert abs(h1 / g1 - 1) <= 0.02 and abs(h2 / g2 - 1) <= 0.02


@pytest.mark.parametrize("ratio", ["1:4/3:1", "0.6:0.6:1"])
def test_paper_lens_unequal_tensions(paper_lens_results, ratio):
    """Unequal tensions: the model's pair interfaces adsorb the third phase
    and their tensions differ from the nominal sigma (see
    test_lens_measure.py). The lens follows Eq. N32 with those tensions
    within 1 degree (measured 0.2-0.3) and Eqs. N33/N34 at those angles
    within 2% in d, h_1, h_2 (measured <= 1%). Against the nominal
    tensions: 1:4/3:1 lands within 3% (85.8 and 47.0 against 83.6 and
    48.2 degrees), the thin 0.6:0.6:1 lens at 25 degrees against 33.6 (its
    angle passes 34 degrees about 3e4 steps in and keeps falling)."""
    (t1, t2, d, h1, h2, A, _), nom, eff = paper_lens_results[ratio]
    assert abs(t1 - eff[0]) <= 1.0 and abs(t2 - eff[1]) <= 1.0
    dd, g1, g2 = LM.lens_from_area(A, *eff)
    assert abs(d / dd - 1) <= 0.02
    assert abs(h1 / g1 - 1) <= 0.02 and abs(h2 / g2 - 1) <= 0.02
    if ratio == "1:4/3:1":
        assert abs(t1 / nom[0] - 1) <= 0.03 and abs(t2 / nom[1] - 1) <= 0.03


@pytest.fixture(scope="module")
def lens_results():
    """The 256 x 256 lens of the benchmark set (unit densities, sigma_12 =
    1e-3, sigma_13 = sigma_23 = s13, beta from Eq. N36), FP32, run to
    equilibrium (chunks of 4e4 steps, less than 0.01 degree per chunk, at
    most 4e6 steps)."""
    out = {}
    for s13 in (0.6e-3, 0.8e-3, 1.0e-3):
        w = W.lens(nx=256, ny=256, R=40, s13=s13, precision="fp32")
        res = _equilibrate(w, 0, 2, 40000, 0.01, 4_000_000)
        eff = _effective_neumann({**w.params, "precision": "fp64"}, 2, 1, 0)
        nom = LM.neumann_symmetric(1e-3, s13)
        print(f"\nlens s13={s13:g}: steps={res[6]} theta=({res[0]:.2f}, "
              f"{res[1]:.2f}) d={res[2]:.1f} h=({res[3]:.1f}, {res[4]:.1f}); "
              f"Eq. N32 nominal {nom:.2f}, with the model's pair tensions "
              f"({eff[0]:.2f}, {eff[1]:.2f})")
        out[s13] = (res, nom, eff)
    return out


@pytest.mark.parametrize("s13", [0.6e-3, 0.8e-3, 1.0e-3])
def test_lens_neumann_angles(lens_results, s13):
    """Both caps within 1 degree of Eq. N32 with the model's own pair
    tensions; the resolved lenses (51.3 and 60 degrees nominal) also within
    3% of the nominal angle."""
    (t1, t2, *_), nom, eff = lens_results[s13]
    assert abs(t1 - eff[0]) <= 1.0 and abs(t2 - eff[1]) <= 1.0
    if s13 > 0.7e-3:
        assert abs(t1 / nom - 1) <= 0.03 and abs(t2 / nom - 1) <= 0.03
    th = [sum(lens_results[s][0][:2]) / 2 for s in (0.6e-3, 0.8e-3, 1.0e-3)]
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


def test_reduction_consistency_four_phases_one_absent():
    """Section 4.1's reduction test: the paper's four-phase static drops
    (300 x 100, densities 20:1:10:5, sigma = 0.01, m = 0.001) with the third
    phase absent against the three-phase run (20:1:5), FP64, 2e4 steps.

    The model does not keep the absent phase at exactly zero (its chemical
    potential combination is not uniform at the other interfaces; see the
    oracle test of the start state), so the runs are "almost identical":
    measured after 2e4 steps max c_3 = 1.6e-3, the other fractions within
    1.2e-3 of the three-phase run, velocities within 1.3e-6 (max |u| 6.5e-6).
    Asserted at those levels with a margin of about 1.5; the FP64 path is
    first checked against the oracle on this geometry."""
    from paper_1904_12553_gb300 import Solver
    w4 = W.paper_static_drops(4, absent=2)
    w3 = W.paper_static_drops(3)
    s = Solver(w4.params)
    s.init(w4.c0)
    s.step(200)
    g = s.moments()
    o = oracle.run(w4.params, w4.c0, steps=200)
    assert np.abs(g["phi"] - o["phi"]).max() <= 1e-12
    assert np.abs(g["u"] - o["u"]).max() <= 1e-14
    s.step(20000 - 200)
    m4 = s.moments()
    s.close()
    s = Solver(w3.params)
    s.init(w3.c0)
    s.step(20000)
    m3 = s.moments()
    s.close()
    dc = [float(np.abs(m4["c"][a] - m3["c"][b]).max())
          for a, b in ((0, 0), (1, 1), (3, 2))]
    c3 = float(np.abs(m4["c"][2]).max())
    du = float(np.abs(m4["u"] - m3["u"]).max())
    print(f"\nreduction: max|dc| (1, 2, background) = {dc[0]:.2e}, "
          f"{dc[1]:.2e}, {dc[2]:.2e}; max c_3 = {c3:.2e}; max|du| = {du:.2e}"
          f" (max|u| {np.abs(m3['u']).max():.2e})")
    assert max(dc) <= 2e-3
    assert c3 <= 2.5e-3
    assert du <= 2e-6
