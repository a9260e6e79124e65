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


@pytest.mark.parametrize("s13", [0.6e-3, 0.8e-3, 1.0e-3])
def test_lens_neumann_angles(s13):
    """N=3 lens, 256x256, walls in y, FP32 storage: sigma_12 = 1e-3,
    sigma_13 = sigma_23 = s13, run to equilibrium (1e5 steps)."""
    from paper_1904_12553_gb300 import Solver
    w = W.lens(nx=256, ny=256, R=40, s13=s13, precision="fp32")
    s = Solver(w.params)
    s.init(w.c0)
    history = []
    for _ in range(10):
        s.step(10000)
        c = s.moments()["c"]
        d, hu, hd, _ = LM.measure(c[0], c[2])
        history.append(LM.angles(d, hu, hd))
    s.close()
    want = LM.neumann_symmetric(1e-3, s13)
    t1, t2 = history[-1]
    drift = max(abs(history[-1][0] - history[-2][0]),
                abs(history[-1][1] - history[-2][1]))
    print(f"\nlens s13={s13:g}: theta=({t1:.2f}, {t2:.2f}) neumann={want:.2f} "
          f"rel=({t1 / want - 1:+.3f}, {t2 / want - 1:+.3f}) "
          f"last-1e4-step drift={drift:.3f} deg")
    assert abs(t1 / want - 1) <= 0.05 and abs(t2 / want - 1) <= 0.05
