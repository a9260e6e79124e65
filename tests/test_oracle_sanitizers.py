"""Memory and undefined-behaviour check of the FP64 CPU oracle.

The oracle (oracle/lbm_oracle.c, oracle/lbm_oracle3d.c) is built a second
time with AddressSanitizer and UndefinedBehaviorSanitizer and driven from a
Python subprocess (sanitizer runtimes preloaded) through oracle.py, over
small ragged grids: every N, periodic and wall boundaries, both gradient
schemes (Eqs. N31 and N40), equal and unequal densities, and D3Q15. Any
out-of-bounds access, use after free or undefined operation ends the run
with a sanitizer report. A control library with a planted one-past-the-end
read shows that the sanitizers are active in that set-up.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = textwrap.dedent("""
    import os, sys
    root, lib = sys.argv[1], sys.argv[2]
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "oracle"))
    import numpy as np
    import oracle
    oracle._LIB_PATH = lib
    from paper_1904_12553_gb300 import workloads as W
    runs = 0
    for N in (2, 3, 4, 5):
        for wall in (0, 1):
            for scheme in (0, 1):
                for rho in (None, [2.0, 1.0, 3.0, 1.5, 2.5][:N]):
                    w = W.random_smooth(10 * N + wall, N, 13, 9, rho=rho, wall_y=wall,
                                        amp_u=0.01, grad_scheme=scheme)
                    o = oracle.run(w.params, w.c0, w.u0, steps=3)
                    assert np.isfinite(o["phi"]).all() and np.isfinite(o["u"]).all()
                    runs += 1
        w3 = W.random_smooth3(N, N, 9, 7, 5, wall_y=N % 2, amp_u=0.01)
        o3 = oracle.run3(w3.params, w3.c0, w3.u0, steps=2)
        assert np.isfinite(o3["phi"]).all()
        runs += 1
    print("runs", runs)
""")

CONTROL = textwrap.dedent("""
    #include <stdlib.h>
    double past_end(int n) {
      double *a = (double *)malloc((size_t)n * sizeof(double));
      for (int i = 0; i < n; ++i) a[i] = i;
      double s = a[n];  /* one past the end */
      free(a);
      return s;
    }
""")


def _runtimes():
    """Paths of gcc's ASan and UBSan runtimes, or None."""
    if shutil.which("gcc") is None:
        return None
    libs = []
    for name in ("libasan.so", "libubsan.so"):
        r = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
        path = r.stdout.strip()
        if r.returncode != 0 or not os.path.isabs(path) or not os.path.exists(path):
            return None
        libs.append(path)
    return libs


def _env(libs):
    env = dict(os.environ)
    env["LD_PRELOAD"] = ":".join(libs)
    env["ASAN_OPTIONS"] = "detect_leaks=0:halt_on_error=1"
    env["UBSAN_OPTIONS"] = "halt_on_error=1:print_stacktrace=1"
    env["OMP_NUM_THREADS"] = "2"
    return env


SAN = ["-fsanitize=address,undefined", "-fno-omit-frame-pointer", "-g", "-O1"]


@pytest.fixture(scope="module")
def runtimes():
    libs = _runtimes()
    if libs is None:
        pytest.skip("gcc sanitizer runtimes not available")
    return libs


def test_sanitizers_catch_a_planted_overrun(runtimes, tmp_path):
    src = tmp_path / "control.c"
    src.write_text(CONTROL)
    lib = tmp_path / "libcontrol.so"
    subprocess.run(["gcc", *SAN, "-fPIC", "-shared", "-o", str(lib), str(src)], check=True)
    code = ("import ctypes as C; l = C.CDLL(%r); l.past_end.restype = C.c_double; "
            "print(l.past_end(4))" % str(lib))
    r = subprocess.run([sys.executable, "-c", code], env=_env(runtimes),
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "runtime error" in r.stderr or "AddressSanitizer" in r.stderr


def test_oracle_runs_clean_under_sanitizers(runtimes, tmp_path):
    lib = tmp_path / "liblbm_oracle.so"
    subprocess.run(["gcc", *SAN, "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                    "-shared", "-o", str(lib), os.path.join(ROOT, "oracle", "lbm_oracle.c"),
                    os.path.join(ROOT, "oracle", "lbm_oracle3d.c"), "-lm"], check=True)
    driver = tmp_path / "drive.py"
    driver.write_text(DRIVER)
    r = subprocess.run([sys.executable, str(driver), ROOT, str(lib)], env=_env(runtimes),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "runtime error" not in r.stderr, r.stderr[-3000:]
    assert "AddressSanitizer" not in r.stderr, r.stderr[-3000:]
    assert "runs 36" in r.stdout
