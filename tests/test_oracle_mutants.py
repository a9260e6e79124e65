"""Planted mistakes: each case copies the oracle's C sources, makes one
plausible mistake in the copy (a dropped term, a wrong sign, index or
factor), builds it, and runs one of the pins against that build, which must
fail. This shows that the pins which fix the oracle catch such a mistake.
The committed oracle is never modified; the copies live in a temporary
directory and run in a subprocess of their own."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
TESTS = os.path.join(ROOT, "tests")

# (name, source file, text in it, planted replacement, pin module, pin, kwargs)
MUTANTS = [
    ("g_eq second-order term dropped (Eq. 25)", "lbm_oracle.c",
     "cu * cu / (2.0 * CS2 * CS2)", "0.0 * cu",
     "test_oracle_pins", "test_geq_moments_appendix_a1a", {}),
    ("h_eq advective term sign (Eq. N25)", "lbm_oracle.c",
     "W[k] * (CX[k] * phi * ux + CY[k] * phi * uy) / CS2;",
     "W[k] * (CX[k] * phi * ux - CY[k] * phi * uy) / CS2;",
     "test_oracle_pins", "test_ch_equilibrium_and_source_moments", {}),
    ("G_k c.F term dropped (Eq. N20_1)", "lbm_oracle.c",
     "G[k] = W[k] * (ugr + cF / CS2 + QT / (2.0 * CS2 * CS2));",
     "G[k] = W[k] * (ugr + QT / (2.0 * CS2 * CS2));",
     "test_oracle_pins", "test_force_distribution_moments_appendix_a1b", {}),
    ("R_k prefactor sign (Eq. N26)", "lbm_oracle.c",
     "R[k] = (1.0 - 1.0 / (2.0 * tau_i))", "R[k] = (1.0 + 1.0 / (2.0 * tau_i))",
     "test_oracle_pins", "test_ch_equilibrium_and_source_moments", {}),
    ("Laplacian centre weight (Eq. N31b)", "lbm_oracle.c",
     "(z[nb(s, x, y, CX[k], CY[k])] - 2.0 * z[n] +",
     "(z[nb(s, x, y, CX[k], CY[k])] - 1.0 * z[n] +",
     "test_oracle_pins", "test_stencils_exact_on_quadratics", {"scheme": 0}),
    ("gradient neighbour index transposed (Eq. N31a)", "lbm_oracle.c",
     "d = (z[nb(s, x, y, CX[k], CY[k])] - z[nb(s, x, y, -CX[k], -CY[k])]) /",
     "d = (z[nb(s, x, y, CX[k], CY[k])] - z[nb(s, x, y, -CY[k], -CX[k])]) /",
     "test_oracle_pins", "test_stencils_exact_on_quadratics", {"scheme": 0}),
    ("h_i(c) factor (rho_i + rho_N)/2 lost (Eq. N17)", "lbm_oracle.c",
     "hf[i] = (p->rho_t[i] + p->rho_t[n]) / 2.0 * s;",
     "hf[i] = (p->rho_t[i] + p->rho_t[n]) * s;",
     "test_oracle_pins", "test_hfun_is_half_dH_dphi", {"N": 3}),
    ("c -> phi inverse sign", "lbm_oracle.c",
     "(p->rho_t[i] - p->rho_t[n])) /", "(p->rho_t[i] + p->rho_t[n])) /",
     "test_oracle_pins", "test_fractions_definitions", {"N": 3}),
    ("lambda right-hand side factor (Eq. N14)", "lbm_oracle.c",
     "b[row] = 4.5 * p->eta * p->eta", "b[row] = 3.0 * p->eta * p->eta",
     "test_oracle_pins", "test_lambda_golden_n3_equal_sigma", {}),
    ("bounce-back keeps the direction (Section 4.2)", "lbm_oracle.c",
     "*kk = OPP[k];", "*kk = k;",
     "test_oracle_pins", "test_channel_flow_between_walls", {"tau_g": 0.8}),
    ("stencil ghost row below the wall wraps around", "lbm_oracle.c",
     "if (yy < 0) yy = 0;", "if (yy < 0) yy += s->ny;",
     "test_oracle_pins", "test_wall_ghost_rows_mirror_the_fluid", {"scheme": 0}),
    ("J~ sign (Eq. N18)", "lbm_oracle.c",
     "Jx -= m->kap[i] * m->p.mob[i] * s->gC[2 * i * V + q];",
     "Jx += m->kap[i] * m->p.mob[i] * s->gC[2 * i * V + q];",
     "test_oracle_pins", "test_mass_flux_and_density_gradient", {"N": 3}),
    ("J~ without the mobility (Eq. N18)", "lbm_oracle.c",
     "Jy -= m->kap[i] * m->p.mob[i] * s->gC[(2 * i + 1) * V + q];",
     "Jy -= m->kap[i] * s->gC[(2 * i + 1) * V + q];",
     "test_oracle_pins", "test_mass_flux_and_density_gradient", {"N": 3}),
    ("grad(rho) coefficient dropped (Eq. N18)", "lbm_oracle.c",
     "rx += m->kap[i] * s->gphi[2 * i * V + q];", "rx += s->gphi[2 * i * V + q];",
     "test_oracle_pins", "test_mass_flux_and_density_gradient", {"N": 3}),
    ("CH relaxation with tau_g instead of tau_i (Eq. N24)", "lbm_oracle.c",
     "double hs = hk - (hk - heq[k]) / m->p.tau[i] + R[k];",
     "double hs = hk - (hk - heq[k]) / tg + R[k];",
     "test_oracle_pins", "test_linear_ch_relaxation_rate", {"tau": 1.3}),
    ("pressure's u.grad(rho) weight (Eq. N23)", "lbm_oracle.c",
     "(sg + 0.5 * ugr + r * s_k(0, ux, uy))", "(sg + 1.5 * ugr + r * s_k(0, ux, uy))",
     "test_oracle_pins", "test_translating_interface_with_density_contrast", {}),
    ("start without (phi u)_prev (reading 8)", "lbm_oracle.c",
     "s->phi_prev[i * V + q] = s->phi[i * V + q];", "s->phi_prev[i * V + q] = 0.0;",
     "test_oracle_pins", "test_uniform_flow_populations_are_stationary", {}),
    ("start with u_prev = 0 (reading 8)", "lbm_oracle.c",
     "s->u_prev[q] = ux;", "s->u_prev[q] = 0.0;",
     "test_oracle_pins", "test_uniform_flow_populations_are_stationary", {}),
    ("kinetic energy without the 1/2", "lbm_oracle.c",
     "e += 0.5 * s->rho[q] * u2;", "e += s->rho[q] * u2;",
     "test_oracle_pins", "test_diagnostics_of_known_states", {}),
    ("a_i of Eq. N30 with tau_i - 1/4", "lbm_oracle.c",
     "m->a[i] = p->mob[i] / (CS2 * (p->tau[i] - 0.5));",
     "m->a[i] = p->mob[i] / (CS2 * (p->tau[i] - 0.25));",
     "test_oracle_pins", "test_linear_ch_relaxation_rate", {"tau": 1.0}),
    ("beta of Eq. N36 with 2 sqrt 2", "lbm_oracle.c",
     "return sqrt(3.0 * sqrt(2.0) * smin * p->eta);", "return sqrt(2.0 * sqrt(2.0) * smin * p->eta);",
     "test_oracle_pins", "test_surface_tension_integral", {}),
    ("mixed gradient upwind weight (Eq. N40)", "lbm_oracle.c",
     "5.0 * z[nb(s, x, y, CX[k], CY[k])] - 3.0 * z[n] -",
     "4.0 * z[nb(s, x, y, CX[k], CY[k])] - 3.0 * z[n] -",
     "test_oracle_pins", "test_stencils_exact_on_quadratics", {"scheme": 1}),
    ("D3Q15 h_eq z term dropped", "lbm_oracle3d.c",
     "CY[k] * phi * u[1] + CZ[k] * phi * u[2]) / CS2;", "CY[k] * phi * u[1]) / CS2;",
     "test_oracle3d_pins", "test_ch3_moments", {}),
    ("D3Q15 G_k c.F term dropped", "lbm_oracle3d.c",
     "G[k] = W[k] * (ugr + cF / CS2 + QT / (2.0 * CS2 * CS2));",
     "G[k] = W[k] * (ugr + QT / (2.0 * CS2 * CS2));",
     "test_oracle3d_pins", "test_force_dist3_moments", {}),
    ("D3Q15 R_k prefactor sign", "lbm_oracle3d.c",
     "R[k] = (1.0 - 1.0 / (2.0 * tau_i))", "R[k] = (1.0 + 1.0 / (2.0 * tau_i))",
     "test_oracle3d_pins", "test_ch3_moments", {}),
    ("D3Q15 J~ sign", "lbm_oracle3d.c",
     "J -= m->kap[i] * m->p.mob[i] * s->gC[(3 * i + a) * V + q];",
     "J += m->kap[i] * m->p.mob[i] * s->gC[(3 * i + a) * V + q];",
     "test_oracle3d_pins", "test_mass_flux_and_density_gradient3", {}),
    ("D3Q15 pressure's u.grad(rho) weight", "lbm_oracle3d.c",
     "(sg + 0.5 * ugr + r * s_k(0, u))", "(sg + 1.5 * ugr + r * s_k(0, u))",
     "test_oracle3d_pins", "test_translating_interface_with_density_contrast3", {}),
    ("D3Q15 gravity dropped", "lbm_oracle3d.c",
     "F[a] = r * m->p.grav[a];", "F[a] = 0.0;",
     "test_oracle3d_pins", "test_channel_flow_between_walls3", {"axis": 0}),
    ("D3Q15 bounce-back keeps the direction", "lbm_oracle3d.c",
     "*kk = opp(k);", "*kk = k;",
     "test_oracle3d_pins", "test_channel_flow_between_walls3", {"axis": 2}),
    ("D3Q15 CH relaxation with tau_g", "lbm_oracle3d.c",
     "hk - (hk - heq[k]) / m->p.tau[i] + R[k];", "hk - (hk - heq[k]) / tg + R[k];",
     "test_oracle3d_pins", "test_linear_ch_relaxation_rate3", {"tau": 1.3}),
    ("D3Q15 surface force sign", "lbm_oracle3d.c",
     "for (int i = 0; i < n; ++i) F[a] += s->C[i * V + q] * s->gphi[(3 * i + a) * V + q];",
     "for (int i = 0; i < n; ++i) F[a] -= s->C[i * V + q] * s->gphi[(3 * i + a) * V + q];",
     "test_oracle3d_pins", "test_laplace_law_cylinder3", {}),
    ("D3Q15 start without (phi u)_prev (reading 8)", "lbm_oracle3d.c",
     "s->phi_prev[i * V + q] = s->phi[i * V + q];", "s->phi_prev[i * V + q] = 0.0;",
     "test_oracle3d_pins", "test_uniform_flow3_populations_are_stationary", {}),
    ("D3Q15 g_eq second-order term dropped", "lbm_oracle3d.c",
     "cu * cu / (2.0 * CS2 * CS2)", "0.0 * cu",
     "test_oracle3d_pins", "test_geq3_moments", {}),
    ("D3Q15 Laplacian centre weight", "lbm_oracle3d.c",
     "- 2.0 * zf[q] +", "- 1.0 * zf[q] +",
     "test_oracle3d_pins", "test_stencils3_exact_on_quadratics", {}),
    ("D3Q15 streaming ignores z", "lbm_oracle3d.c",
     "*q = nb(s, x, y, z, CX[k], CY[k], CZ[k]);", "*q = nb(s, x, y, z, CX[k], CY[k], 0);",
     "test_oracle3d_pins", "test_flat_interface_along_z", {}),
]

_RUNNER = textwrap.dedent("""
    import sys
    sys.path[:0] = [{root!r}, {oracle!r}, {tests!r}]
    import oracle
    oracle._LIB_PATH = {lib!r}
    oracle.build = lambda force=False: oracle._LIB_PATH
    import importlib
    pins = importlib.import_module({module!r})
    try:
        getattr(pins, {pin!r})(**{kwargs!r})
    except AssertionError:
        print("PIN FAILED")
        sys.exit(3)
    print("PIN PASSED")
""")


@pytest.mark.parametrize("name,src,old,new,module,pin,kwargs", MUTANTS,
                         ids=[m[0] for m in MUTANTS])
def test_pin_catches_planted_mistake(tmp_path, name, src, old, new, module, pin, kwargs):
    text = open(os.path.join(ORACLE, src)).read()
    assert text.count(old) == 1, f"planting site of '{name}' not found exactly once"
    for f in ("lbm_oracle.c", "lbm_oracle3d.c"):
        shutil.copy(os.path.join(ORACLE, f), tmp_path / f)
    (tmp_path / src).write_text(text.replace(old, new))
    lib = str(tmp_path / "liblbm_oracle_planted.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                    "-shared", "-o", lib, str(tmp_path / "lbm_oracle.c"),
                    str(tmp_path / "lbm_oracle3d.c"), "-lm"], check=True)
    code = _RUNNER.format(root=ROOT, oracle=ORACLE, tests=TESTS, lib=lib,
                          module=module, pin=pin, kwargs=kwargs)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
    assert r.returncode == 3 and "PIN FAILED" in r.stdout, (name, r.returncode,
                                                            r.stdout[-500:], r.stderr[-2000:])


def test_unplanted_copy_passes(tmp_path):
    """Control: the same harness on an unmodified copy passes the pins."""
    for f in ("lbm_oracle.c", "lbm_oracle3d.c"):
        shutil.copy(os.path.join(ORACLE, f), tmp_path / f)
    lib = str(tmp_path / "liblbm_oracle_copy.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
                    "-shared", "-o", lib, str(tmp_path / "lbm_oracle.c"),
                    str(tmp_path / "lbm_oracle3d.c"), "-lm"], check=True)
    for module, pin, kwargs in {(m[4], m[5], tuple(sorted(m[6].items()))) for m in MUTANTS}:
        code = _RUNNER.format(root=ROOT, oracle=ORACLE, tests=TESTS, lib=lib,
                              module=module, pin=pin, kwargs=dict(kwargs))
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           timeout=600, env=dict(os.environ, OMP_NUM_THREADS="4"))
        assert r.returncode == 0 and "PIN PASSED" in r.stdout, (pin, r.stderr[-2000:])
