"""Pins of the D3Q15 oracle (the 3-D lattice of Section 3.1) against the
moment conditions of the appendix, stencil exactness, conservation and
stationarity (same statements as the 2-D pins, on 15 velocities)."""
import numpy as np
import pytest

import oracle
from paper_1904_12553_gb300 import workloads as W

# D3Q15 velocities as printed in Section 3.1 (columns k = 0..14).
CV = np.array([[0, 1, 0, 0, -1, 0, 0, 1, 1, 1, -1, -1, -1, -1, 1],
               [0, 0, 1, 0, 0, -1, 0, 1, 1, -1, 1, -1, -1, 1, -1],
               [0, 0, 0, 1, 0, 0, -1, 1, -1, 1, 1, -1, 1, -1, -1]],
              dtype=float).T
CS2 = 1.0 / 3.0


def test_geq3_moments():
    rng = np.random.default_rng(0)
    d = np.eye(3)
    for _ in range(30):
        r0, pr, rho = rng.uniform(-2, 2), rng.uniform(-1e-2, 1e-2), rng.uniform(0.5, 9)
        u = rng.uniform(-0.1, 0.1, 3)
        g = oracle.geq3(r0, pr, rho, u)
        assert abs(g.sum() - r0) < 1e-13
        np.testing.assert_allclose(CV.T @ g, rho * u, atol=1e-14 * rho)
        np.testing.assert_allclose(np.einsum("k,ka,kb->ab", g, CV, CV),
                                   pr * d + rho * np.outer(u, u), atol=1e-14 * rho)
        want = rho * CS2 * (np.einsum("ab,c->abc", d, u) + np.einsum("ac,b->abc", d, u)
                            + np.einsum("bc,a->abc", d, u))
        np.testing.assert_allclose(np.einsum("k,ka,kb,kc->abc", g, CV, CV, CV),
                                   want, atol=1e-14 * rho)


def test_force_dist3_moments():
    rng = np.random.default_rng(1)
    for _ in range(30):
        tg = rng.uniform(0.55, 2.0)
        u, F, gr, J = (rng.uniform(-1, 1, 3) * s for s in (0.1, 1e-4, 1.0, 1e-3))
        G = oracle.force_dist3(tg, u, F, gr, J)
        assert abs(G.sum() - u @ gr) < 1e-15
        np.testing.assert_allclose(CV.T @ G, F, atol=1e-17)
        Ju = np.outer(J, u) / (tg - 0.5)
        want = (np.outer(u, F) + np.outer(F, u) + CS2 * np.outer(u, gr)
                + CS2 * np.outer(gr, u) + CS2 * (u @ gr) * np.eye(3) + 0.5 * (Ju + Ju.T))
        np.testing.assert_allclose(np.einsum("k,ka,kb->ab", G, CV, CV), want,
                                   atol=1e-15)


def test_ch3_moments():
    rng = np.random.default_rng(2)
    for _ in range(30):
        a, phi, Ci = rng.uniform(0.1, 3), rng.uniform(-1, 1), rng.uniform(-1e-3, 1e-3)
        u, up = rng.uniform(-0.1, 0.1, 3), rng.uniform(-0.1, 0.1, 3)
        pp, tau = rng.uniform(-1, 1), rng.uniform(0.55, 2)
        h = oracle.heq3(a, phi, Ci, u)
        assert abs(h.sum() - phi) < 1e-15
        np.testing.assert_allclose(CV.T @ h, phi * u, atol=1e-16)
        np.testing.assert_allclose(np.einsum("k,ka,kb->ab", h, CV, CV),
                                   CS2 * a * Ci * np.eye(3), atol=1e-17)
        R = oracle.source3(tau, phi, u, pp, up)
        assert abs(R.sum()) < 1e-17
        np.testing.assert_allclose(CV.T @ R, (1 - 0.5 / tau) * (phi * u - pp * up),
                                   atol=1e-16)


def test_stencils3_exact_on_quadratics():
    rng = np.random.default_rng(3)
    nx, ny, nz = 16, 14, 12
    p = W.base_params3(3, nx, ny, nz, 1e-3)
    s = oracle.OracleSim3D(p)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.astype(float), y.astype(float), z.astype(float)
    A = rng.uniform(-1, 1, (3, 3))
    A = A + A.T
    b = rng.uniform(-1, 1, 3)
    X = np.stack([x, y, z])
    f = 0.5 * np.einsum("aijk,ab,bijk->ijk", X, A, X) + np.einsum("a,aijk->ijk", b, X)
    grad, lap = s.stencils(f)
    sl = (slice(2, nz - 2), slice(2, ny - 2), slice(2, nx - 2))
    want = np.einsum("ab,bijk->aijk", A, X) + b[:, None, None, None]
    for a in range(3):
        np.testing.assert_allclose(grad[a][sl], want[a][sl], atol=1e-10)
    np.testing.assert_allclose(lap[sl], np.trace(A), atol=1e-10)
    s.close()


@pytest.mark.parametrize("wall", [0, 1])
def test_mass_conservation3(wall):
    w = W.random_smooth3(5, 4, 10, 9, 8, rho=[3.0, 1.0, 2.0, 5.0], wall_y=wall,
                         amp_u=0.02, gravity=(0.0, -1e-5, 0.0))
    s = oracle.OracleSim3D(w.params)
    s.init(w.c0, w.u0)
    m0 = s.moments()["phi"].sum((1, 2, 3))
    s.step(60)
    m1 = s.moments()["phi"].sum((1, 2, 3))
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-13 * w.c0[0].size)
    s.close()


def test_quiescent3_stationary():
    N, sh = 3, (6, 7, 5)
    c = np.broadcast_to(np.array([0.2, 0.3, 0.5])[:, None, None, None], (N,) + sh).copy()
    p = W.base_params3(N, sh[2], sh[1], sh[0], 1e-3, rho=[2.0, 1.0, 4.0])
    s = oracle.OracleSim3D(p)
    s.init(c)
    s.step(200)
    m = s.moments()
    assert np.abs(m["u"]).max() <= 1e-18
    assert np.ptp(m["phi"], axis=(1, 2, 3)).max() <= 1e-15
    s.close()


def test_2d_fields_reduce_to_d2q9():
    """A field that does not vary along z does not feel the third
    dimension through the stencils: Eq. N31 on D3Q15 then equals Eq. N31 on
    D2Q9 (both are exact on quadratics and second order; for a smooth
    z-invariant field they agree to the O(h^2) truncation error)."""
    nx, ny = 24, 20
    x = np.arange(nx, dtype=float)
    y = np.arange(ny, dtype=float)[:, None]
    f2 = np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny)
    f3 = np.broadcast_to(f2, (4, ny, nx)).copy()
    s2 = oracle.OracleSim(W.base_params(3, nx, ny, 1e-3))
    s3 = oracle.OracleSim3D(W.base_params3(3, nx, ny, 4, 1e-3))
    g2, l2 = s2.stencils(f2)
    g3, l3 = s3.stencils(f3)
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    assert np.abs(g3[2]).max() < 1e-14
    for a in range(2):
        assert np.abs(g3[a][0] - g2[a]).max() < 0.5 * (kx ** 2 + ky ** 2)
    assert np.abs(l3[0] - l2).max() < 0.5 * (kx ** 2 + ky ** 2)
    s2.close()
    s3.close()


def _flat3(mult, steps):
    """Two flat 1|2 tanh interfaces normal to z (N = 3, equal sigma, width
    W = 4 mult) on a 4 x 4 x 64 mult box, run `steps` steps."""
    import math
    nz, nx, ny = 64 * mult, 4, 4
    eta = math.sqrt(2) * mult
    band = W._layer(nz, 1, nz / 4.0, 3.0 * nz / 4.0, eta)[:, 0]
    c = np.zeros((3, nz, ny, nx))
    c[1] = band[:, None, None]
    c[0] = 1.0 - c[1]
    s = oracle.OracleSim3D(W.base_params3(3, nx, ny, nz, 1e-3, eta=eta))
    s.init(c)
    s.step(steps)
    m = s.moments()
    s.close()
    return band, c, m


def test_flat_interface_along_z():
    """A flat interface normal to z stays put up to the stencil error, which
    falls at least as dx^2 / w^2 when the width doubles (drift 4.4e-3 at
    W = 4 and 3.3e-4 at W = 8 after 2000 steps when this pin was written),
    and follows the D2Q9 oracle's flat interface normal to y: along one axis
    both lattices weigh the neighbouring planes by 1/6 (D3Q15: face 1/9 and
    four corners 1/72; D2Q9: axis 1/9 and two diagonals 1/36), so the
    profiles agree to the lattices' higher-moment differences (7.7e-7 when
    written) where a dropped z term or a wrong weight would show at the
    drift's size."""
    import math
    drifts = []
    for mult in (1, 2):
        band, c, m = _flat3(mult, 2000)
        drifts.append(np.abs(m["c"] - c).max())
        if mult == 1:
            nz = band.size
            c2 = np.zeros((3, nz, 4))
            c2[1] = band[:, None]
            c2[0] = 1.0 - c2[1]
            s2 = oracle.OracleSim(W.base_params(3, 4, nz, 1e-3, eta=math.sqrt(2)))
            s2.init(c2)
            s2.step(2000)
            m2 = s2.moments()
            s2.close()
            assert np.abs(m["c"][:, :, 0, 0] - m2["c"][:, :, 0]).max() < 1e-5
            assert np.ptp(m["c"], axis=(2, 3)).max() < 1e-14
    assert drifts[0] < 1e-2 and drifts[1] < 1e-3, drifts
    assert drifts[0] / drifts[1] > 4.0, drifts


def test_uniform_flow3_is_preserved():
    """A uniform mixture moving at constant velocity stays at equilibrium on
    D3Q15: u is kept in all three components and the fields stay uniform
    (Eq. N22_1, the third-order equilibrium moments and streaming)."""
    N, sh = 3, (5, 6, 7)
    c = np.broadcast_to(np.array([0.2, 0.5, 0.3])[:, None, None, None], (N,) + sh).copy()
    u0 = np.zeros((3,) + sh)
    u0[0], u0[1], u0[2] = 0.03, -0.02, 0.015
    p = W.base_params3(N, sh[2], sh[1], sh[0], 1e-3, rho=[1.0, 4.0, 2.0])
    s = oracle.OracleSim3D(p)
    s.init(c, u0)
    s.step(200)
    m = s.moments()
    for d, v in enumerate((0.03, -0.02, 0.015)):
        np.testing.assert_allclose(m["u"][d], v, atol=1e-15)
    assert np.ptp(m["phi"], axis=(1, 2, 3)).max() <= 1e-14
    s.close()


def test_rho0_is_inert3():
    """On D3Q15 too, rho_0 of Eq. 25 reaches only g_0, which enters neither u
    (c_0 = 0) nor p (Eq. N23 sums k >= 1): outputs are bit-identical."""
    w = W.random_smooth3(9, 3, 8, 7, 6, rho=[2.0, 1.0, 5.0], amp_u=0.01)
    outs = []
    for r0 in (0.0, 1.0, 7.0):
        p = dict(w.params, rho0=r0)
        outs.append(oracle.run3(p, w.c0, w.u0, steps=30))
    for o in outs[1:]:
        for k in ("phi", "u", "p"):
            assert np.array_equal(o[k], outs[0][k])


def test_mass_flux_and_density_gradient3():
    """Eq. N18 on D3Q15 with unequal densities: grad(rho) is Eq. N31a applied
    to the density field and J~ = -sum_i (d rho / d phi_i) m_i grad C_i, with
    d rho / d phi_i read off the density field itself (rho is linear in the
    phi_i, Eqs. N2, N12, N29: a least-squares fit over the grid) instead of
    the oracle's coefficients."""
    N = 3
    w = W.random_smooth3(21, N, 10, 8, 9, rho=[3.0, 1.0, 7.5], amp_u=0.02)
    s = oracle.OracleSim3D(w.params)
    s.init(w.c0, w.u0)
    s.step(3)
    C, J, grho = s.fluxes()
    m = s.moments()
    A = np.column_stack([np.ones(m["rho"].size)] + [m["phi"][i].ravel() for i in range(N - 1)])
    coef, *_ = np.linalg.lstsq(A, m["rho"].ravel(), rcond=None)
    assert np.abs(A @ coef - m["rho"].ravel()).max() < 1e-12
    drho = coef[1:]
    g_field, _ = s.stencils(m["rho"])
    assert np.abs(grho - g_field).max() <= 1e-11 * np.abs(g_field).max()
    mob = np.asarray(w.params["mobility"], dtype=float)
    Jexp = np.zeros_like(J)
    for i in range(N - 1):
        gC, _ = s.stencils(C[i])
        Jexp -= drho[i] * mob[i] * gC
    assert np.abs(J).max() > 0
    assert np.abs(J - Jexp).max() <= 1e-8 * np.abs(Jexp).max()
    s.close()


@pytest.mark.parametrize("axis", [0, 2])
def test_channel_flow_between_walls3(axis):
    """Halfway bounce-back walls in y on D3Q15: a uniform mixture driven by
    a body force rho g along x or z settles on the plane Poiseuille parabola
    u(y) = g (y + 1/2)(ny - 1/2 - y) / (2 nu), nu = (tau_g - 1/2)/3 (Eq.
    N21_1), within 1%, with no flow in the other directions."""
    nx, ny, nz, g, tau_g = 4, 16, 4, 1e-6, 0.8
    grav = [0.0, 0.0, 0.0]
    grav[axis] = g
    c = np.broadcast_to(np.array([0.2, 0.5, 0.3])[:, None, None, None],
                        (3, nz, ny, nx)).copy()
    p = W.base_params3(3, nx, ny, nz, 1e-3, wall_y=1, tau_g=tau_g, gravity=grav)
    s = oracle.OracleSim3D(p)
    s.init(c)
    s.step(6000)
    m = s.moments()
    s.close()
    nu = (tau_g - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    ua = g * y * (ny - y) / (2.0 * nu)
    prof = m["u"][axis][:, :, :]
    for z in range(nz):
        for x in range(nx):
            assert np.abs(prof[z, :, x] - ua).max() <= 1e-2 * ua.max()
    for a in range(3):
        if a != axis:
            assert np.abs(m["u"][a]).max() <= 1e-5 * ua.max()


def test_translating_interface_with_density_contrast3():
    """Galilean invariance on D3Q15: two flat interfaces normal to z between
    pure phases of densities 3 and 1, carried by a uniform flow U along z,
    keep u = U within 3% and p uniform to 2e-3 after 200 steps (the
    u . grad(rho) terms of Eqs. N23 and N20_1 are active)."""
    import math
    nx, ny, nz, U = 4, 4, 64, 0.01
    eta = 2 * math.sqrt(2)
    band = W._layer(nz, 1, nz / 4, 3 * nz / 4, eta)[:, 0]
    c = np.zeros((2, nz, ny, nx))
    c[0] = band[:, None, None]
    c[1] = 1 - c[0]
    u0 = np.zeros((3, nz, ny, nx))
    u0[2] = U
    p = W.base_params3(2, nx, ny, nz, 1e-3, rho=[3.0, 1.0], eta=eta)
    s = oracle.OracleSim3D(p)
    s.init(c, u0)
    s.step(200)
    m = s.moments()
    s.close()
    assert np.abs(m["u"][2] - U).max() <= 0.03 * U
    assert np.abs(m["u"][:2]).max() <= 1e-6 * U
    assert np.ptp(m["p"]) <= 2e-3


def test_laplace_law_cylinder3():
    """A drop column along z (a cylinder of radius R in a two-plane D3Q15
    box) carries the 2-D pressure jump sigma / R (Section 4.1): within 5% at
    W = 4, R = 10 after 4000 steps (0.969 when this pin was written)."""
    n, R, sig, nz = 48, 10.0, 1e-3, 2
    d2 = W.drop(n, n, n / 2, n / 2, R)
    c = np.zeros((2, nz, n, n))
    c[1] = d2[None]
    c[0] = 1 - c[1]
    s = oracle.OracleSim3D(W.base_params3(2, n, n, nz, sig))
    s.init(c)
    s.step(4000)
    m = s.moments()
    s.close()
    y, x = np.mgrid[0:n, 0:n]
    r = np.hypot(x - n / 2, y - n / 2)
    p0 = m["p"][0]
    dp = p0[r < R / 2].mean() - p0[(m["c"][0][0] > 0.999) & (r > R + 10)].mean()
    assert abs(dp / (sig / R) - 1) < 0.05, dp / (sig / R)


@pytest.mark.parametrize("tau", [0.7, 1.3])
def test_linear_ch_relaxation_rate3(tau):
    """On D3Q15, a small cosine mode along z of a uniform binary mixture at
    phi0 = 0.8 decays at the linearised Cahn-Hilliard rate
    m K^2 (beta^2/eta^2 h'(phi0) + lambda K^2), h'(phi0) = -(1 - 3 phi0^2)/4
    (N = 2, unit densities), with lambda and beta from the D2Q9 oracle's
    setup of the same parameters (Eqs. N14, N36) and K^2 from the D3Q15
    Laplacian (Eq. N31b): within 10% whatever tau_i."""
    nx, ny, nz, phi0, eps, M, T = 2, 2, 16, 0.8, 1e-5, 0.1, 3000
    z = np.arange(nz)
    mode = np.cos(2 * np.pi * z / nz)
    p2 = W.base_params(2, 4, 4, 1e-2, tau=tau, tau_g=0.8, mobility=M)
    s2 = oracle.OracleSim(p2)
    k = s2.constants()
    s2.close()
    lam = float(np.ravel(k["lam"])[0])
    bulk = k["beta"] ** 2 / p2["eta"] ** 2
    c1 = np.broadcast_to(((1 + phi0 + eps * mode) / 2)[:, None, None], (nz, ny, nx))
    s = oracle.OracleSim3D(W.base_params3(2, nx, ny, nz, 1e-2, tau=tau, tau_g=0.8,
                                          mobility=M))
    _, lap = s.stencils(np.broadcast_to(mode[:, None, None], (nz, ny, nx)))
    K2 = -lap[0, 0, 0]
    rate = M * K2 * (bulk * (-(1 - 3 * phi0 ** 2) / 4) + lam * K2)
    s.init(np.stack([c1, 1 - c1]))
    s.step(T)
    ph = s.moments()["phi"][0][:, 0, 0]
    s.close()
    amp = 2 * np.mean((ph - ph.mean()) * mode)
    measured = -np.log(amp / eps) / T
    assert abs(measured / rate - 1) < 0.1, (measured, rate)


def test_uniform_flow3_populations_are_stationary():
    """On D3Q15 too a uniform moving mixture is a fixed point of the
    populations from the start state of reading 8 ((phi u)_prev = phi u0, so
    R_k of Eq. N26 vanishes from the first step): h and g after each step
    equal their start values (to roundoff)."""
    N, sh = 3, (5, 6, 7)
    c = np.broadcast_to(np.array([0.2, 0.5, 0.3])[:, None, None, None], (N,) + sh).copy()
    u0 = np.zeros((3,) + sh)
    u0[0], u0[1], u0[2] = 0.03, -0.02, 0.015
    s = oracle.OracleSim3D(W.base_params3(N, sh[2], sh[1], sh[0], 1e-3, rho=[1.0, 4.0, 2.0]))
    s.init(c, u0)
    h0, g0 = s.populations()
    for _ in range(3):
        s.step(1)
        h, g = s.populations()
        assert np.abs(h - h0).max() <= 1e-15
        assert np.abs(g - g0).max() <= 1e-15
    s.close()
