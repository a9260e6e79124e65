"""Lens geometry from volume-fraction fields (liquid lens, Section 4.2).

The paper measures the lens by its length d (distance between the two triple
junctions) and the cap heights h_1, h_2, and converts them to contact angles
theta_i = 2 arctan(2 h_i / d). How the contour and the reference line are
taken is not stated; this helper uses the c_drop = 1/2 contour (linear
interpolation) and, as reference line, the mean height of the c_below = 1/2
level over the columns farthest from the drop.
"""
import math

import numpy as np


def _cross(a, b, lvl=0.5):
    """Fractional position in [0, 1] where a -> b crosses lvl."""
    return (lvl - a) / (b - a)


def level_height(col, lvl=0.5):
    """y of the first crossing of lvl in a column (from below), or None."""
    for y in range(len(col) - 1):
        a, b = col[y], col[y + 1]
        if (a - lvl) * (b - lvl) <= 0 and a != b:
            return y + _cross(a, b, lvl)
    return None


def measure(c_below, c_drop, far_cols=8):
    """Return d, h_up, h_down, y_ref for a lens whose drop fraction is
    ``c_drop`` and whose lower fluid fraction is ``c_below`` ([ny][nx])."""
    ny, nx = c_drop.shape
    cols_with_drop = np.where(c_drop.max(0) > 0.5)[0]
    xc = 0.5 * (cols_with_drop.min() + cols_with_drop.max())
    dist = np.abs(((np.arange(nx) - xc + nx / 2) % nx) - nx / 2)
    far = np.argsort(-dist)[:far_cols]
    ys = [level_height(1.0 - c_below[:, x]) for x in far]
    y_ref = float(np.mean([y for y in ys if y is not None]))
    # d: where the drop contour meets y = y_ref (interpolate rows)
    y0 = int(math.floor(y_ref))
    t = y_ref - y0
    row = (1 - t) * c_drop[y0] + t * c_drop[y0 + 1]
    inside = np.where(row > 0.5)[0]
    xl, xr = inside.min(), inside.max()
    xl_f = xl - 1 + _cross(row[xl - 1], row[xl])
    xr_f = xr + _cross(row[xr], row[xr + 1])
    d = xr_f - xl_f
    # heights: top and bottom of the c_drop = 1/2 contour per column
    top, bot = -np.inf, np.inf
    for x in range(nx):
        col = c_drop[:, x]
        idx = np.where(col > 0.5)[0]
        if len(idx) == 0:
            continue
        ymax, ymin = idx.max(), idx.min()
        if ymax + 1 < ny:
            top = max(top, ymax + _cross(col[ymax], col[ymax + 1]))
        if ymin - 1 >= 0:
            bot = min(bot, ymin - 1 + _cross(col[ymin - 1], col[ymin]))
    return d, top - y_ref, y_ref - bot, y_ref


def contour_points(c, lvl=0.5):
    """Points where the field c crosses lvl along the grid edges (rows and
    columns, linear interpolation), as an array of (x, y)."""
    pts = []
    a, b = c[:, :-1], c[:, 1:]
    yy, xx = np.nonzero((a - lvl) * (b - lvl) < 0)
    t = (lvl - a[yy, xx]) / (b[yy, xx] - a[yy, xx])
    pts.append(np.stack([xx + t, yy.astype(float)], 1))
    a, b = c[:-1, :], c[1:, :]
    yy, xx = np.nonzero((a - lvl) * (b - lvl) < 0)
    t = (lvl - a[yy, xx]) / (b[yy, xx] - a[yy, xx])
    pts.append(np.stack([xx.astype(float), yy + t], 1))
    return np.concatenate(pts)


def fit_circle(p):
    """Least-squares circle x^2 + y^2 = 2 a x + 2 b y + k through points p;
    returns (a, b, r)."""
    A = np.stack([2 * p[:, 0], 2 * p[:, 1], np.ones(len(p))], 1)
    rhs = (p * p).sum(1)
    (a, b, k), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return a, b, math.sqrt(k + a * a + b * b)


def measure_fit(c_below, c_drop, far_cols=8, margin=0.25):
    """Lens length and cap heights from circles fitted to the two caps.

    The c_drop = 1/2 contour points above and below the far-field level of
    the lower fluid (leaving out a band of margin x the cap height around it,
    where the diffuse triple junction rounds the tips) are fitted with one
    circle each; the caps' circles meet at the triple junctions, d is their
    distance and h_1, h_2 the caps' heights above and below that chord.
    Returns d, h_up, h_down, y_chord."""
    d0, hu0, hd0, y_ref = measure(c_below, c_drop, far_cols)
    pts = contour_points(c_drop)
    up = pts[pts[:, 1] > y_ref + max(2.0, margin * hu0)]
    dn = pts[pts[:, 1] < y_ref - max(2.0, margin * hd0)]
    a1, b1, r1 = fit_circle(up)
    a2, b2, r2 = fit_circle(dn)
    # intersections of the two circles
    dx, dy = a2 - a1, b2 - b1
    L = math.hypot(dx, dy)
    t = (r1 * r1 - r2 * r2 + L * L) / (2 * L)
    hh = math.sqrt(max(r1 * r1 - t * t, 0.0))
    mx, my = a1 + t * dx / L, b1 + t * dy / L
    d = 2.0 * hh
    # unit normal of the chord pointing to the upper cap
    nx_, ny_ = dx / L, dy / L
    if ny_ < 0:
        nx_, ny_ = -nx_, -ny_
    h_up = r1 + ((a1 - mx) * nx_ + (b1 - my) * ny_)
    h_down = r2 - ((a2 - mx) * nx_ + (b2 - my) * ny_)
    return d, h_up, h_down, my


def angles(d, h_up, h_down):
    return (math.degrees(2 * math.atan(2 * h_up / d)),
            math.degrees(2 * math.atan(2 * h_down / d)))


def neumann_symmetric(s12, s):
    """Cap angle of a symmetric lens (sigma_13 = sigma_23 = s), Eq. N32."""
    return math.degrees(math.acos(s12 / (2 * s)))


def neumann(s12, s13, s23):
    """Contact angles (theta_1, theta_2) in degrees of a lens of phase 1
    between phase 2 (theta_1 side) and phase 3 (theta_2 side), Eq. N32."""
    t1 = math.acos((s12 ** 2 + s23 ** 2 - s13 ** 2) / (2 * s12 * s23))
    t2 = math.acos((s13 ** 2 + s23 ** 2 - s12 ** 2) / (2 * s13 * s23))
    return math.degrees(t1), math.degrees(t2)


def lens_from_area(A, t1_deg, t2_deg):
    """Length d and cap heights (h_1, h_2) of a lens of area A whose caps
    meet the flat interface at theta_1, theta_2: Eq. N33 solved for d, then
    Eq. N34."""
    th = [math.radians(t1_deg), math.radians(t2_deg)]
    k = sum((t / math.sin(t) - math.cos(t)) / math.sin(t) for t in th)
    d = 2.0 * math.sqrt(A / k)
    h = [0.5 * d * (1 - math.cos(t)) / math.sin(t) for t in th]
    return d, h[0], h[1]


def contour_area(c_drop, lvl=0.5):
    """Area inside the c_drop = lvl contour: per column, the distance
    between the lowest and highest crossing (linear interpolation)."""
    ny, nx = c_drop.shape
    area = 0.0
    for x in range(nx):
        col = c_drop[:, x]
        idx = np.where(col > lvl)[0]
        if len(idx) == 0:
            continue
        ymax, ymin = idx.max(), idx.min()
        top = ymax + (_cross(col[ymax], col[ymax + 1], lvl)
                      if ymax + 1 < ny else 0.5)
        bot = ymin - 1 + (_cross(col[ymin - 1], col[ymin], lvl)
                          if ymin >= 1 else 0.5)
        area += top - bot
    return area


def band_tension(phi, c, lam, beta, eta):
    """Tension of each of the two flat interfaces of a relaxed band (fields
    [.][ny] along y, periodic): the excess of the discrete free energy whose
    variation gives the step's chemical potential (Eqs. N11, N17, N18, N31b
    in one dimension): 1/2 sum_ij lambda_ij dphi_i dphi_j with forward
    differences (their variation is the three-point Laplacian) plus
    beta^2/(2 eta^2) sum_k c_k^2 (1 - c_k)^2 (Eq. N17 is half of the
    derivative of the printed sum), divided by two."""
    dphi = np.roll(phi, -1, axis=1) - phi
    grad = 0.5 * np.einsum("ij,iy,jy->y", lam, dphi, dphi)
    bulk = beta * beta / (2 * eta * eta) * (c * c * (1 - c) ** 2).sum(0)
    return float((grad + bulk).sum() / 2)


def de_gennes_thickness(g, spread, rho1, rho2, rho3, upper=True):
    """Asymptotic thickness of a puddle of fluid 1 floating between fluid 2
    above and fluid 3 below, with spread = s12 + s13 - s23 > 0 (Eq. N37).

    Balancing the hydrostatic pressure across a vertical cut through the
    puddle against the three tensions (Archimedes fixes the immersed part)
    gives H^2 = 2 spread (rho3 - rho2) / (g (rho1 - rho2)(rho3 - rho1)).
    Eq. N37 as printed is its rho2 -> 0 limit (upper=False)."""
    if not upper:
        rho2 = 0.0
    return math.sqrt(2.0 * spread * (rho3 - rho2) /
                     (g * (rho1 - rho2) * (rho3 - rho1)))
