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


def angles(d, h_up, h_down):
    return (math.degrees(2 * math.atan(2 * h_up / d)),
            math.degrees(2 * math.atan(2 * h_down / d)))


def neumann_symmetric(s12, s):
    """Cap angle of a symmetric lens (sigma_13 = sigma_23 = s), Eq. N32."""
    return math.degrees(math.acos(s12 / (2 * s)))


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
