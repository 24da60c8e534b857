"""Oracle contact angle of a sessile droplet (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may
import this module.

Independent of the product's circle fit: the droplet is taken as a circular
cap (the static shape with no gravity) fixed by two measurements of the
rho = (rho_L + rho_V)/2 contour, its apex height H above the wall line and
its chord 2c on an integer row y_e above the wall. A circle through the apex
and both chord ends has radius R = (c^2 + (H - y_e)^2) / (2 (H - y_e)) and
centre height y_c = H - R; the angle through the liquid at the wall line y_w
is arccos((y_w - y_c) / R) (Sec. 3.3 quotes angles "defined in the liquid
phase"). Contour positions come from linear interpolation between the two
cells that straddle the mid density, scanning outward from the droplet's
centre column along the chord row and upward along the centre column.
"""

from __future__ import annotations

import math

import numpy as np


def _crossing(v0: float, v1: float, level: float) -> float:
    """Fraction t in [0, 1] where the segment v0 -> v1 meets level."""
    return (v0 - level) / (v0 - v1)


def contact_angle_cap(rho, rho_l: float, rho_v: float, wall_y: float = 0.0, chord_row: int = 3) -> float:
    """Contact angle in degrees, through the liquid as Sec. 3.3 defines it,
    of the one droplet on the bottom wall of rho[y, x] (periodic in x), by
    the apex-and-chord cap construction."""
    rho = np.asarray(rho, dtype=np.float64)
    Ly, Lx = rho.shape
    level = 0.5 * (rho_l + rho_v)
    row = rho[chord_row]
    inside = row > level
    if not inside.any() or inside.all():
        raise ValueError("chord row does not cut the droplet")
    # start from the middle of the longest run of liquid cells on the chord row
    best_len, best_start = 0, 0
    for s in range(Lx):
        if inside[s] and not inside[s - 1]:
            n = 0
            while inside[(s + n) % Lx]:
                n += 1
            if n > best_len:
                best_len, best_start = n, s
    left_cell = best_start                  # first liquid cell of the run
    right_cell = best_start + best_len - 1  # last liquid cell (unwrapped)
    # left crossing between left_cell - 1 (vapour) and left_cell (liquid)
    tl = _crossing(row[(left_cell - 1) % Lx], row[left_cell % Lx], level)
    x_left = left_cell - 1 + tl
    tr = _crossing(row[right_cell % Lx], row[(right_cell + 1) % Lx], level)
    x_right = right_cell + tr
    c = 0.5 * (x_right - x_left)
    xm = 0.5 * (x_right + x_left)
    # apex: upward along the column nearest the centre, first liquid -> vapour
    col = rho[:, int(round(xm)) % Lx]
    H = None
    for y in range(chord_row, Ly - 1):
        if col[y] > level >= col[y + 1]:
            H = y + _crossing(col[y], col[y + 1], level)
            break
    if H is None:
        raise ValueError("no apex found above the chord row")
    h = H - chord_row
    R = (c * c + h * h) / (2.0 * h)
    yc = H - R
    cosang = max(-1.0, min(1.0, (wall_y - yc) / R))
    return math.degrees(math.acos(cosang))


def cap_density(Lx: int, Ly: int, rho_l: float, rho_v: float, R: float, angle_deg: float, wall_y: float = 0.0,
                width: float = 5.0) -> np.ndarray:
    """A droplet whose mid-density contour is exactly the circle of radius R
    meeting the wall line at the given angle (through the liquid): centre at
    (Lx/2, wall_y - R cos(angle)), tanh profile of the distance to it. The
    known-answer input of the angle pins (geometry only, no method
    arithmetic)."""
    yc = wall_y - R * math.cos(math.radians(angle_deg))
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    r = np.hypot(x - 0.5 * Lx, y - yc)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - R) / width)
