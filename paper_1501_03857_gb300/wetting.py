"""Wettability calibration: the static contact angle of a sessile droplet as a
function of the fluid-solid interaction strength G_w of Eq. 22.

Sec. 3.3 tunes the heating surface's wettability with G_w and quotes the
resulting static contact angles (defined in the liquid phase, at T_s); to run
a boiling curve at prescribed angles one needs the inverse map angle -> G_w.
This module measures it with the library's own step: droplets standing on the
bottom wall relax at T = T_s (thermal step off, no gravity) in one batched
launch per step, and the angle is read from the density field.

Contact angle from a density field: the interface is the rho = (rho_L +
rho_V)/2 contour, located to sub-cell accuracy by linear interpolation
between neighbouring cells (along y and along x). A circle is fitted to the
contour points at least `skip` cells above the wall (the first rows are
shaped by the wall treatment) by algebraic least squares (Kasa, IEEE Trans.
Instrum. Meas. 25, 1976: minimise sum (x^2 + y^2 + D x + E y + F)^2, linear
in D, E, F). With centre height y_c and radius R the angle through the liquid
at the wall line y = y_w is arccos((y_w - y_c) / R): a centre on the wall
gives 90 deg, a centre below it a wetting (< 90 deg) droplet. The wall line is
the wall node row y_w = 0 (Zou-He wet nodes sit on the boundary).
"""

from __future__ import annotations

import math
from dataclasses import replace

import numpy as np

from . import inputs, lb


def interface_points(rho: np.ndarray, level: float, periodic_x: bool = True):
    """(x, y) of the sub-cell crossings of `level` between vertically and
    horizontally adjacent cells of rho[y, x]."""
    rho = np.asarray(rho, dtype=np.float64)
    d = rho - level
    xs, ys = [], []
    a, b = d[:-1, :], d[1:, :]
    j, i = np.nonzero(a * b < 0)
    t = a[j, i] / (a[j, i] - b[j, i])
    xs.append(i.astype(np.float64))
    ys.append(j + t)
    if periodic_x:
        a, b = d, np.roll(d, -1, axis=1)
    else:
        a, b = d[:, :-1], d[:, 1:]
    j, i = np.nonzero(a * b < 0)
    t = a[j, i] / (a[j, i] - b[j, i])
    xs.append(i + t)
    ys.append(j.astype(np.float64))
    return np.concatenate(xs), np.concatenate(ys)


def fit_circle(x: np.ndarray, y: np.ndarray):
    """Algebraic least-squares circle through the points: (xc, yc, R)."""
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    rhs = -(x * x + y * y)
    (D, E, F), *_ = np.linalg.lstsq(A, rhs, rcond=None)
    xc, yc = -D / 2.0, -E / 2.0
    return xc, yc, math.sqrt(max(xc * xc + yc * yc - F, 0.0))


def contact_angle(rho: np.ndarray, rho_l: float, rho_v: float, wall_y: float = 0.0, skip: float = 3.0) -> dict:
    """Static contact angle (degrees, through the liquid) of the single droplet
    standing on the bottom wall of rho[y, x]; periodic in x. Returns the angle
    with the fitted circle (xc, yc, R) and the number of contour points."""
    Ly, Lx = np.shape(rho)
    x, y = interface_points(rho, 0.5 * (rho_l + rho_v))
    if x.size == 0:
        raise ValueError("no liquid-vapour interface in the field")
    # unwrap x around the droplet: centre the liquid's column of mass at Lx/2
    liquid = np.asarray(rho) > 0.5 * (rho_l + rho_v)
    cols = np.nonzero(liquid.any(axis=0))[0]
    ang = 2 * np.pi * cols / Lx
    cx = (math.atan2(np.sin(ang).mean(), np.cos(ang).mean()) / (2 * np.pi) * Lx) % Lx
    x = (x - cx + 0.5 * Lx) % Lx - 0.5 * Lx
    keep = y >= wall_y + skip
    if keep.sum() < 8:
        raise ValueError("too few interface points above the wall for a circle fit")
    xc, yc, R = fit_circle(x[keep], y[keep])
    c = (wall_y - yc) / R
    theta = math.degrees(math.acos(min(1.0, max(-1.0, c))))
    return {"angle_deg": theta, "xc": xc + cx, "yc": yc, "R": R, "points": int(keep.sum())}


def droplet_config(Lx: int = 240, Ly: int = 120, ghost_layer: bool = False, **kw) -> lb.Config:
    """The calibration case: walls in y, thermal step off (T = T_s everywhere),
    no gravity, no noise; the other parameters are the paper's (Sec. 3.1)."""
    base = lb.Config(Lx=Lx, Ly=Ly, bc_y=lb.BC_WALLS, ghost_layer=ghost_layer, isothermal=True, g=0.0,
                     noise_amp=0.0, pool_height=Ly / 2)
    return replace(base, **kw)


def run_droplets(gw_values, cfg: lb.Config | None = None, radius: float = 40.0, steps: int = 40000,
                 checkpoints=None, stream=None) -> dict:
    """Relax one sessile droplet per G_w (all in one batched launch per step)
    and measure the contact angles. checkpoints: step counts (<= steps) at
    which the angles are also recorded, to show convergence. Returns
    {"Gw": [...], "angle_deg": [...], "history": {step: [...]}}."""
    cfg = cfg or droplet_config()
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.sessile_density(cfg.Lx, cfg.Ly, rl, rv, radius)
    gw_values = [float(g) for g in gw_values]
    batch = lb.Batch([{"cfg": cfg, "Gw": g, "rho0": rho0} for g in gw_values], stream=stream)
    marks = sorted(set(int(s) for s in (checkpoints or [])) | {int(steps)})
    history, done = {}, 0
    try:
        for m in marks:
            if m > done:
                batch.step(m - done)
                done = m
            angles = []
            for i in range(len(gw_values)):
                rho = batch.fields(i, ("rho",))["rho"]
                angles.append(contact_angle(rho, rl, rv)["angle_deg"])
            history[m] = angles
    finally:
        batch.close()
    return {"Gw": gw_values, "angle_deg": history[marks[-1]], "history": history,
            "radius0": radius, "steps": steps, "Lx": cfg.Lx, "Ly": cfg.Ly, "ghost_layer": bool(cfg.ghost_layer)}


def gw_for_angle(angle_deg, gw_table, angle_table):
    """G_w giving the contact angle(s) `angle_deg`, by linear interpolation in a
    measured table; the table must be strictly increasing in angle and the
    targets inside its range."""
    gw = np.asarray(gw_table, dtype=np.float64)
    an = np.asarray(angle_table, dtype=np.float64)
    order = np.argsort(gw)
    gw, an = gw[order], an[order]
    if np.any(np.diff(an) <= 0):
        raise ValueError("contact angle is not strictly increasing with G_w in the table")
    tgt = np.asarray(angle_deg, dtype=np.float64)
    if np.any(tgt < an[0]) or np.any(tgt > an[-1]):
        raise ValueError(f"target angle outside the calibrated range [{an[0]:.1f}, {an[-1]:.1f}] deg")
    return np.interp(tgt, an, gw)
