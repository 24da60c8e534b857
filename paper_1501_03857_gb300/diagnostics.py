"""Diagnostics of a boiling domain (Sec. 3.2): the pressure field, the vapour
bubbles in it, the Young-Laplace pressure jump of each and its fit.

Sec. 3.2 explains the shrinkage of a rising bubble that merges into the
vapour above the pool by the Young-Laplace law, delta p = (surface tension) /
r in two dimensions, and follows the pressure at the centre of the top wall
(Fig. 3; `Simulation.set_probes` records it on the device every step). These
host-side tools work on fields read back with `Simulation.fields`:

* pressure(cfg, rho, T): the Peng-Robinson pressure of Eq. 21 (computed by the
  library's host EOS, FP64);
* bubbles(rho, ...): connected vapour regions (rho below the mid density,
  4-connected, periodic in x and optionally in y), with area, equivalent
  radius sqrt(area / pi) and centroid;
* laplace_jump(p, bubble, ...): pressure in the vapour core (within 2 cells
  of the centroid) minus the bulk liquid's (10 cells or more beyond r_eq);
* laplace_fit(radii, jumps): least-squares delta p = s / r + c; for static
  bubbles s is the surface tension and c ~ 0.
"""

from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

from . import lb


def pressure(cfg: lb.Config, rho: np.ndarray, T: np.ndarray) -> np.ndarray:
    """p_EOS(rho, T) of Eq. 21 (FP64) for the fields of `Simulation.fields`."""
    return lb.eos_pressure(cfg, rho, T)


def _merge_seam(lab: np.ndarray, axis: int) -> np.ndarray:
    """Join labels that touch across the periodic boundary along `axis`."""
    first = np.take(lab, 0, axis=axis)
    last = np.take(lab, -1, axis=axis)
    parent = {}

    def find(a):
        while parent.get(a, a) != a:
            a = parent[a]
        return a

    for a, b in zip(first.ravel(), last.ravel()):
        if a and b:
            ra, rb = find(int(a)), find(int(b))
            if ra != rb:
                parent[max(ra, rb)] = min(ra, rb)
    if not parent:
        return lab
    lut = np.arange(lab.max() + 1)
    for a in range(1, lab.max() + 1):
        lut[a] = find(a)
    return lut[lab]


def _periodic_mean(coord: np.ndarray, period: int) -> float:
    ang = 2.0 * np.pi * coord / period
    return (math.atan2(np.sin(ang).mean(), np.cos(ang).mean()) / (2.0 * np.pi) * period) % period


def bubbles(rho: np.ndarray, rho_l: float, rho_v: float, periodic_y: bool = False, exclude_walls: bool = True,
            min_cells: int = 12) -> list:
    """Connected vapour regions of rho[y, x] below (rho_l + rho_v) / 2.
    With exclude_walls, regions touching the first or last row (vapour films
    on the heated wall, the vapour space under the top wall) are dropped.
    Returns dicts with label, cells, r_eq, xc, yc (centroid, periodic in x),
    and the boolean mask."""
    rho = np.asarray(rho)
    Ly, Lx = rho.shape
    vap = rho < 0.5 * (rho_l + rho_v)
    lab, n = ndimage.label(vap)
    lab = _merge_seam(lab, axis=1)
    if periodic_y:
        lab = _merge_seam(lab, axis=0)
    out = []
    for k in np.unique(lab):
        if k == 0:
            continue
        m = lab == k
        ys, xs = np.nonzero(m)
        if ys.size < min_cells:
            continue
        if exclude_walls and not periodic_y and (ys.min() == 0 or ys.max() == Ly - 1):
            continue
        out.append({"label": int(k), "cells": int(ys.size), "r_eq": math.sqrt(ys.size / math.pi),
                    "xc": _periodic_mean(xs, Lx), "yc": _periodic_mean(ys, Ly) if periodic_y else float(ys.mean()),
                    "mask": m})
    return out


def bubble_count(rho: np.ndarray, rho_l: float, rho_v: float, periodic_y: bool = False, exclude_walls: bool = True,
                 min_cells: int = 12) -> int:
    """len(bubbles(rho, rho_l, rho_v, ...)) with the same arguments, from one
    labelling and the labels' cell counts, without the per-bubble records
    (about 1 ms instead of 9 on the 600 x 150 pool: the boiling-curve runs
    sample it thousands of times)."""
    rho = np.asarray(rho)
    vap = rho < 0.5 * (rho_l + rho_v)
    lab, _ = ndimage.label(vap)
    lab = _merge_seam(lab, axis=1)
    if periodic_y:
        lab = _merge_seam(lab, axis=0)
    keep = np.bincount(lab.ravel()) >= min_cells
    keep[0] = False
    if exclude_walls and not periodic_y:
        keep[lab[0]] = False
        keep[lab[-1]] = False
    return int(keep.sum())


def _distance(shape, xc: float, yc: float, periodic_y: bool) -> np.ndarray:
    Ly, Lx = shape
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    dx = np.abs(x - xc)
    dx = np.minimum(dx, Lx - dx)
    dy = np.abs(y - yc)
    if periodic_y:
        dy = np.minimum(dy, Ly - dy)
    return np.hypot(dx, dy)


def laplace_jump(p: np.ndarray, bubble: dict, inner: float = 2.0, gap: float = 10.0,
                 periodic_y: bool = False) -> float:
    """Inside minus outside pressure of one bubble: mean p over the cells
    within `inner` of its centroid (the vapour core), minus mean p over the
    cells at least r_eq + gap from it (bulk liquid, clear of the interface's
    tails: a tanh profile of width 5 is still 4 % of the jump 4 cells out)."""
    d = _distance(p.shape, bubble["xc"], bubble["yc"], periodic_y)
    core = d <= inner
    bulk = d >= bubble["r_eq"] + gap
    if not core.any() or not bulk.any():
        raise ValueError("bubble too small or domain too small for a pressure jump")
    return float(p[core].mean() - p[bulk].mean())


def laplace_fit(radii, jumps) -> dict:
    """Least squares jumps = s / r + c over the bubbles: s (surface tension
    for static bubbles), c and the coefficient of determination r2."""
    inv = 1.0 / np.asarray(radii, dtype=np.float64)
    dp = np.asarray(jumps, dtype=np.float64)
    A = np.stack([inv, np.ones_like(inv)], axis=1)
    (s, c), *_ = np.linalg.lstsq(A, dp, rcond=None)
    pred = A @ np.array([s, c])
    ss = float(np.sum((dp - dp.mean()) ** 2))
    r2 = 1.0 - float(np.sum((dp - pred) ** 2)) / ss if ss > 0 else 1.0
    return {"surface_tension": float(s), "intercept": float(c), "r2": r2}
