"""Seeded synthetic inputs for the boiling workloads.

This module holds none of the method's arithmetic: only a counter-based random
number generator (splitmix64, Steele, Lea and Flood, OOPSLA 2014) and geometric
density layouts (a liquid pool under vapour, vapour bubbles in liquid, a
droplet, a flat slab) built from coexistence densities that the caller passes
in as numbers. Both the CUDA path and the FP64 oracle are fed the same arrays
from here; the library's own C host code implements the same generator for
``lb_init`` calls without an explicit density field.

Layouts follow the paper's set-up (Sec. 3.1: liquid below y0, vapour above,
periodic in x) with a tanh interface of width 5 lattice units and a relative
density noise of +-amp ("small fluctuations", Sec. 3.2), drawn per cell from
counter ``y * Lx + x`` of the stream keyed by ``seed``.
"""

from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
D2Q9_WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """n-th output of the splitmix64 sequence started at ``seed``:
    mix(seed + (n + 1) * GAMMA) with the published finaliser."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counter, dtype=np.uint64) + np.uint64(1)) * GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of splitmix64."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def cell_noise(Lx: int, Ly: int, seed: int, y0: int = 0) -> np.ndarray:
    """Uniform [-1, 1) per cell, counter y * Lx + x, for rows y0 .. y0 + Ly - 1."""
    n = (np.arange(Lx * Ly, dtype=np.uint64) + np.uint64(y0 * Lx)).reshape(Ly, Lx)
    return 2.0 * uniform01(seed, n) - 1.0


def _finish(rho: np.ndarray, noise_amp: float, seed: int, y0: int = 0) -> np.ndarray:
    Ly, Lx = rho.shape
    if noise_amp:
        rho = rho * (1.0 + noise_amp * cell_noise(Lx, Ly, seed, y0))
    return rho.astype(np.float32)


def pool_density(Lx, Ly, rho_l, rho_v, pool_height, width=5.0, noise_amp=1e-4, seed=1, rows=None):
    """Liquid below y = pool_height, vapour above (Sec. 3.1), tanh interface.
    rows = (y0, y1) returns only rows y0 .. y1 - 1 of the Ly-row field (the
    same values; for fields too large to build at once)."""
    y0, y1 = (0, Ly) if rows is None else rows
    y = np.arange(y0, y1, dtype=np.float64)[:, None]
    prof = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (y - pool_height) / width)
    return _finish(np.broadcast_to(prof, (y1 - y0, Lx)).copy(), noise_amp, seed, y0)


def slab_density(Lx, Ly, rho_l, rho_v, y0, y1, width=5.0, noise_amp=0.0, seed=1):
    """Flat liquid slab y0 <= y < y1 in vapour (for periodic-y tests)."""
    y = np.arange(Ly, dtype=np.float64)[:, None]
    prof = rho_v + 0.5 * (rho_l - rho_v) * (np.tanh(2.0 * (y - y0) / width) - np.tanh(2.0 * (y - y1) / width))
    return _finish(np.broadcast_to(prof, (Ly, Lx)).copy(), noise_amp, seed)


def droplet_density(Lx, Ly, rho_l, rho_v, radius, cx=None, cy=None, width=5.0, noise_amp=0.0, seed=1):
    """Circular liquid droplet in vapour, centred in the box by default."""
    cx = (Lx - 1) / 2.0 if cx is None else cx
    cy = (Ly - 1) / 2.0 if cy is None else cy
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    r = np.hypot(x - cx, y - cy)
    rho = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - radius) / width)
    return _finish(rho, noise_amp, seed)


def sessile_density(Lx, Ly, rho_l, rho_v, radius, cx=None, cy=0.0, width=5.0, noise_amp=0.0, seed=1):
    """A liquid circle of the given radius centred at (cx, cy) in vapour, for a
    droplet on the bottom wall (cy = 0: a half disc standing on the wall row);
    tanh interface, periodic in x (minimum-image distance)."""
    cx = Lx / 2.0 if cx is None else cx
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    dx = np.abs(x - cx)
    dx = np.minimum(dx, Lx - dx)
    r = np.hypot(dx, y - cy)
    rho = 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r - radius) / width)
    return _finish(rho, noise_amp, seed)


def bubble_layout(Lx, Ly, n_bubbles, r_min, r_max, seed, wall_gap=3, max_tries=200000):
    """Non-overlapping circles (cx, cy, r), radius uniform in [r_min, r_max],
    centres uniform, rejection-sampled with draws from the seed's stream."""
    out = []
    k = 0
    while len(out) < n_bubbles and k < max_tries:
        u = uniform01(seed, np.arange(3 * k, 3 * k + 3, dtype=np.uint64))
        k += 1
        r = r_min + (r_max - r_min) * u[0]
        cx = u[1] * Lx
        cy = (r + wall_gap) + u[2] * max(Ly - 2 * (r + wall_gap), 0.0)
        ok = True
        for (bx, by, br) in out:
            dx = abs(cx - bx)
            dx = min(dx, Lx - dx)
            if dx * dx + (cy - by) ** 2 < (r + br + 2.0) ** 2:
                ok = False
                break
        if ok:
            out.append((cx, cy, r))
    return out


def bubble_density(Lx, Ly, rho_l, rho_v, n_bubbles=256, r_min=20.0, r_max=60.0, seed=4,
                   width=5.0, noise_amp=1e-4, noise_seed=None):
    """Vapour bubbles in saturated liquid (a seeded bubble array): each bubble
    is a tanh well; periodic in x."""
    rho = np.full((Ly, Lx), float(rho_l))
    y = np.arange(Ly, dtype=np.float64)[:, None]
    for (cx, cy, r) in bubble_layout(Lx, Ly, n_bubbles, r_min, r_max, seed):
        x0 = int(np.floor(cx - r - 4 * width))
        x1 = int(np.ceil(cx + r + 4 * width)) + 1
        y0 = max(int(np.floor(cy - r - 4 * width)), 0)
        y1 = min(int(np.ceil(cy + r + 4 * width)) + 1, Ly)
        xs = np.arange(x0, x1)
        xx = xs.astype(np.float64)[None, :]
        yy = y[y0:y1]
        d = np.hypot(xx - cx, yy - cy)
        dip = 0.5 * (rho_l - rho_v) * (1.0 - np.tanh(2.0 * (d - r) / width))
        cols = np.mod(xs, Lx)
        rho[y0:y1, cols] = np.minimum(rho[y0:y1, cols], rho_l - dip)
    return _finish(rho, noise_amp, seed if noise_seed is None else noise_seed)


def random_state(Lx, Ly, rho_l, rho_v, pool_height, seed, pop_amp=0.05, rho_amp=0.02,
                 theta_max=0.01):
    """A random but physical state for one-step kernel parity: a pool density
    with +-rho_amp relative noise, populations w_a rho (1 +- pop_amp), and a
    temperature offset theta in [0, theta_max). Returns (rho0, fpost, theta) as
    float32 arrays; rho0 is the density the populations were built from."""
    rho0 = pool_density(Lx, Ly, rho_l, rho_v, pool_height, noise_amp=rho_amp, seed=seed).astype(np.float64)
    n = np.arange(9 * Lx * Ly, dtype=np.uint64).reshape(9, Ly, Lx)
    u = 2.0 * uniform01(seed + 1, n) - 1.0
    f = D2Q9_WEIGHTS[:, None, None] * rho0[None] * (1.0 + pop_amp * u)
    th = theta_max * uniform01(seed + 2, np.arange(Lx * Ly, dtype=np.uint64).reshape(Ly, Lx))
    return rho0.astype(np.float32), f.astype(np.float32), th.astype(np.float32)


def boiling_curve_batch(n=48, seed=3, superheat_range=(0.02, 0.4), n_wettability=5,
                        lx_range=(200, 400), ly_range=(200, 600), step=8):
    """The points of a batched boiling curve: instance i has superheat
    fraction s_i = lo + (hi - lo) i/(n-1) (of T_c), wettability index
    i mod n_wettability, and a domain size drawn uniformly from the multiples
    of `step` in the given ranges (two draws of the seed's stream per
    instance). Returns a list of dicts (Lx, Ly, superheat_frac, wet_index)."""
    out = []
    nx = (lx_range[1] - lx_range[0]) // step + 1
    ny = (ly_range[1] - ly_range[0]) // step + 1
    u = uniform01(seed, np.arange(2 * n, dtype=np.uint64))
    for i in range(n):
        Lx = lx_range[0] + step * min(int(u[2 * i] * nx), nx - 1)
        Ly = ly_range[0] + step * min(int(u[2 * i + 1] * ny), ny - 1)
        frac = superheat_range[0] + (superheat_range[1] - superheat_range[0]) * i / max(n - 1, 1)
        out.append({"Lx": Lx, "Ly": Ly, "superheat_frac": frac, "wet_index": i % n_wettability})
    return out
