"""Host diagnostics (Sec. 3.2: pressure, bubbles, Young-Laplace) on the CPU:
the library's EOS pressure against the oracle's Eq. 21, bubble detection on
synthetic fields with known geometry, and the Laplace jump and fit on exact
data. The probe and the GPU-vs-oracle Laplace comparison are GPU tests."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import diagnostics as D, lb

F64 = torch.float64


def test_eos_pressure_matches_oracle():
    cfg = lb.Config()
    Tc = lb.critical_temperature(cfg)
    rng = np.random.default_rng(7)
    rho = rng.uniform(0.2, 7.5, 500).astype(np.float32)
    T = (Tc * rng.uniform(0.7, 1.1, 500)).astype(np.float32)
    got = lb.eos_pressure(cfg, rho, T)
    ref = O.pr_pressure(torch.tensor(rho, dtype=F64), torch.tensor(T, dtype=F64), cfg.a, cfg.b, cfg.R, cfg.omega,
                        O.critical_temperature(cfg.a, cfg.b, cfg.R)).numpy()
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-14)


def test_eos_pressure_equal_at_coexistence():
    """Maxwell's construction gives one pressure for both phases (to the
    FP32 rounding of the density and temperature the call takes)."""
    cfg = lb.Config()
    rv, rl = lb.coexistence(cfg)
    Ts = cfg.Ts_over_Tc * lb.critical_temperature(cfg)
    p = D.pressure(cfg, np.array([rv, rl], dtype=np.float64), np.full(2, Ts))
    assert abs(p[0] - p[1]) < 1e-5 * abs(p[0])


def disc_field(Lx, Ly, discs, rho_l=6.5, rho_v=0.38):
    """Liquid with sharp vapour discs (cx, cy, r), periodic in x."""
    y, x = np.mgrid[0:Ly, 0:Lx].astype(np.float64)
    rho = np.full((Ly, Lx), rho_l)
    for cx, cy, r in discs:
        dx = np.abs(x - cx)
        dx = np.minimum(dx, Lx - dx)
        rho[np.hypot(dx, y - cy) < r] = rho_v
    return rho


def test_bubbles_geometry_and_seam():
    """Three vapour discs: one across the x seam, one touching the heated
    wall (dropped as a wall film), one interior; areas give r_eq within the
    pixelisation, centroids are found across the seam."""
    rho = disc_field(200, 100, [(2.0, 50.0, 12.0), (100.0, 6.0, 10.0), (120.0, 60.0, 15.0)])
    bs = D.bubbles(rho, 6.5, 0.38)
    assert len(bs) == 2
    bs.sort(key=lambda b: b["r_eq"])
    seam, inner = bs
    assert abs(seam["r_eq"] - 12.0) < 0.3 and abs(inner["r_eq"] - 15.0) < 0.3
    d = abs(seam["xc"] - 2.0)
    assert min(d, 200 - d) < 0.5 and abs(seam["yc"] - 50.0) < 0.5
    assert abs(inner["xc"] - 120.0) < 0.5 and abs(inner["yc"] - 60.0) < 0.5
    assert len(D.bubbles(rho, 6.5, 0.38, exclude_walls=False)) == 3


def test_laplace_jump_exact():
    rho = disc_field(120, 120, [(60.0, 60.0, 20.0)])
    y, x = np.mgrid[0:120, 0:120].astype(np.float64)
    d = np.hypot(x - 60.0, y - 60.0)
    # core value inside, bulk value far out, anything in between
    p = np.where(d <= 2.0, 0.031, np.where(d >= 29.0, 0.027, 0.5))
    b = D.bubbles(rho, 6.5, 0.38)[0]
    assert abs(D.laplace_jump(p, b) - 0.004) < 1e-15


def test_laplace_fit_exact_and_noisy():
    r = np.array([8.0, 10.0, 13.0, 17.0, 22.0])
    fit = D.laplace_fit(r, 0.3 / r + 1e-5)
    assert abs(fit["surface_tension"] - 0.3) < 1e-12 and abs(fit["intercept"] - 1e-5) < 1e-12
    assert fit["r2"] > 1 - 1e-12
    noisy = 0.3 / r * (1 + 0.2 * np.array([1, -1, 1, -1, 1]))
    assert D.laplace_fit(r, noisy)["r2"] < 0.99


def test_bubble_count_equals_bubbles():
    """bubble_count gives len(bubbles(...)) for the same arguments on random
    two-phase fields: periodic and wall-bounded y, walls excluded or not,
    several size thresholds."""
    rng = np.random.default_rng(5)
    rl, rv = 6.5, 0.38
    for _ in range(60):
        Ly, Lx = int(rng.integers(5, 60)), int(rng.integers(5, 90))
        rho = np.where(rng.random((Ly, Lx)) < rng.uniform(0.2, 0.7), rv, rl)
        for per in (False, True):
            for ex in (False, True):
                for mc in (1, 4, 12):
                    assert D.bubble_count(rho, rl, rv, periodic_y=per, exclude_walls=ex, min_cells=mc) == len(
                        D.bubbles(rho, rl, rv, periodic_y=per, exclude_walls=ex, min_cells=mc))
