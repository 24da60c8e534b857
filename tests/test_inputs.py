"""The seeded input recipes on the CPU: the 4096 x 4096 bubble array (256
non-overlapping bubbles, radii in [20, 60], clear of the walls), its density
field, and the 48-instance boiling-curve batch (sizes, superheats,
wettability indices)."""

import numpy as np
import pytest

from paper_1501_03857_gb300 import inputs

RL, RV = 6.498946, 0.379679


@pytest.fixture(scope="module")
def layout():
    return inputs.bubble_layout(4096, 4096, 256, 20.0, 60.0, seed=4)


def test_bubble_layout_count_radii_and_walls(layout):
    assert len(layout) == 256
    r = np.array([b[2] for b in layout])
    assert r.min() >= 20.0 and r.max() <= 60.0
    assert r.max() - r.min() > 30.0  # the radii spread over the range
    for cx, cy, rr in layout:
        assert 0.0 <= cx < 4096.0
        assert cy - rr >= 3.0 - 1e-9 and cy + rr <= 4096 - 3.0 + 1e-9


def test_bubbles_do_not_overlap_across_the_periodic_seam(layout):
    b = np.array(layout)
    dx = np.abs(b[:, None, 0] - b[None, :, 0])
    dx = np.minimum(dx, 4096.0 - dx)
    d = np.hypot(dx, b[:, None, 1] - b[None, :, 1])
    gap = d - (b[:, None, 2] + b[None, :, 2])
    np.fill_diagonal(gap, np.inf)
    assert gap.min() >= 2.0


def test_bubble_density_small_case():
    Lx, Ly = 400, 300
    lay = inputs.bubble_layout(Lx, Ly, 6, 20.0, 30.0, seed=4)
    rho = inputs.bubble_density(Lx, Ly, RL, RV, n_bubbles=6, r_min=20.0, r_max=30.0, seed=4, noise_amp=0.0)
    assert rho.shape == (Ly, Lx)
    assert rho.max() <= RL + 1e-12 and rho.min() >= RV - 1e-12
    for cx, cy, r in lay:
        assert abs(rho[int(round(cy)), int(round(cx)) % Lx] - RV) < 0.05 * (RL - RV)
    yy, xx = np.mgrid[0:Ly, 0:Lx]
    far = np.ones((Ly, Lx), bool)
    for cx, cy, r in lay:
        dx = np.abs(xx - cx)
        dx = np.minimum(dx, Lx - dx)
        far &= np.hypot(dx, yy - cy) > r + 20
    assert far.any() and np.allclose(rho[far], RL, rtol=1e-6)


def test_boiling_curve_batch_recipe():
    b = inputs.boiling_curve_batch()
    assert len(b) == 48
    for i, d in enumerate(b):
        assert 200 <= d["Lx"] <= 400 and d["Lx"] % 8 == 0
        assert 200 <= d["Ly"] <= 600 and d["Ly"] % 8 == 0
        assert d["wet_index"] == i % 5
    s = np.array([d["superheat_frac"] for d in b])
    assert s[0] == pytest.approx(0.02) and s[-1] == pytest.approx(0.4)
    assert np.allclose(np.diff(s), (0.4 - 0.02) / 47)
    cells = sum(d["Lx"] * d["Ly"] for d in b)
    assert 48 * 200 * 200 <= cells <= 48 * 400 * 600
    assert len({(d["Lx"], d["Ly"]) for d in b}) > 40  # uneven sizes
    assert b == inputs.boiling_curve_batch()  # seeded
