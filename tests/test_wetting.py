"""Contact-angle measurement and wettability calibration (Eq. 22, Sec. 3.3),
on the CPU: both angle methods against circular caps of known angle, the
angle -> G_w inversion, and the oracle's sessile droplets against the angles
the paper prints."""

import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import inputs, wetting as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RL, RV = 6.498946, 0.379679


def paper_values():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


@pytest.mark.parametrize("R", [30.0, 60.0])
@pytest.mark.parametrize("angle", [30.0, 45.0, 60.0, 90.0, 120.0, 150.0, 160.0])
def test_cap_angle_both_methods(R, angle):
    """A droplet whose mid-density contour is exactly a circle meeting the
    wall at a known angle: the circle fit and the apex-chord construction
    both return that angle."""
    rho = O.cap_density(300, 160, RL, RV, R, angle)
    assert abs(W.contact_angle(rho, RL, RV)["angle_deg"] - angle) < 0.1
    assert abs(O.contact_angle_cap(rho, RL, RV) - angle) < 0.1


def test_cap_angle_across_periodic_seam():
    """A droplet centred on the x-periodic seam reads the same angle."""
    rho = O.cap_density(300, 160, RL, RV, 40.0, 70.0)
    shifted = np.roll(rho, 150, axis=1)
    assert abs(W.contact_angle(shifted, RL, RV)["angle_deg"] - 70.0) < 0.1
    assert abs(O.contact_angle_cap(shifted, RL, RV) - 70.0) < 0.1


def test_wall_line_matters():
    """Reading the same field against a wall line half a cell higher changes
    a 45 deg angle by more than the method error (the wall line is not a
    free parameter)."""
    rho = O.cap_density(300, 160, RL, RV, 40.0, 45.0)
    a0 = W.contact_angle(rho, RL, RV, wall_y=0.0)["angle_deg"]
    a1 = W.contact_angle(rho, RL, RV, wall_y=0.5)["angle_deg"]
    assert abs(a1 - a0) > 0.5


def test_gw_for_angle_interpolates_and_checks():
    gw = [0.0, 0.1, 0.2, 0.3]
    an = [44.0, 55.0, 77.0, 108.0]
    assert np.allclose(W.gw_for_angle([44.0, 55.0, 108.0], gw, an), [0.0, 0.1, 0.3])
    assert abs(float(W.gw_for_angle(66.0, gw, an)) - 0.15) < 1e-12
    # unsorted input is sorted by G_w first
    assert abs(float(W.gw_for_angle(66.0, gw[::-1], an[::-1])) - 0.15) < 1e-12
    with pytest.raises(ValueError):
        W.gw_for_angle(120.0, gw, an)
    with pytest.raises(ValueError):
        W.gw_for_angle(50.0, gw, [44.0, 60.0, 58.0, 108.0])


def test_sessile_density_is_a_half_disc():
    rho = inputs.sessile_density(120, 60, RL, RV, 20.0)
    assert rho.dtype == np.float32
    assert rho[0, 60] > 0.99 * RL and rho[0, 5] < 1.01 * RV
    assert abs(O.contact_angle_cap(rho.astype(np.float64), RL, RV) - 90.0) < 1.0


@pytest.mark.slow
def test_oracle_droplets_match_paper_angles():
    """FP64 oracle, sessile droplets at T_s (thermal step off, g = 0) on a
    72 x 40 domain, 3000 steps from a half disc of radius 16: the static
    angles at G_w = 0 and 0.105 are the paper's within its "around", and the
    angle grows with G_w."""
    torch.set_num_threads(min(8, os.cpu_count() or 1))
    pv = paper_values()
    angles = {}
    for gw in (0.0, 0.105):
        P = O.Params(Lx=72, Ly=40, isothermal=True, g=0.0, Gw=gw)
        P.finalize()
        rho0 = torch.tensor(inputs.sessile_density(72, 40, P.rho_l, P.rho_v, 16.0), dtype=torch.float64)
        P.finalize(rho0=rho0)
        f, th = O.initial_state(rho0, P)
        for _ in range(3000):
            f, th, _ = O.step(f, th, P)
        angles[gw] = O.contact_angle_cap(f.sum(0).numpy(), P.rho_l, P.rho_v)
    for gw, key in ((0.0, "angle_gw_0"), (0.105, "angle_gw_0.105")):
        ref, tol = pv[key]
        assert abs(angles[gw] - ref) < tol, (gw, angles[gw], ref)
    assert angles[0.105] > angles[0.0] + 5.0
