"""GPU wettability calibration (Eq. 22, Sec. 3.3): sessile droplets through
the batched C-ABI path against the paper's printed contact angles, and one
droplet against the FP64 oracle step for step."""

import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import inputs
from parity_util import norm_err, oracle_initial_fp32, oracle_params, run_oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_values():
    out = {}
    for line in open(os.path.join(GOLDEN, "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v, tol = line.split()
            out[k] = (float(v), float(tol))
    return out


@pytest.fixture(scope="module")
def W():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import wetting
    return wetting


def test_calibration_matches_paper_angles(W):
    """240 x 120 droplets (half disc of radius 40) at T_s, 20000 steps, in one
    batch: G_w = 0, 0.065, 0.105 give the paper's 44.5, 50 and 55.5 deg
    within its "around"; the angles have settled (change < 0.2 deg over the
    last 10000 steps) and increase with G_w."""
    pv = paper_values()
    r = W.run_droplets([0.0, 0.065, 0.105], W.droplet_config(240, 120), radius=40.0, steps=20000,
                       checkpoints=[10000])
    got = r["angle_deg"]
    for a, key in zip(got, ("angle_gw_0", "angle_gw_0.065", "angle_gw_0.105")):
        ref, tol = pv[key]
        assert abs(a - ref) < tol, (key, a, ref)
    assert got[0] < got[1] < got[2]
    assert max(abs(a - b) for a, b in zip(r["history"][10000], got)) < 0.2


def test_gw_for_angle_round_trip(W):
    """G_w read off a measured table reproduces the target angle when the
    droplet is relaxed at that G_w (interpolation error of the table)."""
    cfg = W.droplet_config(240, 120)
    table = W.run_droplets([0.1, 0.15, 0.2, 0.25], cfg, radius=40.0, steps=20000)
    g = float(W.gw_for_angle(70.0, table["Gw"], table["angle_deg"]))
    check = W.run_droplets([g], cfg, radius=40.0, steps=20000)
    assert abs(check["angle_deg"][0] - 70.0) < 1.0


def test_droplet_matches_oracle(W):
    """A 72 x 40 sessile droplet (G_w = 0.105, T_s, g = 0), 3000 steps from
    the same FP32 state: density field within 1e-4 of the FP64 oracle (the
    droplet relaxes towards a steady state, so the error does not grow), and
    the angles read by the two independent methods within 0.1 deg of each
    other and of the oracle field's."""
    from paper_1501_03857_gb300 import lb
    torch.set_num_threads(min(8, os.cpu_count() or 1))
    cfg = W.droplet_config(72, 40)
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.sessile_density(72, 40, rl, rv, 16.0)
    sim = lb.Simulation(cfg, Gw=0.105, rho0=rho0)
    P = oracle_params(cfg, rho0, Gw=0.105)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim.set_state(f0, th0)
    sim.step(3000)
    fg, _ = sim.get_state()
    fr, _, _ = run_oracle(f0, th0, P, 3000)
    rho_g = fg.astype(np.float64).sum(axis=0)
    rho_r = fr.sum(0).numpy()
    assert norm_err(rho_g, rho_r) < 1e-4
    a_gpu = W.contact_angle(rho_g, P.rho_l, P.rho_v)["angle_deg"]
    a_ref = O.contact_angle_cap(rho_r, P.rho_l, P.rho_v)
    assert abs(a_gpu - a_ref) < 0.1
    sim.close()
