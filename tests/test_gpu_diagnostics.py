"""GPU diagnostics (Sec. 3.2, Fig. 3): the device pressure probes against the
FP64 oracle step by step (plain and graph-replayed steps, ring wrap-around),
and the Young-Laplace law of static bubbles measured on GPU fields against
the oracle's own measurement of the same bubbles."""

import math
import os

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import inputs
from parity_util import oracle_initial_fp32, oracle_params

pytestmark = pytest.mark.gpu
F64 = torch.float64


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def test_probes_match_oracle(lb):
    """Probes at the centre of the top wall (Fig. 3's point), on the heated
    wall row and in the bulk of a heated pool: after 40 steps (32 replayed
    from a captured graph, 8 plain) a 16-record ring holds the last 16 steps
    in order, equal to the oracle's rho^t, T^t and p_EOS(rho^t, T^t) there."""
    Lx, Ly = 64, 48
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=lb.BC_WALLS, pool_height=20.0, noise_amp=1e-3, seed=3)
    Tc = lb.critical_temperature(cfg)
    sh = 0.1 * Tc
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 20.0, noise_amp=1e-3, seed=3)
    sim = lb.Simulation(cfg, superheat=sh, rho0=rho0)
    P = oracle_params(cfg, rho0, superheat=sh)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim.set_state(f0, th0)
    pts = [(Lx // 2, Ly - 1), (10, 0), (50, 20)]
    sim.set_probes(pts, capacity=16)
    sim.step(40)
    r = sim.probe_read()
    assert r["count"] == 40 and r["p"].shape == (3, 16)
    f, th = torch.tensor(f0, dtype=F64), torch.tensor(th0, dtype=F64)
    ref = []
    for _ in range(40):
        fn, thn, info = O.step(f, th, P)
        rho = info.fields.rho
        rec = []
        for x, y in pts:
            T = P.Ts + float(th[y, x])
            p = float(O.pr_pressure(rho[y, x], torch.tensor(T, dtype=F64), P.a, P.b, P.R, P.omega, P.Tc))
            rec.append((float(rho[y, x]), T, p))
        ref.append(rec)
        f, th = fn, thn
    ref = np.array(ref[-16:]).transpose(1, 0, 2)  # [probe][step][rho, T, p]
    err_rho = np.max(np.abs(r["rho"] / ref[..., 0] - 1))
    err_T = np.max(np.abs(r["T"] / ref[..., 1] - 1))
    # p is a difference of O(1) terms (~60x cancellation in the liquid), so
    # it is compared against the pressure scale p(T_s) of the coexistence
    err_p = np.max(np.abs(r["p"] - ref[..., 2])) / abs(ref[0, 0, 2])
    assert err_rho < 2e-6 and err_T < 1e-6 and err_p < 1e-4
    # removing the probes stops the recording; setting them again restarts it
    sim.set_probes([])
    sim.step(3)
    sim.set_probes(pts[:1], capacity=8)
    sim.step(5)
    assert sim.probe_read()["count"] == 5
    sim.close()


def test_probe_rejects_bad_points(lb):
    cfg = lb.Config(Lx=32, Ly=24, pool_height=10.0)
    sim = lb.Simulation(cfg)
    with pytest.raises(lb.LBError):
        sim.set_probes([(32, 0)])
    with pytest.raises(lb.LBError):
        sim.set_probes([(0, -1)])
    with pytest.raises(lb.LBError):
        sim.set_probes([(1, 1)] * (lb.PROBE_MAX + 1))
    sim.close()


def test_laplace_law_static_bubbles(lb):
    """Young-Laplace (Sec. 3.2): static vapour bubbles of radius 15-30 (well
    above the interface width, where the sharp-interface law applies) in
    saturated liquid, periodic 128 x 128 at T_s without gravity, relaxed
    20000 steps in one batch; the jump read from the GPU fields by the bubble
    and pressure diagnostics is delta p = s / r with R^2 > 0.99 and an
    intercept below 5 % of the largest jump."""
    from paper_1501_03857_gb300 import diagnostics as D
    L = 128
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_PERIODIC, isothermal=True, g=0.0, noise_amp=0.0)
    rv, rl = lb.coexistence(cfg)
    Ts = cfg.Ts_over_Tc * lb.critical_temperature(cfg)
    radii = (15.0, 20.0, 25.0, 30.0)
    batch = lb.Batch([{"cfg": cfg, "rho0": inputs.droplet_density(L, L, rv, rl, R)} for R in radii])
    batch.step(20000)
    r_eq, dp = [], []
    for i in range(len(radii)):
        f, _ = batch.get_state(i)
        rho = f.astype(np.float64).sum(axis=0)
        bs = D.bubbles(rho, rl, rv, periodic_y=True)
        assert len(bs) == 1
        r_eq.append(bs[0]["r_eq"])
        dp.append(D.laplace_jump(D.pressure(cfg, rho, np.full_like(rho, Ts)), bs[0], periodic_y=True))
    batch.close()
    fit = D.laplace_fit(r_eq, dp)
    print("laplace", r_eq, dp, fit)
    assert fit["surface_tension"] > 0 and fit["r2"] > 0.99, fit
    assert abs(fit["intercept"]) < 0.05 * max(dp), fit


def test_bubble_diagnostics_gpu_vs_oracle(lb):
    """One vapour bubble (radius 10, periodic 48 x 48, T_s, 1500 steps) run
    by the GPU and by the FP64 oracle from the same FP32 state: the bubble
    diagnostics read the same radius (0.05 cells) and pressure jump (0.5 %)
    from both fields."""
    from paper_1501_03857_gb300 import diagnostics as D
    torch.set_num_threads(min(8, os.cpu_count() or 1))
    L = 48
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_PERIODIC, isothermal=True, g=0.0, noise_amp=0.0)
    rv, rl = lb.coexistence(cfg)
    Ts = cfg.Ts_over_Tc * lb.critical_temperature(cfg)
    rho0 = inputs.droplet_density(L, L, rv, rl, 10.0)
    P = oracle_params(cfg, rho0)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(1500)
    fg, _ = sim.get_state()
    sim.close()
    f, th = torch.tensor(f0, dtype=F64), torch.tensor(th0, dtype=F64)
    for _ in range(1500):
        f, th, _ = O.step(f, th, P)
    out = []
    for rho in (fg.astype(np.float64).sum(axis=0), f.sum(0).numpy()):
        b = D.bubbles(rho, rl, rv, periodic_y=True)
        assert len(b) == 1
        out.append((b[0]["r_eq"], D.laplace_jump(D.pressure(cfg, rho, np.full_like(rho, Ts)), b[0],
                                                 periodic_y=True)))
    (rg, dg), (ro, do) = out
    assert abs(rg - ro) < 0.05
    assert abs(dg - do) < 5e-3 * abs(do)
