"""GPU parity: the CUDA step, called through the C ABI, against the FP64
oracle on the same seeded inputs.

Tolerances (normalised max-norm error, max|gpu - oracle| / max|oracle| per
field) follow from FP32 storage and arithmetic: one step from an FP32 state
carries a few ulp (2^-24 ~ 6e-8) of rounding per operation through about a
hundred dependent operations, so 2e-6; after 200 steps the required bound
is 1e-5.
"""

import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_1501_03857_gb300 import inputs
from parity_util import norm_err, oracle_fields, oracle_initial_fp32, oracle_params, rel_err, run_oracle, theta_err

pytestmark = pytest.mark.gpu

TOL_ONE_STEP = 2e-6
TOL_200 = 1e-5


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def coex(lb, cfg):
    return lb.coexistence(cfg)


CASES = [
    # (Lx, Ly, bc, ghost, Gw, isothermal)
    (8, 6, 0, False, 0.0, False),
    (33, 17, 0, False, 0.08, False),
    (33, 17, 1, False, 0.0, False),
    (33, 17, 2, False, 0.0, False),
    (40, 12, 0, True, 0.0, False),
    (21, 9, 0, False, 0.0, True),
    (300, 70, 0, False, 0.105, False),
    (517, 41, 1, False, 0.065, False),
    (130, 23, 1, True, 0.05, False),   # outflow top with the ghost layer, two strips, ragged
    (229, 31, 2, False, 0.0, True),    # periodic, thermal step off, three strips, ragged
]


@pytest.mark.parametrize("Lx,Ly,bc,ghost,Gw,iso", CASES)
def test_one_step_from_random_state(lb, Lx, Ly, bc, ghost, Gw, iso):
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, ghost_layer=ghost, isothermal=iso)
    rv, rl = coex(lb, cfg)
    rho0, f0, th0 = inputs.random_state(Lx, Ly, rl, rv, Ly * 0.45, seed=Lx * 1000 + Ly)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=Gw, rho0=rho0)
    sim.set_launch(0, 6)  # several segments even on small grids
    sim.set_state(f0, th0)
    sim.step(1)
    fg, tg = sim.get_state()
    P = oracle_params(cfg, rho0, superheat=0.012, Gw=Gw)
    fr, tr, qs = run_oracle(f0, th0, P, 1)
    assert norm_err(fg, fr.numpy()) < TOL_ONE_STEP
    assert theta_err(tg, tr.numpy(), 0.012) < TOL_ONE_STEP
    if bc != 2:
        h = sim.heat_flux()
        assert h["n"] == 1
        assert abs(h["q_inst"] - qs[0]) <= 1e-5 * abs(qs[0]) + 1e-12


MINIMAL = [(1, 3, 0, False, 0.0, False), (1, 9, 2, False, 0.0, False), (2, 3, 1, False, 0.05, False),
           (5, 4, 0, True, 0.0, False), (3, 5, 2, False, 0.0, True)]


@pytest.mark.parametrize("Lx,Ly,bc,ghost,Gw,iso", MINIMAL)
def test_one_step_minimal_grids(lb, Lx, Ly, bc, ghost, Gw, iso):
    """The smallest grids the library accepts (one column, three rows, every
    boundary treatment) against the oracle, after the bounds-checked build
    ran them without a flag (test_gpu_checked.py)."""
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, ghost_layer=ghost, isothermal=iso)
    rv, rl = coex(lb, cfg)
    rho0, f0, th0 = inputs.random_state(Lx, Ly, rl, rv, Ly * 0.45, seed=Lx * 1000 + Ly)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=Gw, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(1)
    fg, tg = sim.get_state()
    sim.close()
    P = oracle_params(cfg, rho0, superheat=0.012, Gw=Gw)
    fr, tr, _ = run_oracle(f0, th0, P, 1)
    assert norm_err(fg, fr.numpy()) < TOL_ONE_STEP
    assert theta_err(tg, tr.numpy(), 0.012) < TOL_ONE_STEP


def config1(lb, outflow=True):
    """100 x 100 pool, a = 2/49, superheat 0.1 Tc, pool to y = 40, noise 1e-4,
    seed 1, g = 3e-5 (the small FP64 configuration)."""
    cfg = lb.Config(Lx=100, Ly=100, a=2 / 49, bc_y=1 if outflow else 0, pool_height=40.0, noise_amp=1e-4, seed=1)
    Tc = lb.critical_temperature(cfg)
    return cfg, 0.1 * Tc


@pytest.mark.parametrize("outflow", [True, False])
def test_200_steps_config1(lb, outflow):
    cfg, sh = config1(lb, outflow)
    rv, rl = coex(lb, cfg)
    rho0 = inputs.pool_density(cfg.Lx, cfg.Ly, rl, rv, cfg.pool_height, noise_amp=cfg.noise_amp, seed=cfg.seed)
    P = oracle_params(cfg, rho0, superheat=sh)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, superheat=sh, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(200)
    fg, tg = sim.get_state()
    fr, tr, qs = run_oracle(f0, th0, P, 200)
    errs = {"f": norm_err(fg, fr.numpy()), "theta": theta_err(tg, tr.numpy(), sh)}
    fl = sim.fields()
    rr, vxr, vyr, Tr = oracle_fields(fr, tr, P)
    # velocity components are normalised by the speed scale max|v| (u_x alone
    # is ~1e-6 while |v| ~ 1e-2 here, so its own maximum is no scale)
    vs = float(np.hypot(vxr, vyr).max())
    errs.update(rho=norm_err(fl["rho"], rr), ux=norm_err(fl["ux"], vxr, vs), uy=norm_err(fl["uy"], vyr, vs))
    # per-element relative errors where the field is strictly positive: the
    # populations span 0.011 (vapour diagonal) to 2.9 (liquid rest) and the
    # density 0.38 to 6.5, so the normalised errors above alone would let
    # the small values be off by 100 x more
    fref = fr.numpy()
    assert float(fref.min()) > 0 and float(rr.min()) > 0
    errs.update(f_rel=rel_err(fg, fref), rho_rel=rel_err(fl["rho"], rr))
    print("200 steps, outflow" if outflow else "200 steps, walls", {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < TOL_200, (k, v, errs)
    h = sim.heat_flux()
    assert h["n"] == 200
    assert abs(h["q_mean"] / np.mean(qs) - 1) < 1e-5


@pytest.mark.parametrize("outflow", [True, False])
def test_2000_steps_config1_long_run(lb, outflow):
    """The 100 x 100 configuration (walls, superheat 0.1 T_c) for 2000 steps,
    ten times the 200-step horizon, GPU against the FP64 oracle: no bubble
    has nucleated yet, so the run is still deterministic and the fields stay
    within the same 1e-5 bound (measured f 1e-6, theta 3e-6) and the mean
    wall heat flux of the second half within 1e-4 (measured 7e-7), far
    inside the 2 % statistical bound meant for chaotic runs."""
    import os
    torch.set_num_threads(min(16, os.cpu_count() or 1))
    cfg, sh = config1(lb, outflow=outflow)
    rv, rl = coex(lb, cfg)
    rho0 = inputs.pool_density(cfg.Lx, cfg.Ly, rl, rv, cfg.pool_height, noise_amp=cfg.noise_amp, seed=cfg.seed)
    P = oracle_params(cfg, rho0, superheat=sh)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, superheat=sh, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(1000)
    sim.heat_flux(reset=True)
    sim.step(1000)
    h = sim.heat_flux()
    fg, tg = sim.get_state()
    sim.close()
    fr, tr, qs = run_oracle(f0, th0, P, 2000)
    q_ref = float(np.mean(qs[1000:]))
    ef, et = norm_err(fg, fr.numpy()), theta_err(tg, tr.numpy(), sh)
    print(f"2000 steps: q rel {abs(h['q_mean'] / q_ref - 1):.2e}, f {ef:.2e}, theta {et:.2e}")
    assert abs(h["q_mean"] / q_ref - 1) < 1e-4
    assert ef < TOL_200 and et < TOL_200


def test_200_steps_paper_scale_300x400(lb):
    """The paper-scale single-run configuration: 300 x 400, walls, bottom
    superheat 0.2 T_c, wettability G_w = 0.125 (near the 60 deg point of the
    contact-angle calibration; any fixed value serves for parity), liquid
    pool to y = 100 with 1e-4 noise (seed 2), the paper's EOS (a = 3/49):
    200 steps against the oracle within the 1e-5 bound, heat flux within
    1e-5."""
    import os
    torch.set_num_threads(min(16, os.cpu_count() or 1))
    cfg = lb.Config(Lx=300, Ly=400, bc_y=lb.BC_WALLS, pool_height=100.0, noise_amp=1e-4, seed=2)
    sh, gw = 0.2 * lb.critical_temperature(cfg), 0.125
    rv, rl = coex(lb, cfg)
    rho0 = inputs.pool_density(cfg.Lx, cfg.Ly, rl, rv, cfg.pool_height, noise_amp=cfg.noise_amp, seed=cfg.seed)
    P = oracle_params(cfg, rho0, superheat=sh, Gw=gw)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, superheat=sh, Gw=gw, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(200)
    fg, tg = sim.get_state()
    h = sim.heat_flux()
    sim.close()
    fr, tr, qs = run_oracle(f0, th0, P, 200)
    assert norm_err(fg, fr.numpy()) < TOL_200
    assert theta_err(tg, tr.numpy(), sh) < TOL_200
    assert abs(h["q_mean"] / np.mean(qs) - 1) < 1e-5


SHAPES = ((0, 0), (64, 1), (128, 5), (256, 57), (64, 1000), (128, 13))


def test_launch_shape_does_not_change_results(lb):
    """Each cell's arithmetic is the same whatever the strip width and segment
    height, so the results are bit-identical across launch shapes."""
    cfg = lb.Config(Lx=263, Ly=57, bc_y=0)
    rv, rl = coex(lb, cfg)
    rho0, f0, th0 = inputs.random_state(cfg.Lx, cfg.Ly, rl, rv, 25, seed=5)
    ref = None
    for bx, seg in SHAPES:
        sim = lb.Simulation(cfg, superheat=0.01, Gw=0.05, rho0=rho0)
        sim.set_launch(bx, seg)
        sim.set_state(f0, th0)
        sim.step(3)
        fg, tg = sim.get_state()
        if ref is None:
            ref = (fg, tg)
        else:
            assert np.array_equal(fg, ref[0]) and np.array_equal(tg, ref[1]), (bx, seg)


def test_heat_flux_is_reproducible(lb):
    """Two runs of the same wide domain (38 column strips, so 38 blocks add
    to q(t) every step, finishing in whatever order the GPU schedules them)
    give identical heat-flux statistics: each strip's sum has its own slot
    and the slots are folded in strip order."""
    cfg = lb.Config(Lx=4096, Ly=48, bc_y=0, pool_height=20, noise_amp=1e-3, seed=7)
    out = []
    for _ in range(2):
        sim = lb.Simulation(cfg, superheat=0.02, Gw=0.05)
        sim.step(70)
        out.append(sim.heat_flux())
        sim.close()
    assert out[0]["n"] == 70
    assert out[0]["q_mean"] == out[1]["q_mean"] and out[0]["q_std"] == out[1]["q_std"]
    assert out[0]["q_inst"] == out[1]["q_inst"]


def test_fields_and_mass_match_oracle(lb):
    cfg = lb.Config(Lx=64, Ly=48, bc_y=0, pool_height=20)
    rv, rl = coex(lb, cfg)
    rho0, f0, th0 = inputs.random_state(cfg.Lx, cfg.Ly, rl, rv, 20, seed=9)
    sim = lb.Simulation(cfg, superheat=0.01, Gw=0.1, rho0=rho0)
    sim.set_state(f0, th0)
    fl = sim.fields()
    P = oracle_params(cfg, rho0, superheat=0.01, Gw=0.1)
    rr, vxr, vyr, Tr = oracle_fields(torch.tensor(f0, dtype=torch.float64), torch.tensor(th0, dtype=torch.float64), P)
    assert norm_err(fl["rho"], rr) < TOL_ONE_STEP
    vs = float(np.hypot(vxr, vyr).max())
    assert norm_err(fl["ux"], vxr, vs) < 1e-5
    assert norm_err(fl["uy"], vyr, vs) < 1e-5
    assert norm_err(fl["T"], Tr) < 1e-6
    assert abs(sim.mass() / float(np.asarray(f0, np.float64).sum()) - 1) < 1e-12


def test_mass_conserved_periodic(lb):
    """Fully periodic: mass is conserved to FP32 rounding (FP64 sum)."""
    cfg = lb.Config(Lx=128, Ly=96, bc_y=2, g=0.0)
    rv, rl = coex(lb, cfg)
    rho0 = inputs.droplet_density(128, 96, rl, rv, 20, noise_amp=1e-3, seed=2)
    sim = lb.Simulation(cfg, rho0=rho0)
    m0 = sim.mass()
    sim.step(2000)
    sim.sync()
    assert abs(sim.mass() / m0 - 1) < 1e-5


def test_eos_domain_and_nonfinite_flags(lb):
    """A density beyond the EOS limit (psi argument < 0) and a NaN, both
    planted on the host, come back as LB_E_EOS_DOMAIN and LB_E_NONFINITE at
    the next synchronising call; the context stays usable."""
    cfg = lb.Config(Lx=16, Ly=8, bc_y=2)
    rv, rl = coex(lb, cfg)
    P = oracle_params(cfg, np.full((8, 16), rl, dtype=np.float32))
    rho_bad = 9.9
    T = torch.tensor([P.Ts], dtype=torch.float64)
    assert bool(O.pseudopotential(torch.tensor([rho_bad], dtype=torch.float64), T, P)[1][0])
    sim = lb.Simulation(cfg, rho0=np.full((8, 16), rl, dtype=np.float32))
    f, th = sim.get_state()
    sim.set_state(f * np.float32(rho_bad / rl), th)
    sim.step(1)
    with pytest.raises(lb.LBError) as ei:
        sim.sync()
    assert ei.value.code == -3
    sim.sync()  # the flag was cleared by the report
    f3 = f.copy()
    f3[0, 2, 2] = np.nan
    sim.set_state(f3, th)
    sim.step(1)
    with pytest.raises(lb.LBError) as ei:
        sim.sync()
    assert ei.value.code == -4
    sim.set_state(f, th)
    sim.step(1)
    sim.sync()


def test_save_load_roundtrip(lb):
    cfg = lb.Config(Lx=50, Ly=30, bc_y=0, pool_height=12)
    sim = lb.Simulation(cfg, superheat=0.01)
    sim.step(10)
    blob = sim.save()
    sim.step(5)
    f1, t1 = sim.get_state()
    q1 = sim.heat_flux()
    sim.load(blob)
    assert sim.info()["steps"] == 10
    sim.step(5)
    f2, t2 = sim.get_state()
    assert np.array_equal(f1, f2) and np.array_equal(t1, t2)
    q2 = sim.heat_flux()
    assert q2 == q1  # the heat flux is folded in a fixed order
    # the blob also carries the wall temperature and G_w: settings changed
    # after the save are undone by the load
    sim.load(blob)
    sim.set_wall_temperature(0.05, 0.01 * np.cos(np.arange(50)))
    sim.set_wettability(0.1)
    sim.step(3)
    sim.load(blob)
    sim.step(5)
    f3, t3 = sim.get_state()
    assert np.array_equal(f1, f3) and np.array_equal(t1, t3)
    assert sim.heat_flux() == q1


def test_wall_temperature_profile_and_superheat_step(lb):
    """Per-x wall profile and the superheat step of Sec. 3.2 match the oracle."""
    cfg = lb.Config(Lx=40, Ly=20, bc_y=0, pool_height=10)
    rv, rl = coex(lb, cfg)
    rho0 = inputs.pool_density(40, 20, rl, rv, 10, noise_amp=1e-3, seed=4)
    prof = 0.004 * np.sin(2 * math.pi * np.arange(40) / 40)
    P = oracle_params(cfg, rho0, superheat=0.01, profile=prof)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, superheat=0.01, profile=prof, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(20)
    sim.set_wall_temperature(0.02, prof)
    sim.step(20)
    f, th, _ = run_oracle(f0, th0, P, 20)
    P.theta_b = torch.tensor(0.02 + prof, dtype=torch.float64)
    th = th.clone()
    th[0] = P.theta_b
    fr, tr, _ = run_oracle(f.numpy(), th.numpy(), P, 20)
    fg, tg = sim.get_state()
    assert norm_err(fg, fr.numpy()) < 1e-5
    assert theta_err(tg, tr.numpy(), 0.02) < 1e-5


def test_full_size_sampled_rows(lb):
    """4096 x 4096 bubble domain, one step in the benchmark's launch shape:
    bands of rows (bottom wall, middle, top wall) against the oracle run on
    the band alone; rows at least 7 away from a band's artificial edge depend
    only on data inside the band."""
    L = 4096
    cfg = lb.Config(Lx=L, Ly=L, bc_y=0)
    rv, rl = coex(lb, cfg)
    rho0 = inputs.bubble_density(L, L, rl, rv, n_bubbles=256, r_min=20, r_max=60, seed=4)
    sim = lb.Simulation(cfg, superheat=0.1 * lb.critical_temperature(cfg), Gw=0.0, rho0=rho0)
    rho_ave = float(np.asarray(rho0, np.float64).mean())
    P = oracle_params(cfg, None, superheat=0.1 * lb.critical_temperature(cfg), rho_ave=rho_ave)
    # the initial state of both sides: the oracle's equilibrium of rho0, in FP32
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim.set_state(f0, th0)
    sim.step(1)
    fg, tg = sim.get_state()
    band = 16
    for y0, bc in ((0, 0), (2000, 2), (L - band, 0)):
        Pb = oracle_params(lb.Config(Lx=L, Ly=band, bc_y=bc), None, superheat=P.theta_b[0].item(), rho_ave=rho_ave)
        fr, tr, qs = run_oracle(f0[:, y0:y0 + band], th0[y0:y0 + band], Pb, 1)
        if y0 == 0:
            rows = list(range(0, band - 7))
            q = sim.heat_flux()["q_inst"]
            assert abs(q - qs[0]) <= 1e-5 * abs(qs[0])
        elif y0 == L - band:
            rows = list(range(7, band))
        else:
            rows = list(range(7, band - 7))
        assert norm_err(fg[:, y0 + rows[0]:y0 + rows[-1] + 1], fr.numpy()[:, rows[0]:rows[-1] + 1]) < TOL_ONE_STEP
        assert theta_err(tg[y0 + rows[0]:y0 + rows[-1] + 1], tr.numpy()[rows[0]:rows[-1] + 1],
                         P.theta_b[0].item()) < TOL_ONE_STEP


def test_maximum_size_sampled_rows(lb):
    """The largest grid the 32-bit population offsets allow (16384 x 14563,
    238.6 M cells, 19 GB of state), a pool initialised on the device from its
    density, one step in the default launch shape: bands of rows (heated
    wall, the interface in the middle, top wall) against the oracle run on
    the band alone from the same densities; rows at least 7 away from a
    band's artificial edge depend only on data inside the band."""
    Lx, Ly, band = 16384, 14563, 16
    y_if = 7000.5
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=0)
    rv, rl = coex(lb, cfg)
    sh = 0.1 * lb.critical_temperature(cfg)
    rho0 = np.empty((Ly, Lx), dtype=np.float32)
    for y0 in range(0, Ly, 1024):  # row chunks keep the host temporaries small
        y1 = min(y0 + 1024, Ly)
        rho0[y0:y1] = inputs.pool_density(Lx, Ly, rl, rv, y_if, noise_amp=1e-3, seed=11, rows=(y0, y1))
    rho_ave = float(rho0.astype(np.float64).mean())
    sim = lb.Simulation(cfg, superheat=sh, rho0=rho0)
    sim.step(1)
    fg = torch.empty((9, Ly, Lx), dtype=torch.float32, device="cuda")
    tg = torch.empty((Ly, Lx), dtype=torch.float32, device="cuda")
    sim.get_state_device(fg, tg)
    q = sim.heat_flux()["q_inst"]
    sim.close()
    for y0, bc in ((0, 0), (int(y_if) - band // 2, 2), (Ly - band, 0)):
        Pb = oracle_params(lb.Config(Lx=Lx, Ly=band, bc_y=bc), None, superheat=sh, rho_ave=rho_ave)
        rb = torch.tensor(rho0[y0:y0 + band], dtype=torch.float64)
        f0, th0 = O.initial_state(rb, Pb)
        fr, tr, qs = run_oracle(f0.numpy().astype(np.float32), th0.numpy().astype(np.float32), Pb, 1)
        if y0 == 0:
            rows = list(range(0, band - 7))
            assert abs(q - qs[0]) <= 1e-5 * abs(qs[0])
        elif y0 == Ly - band:
            rows = list(range(7, band))
        else:
            rows = list(range(7, band - 7))
        r0, r1 = rows[0], rows[-1] + 1
        got_f = fg[:, y0 + r0:y0 + r1].cpu().numpy()
        got_t = tg[y0 + r0:y0 + r1].cpu().numpy()
        assert norm_err(got_f, fr.numpy()[:, r0:r1]) < TOL_ONE_STEP
        assert theta_err(got_t, tr.numpy()[r0:r1], sh) < TOL_ONE_STEP
