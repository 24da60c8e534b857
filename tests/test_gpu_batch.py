"""The batched form: several uneven-size simulations advanced by one launch
per step (with captured graphs for runs of 32 steps) give bit-identical
results to stepping each instance alone, for odd and even step counts. The
heat flux is folded from fixed per-strip slots in strip order, so with the
same block size (the same strips) its statistics are identical too."""

import numpy as np
import pytest
import torch

from paper_1501_03857_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = [(64, 40), (100, 64), (48, 96), (130, 50), (72, 72)]


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def make_instances(lb):
    out = []
    for i, (Lx, Ly) in enumerate(SIZES):
        cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=lb.BC_WALLS if i % 2 == 0 else lb.BC_TOP_OUTFLOW,
                        pool_height=0.4 * Ly)
        rv, rl = lb.coexistence(cfg)
        rho0 = inputs.pool_density(Lx, Ly, rl, rv, 0.4 * Ly, noise_amp=1e-3, seed=10 + i)
        out.append({"cfg": cfg, "superheat": 0.005 * (i + 1), "Gw": 0.03 * i, "rho0": rho0})
    return out


@pytest.mark.parametrize("shape", [(128, 0), (64, 16)])
def test_batch_equals_single_instances(lb, shape):
    insts = make_instances(lb)
    batch = lb.Batch(insts)
    batch.set_launch(*shape)
    for n in (3, 32, 5, 40):  # odd counts, one graph chunk, a chunk plus remainder
        batch.step(n)
    batch.sync()
    q = batch.heat_flux()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.set_launch(shape[0], 0)
        sim.step(80)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        hs = sim.heat_flux()
        assert q["n"][i] == hs["n"] == 80
        assert q["q_mean"][i] == hs["q_mean"] and q["q_std"][i] == hs["q_std"]
        # macroscopic fields of the instance (lb_batch_fields) equal the
        # single run's (lb_fields); a subset is computed when asked
        fb_all = batch.fields(i)
        fs_all = sim.fields()
        for k in ("rho", "ux", "uy", "T"):
            assert np.array_equal(fb_all[k], fs_all[k]), (i, k)
        assert set(batch.fields(i, ("rho",))) == {"rho"}
        sim.close()


def test_batch_with_different_model_constants(lb):
    """Instances that differ in a model constant (sigma of Eq. 8, gravity of
    Eq. 9) run with the constants taken from each instance's own record
    rather than shared launch parameters; the results are still
    bit-identical to stepping each instance alone."""
    insts = make_instances(lb)[:3]
    from dataclasses import replace
    insts[1]["cfg"] = replace(insts[1]["cfg"], sigma=1.1)
    insts[2]["cfg"] = replace(insts[2]["cfg"], g=2e-5)
    batch = lb.Batch(insts)
    batch.set_launch(64, 0)
    batch.step(37)
    batch.sync()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.step(37)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        sim.close()
    batch.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_parameter_changes_follow_instances(lb, persistent):
    insts = make_instances(lb)[:3]
    batch = lb.Batch(insts)
    if persistent:
        batch.set_persistent(1)  # 33 steps after the change: one 32-step launch and one of 1
    batch.step(7)
    batch.set_wall_temperature(1, 0.03)
    batch.set_wettability(2, 0.1)
    batch.step(33)
    sims = []
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.step(7)
        if i == 1:
            sim.set_wall_temperature(0.03)
        if i == 2:
            sim.set_wettability(0.1)
        sim.step(33)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i


def test_tune_batch_keeps_state(lb):
    from paper_1501_03857_gb300 import tune
    insts = make_instances(lb)[:2]
    batch = lb.Batch(insts)
    batch.step(4)
    before = [batch.get_state(i) for i in range(2)]
    bx, seg, ms, tpb = tune.tune_batch(batch, candidates=((64, 0), (128, 0), (64, 0, 2)), steps=2)
    assert bx in (64, 128) and ms > 0 and tpb in (0, 2)
    after = [batch.get_state(i) for i in range(2)]
    for (f0, t0), (f1, t1) in zip(before, after):
        assert np.array_equal(f0, f1) and np.array_equal(t0, t1)


# ---- the persistent batch: one cooperative launch per run of 32 steps ------

@pytest.mark.parametrize("block_x,tpb", [(64, 1), (64, 2), (128, 3)])
def test_persistent_batch_equals_single_instances(lb, block_x, tpb):
    """Every instance advanced by the persistent launches (tiles dealt out to
    one co-resident grid, a tile waiting for its instance's previous step)
    is bit-identical to the instance stepped alone, heat-flux statistics
    included, for runs below, at and above the 32 steps of one launch."""
    insts = make_instances(lb)
    batch = lb.Batch(insts)
    batch.set_launch(block_x, 0)
    batch.set_persistent(tpb)
    for n in (3, 32, 5, 40):
        batch.step(n)
    batch.sync()
    q = batch.heat_flux()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.set_launch(block_x, 0)
        sim.step(80)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        hs = sim.heat_flux()
        assert q["n"][i] == hs["n"] == 80
        assert q["q_mean"][i] == hs["q_mean"] and q["q_std"][i] == hs["q_std"]
        sim.close()
    batch.close()


def test_persistent_batch_with_different_model_constants(lb):
    """Instances that differ in sigma and gravity take every constant from
    their own record in the persistent kernel too."""
    insts = make_instances(lb)[:3]
    from dataclasses import replace
    insts[1]["cfg"] = replace(insts[1]["cfg"], sigma=1.1)
    insts[2]["cfg"] = replace(insts[2]["cfg"], g=2e-5)
    batch = lb.Batch(insts)
    batch.set_launch(64, 0)
    batch.set_persistent(2)
    batch.step(37)
    batch.sync()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.step(37)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        sim.close()
    batch.close()


def test_persistent_wait_limit_reports_timeout_and_recovers(lb):
    """A wait limit of one poll makes the tiles' waits for the rest of their
    instance run out: the launch ends, LB_E_TIMEOUT is reported, the context
    stays usable, and with the default limit and the states reset the batch
    again equals the single runs."""
    insts = make_instances(lb)
    batch = lb.Batch(insts)
    batch.set_launch(64, 8)  # many tiles per instance
    init = [batch.get_state(i) for i in range(len(insts))]
    batch.set_persistent(1, wait_limit=1)
    batch.step(32)
    with pytest.raises(lb.LBError) as ei:
        batch.sync()
    assert ei.value.code == -5
    batch.sync()  # reported once, then cleared
    batch.set_persistent(1)
    for i, (f0, t0) in enumerate(init):
        batch.set_state(i, f0, t0)
    batch.step(33)
    batch.sync()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.step(33)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        sim.close()
    batch.close()


@pytest.mark.parametrize("tpb", [0, 2])
def test_batch_instance_matches_oracle(lb, tpb):
    """One instance of an uneven batch (one launch per step, and the
    persistent launch) against the FP64 oracle directly: 40 steps of a
    heated pool with wettability, within the 1e-5 bound of the parity tests
    (normalised, and per element for the populations)."""
    import oracle as O
    from parity_util import norm_err, oracle_initial_fp32, oracle_params, rel_err, run_oracle, theta_err
    insts = make_instances(lb)[:3]
    d = insts[1]
    cfg = d["cfg"]
    P = oracle_params(cfg, d["rho0"], superheat=d["superheat"], Gw=d["Gw"])
    f0, th0 = oracle_initial_fp32(d["rho0"], P)
    batch = lb.Batch(insts)
    batch.set_launch(64, 0)
    batch.set_persistent(tpb)
    batch.set_state(1, f0, th0)
    batch.step(40)
    fb, tb = batch.get_state(1)
    q = batch.heat_flux()
    batch.close()
    fr, tr, qs = run_oracle(f0, th0, P, 40)
    assert norm_err(fb, fr.numpy()) < 1e-5
    assert rel_err(fb, fr.numpy()) < 1e-5
    assert theta_err(tb, tr.numpy(), d["superheat"]) < 1e-5
    assert abs(q["q_mean"][1] / np.mean(qs) - 1) < 1e-5


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_of_every_grid_option_equals_single_instances(lb, persistent):
    """Instances with the ghost layer (walls and outflow top), periodic y and
    the thermal step off, mixed in one batch, give the single-instance
    results bit for bit, heat-flux statistics included."""
    opts = [dict(bc_y=lb.BC_WALLS, ghost_layer=True), dict(bc_y=lb.BC_TOP_OUTFLOW, ghost_layer=True),
            dict(bc_y=lb.BC_PERIODIC), dict(bc_y=lb.BC_WALLS, isothermal=True),
            dict(bc_y=lb.BC_TOP_OUTFLOW, isothermal=True, ghost_layer=True)]
    sizes = [(56, 30), (90, 41), (48, 36), (120, 25), (33, 50)]
    insts = []
    for i, (o, (Lx, Ly)) in enumerate(zip(opts, sizes)):
        cfg = lb.Config(Lx=Lx, Ly=Ly, pool_height=0.4 * Ly, **o)
        rv, rl = lb.coexistence(cfg)
        rho0 = inputs.pool_density(Lx, Ly, rl, rv, 0.4 * Ly, noise_amp=1e-3, seed=30 + i)
        insts.append({"cfg": cfg, "superheat": 0.004 * (i + 2), "Gw": 0.02 * i, "rho0": rho0})
    batch = lb.Batch(insts)
    batch.set_launch(64, 0)  # the single instances' block size: the same strips, the same heat-flux fold
    if persistent:
        batch.set_persistent(2)
    batch.step(37)  # one 32-step run and a remainder of 5
    batch.sync()
    q = batch.heat_flux()
    for i, d in enumerate(insts):
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], rho0=d["rho0"])
        sim.set_launch(64, 0)
        sim.step(37)
        fs, ts = sim.get_state()
        fb, tb = batch.get_state(i)
        assert np.array_equal(fs, fb) and np.array_equal(ts, tb), i
        hs = sim.heat_flux()
        assert q["n"][i] == hs["n"] and q["q_mean"][i] == hs["q_mean"] and q["q_std"][i] == hs["q_std"], i
        sim.close()
    batch.close()
