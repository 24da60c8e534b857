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


def test_batch_parameter_changes_follow_instances(lb):
    insts = make_instances(lb)[:3]
    batch = lb.Batch(insts)
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
    bx, seg, ms = tune.tune_batch(batch, candidates=((64, 0), (128, 0)), steps=2)
    assert bx in (64, 128) and ms > 0
    after = [batch.get_state(i) for i in range(2)]
    for (f0, t0), (f1, t1) in zip(before, after):
        assert np.array_equal(f0, f1) and np.array_equal(t0, t1)
