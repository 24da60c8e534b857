"""Degenerate calls of the boundary on the GPU: zero steps, the heat-flux
record before any step, and adjoint windows of one step or shorter than the
checkpoint interval. Each either leaves the state exactly as it was or gives
exactly what the general path gives. With every step stored, the adjoint's
forward pass runs in its own buffers and copies the window's last state
(populations and theta) back into the simulation; the state comparison
checks that copy."""

import numpy as np
import pytest
import torch

from paper_1501_03857_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def pool(lb, Lx=40, Ly=24, bc=None, seed=2):
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=lb.BC_WALLS if bc is None else bc, pool_height=0.45 * Ly)
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 0.45 * Ly, noise_amp=1e-3, seed=seed)
    return cfg, rho0


def test_zero_steps_change_nothing(lb):
    cfg, rho0 = pool(lb)
    sim = lb.Simulation(cfg, superheat=0.01, Gw=0.05, rho0=rho0)
    q0 = sim.heat_flux()
    assert q0["n"] == 0 and q0["q_mean"] == 0.0 and q0["q_std"] == 0.0  # no sample yet
    sim.step(5)
    f0, t0 = sim.get_state()
    q5 = sim.heat_flux()
    sim.step(0)
    f1, t1 = sim.get_state()
    q = sim.heat_flux()
    assert np.array_equal(f0, f1) and np.array_equal(t0, t1)
    assert q == q5 and q["n"] == 5
    with pytest.raises(RuntimeError):
        sim.step(-1)
    sim.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_zero_batch_steps_change_nothing(lb, persistent):
    insts = []
    for i, (Lx, Ly) in enumerate([(40, 24), (70, 30)]):
        cfg, rho0 = pool(lb, Lx, Ly, seed=5 + i)
        insts.append({"cfg": cfg, "superheat": 0.01, "Gw": 0.02 * i, "rho0": rho0})
    batch = lb.Batch(insts)
    if persistent:
        batch.set_persistent(1)
    batch.step(3)
    batch.sync()
    before = [batch.get_state(i) for i in range(2)]
    q3 = batch.heat_flux()
    batch.step(0)
    batch.sync()
    q = batch.heat_flux()
    for i in range(2):
        f, t = batch.get_state(i)
        assert np.array_equal(f, before[i][0]) and np.array_equal(t, before[i][1])
    assert all(np.array_equal(q[k], q3[k]) for k in q) and list(q["n"]) == [3, 3]


@pytest.mark.parametrize("n,ckpt", [(1, 1), (1, 4), (3, 5), (3, 3)])
def test_short_adjoint_windows_equal_every_step_stored(lb, n, ckpt):
    """One step, and windows no longer than the interval (one segment, one
    checkpoint): the same J and gradients as storing every step, bit for bit,
    and the simulation advances by the window either way."""
    cfg, rho0 = pool(lb, bc=lb.BC_TOP_OUTFLOW)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=0.05, rho0=rho0)
    sim.step(4)
    blob = sim.save()
    q4 = sim.heat_flux()
    J, dTb, dGw = sim.adjoint(n, ckpt)
    assert sim.heat_flux() == q4 and sim.info()["steps"] == 4 + n  # accumulators untouched, steps advanced
    fa, ta = sim.get_state()
    sim.load(blob)
    J1, dTb1, dGw1 = sim.adjoint(n, 1)
    fb, tb = sim.get_state()
    sim.load(blob)
    sim.step(n)
    fc, tc = sim.get_state()
    assert J == J1 and dGw == dGw1 and np.array_equal(dTb, dTb1)
    assert np.isfinite(J) and J != 0.0 and np.any(dTb != 0.0)
    assert np.array_equal(fa, fb) and np.array_equal(fa, fc) and np.array_equal(ta, tc)
    with pytest.raises(RuntimeError):
        sim.adjoint(0, 1)
    sim.close()


@pytest.mark.parametrize("ckpt", [1, 3])
def test_adjoint_window_records_probes_once(lb, ckpt):
    """Probes record each step of the adjoint's forward pass once, with the
    values plain steps record; the segment replays of the reverse sweep add
    no records."""
    cfg, rho0 = pool(lb)
    pts = [(3, 2), (20, 10), (39, 22)]
    sim = lb.Simulation(cfg, superheat=0.012, Gw=0.05, rho0=rho0)
    sim.step(2)
    blob = sim.save()
    sim.set_probes(pts, capacity=32)
    sim.adjoint(7, ckpt)
    ra = sim.probe_read()
    sim.load(blob)
    sim.set_probes(pts, capacity=32)
    sim.step(7)
    rb = sim.probe_read()
    assert ra["count"] == rb["count"] == 7
    for k in ("rho", "T", "p"):
        assert ra[k].shape == (3, 7) and np.array_equal(ra[k], rb[k]), k
    sim.close()


def test_adjoint_does_not_depend_on_the_launch_shape(lb):
    """The replayed forward steps are launch-shape independent, so J and the
    gradients are the same under another block size and segment height."""
    cfg, rho0 = pool(lb, Lx=150, Ly=40)
    out = []
    for shape in ((0, 0), (128, 7), (64, 3)):
        sim = lb.Simulation(cfg, superheat=0.012, Gw=0.05, rho0=rho0)
        sim.set_launch(*shape)
        sim.step(3)
        out.append(sim.adjoint(9, 4))
        sim.close()
    for J, dTb, dGw in out[1:]:
        assert J == out[0][0] and np.array_equal(dTb, out[0][1])
        assert abs(dGw - out[0][2]) <= 1e-12 * abs(out[0][2])


def test_simulations_on_two_streams_are_independent(lb):
    """Two simulations on their own CUDA streams, stepped in turns (runs of 32
    steps replayed from graphs and single steps), each end where it ends when
    run alone: handles share no device state."""
    cases = [pool(lb, Lx=90, Ly=36, seed=1), pool(lb, Lx=64, Ly=48, bc=lb.BC_TOP_OUTFLOW, seed=2)]
    solo = []
    for cfg, rho0 in cases:
        sim = lb.Simulation(cfg, superheat=0.01, Gw=0.03, rho0=rho0)
        sim.step(70)
        solo.append(sim.get_state() + (sim.heat_flux(),))
        sim.close()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sims = [lb.Simulation(cfg, superheat=0.01, Gw=0.03, rho0=rho0, stream=s) for (cfg, rho0), s in zip(cases, streams)]
    for n in (33, 1, 36):
        for sim in sims:
            sim.step(n)
    for sim, (f, t, q) in zip(sims, solo):
        f2, t2 = sim.get_state()
        assert np.array_equal(f, f2) and np.array_equal(t, t2)
        assert sim.heat_flux() == q
        sim.close()


def test_calls_after_close_raise(lb):
    """A closed simulation or batch has no handle: every call is rejected by
    the library's null-handle check (an LBError), nothing reaches the device,
    and closing twice is harmless."""
    cfg, rho0 = pool(lb)
    sim = lb.Simulation(cfg, superheat=0.01, rho0=rho0)
    sim.step(2)
    sim.close()
    sim.close()
    for call in (lambda: sim.step(1), sim.heat_flux, sim.get_state, sim.sync, lambda: sim.adjoint(2, 1)):
        with pytest.raises(lb.LBError):
            call()
    batch = lb.Batch([{"cfg": cfg, "rho0": rho0}])
    batch.step(2)
    batch.close()
    batch.close()
    for call in (lambda: batch.step(1), batch.heat_flux, batch.sync):
        with pytest.raises(lb.LBError):
            call()


@pytest.mark.parametrize("ckpt", [1, 3])
def test_adjoint_reports_faults_in_its_window(lb, ckpt):
    """A density beyond the EOS limit (rho = 9.9 > the domain of psi, as in
    the step's own flag test) and a NaN population, planted on the host in
    the window-start state, make lb_adjoint return LB_E_EOS_DOMAIN and
    LB_E_NONFINITE; the simulation's own flags stay clear, and after a good
    state is set the same call succeeds."""
    cfg, rho0 = pool(lb)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=0.05, rho0=rho0)
    f, th = sim.get_state()
    rl = lb.coexistence(cfg)[1]
    bad = f.copy()
    bad[:, 3:6, 10:14] *= np.float32(9.9 / rl)  # liquid cells pushed past the EOS domain
    nan = f.copy()
    nan[4, 8, 8] = np.nan
    for state, code in ((bad, -3), (nan, -4)):
        sim.set_state(state, th)
        with pytest.raises(lb.LBError) as ei:
            sim.adjoint(1, ckpt)  # one step: the planted fault, before it can turn into another
        assert ei.value.code == code
        sim.sync()  # the simulation's own accumulator saw nothing
    sim.set_state(f, th)
    J, dTb, dGw = sim.adjoint(4, ckpt)
    assert np.isfinite(J) and np.all(np.isfinite(dTb)) and np.isfinite(dGw)
    sim.close()
