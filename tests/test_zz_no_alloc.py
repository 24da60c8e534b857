"""lb_fields_noalloc, the entry point for callers that cannot allocate device
memory (code inside another framework's memory pool or allocator hook,
processes not allowed to allocate after start-up, real-time loops that must
not touch the allocator). It computes the same macroscopic fields as
lb_fields from a device-resident state, with its scratch in a static device
array inside the library instead of a workspace. The test compares it with
lb_fields on two calls in a row (the second call sees the scratch the first
one left behind). This file is collected last on purpose."""

import numpy as np
import pytest
import torch

from paper_1501_03857_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 2e-6  # the one-step parity tolerance of the other GPU tests


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


def _norm_err(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / (s if s > 0 else 1.0))


@pytest.mark.parametrize("bc,ghost", [(0, False), (2, False), (0, True)])
def test_noalloc_fields_match_lb_fields_on_two_calls(lb, bc, ghost):
    Lx, Ly = 200, 96
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, ghost_layer=ghost)
    rv, rl = lb.coexistence(cfg)
    rho0, f0, th0 = inputs.random_state(Lx, Ly, rl, rv, 40, seed=21)
    Gw = 0.065
    sim = lb.Simulation(cfg, superheat=0.01, Gw=Gw, rho0=rho0)
    sim.set_state(f0, th0)
    rho_ave = float(np.asarray(rho0, np.float64).mean())
    dev = dict(dtype=torch.float32, device="cuda")
    f = torch.empty(9, Ly, Lx, **dev)
    th = torch.empty(Ly, Lx, **dev)
    for call in range(2):
        sim.get_state_device(f, th)
        ref = [torch.empty(Ly, Lx, **dev) for _ in range(4)]
        sim.fields_device(*ref)
        out = [torch.full((Ly, Lx), float("nan"), **dev) for _ in range(4)]
        torch.cuda.synchronize()
        before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
        lb.fields_noalloc(cfg, Gw, rho_ave, f, th, *out)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may place the library's static array (lazy
            # module loading); the second must not take any device memory
            assert (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()) == before
        for name, a, b in zip(("rho", "ux", "uy", "T"), out, ref):
            assert torch.isfinite(a).all(), (call, name)
            assert _norm_err(a, b) <= TOL, (call, name, _norm_err(a, b))
        sim.step(5)  # a different state for the second call


def test_noalloc_tall_grid_matches_lb_fields(lb):
    """A grid taller than the 65535 blocks a launch takes in y (2 x 70000
    cells, within the scratch): the per-cell kernels loop over rows."""
    Lx, Ly = 2, 70000
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=0, pool_height=30000)
    rho0 = lb.initial_density(cfg)
    sim = lb.Simulation(cfg, superheat=0.01, rho0=rho0)
    sim.step(3)
    dev = dict(dtype=torch.float32, device="cuda")
    f = torch.empty(9, Ly, Lx, **dev)
    th = torch.empty(Ly, Lx, **dev)
    sim.get_state_device(f, th)
    ref = [torch.empty(Ly, Lx, **dev) for _ in range(4)]
    sim.fields_device(*ref)
    out = [torch.full((Ly, Lx), float("nan"), **dev) for _ in range(4)]
    lb.fields_noalloc(cfg, 0.0, float(np.asarray(rho0, np.float64).mean()), f, th, *out)
    torch.cuda.synchronize()
    for name, a, b in zip(("rho", "ux", "uy", "T"), out, ref):
        assert torch.isfinite(a).all(), name
        assert _norm_err(a, b) <= TOL, (name, _norm_err(a, b))
    sim.close()


def test_noalloc_refuses_a_capturing_stream(lb):
    """The call synchronises its stream, which a stream under capture does
    not allow: it returns LB_E_INVAL without enqueuing anything, and the
    caller's capture stays valid and can be completed and replayed."""
    Lx, Ly = 32, 16
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=0)
    dev = dict(dtype=torch.float32, device="cuda")
    f = torch.full((9, Ly, Lx), 0.5, **dev)
    th = torch.zeros(Ly, Lx, **dev)
    x = torch.zeros(4, **dev)
    lb.fields_noalloc(cfg, 0.0, 4.5, f, th, torch.empty(Ly, Lx, **dev))  # set-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    out = torch.empty(Ly, Lx, **dev)
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        with pytest.raises(lb.LBError) as ei:
            lb.fields_noalloc(cfg, 0.0, 4.5, f, th, out, stream=s)
        x.add_(1.0)
    assert ei.value.code == -1 and "captured" in str(ei.value)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(x, torch.full((4,), 2.0, **dev))


def test_noalloc_rejects_grids_above_its_scratch(lb):
    cfg = lb.Config(Lx=1024, Ly=1024)
    assert cfg.Lx * cfg.Ly > lb.NOALLOC_MAX_CELLS
    dev = dict(dtype=torch.float32, device="cuda")
    f = torch.zeros(9, cfg.Ly, cfg.Lx, **dev)
    th = torch.zeros(cfg.Ly, cfg.Lx, **dev)
    with pytest.raises(lb.LBError) as ei:
        lb.fields_noalloc(cfg, 0.0, 3.0, f, th)
    assert ei.value.code == -1 and "LB_NOALLOC_MAX_CELLS" in str(ei.value)
