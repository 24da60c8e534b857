"""The hand-written discrete adjoint against the FP64 oracle: gradients of
the window-averaged wall heat flux with respect to the wall temperature
profile and G_w, compared with the oracle's autograd adjoint and with FP64
central differences of the oracle (required agreement: 1e-3 relative)."""

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


def setup(lb, Lx=24, Ly=16, superheat=0.012, Gw=0.05, seed=3, bc=None, ghost=False):
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=lb.BC_WALLS if bc is None else bc, pool_height=0.45 * Ly, ghost_layer=ghost)
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 0.45 * Ly, noise_amp=1e-2, seed=seed)
    prof = superheat + 0.003 * np.sin(2 * np.pi * np.arange(Lx) / Lx)
    P = oracle_params(cfg, rho0, superheat=0.0, profile=prof, Gw=Gw)
    f0, th0 = oracle_initial_fp32(rho0, P)
    return cfg, rho0, prof, P, f0, th0


def oracle_J(P, f0, th0, tb, gw, n):
    """J(theta_b, G_w) of the oracle with the window-start wall row = theta_b."""
    P.theta_b = tb
    P.Gw = gw
    f = torch.tensor(f0, dtype=F64)
    th = torch.cat([tb.view(1, -1), torch.tensor(th0[1:], dtype=F64)], 0)
    qs = []
    for _ in range(n):
        f, th, info = O.step(f, th, P)
        qs.append(info.q)
    return torch.stack(qs).mean()


def gpu_adjoint(lb, cfg, rho0, prof, Gw, f0, th0, n, ckpt):
    sim = lb.Simulation(cfg, superheat=0.0, profile=prof, Gw=Gw, rho0=rho0)
    sim.set_state(f0, th0)
    return sim.adjoint(n, ckpt)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("ckpt", [5, 1])
@pytest.mark.parametrize("Lx,Ly,outflow", [(24, 16, False), (24, 16, True), (24, 17, False), (24, 17, True),
                                           (130, 17, True)])
def test_adjoint_matches_oracle_autograd(lb, Lx, Ly, outflow, ckpt):
    """Walls, and the outflow top (whose top row pulls populations 4, 7, 8
    from itself, so their f* has two consumers). The reverse kernels march
    segments of 4 rows here: with Ly = 17 the top row would be a segment of
    its own and is joined to the one below; Lx = 130 takes two column strips
    of each reverse kernel. Checkpoints every 5 steps (segments replayed) and
    every step (every step stored by the forward pass)."""
    n = 12
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=Lx, Ly=Ly, bc=lb.BC_TOP_OUTFLOW if outflow else None)
    tb = torch.tensor(prof, dtype=F64, requires_grad=True)
    gw = torch.tensor(0.05, dtype=F64, requires_grad=True)
    Jo = oracle_J(P, f0, th0, tb, gw, n)
    gtb, ggw = torch.autograd.grad(Jo, (tb, gw))
    J, dTb, dGw = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, n, ckpt=ckpt)
    print(f"J rel {abs(J / float(Jo) - 1):.2e} dTb rel {rel(dTb, gtb.numpy()):.2e} "
          f"dGw rel {abs(dGw / float(ggw) - 1):.2e}")
    assert abs(J / float(Jo) - 1) < 1e-5
    assert rel(dTb, gtb.numpy()) < 1e-3, rel(dTb, gtb.numpy())
    assert abs(dGw / float(ggw) - 1) < 1e-3, (dGw, float(ggw))


@pytest.mark.parametrize("Lx,Ly,outflow,ckpt", [(24, 16, False, 5), (24, 17, True, 1), (130, 16, False, 1),
                                                (130, 17, True, 4), (3, 5, False, 2)])
def test_adjoint_ghost_layer_matches_oracle_autograd(lb, Lx, Ly, outflow, ckpt):
    """The ghost-layer option (F_m also on the wall rows, from a ghost row
    that copies the wall row's psi): walls and outflow top, both modes."""
    n = 10
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=Lx, Ly=Ly, bc=lb.BC_TOP_OUTFLOW if outflow else None, ghost=True)
    assert P.ghost
    tb = torch.tensor(prof, dtype=F64, requires_grad=True)
    gw = torch.tensor(0.05, dtype=F64, requires_grad=True)
    Jo = oracle_J(P, f0, th0, tb, gw, n)
    gtb, ggw = torch.autograd.grad(Jo, (tb, gw))
    J, dTb, dGw = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, n, ckpt=ckpt)
    print(f"ghost {Lx}x{Ly}: J rel {abs(J / float(Jo) - 1):.2e} dTb rel {rel(dTb, gtb.numpy()):.2e} "
          f"dGw rel {abs(dGw / float(ggw) - 1):.2e}")
    assert abs(J / float(Jo) - 1) < 1e-5
    assert rel(dTb, gtb.numpy()) < 1e-3, rel(dTb, gtb.numpy())
    assert abs(dGw / float(ggw) - 1) < 1e-3, (dGw, float(ggw))


@pytest.mark.parametrize("Lx,Ly,outflow,ckpt", [(1, 3, False, 1), (1, 3, True, 3), (2, 4, True, 1), (2, 5, False, 2),
                                                (5, 5, True, 4), (3, 9, False, 1)])
def test_adjoint_small_grids_match_oracle_autograd(lb, Lx, Ly, outflow, ckpt):
    """The smallest grids: one or two columns (every lane of a reverse
    kernel's strip wraps onto them), three rows (both walls next to the one
    fluid row), walls and outflow top, both adjoint modes."""
    n = 6
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=Lx, Ly=Ly, bc=lb.BC_TOP_OUTFLOW if outflow else None)
    tb = torch.tensor(prof, dtype=F64, requires_grad=True)
    gw = torch.tensor(0.05, dtype=F64, requires_grad=True)
    Jo = oracle_J(P, f0, th0, tb, gw, n)
    gtb, ggw = torch.autograd.grad(Jo, (tb, gw))
    J, dTb, dGw = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, n, ckpt=ckpt)
    print(f"{Lx}x{Ly}: J rel {abs(J / float(Jo) - 1):.2e} dTb rel {rel(dTb, gtb.numpy()):.2e} "
          f"dGw {dGw:.3e} oracle {float(ggw):.3e}")
    assert abs(J / float(Jo) - 1) < 1e-5
    assert rel(dTb, gtb.numpy()) < 1e-3, rel(dTb, gtb.numpy())
    assert abs(dGw - float(ggw)) <= 1e-3 * abs(float(ggw)) + 1e-12, (dGw, float(ggw))


def test_adjoint_matches_central_differences(lb):
    """Central differences (h = 1e-4) of the FP64 oracle on single cells of
    T_b, the uniform T_b mode and G_w."""
    n = 30
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=32, Ly=20, seed=5)
    J, dTb, dGw = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, n, ckpt=7)
    h = 1e-4
    tb0 = torch.tensor(prof, dtype=F64)
    Jf = lambda tb, gw: float(oracle_J(P, f0, th0, tb, torch.tensor(gw, dtype=F64), n))
    for x in (0, 9, 31):
        e = torch.zeros(cfg.Lx, dtype=F64)
        e[x] = h
        fd = (Jf(tb0 + e, 0.05) - Jf(tb0 - e, 0.05)) / (2 * h)
        print(f"x={x} adjoint {dTb[x]:.6e} fd {fd:.6e} rel {abs(dTb[x] - fd) / abs(fd):.2e}")
        assert abs(dTb[x] - fd) <= 1e-3 * abs(fd) + 1e-9, (x, dTb[x], fd)
    fd = (Jf(tb0 + h, 0.05) - Jf(tb0 - h, 0.05)) / (2 * h)
    assert abs(dTb.sum() - fd) <= 1e-3 * abs(fd), (dTb.sum(), fd)
    fd = (Jf(tb0, 0.05 + h) - Jf(tb0, 0.05 - h)) / (2 * h)
    assert abs(dGw - fd) <= 1e-3 * abs(fd), (dGw, fd)


def test_checkpoint_interval_does_not_change_gradients(lb):
    n = 20
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=30, Ly=14, seed=7)
    a = gpu_adjoint(lb, cfg, rho0, prof, 0.08, f0, th0, n, ckpt=1)
    b = gpu_adjoint(lb, cfg, rho0, prof, 0.08, f0, th0, n, ckpt=6)
    c = gpu_adjoint(lb, cfg, rho0, prof, 0.08, f0, th0, n, ckpt=100)
    for other in (b, c):
        assert other[0] == a[0]
        assert np.array_equal(other[1], a[1])
        assert abs(other[2] - a[2]) <= 1e-12 * abs(a[2])


def test_autograd_function(lb):
    cfg, rho0, prof, P, f0, th0 = setup(lb, Lx=20, Ly=12, seed=9)
    sim = lb.Simulation(cfg, superheat=0.0, profile=prof, Gw=0.05, rho0=rho0)
    sim.set_state(f0, th0)
    blob = sim.save()
    Tb = torch.tensor(prof, dtype=F64, requires_grad=True)
    Gw = torch.tensor(0.05, dtype=F64, requires_grad=True)
    J = lb.heat_flux_window(Tb, Gw, sim, blob, 10, 4)
    J.backward()
    _, dTb, dGw = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, 10, 4)
    assert np.allclose(Tb.grad.numpy(), dTb, rtol=1e-12, atol=0)
    assert abs(float(Gw.grad) - dGw) <= 1e-12 * abs(dGw)
    # without an interval the wrapper lets the library pick it (every step
    # stored here): the same J and gradients as an explicit interval of 1
    Tb2 = torch.tensor(prof, dtype=F64, requires_grad=True)
    Gw2 = torch.tensor(0.05, dtype=F64, requires_grad=True)
    J2 = lb.heat_flux_window(Tb2, Gw2, sim, blob, 10)
    J2.backward()
    J1, dTb1, dGw1 = gpu_adjoint(lb, cfg, rho0, prof, 0.05, f0, th0, 10, 1)
    assert float(J2) == J1
    assert np.allclose(Tb2.grad.numpy(), dTb1, rtol=1e-12, atol=0)
    assert abs(float(Gw2.grad) - dGw1) <= 1e-12 * abs(dGw1)


@pytest.mark.parametrize("L", [256, 512])
def test_gradient_direction_at_bench_scale(lb, L):
    """The whole dJ/dT_b(x) vector on the 256 x 256 boiling domain of the
    benchmark (500-step window after a 200-step transient, checkpoint every
    100): the FP32 forward's central difference along the normalised
    gradient g/|g| equals |g| within the 1e-3 bound, and along a direction
    orthogonal to g it is small against |g|. Also at 512 x 512, where each
    reverse kernel marches several column strips and many segments."""
    n = 500
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_WALLS, pool_height=0.4 * L, seed=5)
    sh, gw = 0.1 * lb.critical_temperature(cfg), 0.065
    sim = lb.Simulation(cfg, superheat=sh, Gw=gw)
    sim.step(200)
    blob = sim.save()
    J, g, _ = sim.adjoint(n, 100)
    norm = float(np.linalg.norm(g))
    d = g / norm

    def J_of(profile):
        sim.load(blob)
        sim.set_wall_temperature(sh, profile)
        sim.heat_flux(reset=True)
        sim.step(n)
        return sim.heat_flux()["q_mean"]

    h = 1e-4
    along = (J_of(h * d) - J_of(-h * d)) / (2 * h)
    assert abs(along / norm - 1) < 1e-3, (along, norm)
    rng = np.random.default_rng(0)
    o = rng.standard_normal(L)
    o -= (o @ d) * d
    o /= np.linalg.norm(o)
    across = (J_of(h * o) - J_of(-h * o)) / (2 * h)
    assert abs(across - float(g @ o)) < 1e-3 * norm, (across, float(g @ o), norm)
    sim.close()


def test_adjoint_256_window_against_fp64_reference(lb):
    """The gradient of the benchmark window (256 x 256 boiling domain, 200
    steps from the pool, then a 2000-step window, checkpoint every 100)
    against FP64 reference gradients of the oracle (central differences
    at h = 2e-4 and 1e-4, Richardson-extrapolated; tests/golden/
    adjoint_256_gradients.txt, written from the oracle alone): dJ/dG_w and
    the uniform T_b mode within 1e-3, J within 1e-5."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "adjoint_256_gradients.txt")
    ref = {}
    for line in open(path):
        p = line.split("#")[0].split()
        if len(p) == 2:
            ref[p[0]] = float(p[1])
    L = 256
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_WALLS, pool_height=0.4 * L, seed=5)
    sh = 0.1 * lb.critical_temperature(cfg)
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(L, L, rl, rv, 0.4 * L, noise_amp=1e-4, seed=5)
    P = oracle_params(cfg, rho0, superheat=sh, Gw=0.065)
    f0, th0 = oracle_initial_fp32(rho0, P)
    sim = lb.Simulation(cfg, superheat=sh, Gw=0.065, rho0=rho0)
    sim.set_state(f0, th0)
    sim.step(200)
    J, dTb, dGw = sim.adjoint(2000, 100)
    sim.close()
    eJ, eG, eT = abs(J / ref["J"] - 1), abs(dGw / ref["dGw"] - 1), abs(float(dTb.sum()) / ref["dTb_uniform"] - 1)
    print(f"256^2 window: J rel {eJ:.2e}, dJ/dG_w rel {eG:.2e}, uniform dJ/dT_b rel {eT:.2e} "
          f"(Richardson vs h = 1e-4 alone: {abs(ref['dGw'] / ref['dGw_h1e-4'] - 1):.1e}, "
          f"{abs(ref['dTb_uniform'] / ref['dTb_uniform_h1e-4'] - 1):.1e})")
    assert eJ < 1e-5
    assert eG < 1e-3 and eT < 1e-3


def test_checkpoint_interval_for_a_memory_budget(lb):
    """lb_adjoint_pick_ckpt: every step stored when its scratch fits the
    budget; else the interval of smallest scratch, which fits and equals
    lb_adjoint_scratch_bytes for it; an error when nothing fits. The picked
    interval's adjoint is the one run with that interval given explicitly."""
    cfg, rho0, prof, P, f0, th0 = setup(lb)
    sim = lb.Simulation(cfg, superheat=0.0, profile=prof, Gw=0.05, rho0=rho0)
    n = 40
    all_steps = sim.adjoint_scratch_bytes(n, 1)
    assert sim.adjoint_ckpt(n, all_steps) == 1
    c = sim.adjoint_ckpt(n, all_steps - 1)
    sizes = {k: sim.adjoint_scratch_bytes(n, k) for k in range(2, n + 1)}
    assert c >= 2 and sizes[c] == min(sizes.values()) and sizes[c] < all_steps
    assert sim.adjoint_ckpt(n, sizes[c]) == c
    with pytest.raises(RuntimeError):
        sim.adjoint_ckpt(n, sizes[c] - 1)
    with pytest.raises(RuntimeError):
        sim.adjoint_ckpt(1, sim.adjoint_scratch_bytes(1, 1) - 1)
    sim.set_state(f0, th0)
    J, dTb, dGw = sim.adjoint(12)  # default budget: half the free memory, every step stored
    sim.set_state(f0, th0)
    J1, dTb1, dGw1 = sim.adjoint(12, 1)
    assert J == J1 and dGw == dGw1 and np.array_equal(dTb, dTb1)
    sim.close()
