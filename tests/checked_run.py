"""Helper of test_gpu_checked.py (not a test module): steps the cases given
on the command line, the batches and the adjoints below with whichever
library LBBOIL_LIB selects and saves the resulting states and gradients to
an .npz file. Every run ends with a synchronising call, which raises if the
checked build flagged an address outside its buffer."""

import json
import sys

import numpy as np

from paper_1501_03857_gb300 import inputs, lb


def run(case):
    Lx, Ly, bc, ghost, gw, iso, steps, bx, seg = case
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, ghost_layer=bool(ghost), isothermal=bool(iso))
    rv, rl = lb.coexistence(cfg)
    rho0, f0, th0 = inputs.random_state(Lx, Ly, rl, rv, Ly * 0.45, seed=Lx * 1000 + Ly)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=gw, rho0=rho0)
    sim.set_launch(bx, seg)
    sim.set_state(f0, th0)
    sim.step(steps)
    sim.sync()
    f, th = sim.get_state()
    sim.close()
    return f, th


def run_batch(shapes, block_x=64, seg=0, vary=False, tpb=0):
    insts = []
    for i, (Lx, Ly, bc) in enumerate(shapes):
        # vary: instances differ in sigma, so the step reads every constant
        # from its instance's record instead of shared launch parameters
        cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, pool_height=0.4 * Ly, seed=20 + i,
                        sigma=1.2 + (0.05 * (i % 2) if vary else 0.0))
        insts.append({"cfg": cfg, "superheat": 0.01, "Gw": 0.05 * (i % 3)})
    b = lb.Batch(insts)
    b.set_launch(block_x, seg)
    b.set_persistent(tpb)  # 0: one launch per step; >= 1: the persistent launch
    b.step(37)
    b.sync()
    out = [b.get_state(i) for i in range(b.n)]
    b.close()
    return out


# adjoints (Lx, Ly, bc, nsteps, ckpt_every): odd sizes, one and two columns,
# three rows, several strips and segments of both reverse kernels, walls and
# outflow top, segments replayed and every step stored
ADJOINTS = [(1, 3, 0, 6, 1), (2, 4, 1, 6, 3), (17, 9, 0, 8, 1), (33, 17, 1, 8, 5), (130, 17, 0, 6, 4),
            (257, 40, 1, 5, 1), (300, 70, 0, 5, 2), (45, 13, 0, 6, 1, 1), (131, 21, 1, 6, 3, 1)]  # ..., ghost layer


def run_adjoint(case):
    Lx, Ly, bc, n, ck = case[:5]
    ghost = bool(case[5]) if len(case) > 5 else False
    cfg = lb.Config(Lx=Lx, Ly=Ly, bc_y=bc, pool_height=0.45 * Ly, ghost_layer=ghost)
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(Lx, Ly, rl, rv, 0.45 * Ly, noise_amp=1e-2, seed=Lx + 7 * Ly)
    sim = lb.Simulation(cfg, superheat=0.012, Gw=0.05, rho0=rho0)
    J, dTb, dGw = sim.adjoint(n, ck)
    sim.close()
    return np.concatenate([[J, dGw], dTb])


def random_batch(seed=11, n=12):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(1, 200)), int(rng.integers(3, 90)), int(rng.integers(0, 3))) for _ in range(n)]


if __name__ == "__main__":
    cases = json.loads(sys.argv[1])
    res = {}
    for k, c in enumerate(cases):
        res[f"f{k}"], res[f"t{k}"] = run(c)
    batches = [(((40, 30, 0), (57, 23, 1), (33, 48, 2)), 64, 0, False, 0), (random_batch(), 128, 0, False, 0),
               (random_batch(12, 9), 64, 5, False, 0), (random_batch(13, 7), 64, 0, True, 0),
               (random_batch(14, 5), 128, 7, True, 0),
               # the persistent launch: one and several tiles per block
               (random_batch(15, 10), 64, 0, False, 1), (random_batch(16, 8), 128, 6, False, 2),
               (random_batch(17, 6), 64, 0, True, 1), (random_batch(18, 4), 64, 3, False, 3)]
    for j, (shapes, bx, seg, vary, tpb) in enumerate(batches):
        for k, (f, t) in enumerate(run_batch(shapes, bx, seg, vary, tpb)):
            res[f"b{j}f{k}"], res[f"b{j}t{k}"] = f, t
    for k, c in enumerate(ADJOINTS):
        res[f"adj{k}"] = run_adjoint(c)
    np.savez(sys.argv[2], **res)
