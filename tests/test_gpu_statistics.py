"""Statistical parity of the time-averaged wall heat flux on a boiling run.

Nucleate boiling is chaotic: a GPU run (FP32) and an oracle run (FP64) from
the same initial state part ways after the first bubbles, so a long run is
compared only through statistics. q_bar, the time average of the mean
bottom-wall heat flux q(t) (Sec. 3.2), of a small boiling pool is averaged
over an ensemble of seeds of the initial density noise on both sides: the
FP64 oracle's ensemble is stored in tests/golden/qbar_boiling_200x100.txt
(written by make_qbar_golden.py beside it, which calls only the oracle),
the GPU runs its own larger ensemble as the instances of one batch. The two
ensemble means must agree within 2 %; the combined standard error of the
difference is printed with them.
"""

import os

import numpy as np
import pytest
import torch

from paper_1501_03857_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "qbar_boiling_200x100.txt")
GPU_SEEDS = 512


def read_golden(path=GOLDEN):
    """{"mean", "sem", "nseeds", "runs": {seed: q_bar}} of the stored file."""
    out = {"runs": {}}
    for line in open(path):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "seed":
            out["runs"][int(line[1])] = float(line[2])
        elif line[0] == "seeds":
            out["nseeds"] = int(line[1])
        else:
            out[line[0]] = float(line[1])
    return out


@pytest.fixture(scope="module")
def lb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import lb as lbmod
    return lbmod


@pytest.mark.parametrize("tpb", [0, 1])
def test_time_averaged_heat_flux_matches_oracle_ensemble(lb, tpb):
    """200 x 100 pool, liquid below y = 60, superheat 0.02 (nucleate
    boiling), q_bar over steps 10000-29999: the mean over 512 GPU runs
    (one launch per step, and the persistent launch) against the mean over
    the oracle's runs, within 2 %."""
    g = read_golden()
    cfg = lb.Config(Lx=200, Ly=100, bc_y=lb.BC_WALLS, pool_height=60.0, noise_amp=1e-4)
    rv, rl = lb.coexistence(cfg)
    insts = [{"cfg": cfg, "superheat": 0.02,
              "rho0": inputs.pool_density(cfg.Lx, cfg.Ly, rl, rv, 60.0, noise_amp=1e-4, seed=sd)}
             for sd in range(1, GPU_SEEDS + 1)]
    batch = lb.Batch(insts)
    batch.set_persistent(tpb)
    batch.step(10000)
    batch.heat_flux(reset=True)
    batch.step(20000)
    q = batch.heat_flux()
    batch.close()
    assert (q["n"] == 20000).all()
    qg = q["q_mean"]
    mg, sg = float(qg.mean()), float(qg.std(ddof=1) / np.sqrt(len(qg)))
    mo, so = g["mean"], g["sem"]
    rel = mg / mo - 1.0
    comb = float(np.hypot(sg, so)) / mo
    same = sorted(g["runs"])
    mg_same = float(np.mean([qg[s - 1] for s in same]))
    print(f"q_bar GPU {mg:.5e} +- {sg:.1e} ({len(qg)} runs), oracle {mo:.5e} +- {so:.1e} ({len(same)} runs): "
          f"difference {100 * rel:+.2f} % (combined standard error {100 * comb:.2f} %); "
          f"GPU mean over the oracle's seeds {mg_same:.5e} ({100 * (mg_same / mo - 1):+.2f} %)")
    assert abs(rel) <= 0.02
