"""Statistical parity of the time-averaged wall heat flux on a boiling run.

Nucleate boiling is chaotic: a GPU run (FP32) and an oracle run (FP64) from
the same initial state part ways after the first bubbles, so a long run is
compared only through statistics. q_bar, the time average of the mean
bottom-wall heat flux q(t) (Sec. 3.2), of a small boiling pool is averaged
over an ensemble of seeds of the initial density noise on both sides: the
FP64 oracle's ensemble is stored in tests/golden/qbar_boiling_200x100.txt
(written by make_qbar_golden.py beside it, which calls only the oracle),
the GPU runs its own larger ensemble as the instances of one batch.

The ensemble has a long low tail. Most runs boil in the nucleate regime
(q_bar 1.13e-3 to 1.35e-3 in 58 of the oracle's 70 runs); about one in six
stays for part of the window under the vapour blanket that the first burst
of bubbles spreads over the wall (q_bar 0.59e-3 to 0.96e-3). The all-run mean
therefore carries the binomial noise of how many runs fall in the tail
(16 % run-to-run spread against 5.3 % within the nucleate runs). So the
comparison is: the mean q_bar of the runs above Q_GAP (the nucleate runs)
within 2 % (the scope's bound), and the fraction of runs below it within
three standard errors of the difference of two binomial fractions. The
all-run means and their standard errors are printed beside them.
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


Q_GAP = 1.0e-3  # between the oracle's blanketed runs (highest 0.96e-3) and its nucleate runs (lowest 1.13e-3)


@pytest.mark.parametrize("tpb", [0, 1])
def test_time_averaged_heat_flux_matches_oracle_ensemble(lb, tpb):
    """200 x 100 pool, liquid below y = 60, superheat 0.02 (nucleate
    boiling), q_bar over steps 10000-29999 of 512 GPU runs (one launch per
    step, and the persistent launch) against the oracle's runs."""
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
    qg = np.asarray(q["q_mean"])
    qo = np.array([g["runs"][k] for k in sorted(g["runs"])])
    sem = lambda v: float(v.std(ddof=1) / np.sqrt(len(v)))
    hg, ho = qg[qg > Q_GAP], qo[qo > Q_GAP]
    fg, fo = 1 - len(hg) / len(qg), 1 - len(ho) / len(qo)
    rel = hg.mean() / ho.mean() - 1.0
    comb = float(np.hypot(sem(hg), sem(ho))) / ho.mean()
    fp = (fg * len(qg) + fo * len(qo)) / (len(qg) + len(qo))
    fsd = float(np.sqrt(fp * (1 - fp) * (1 / len(qg) + 1 / len(qo))))
    same = sorted(g["runs"])
    print(f"all runs: GPU {qg.mean():.5e} +- {sem(qg):.1e} ({len(qg)}), oracle {qo.mean():.5e} +- {sem(qo):.1e} "
          f"({len(qo)}); nucleate runs: GPU {hg.mean():.5e}, oracle {ho.mean():.5e}, difference {100 * rel:+.2f} % "
          f"(combined standard error {100 * comb:.2f} %); blanketed fraction GPU {fg:.3f}, oracle {fo:.3f} "
          f"(sd of the difference {fsd:.3f}); in the gap: GPU {int(((qg > 0.85e-3) & (qg < 1.1e-3)).sum())}; "
          f"same seeds, GPU mean {np.mean([qg[s - 1] for s in same]):.5e}")
    assert abs(rel) <= 0.02
    assert abs(fg - fo) <= 3 * fsd
