"""Write tests/golden/qbar_boiling_200x100.txt: the time-averaged bottom-wall
heat flux q_bar (Sec. 3.2: q(t) is the mean over x of q_w = -lambda dT/dy at
the heated wall, q_bar its time average) of a small boiling pool, run by the
FP64 oracle once per seed of the pool's initial density noise.

Only oracle/ (the method) and paper_1501_03857_gb300/inputs.py (seeded
layouts, no method arithmetic) are used. Nucleate boiling is chaotic, so a
GPU run and an oracle run from the same state part ways after the first
bubbles and only the statistics of q_bar can be compared: the file holds
every seed's q_bar and the ensemble mean with its standard error.

Workload: 200 x 100 cells, walls in y, the paper's EOS and transport
parameters (Sec. 3.1, after Eq. 21), liquid pool below y = 60 with relative
density noise 1e-4, bottom-wall superheat Delta T = 0.02 (lattice units,
nucleate boiling: the first bubbles appear after 2000-4000 steps), 30000
steps; q_bar is the mean of q(t) over steps t = 10000 .. 29999.

Usage: python tests/golden/make_qbar_golden.py [first_seed last_seed] [nprocs]
runs the seeds first_seed..last_seed (default 1..70) and merges them with
the runs already in the file (35 seeds on 7 single-threaded processes take
about 55 minutes).
"""

import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qbar_boiling_200x100.txt")
LX, LY, POOL, NOISE, SUPERHEAT = 200, 100, 60.0, 1e-4, 0.02
STEPS, T0 = 30000, 10000


def run_seed(seed):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    torch.set_num_threads(1)
    import oracle as O
    from paper_1501_03857_gb300 import inputs
    P = O.Params(Lx=LX, Ly=LY)
    Tc = O.critical_temperature(P.a, P.b, P.R)
    rv, rl = O.maxwell_coexistence(P.a, P.b, P.R, P.omega, P.Ts_over_Tc * Tc)
    rho0 = torch.tensor(inputs.pool_density(LX, LY, rl, rv, POOL, noise_amp=NOISE, seed=seed), dtype=torch.float64)
    P.finalize(rho0=rho0, superheat=SUPERHEAT, rho_v=rv, rho_l=rl)
    f, th = O.initial_state(rho0, P)
    qs = np.empty(STEPS)
    for n in range(STEPS):
        f, th, info = O.step(f, th, P)
        qs[n] = float(info.q)
    return seed, float(qs[T0:].mean()), float(qs[:T0].mean())


def main():
    first = int(sys.argv[1]) if len(sys.argv) > 2 else 1
    last = int(sys.argv[2]) if len(sys.argv) > 2 else 70
    nprocs = int(sys.argv[3]) if len(sys.argv) > 3 else 7
    runs = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            p = line.split()
            if p and p[0] == "seed":
                runs[int(p[1])] = float(p[2])
    todo = [sd for sd in range(first, last + 1) if sd not in runs]
    t0 = time.time()
    if todo:
        with mp.get_context("spawn").Pool(nprocs) as pool:
            for sd, qb, _ in pool.map(run_seed, todo, chunksize=1):
                runs[sd] = qb
    import numpy as np
    q = np.array([runs[k] for k in sorted(runs)])
    mean, sem = q.mean(), q.std(ddof=1) / np.sqrt(len(q))
    with open(OUT, "w") as fh:
        fh.write("# Time-averaged bottom-wall heat flux q_bar (Sec. 3.2) of a boiling pool, FP64 oracle,\n")
        fh.write("# one run per seed of the initial density noise; written by make_qbar_golden.py\n")
        fh.write(f"# Lx {LX} Ly {LY} walls, paper EOS and transport (Sec. 3.1), pool_height {POOL}, "
                 f"noise_amp {NOISE}, superheat {SUPERHEAT}\n")
        fh.write(f"# steps {STEPS}, q_bar over steps {T0}..{STEPS - 1}; single-threaded runs of about 10 minutes "
                 f"each (the last {len(todo)} in {time.time() - t0:.0f} s on {nprocs} processes)\n")
        fh.write(f"mean {mean:.9e}\nsem {sem:.9e}\nseeds {len(q)}\n")
        for sd in sorted(runs):
            fh.write(f"seed {sd} {runs[sd]:.9e}\n")
    print(f"q_bar mean {mean:.6e} sem {sem:.3e} ({100 * sem / mean:.2f} %) over {len(q)} seeds")


if __name__ == "__main__":
    main()
