"""Write tests/golden/adjoint_256_gradients.txt: FP64 reference gradients of
the window-averaged bottom-wall heat flux J = (1/S) sum_n q(t_n) (Sec. 3.2)
on the 256 x 256 boiling domain, by central differences of the FP64 oracle
with Richardson extrapolation, so the reference carries neither FP32
rounding nor a first-order h^2 term.

Only oracle/ (the method) and paper_1501_03857_gb300/inputs.py (seeded
layouts, no method arithmetic) are used. Workload: 256 x 256 cells, walls in
y, the paper's EOS and transport (Sec. 3.1, after Eq. 21), liquid pool
below y = 102.4 with relative density noise 1e-4 (seed 5), bottom-wall
superheat 0.1 T_c, G_w = 0.065 (Eq. 22). The oracle runs 200 steps from
the pool; the window is the next 2000 steps. The window-start state is held
fixed except its bottom wall row, which is T_b (the gradient's definition).

For p = G_w and for the uniform shift of T_b(x): D(h) = (J(p + h) -
J(p - h)) / (2 h) at h = 2e-4 and 1e-4, and the extrapolated value
(4 D(h/2) - D(h)) / 3, whose error is O(h^4).

Usage: python tests/golden/make_adjoint_golden.py [threads]  (about 40
minutes on 8 threads)
"""

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_256_gradients.txt")
L, POOL, NOISE, SEED, GW = 256, 0.4 * 256, 1e-4, 5, 0.065
PRE, WINDOW = 200, 2000


def main():
    import numpy as np
    import torch
    torch.set_num_threads(int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1))
    import oracle as O
    from paper_1501_03857_gb300 import inputs
    t0 = time.time()
    P = O.Params(Lx=L, Ly=L, Gw=GW)
    Tc = O.critical_temperature(P.a, P.b, P.R)
    rv, rl = O.maxwell_coexistence(P.a, P.b, P.R, P.omega, P.Ts_over_Tc * Tc)
    sh = 0.1 * Tc
    rho0 = torch.tensor(inputs.pool_density(L, L, rl, rv, POOL, noise_amp=NOISE, seed=SEED), dtype=torch.float64)
    P.finalize(rho0=rho0, superheat=sh, rho_v=rv, rho_l=rl)
    f, th = O.initial_state(rho0, P)
    for _ in range(PRE):
        f, th, _ = O.step(f, th, P)
    f0, th0 = f, th

    def J(dtb=0.0, dgw=0.0):
        P.theta_b = torch.full((L,), sh + dtb, dtype=torch.float64)
        P.Gw = GW + dgw
        f, th = f0.clone(), th0.clone()
        th[0] = P.theta_b
        acc = 0.0
        for _ in range(WINDOW):
            f, th, info = O.step(f, th, P)
            acc += float(info.q)
        return acc / WINDOW

    Jv = J()
    res = {}
    for name, kw in (("Gw", "dgw"), ("Tb_uniform", "dtb")):
        D = {}
        for h in (2e-4, 1e-4):
            D[h] = (J(**{kw: h}) - J(**{kw: -h})) / (2 * h)
        res[name] = (D[2e-4], D[1e-4], (4 * D[1e-4] - D[2e-4]) / 3)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle reference gradients of J = window mean of q(t) (Sec. 3.2) on the 256 x 256\n")
        fh.write("# boiling domain; written by make_adjoint_golden.py\n")
        fh.write(f"# pool_height {POOL}, noise_amp {NOISE}, seed {SEED}, superheat 0.1 Tc = {sh:.9e}, Gw {GW}; "
                 f"{PRE} steps, then a window of {WINDOW}; wall time {time.time() - t0:.0f} s\n")
        fh.write(f"J {Jv:.12e}\n")
        for name, (d1, d2, dr) in res.items():
            fh.write(f"# {name}: central differences at h = 2e-4 and 1e-4, then Richardson\n")
            fh.write(f"d{name}_h2e-4 {d1:.12e}\nd{name}_h1e-4 {d2:.12e}\nd{name} {dr:.12e}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
