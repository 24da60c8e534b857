"""Benchmark of the fused hybrid thermal LB boiling step (one JSON line).

Workload: the 4096 x 4096 bubble-array boiling domain (walls in y, heated
bottom at superheat 0.1 T_c, 256 vapour bubbles of radius 20-60 in saturated
liquid at 0.86 T_c, paper EOS a = 3/49). A "step" is one time step of the
whole path: stream + collide + forces, RK4 temperature, wall heat flux.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value      MLUPS (lattice-cell updates per microsecond) over all ranks, device
           time of the timed steps with the state resident in HBM (the state,
           1.34 GB, is larger than L2, so no flush is needed).
e2e        the same metric through the public API with host buffers: every
           step uploads the wall temperature profile from host memory, steps,
           and reads the heat-flux accumulators back (synchronising).
roofline   the fused kernel's algorithmic 80 B per cell update (9 populations
           and theta, each read and written once) over its average CUDA-event
           duration, against the measured HBM copy bandwidth.
cpu_baseline / --impl reference
           the FP64 oracle on the host cores, on a bounded band of rows of the
           same workload.
batched    48 boiling-curve instances (contact angles 40-150 deg through the
           sessile-droplet G_w calibration) in one launch per step against
           the same instances stepped one after another.
adjoint    gradient of the window-mean wall heat flux: cost against the
           forward steps and agreement with finite differences (256 x 256),
           and the reverse sweep's roofline on a 2048 x 2048 domain.
experiments the boiling curves and regimes of Sec. 3.2-3.3 and Fig. 3's
           top-wall pressure on the paper's 600 x 150 pool.
Multi-GPU (torchrun): independent replicas, one domain per rank (weak scaling).
"""

from __future__ import annotations

import argparse
import datetime
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % HBM roofline (fwd, adjoint); boiling-curve sims/hour batched vs plain"
L = 4096
BYTES_PER_LU = 80  # 9 populations + theta, FP32, read + write
WORKLOAD = {"workload": "boiling domain 4096x4096, 256 vapour bubbles r=20-60, walls in y, "
                        "heated bottom superheat 0.1Tc, Ts=0.86Tc, PR a=3/49 b=2/21 omega=0.344",
            "Lx": L, "Ly": L, "state_bytes": None, "l2": "inputs larger than L2 (no flush)"}


def workload_config():
    from paper_1501_03857_gb300 import lb
    return lb.Config(Lx=L, Ly=L, bc_y=lb.BC_WALLS)


def workload_rho0(cfg, rv, rl):
    from paper_1501_03857_gb300 import inputs
    return inputs.bubble_density(cfg.Lx, cfg.Ly, rl, rv, n_bubbles=256, r_min=20.0, r_max=60.0, seed=4)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples (every 50 ms) kept only while the
    timed region runs (host wall-clock window given to stop())."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i", str(index),
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # let nvidia-smi start sampling before the timed region
        except OSError:
            self.proc = None

    def stop(self, t0: float, t1: float):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        return self.summarise(out, t0, t1)

    @staticmethod
    def summarise(out: str, t0: float, t1: float):
        """Median SM clock, the largest maximum clock and the active throttle
        reasons over the samples inside [t0, t1] (25 ms slack)."""
        rows = []
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 - 0.025 <= r[0] <= t1 + 0.025]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = set()
        for r in inside:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm = [r[1] for r in inside]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(r[2] for r in rows) if rows else None,
                "reasons": sorted(reasons), "samples": len(sm), "window_s": t1 - t0}


# rows of the workload's bottom band (full 4096 width) that the FP64 oracle
# steps: the same band for the cpu_baseline block and the reference arm
CPU_BAND_ROWS = 32


def oracle_band(rows: int = CPU_BAND_ROWS):
    """The workload's bottom band of `rows` rows for the FP64 oracle: its
    parameters (rho_ave of the whole domain) and initial state."""
    import torch
    import oracle as O
    from paper_1501_03857_gb300 import inputs
    a, b, R, om = 3 / 49, 2 / 21, 1.0, 0.344
    Tc = O.critical_temperature(a, b, R)
    rv, rl = O.maxwell_coexistence(a, b, R, om, 0.86 * Tc)
    rho_full = inputs.bubble_density(L, L, rl, rv, n_bubbles=256, r_min=20.0, r_max=60.0, seed=4)
    rho0 = torch.tensor(rho_full[:rows], dtype=torch.float64)
    P = O.Params(Lx=L, Ly=rows, a=a, b=b, R=R, omega=om)
    P.finalize(rho0=rho0, superheat=0.1 * Tc, rho_v=rv, rho_l=rl)
    P.rho_ave = float(np.asarray(rho_full, np.float64).mean())
    f, th = O.initial_state(rho0, P)
    return P, f, th


def cpu_baseline(seconds: float = 12.0, rows: int = CPU_BAND_ROWS):
    """The FP64 oracle on a band of `rows` rows (full 4096 width, the bottom
    wall band) of the workload, for about `seconds` of CPU time."""
    import torch
    import oracle as O
    from paper_1501_03857_gb300 import inputs
    cores = os.cpu_count() or 1
    torch.set_num_threads(cores)
    a, b, R, om = 3 / 49, 2 / 21, 1.0, 0.344
    P, f, th = oracle_band(rows)
    f, th, _ = O.step(f, th, P)  # warm-up
    n, t0 = 0, time.perf_counter()
    while True:
        f, th, _ = O.step(f, th, P)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds and n >= 2:
            break
    mlups = n * L * rows / el / 1e6
    threads = torch.get_num_threads()

    def timed(fn, budget):
        k, t0 = 0, time.perf_counter()
        while True:
            fn()
            k += 1
            dt = time.perf_counter() - t0
            if dt > budget and k >= 2:
                return k, dt

    # the same band on one thread
    torch.set_num_threads(1)
    state = [f, th]

    def one():
        state[0], state[1], _ = O.step(state[0], state[1], P)

    k1, t1 = timed(one, 3.0)
    # the small 100 x 100 configuration (a = 2/49, pool to y = 40), all cores
    torch.set_num_threads(threads)
    a2 = 2 / 49
    Tc2 = O.critical_temperature(a2, b, R)
    rv2, rl2 = O.maxwell_coexistence(a2, b, R, om, 0.86 * Tc2)
    r2 = torch.tensor(inputs.pool_density(100, 100, rl2, rv2, 40.0, seed=1), dtype=torch.float64)
    P2 = O.Params(Lx=100, Ly=100, a=a2, b=b, R=R, omega=om)
    P2.finalize(rho0=r2, superheat=0.1 * Tc2, rho_v=rv2, rho_l=rl2)
    st2 = list(O.initial_state(r2, P2))

    def small():
        st2[0], st2[1], _ = O.step(st2[0], st2[1], P2)

    k2, t2 = timed(small, 3.0)
    return {"value": mlups, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"FP64 oracle (PyTorch CPU), {n} steps of a {L}x{rows} bottom band of the workload, "
                      f"{el:.1f} s",
            "single_thread": {"value": k1 * L * rows / t1 / 1e6, "unit": "MLUPS", "cores": 1,
                              "sample": f"{k1} steps of the same band, {t1:.1f} s"},
            "config_100x100": {"value": k2 * 100 * 100 / t2 / 1e6, "unit": "MLUPS", "cores": threads,
                               "sample": f"{k2} steps of the 100 x 100 pool (a = 2/49), {t2:.1f} s"}}


# The batched curve's surfaces, by static contact angle; their G_w come from
# the sessile-droplet calibration run by wettability_calibration.
CURVE_ANGLES = (40.0, 60.0, 90.0, 120.0, 150.0)  # static contact angles of the curve's surfaces, deg
CURVE_STEPS = 50000  # steps of one boiling-curve simulation
CAL_LADDER = tuple(round(-0.125 + 0.025 * k, 3) for k in range(22))  # G_w -0.125 .. 0.4


def wettability_calibration(torch, lb):
    """Static contact angle vs G_w (Eq. 22) from sessile droplets relaxed at
    T_s on a 240 x 120 domain (all ladder points in one batched run of 20000
    steps), and the G_w of each of the curve's contact angles."""
    from paper_1501_03857_gb300 import wetting
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    st = torch.cuda.current_stream()
    ev[0].record(st)
    r = wetting.run_droplets(CAL_LADDER, wetting.droplet_config(240, 120), radius=40.0, steps=20000,
                             checkpoints=[10000], stream=st)
    ev[1].record(st)
    torch.cuda.synchronize()
    gw, an = list(r["Gw"]), list(r["angle_deg"])
    # the monotone part of the table (a droplet near detachment reads noisily)
    n = 1
    while n < len(an) and an[n] > an[n - 1] and an[n - 1] < 170.0:
        n += 1
    targets = wetting.gw_for_angle(CURVE_ANGLES, gw[:n], an[:n])
    drift = max(abs(a - b) for a, b in zip(r["history"][10000][:n], an[:n]))
    return {"grid": "240x120", "radius0": 40.0, "steps": 20000, "Gw": gw, "angle_deg": [round(a, 3) for a in an],
            "max_change_10k_to_20k_deg": drift, "curve_angles_deg": list(CURVE_ANGLES),
            "curve_Gw": [float(g) for g in targets], "ms": ev[0].elapsed_time(ev[1])}


def batched_curve(torch, lb, gw_of_angle, steps_batch=64, steps_seq=32, dist=None):
    """48 boiling-curve instances (uneven 200-400 x 200-600 domains, superheat
    0.02-0.4 Tc, contact angles 40-150 deg through the calibrated G_w of
    gw_of_angle) in one launch per step vs. the same instances stepped one
    after another through the plain path. With N ranks (dist) the instances
    are dealt out to the ranks (replicas.shard): each rank times its share,
    and the job's times are the slowest rank's."""
    from paper_1501_03857_gb300 import inputs, replicas, tune
    rank, world = (dist.get_rank(), dist.get_world_size()) if dist is not None else (0, 1)
    pts = replicas.shard(list(enumerate(inputs.boiling_curve_batch(48, seed=3))), rank, world)
    n_all = 48
    insts = []
    for i, d in pts:
        cfg = lb.Config(Lx=d["Lx"], Ly=d["Ly"], bc_y=lb.BC_WALLS, pool_height=0.4 * d["Ly"], seed=100 + i)
        Tc = lb.critical_temperature(cfg)
        insts.append({"cfg": cfg, "superheat": d["superheat_frac"] * Tc, "Gw": gw_of_angle[d["wet_index"]]})
    cells = sum(d["cfg"].Lx * d["cfg"].Ly for d in insts)
    st = torch.cuda.current_stream()
    batch = lb.Batch(insts, stream=st)
    # every candidate launch (one launch per step, and the persistent launch
    # with 1-4 tiles per block) timed; the fastest is the batched figure
    cands = tune.time_batch_candidates(batch)
    best_step = min((v, k) for k, v in cands.items() if k[2] == 0)
    best_pers = min(((v, k) for k, v in cands.items() if k[2] > 0), default=None)
    bx, seg, _, tpb = tune.tune_batch(batch)
    batch.step(GRAPH_WARM)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(st)
    batch.step(steps_batch)
    ev[1].record(st)
    torch.cuda.synchronize()
    t_b = ev[0].elapsed_time(ev[1]) / steps_batch
    batch.sync()
    info = batch.info()
    batch.close()
    t_seq = 0.0
    for d in insts:
        sim = lb.Simulation(d["cfg"], superheat=d["superheat"], Gw=d["Gw"], stream=st)
        sim.step(3)
        torch.cuda.synchronize()
        ev[0].record(st)
        sim.step(steps_seq)
        ev[1].record(st)
        torch.cuda.synchronize()
        t_seq += ev[0].elapsed_time(ev[1]) / steps_seq
        sim.close()
    t_b = replicas.max_over_ranks(t_b, dist, device="cuda")
    t_seq = replicas.max_over_ranks(t_seq, dist, device="cuda")
    cells = int(round(replicas.max_over_ranks(cells, dist, device="cuda")))  # the largest share
    sph = lambda t: n_all * 3600.0 / (CURVE_STEPS * t * 1e-3)
    return {"instances": n_all, "ranks": world, "instances_per_rank_max": len(insts),
            "cells_largest_share": cells, "steps_per_sim": CURVE_STEPS,
            "ms_per_step_batched": t_b, "ms_per_step_sequential": t_seq,
            "sims_per_hour_batched": sph(t_b), "sims_per_hour_sequential": sph(t_seq),
            "speedup": t_seq / t_b, "mlups_batched": cells / (t_b * 1e3) * world,
            "launch": {"block_x": bx, "seg_rows": seg, "tiles_per_block": tpb, "blocks": info["blocks"],
                       "mode": ("persistent: one cooperative launch per 32 steps" if tpb
                                else "one launch per step") + ", replayed from captured graphs"},
            "tuner_ms_per_step": {"per_step_launch": {"ms": best_step[0], "block_x": best_step[1][0],
                                                      "seg_rows": best_step[1][1]},
                                  "persistent": None if best_pers is None else
                                  {"ms": best_pers[0], "block_x": best_pers[1][0], "tiles_per_block": best_pers[1][2]}}}


GRAPH_WARM = 32


def adjoint_window(torch, lb, L=256, nsteps=2000, ckpt=100):
    """Gradient of the mean wall heat flux over a 2000-step window of a 256 x 256
    boiling domain w.r.t. the 256-cell wall temperature profile and G_w
    (checkpoint every 100 steps): cost against the forward steps alone, and a
    check against central differences of the same FP32 forward (uniform T_b
    mode and G_w, h = 1e-4). The timed adjoint call follows an untimed one, so
    graph capture and scratch allocation are not in it."""
    from paper_1501_03857_gb300 import inputs
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_WALLS, pool_height=0.4 * L, seed=5)
    Tc = lb.critical_temperature(cfg)
    sh, Gw = 0.1 * Tc, 0.065
    rv, rl = lb.coexistence(cfg)
    rho0 = inputs.pool_density(L, L, rl, rv, 0.4 * L, noise_amp=1e-4, seed=5)
    st = torch.cuda.current_stream()
    sim = lb.Simulation(cfg, superheat=sh, Gw=Gw, rho0=rho0, stream=st)
    sim.step(200)  # leave the initial transient
    blob = sim.save()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def forward_J(dtb=0.0, dgw=0.0):
        sim.load(blob)
        sim.set_wall_temperature(sh + dtb)
        sim.set_wettability(Gw + dgw)
        sim.heat_flux(reset=True)
        sim.step(nsteps)
        return sim.heat_flux()["q_mean"]

    forward_J()  # warm-up
    sim.load(blob)
    sim.set_wall_temperature(sh)
    sim.set_wettability(Gw)
    torch.cuda.synchronize()
    ev[0].record(st)
    sim.step(nsteps)
    ev[1].record(st)
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1])
    sim.load(blob)
    sim.adjoint(nsteps, ckpt)  # warm-up: captures the segment graphs
    sim.load(blob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, dTb, dGw = sim.adjoint(nsteps, ckpt)
    t_adj = (time.perf_counter() - t0) * 1e3
    # the same window with every step stored (checkpoint every step: no
    # replay, about 20 planes of scratch per step), timed the same way
    sim.load(blob)
    sim.adjoint(nsteps, 1)
    sim.load(blob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J1, dTb1, dGw1 = sim.adjoint(nsteps, 1)
    t_all = (time.perf_counter() - t0) * 1e3
    store_all = {"ckpt_every": 1, "ms_adjoint_total": t_all, "cost_ratio": t_all / t_fwd,
                 "scratch_gb": sim.adjoint_scratch_bytes(nsteps, 1) / 1e9,
                 "same_gradients": bool(J1 == J and np.array_equal(dTb1, dTb) and dGw1 == dGw)}
    default_ckpt = sim.adjoint_ckpt(nsteps)  # the interval sim.adjoint(nsteps) picks here
    h = 1e-4
    fd_tb = (forward_J(dtb=h) - forward_J(dtb=-h)) / (2 * h)
    fd_gw = (forward_J(dgw=h) - forward_J(dgw=-h)) / (2 * h)
    sim.close()
    # the FP64 reference gradients of this window (tests/golden, written from
    # the oracle by central differences with Richardson extrapolation)
    ref = {}
    gp = os.path.join(ROOT, "tests", "golden", "adjoint_256_gradients.txt")
    if L == 256 and nsteps == 2000 and os.path.exists(gp):
        for line in open(gp):
            p = line.split("#")[0].split()
            if len(p) == 2:
                ref[p[0]] = float(p[1])
    fp64 = None
    if ref:
        fp64 = {"J": ref["J"], "dJ_dGw": ref["dGw"], "dJ_dTb_uniform": ref["dTb_uniform"],
                "rel_err_J": abs(J / ref["J"] - 1), "rel_err_Gw": abs(dGw / ref["dGw"] - 1),
                "rel_err_uniform": abs(float(dTb.sum()) / ref["dTb_uniform"] - 1),
                "what": "FP64 oracle central differences, h = 2e-4 and 1e-4, Richardson-extrapolated"}
    return {"grid": f"{L}x{L}", "steps": nsteps, "ckpt_every": ckpt, "default_ckpt_every": default_ckpt,
            "J": J, "vs_fp64_reference": fp64,
            "ms_forward": t_fwd, "ms_adjoint_total": t_adj, "cost_ratio": t_adj / t_fwd,
            "store_every_step": store_all,
            "mlups_adjoint": L * L * nsteps / (t_adj * 1e-3) / 1e6,
            "mlups_forward": L * L * nsteps / (t_fwd * 1e-3) / 1e6,
            "dJ_dTb_uniform": float(dTb.sum()), "fd_uniform": fd_tb,
            "rel_err_uniform": abs(float(dTb.sum()) - fd_tb) / abs(fd_tb),
            "dJ_dGw": dGw, "fd_Gw": fd_gw, "rel_err_Gw": abs(dGw - fd_gw) / abs(fd_gw),
            "fd": "central differences of the FP32 GPU forward, h = 1e-4"}


CURVE_SUPERHEATS = (0.008, 0.01, 0.0137, 0.0165, 0.019, 0.021, 0.023, 0.025, 0.027, 0.029, 0.032, 0.035)
CURVE_SEEDS = (1, 2, 3)  # seeds of the pool's initial noise averaged per case


def paper_experiments(torch, dist=None):
    """The boiling curves of Sec. 3.2-3.3 on the paper's 600 x 150 pool (12
    superheats x G_w 0, 0.065, 0.105 x 3 seeds of the initial noise in one
    batch; 20000 steps at the base superheat, switch, 5000 settling, 15000
    averaged; case statistics are seed-ensemble means) and Fig. 3's top-wall
    pressure; compact summary and wall time. With N ranks (dist) the curve's
    runs are dealt out to the ranks and gathered back."""
    from paper_1501_03857_gb300 import experiments as E, replicas
    t0 = time.perf_counter()
    r = E.boiling_curve(CURVE_SUPERHEATS, Gw_values=(0.0, 0.065, 0.105), seeds=CURVE_SEEDS, dist=dist)
    t_curve = replicas.max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
    curves = {}
    for gw, c in r["curves"].items():
        grp = [x for x in r["cases"] if x["Gw"] == gw]
        curves[str(gw)] = dict(c, superheats=[x["superheat"] for x in grp], q_mean=[x["q_mean"] for x in grp],
                               q_sem=[x["q_sem"] for x in grp], regimes=[x["regime"] for x in grp])
    t0 = time.perf_counter()
    tp = E.top_wall_pressure((0.0137, 0.0165))
    t_top = time.perf_counter() - t0
    steps = r["t_switch"] + r["t_settle"] + r["t_avg"]
    sims = len(r["cases"]) * len(r["seeds"])
    return {"grid": "600x150", "cases": len(r["cases"]), "seeds": r["seeds"], "simulations": sims, "ranks": r["ranks"],
            "steps_per_case": steps, "s_curves": t_curve, "sims_per_hour": sims * 3600.0 / t_curve, "curves": curves,
            "top_wall_pressure": {str(k): v["p_top"] for k, v in tp["cases"].items()}, "s_top_wall_pressure": t_top}


# Algorithmic bytes per lattice update of one reverse step: the stored state
# (9 populations + theta) read once and the adjoint state read and written
# once, plus the forward recomputation of the step from its checkpoint.
ADJ_BYTES_PER_LU = 40 + 80 + 80


def adjoint_roofline(torch, lb, L=2048, nsteps=16, ckpt=8):
    """The adjoint on a domain larger than L2 (2048 x 2048: 168 MB per state):
    reverse-sweep time per step = (adjoint call - forward steps) / nsteps, and
    its HBM roofline at ADJ_BYTES_PER_LU."""
    cfg = lb.Config(Lx=L, Ly=L, bc_y=lb.BC_WALLS, pool_height=0.4 * L, seed=5)
    Tc = lb.critical_temperature(cfg)
    st = torch.cuda.current_stream()
    sim = lb.Simulation(cfg, superheat=0.1 * Tc, Gw=0.065, stream=st)
    sim.step(20)
    blob = sim.save()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sim.step(nsteps)
    sim.load(blob)
    torch.cuda.synchronize()
    ev[0].record(st)
    sim.step(nsteps)
    ev[1].record(st)
    torch.cuda.synchronize()
    t_fwd = ev[0].elapsed_time(ev[1])
    sim.load(blob)
    sim.adjoint(nsteps, ckpt)  # warm-up: graph capture, scratch
    sim.load(blob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.adjoint(nsteps, ckpt)
    t_adj = (time.perf_counter() - t0) * 1e3
    # every step stored (checkpoint every step: no replay)
    sim.load(blob)
    sim.adjoint(nsteps, 1)
    sim.load(blob)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.adjoint(nsteps, 1)
    t_all = (time.perf_counter() - t0) * 1e3
    scratch_all = sim.adjoint_scratch_bytes(nsteps, 1)
    default_ckpt = sim.adjoint_ckpt(nsteps)  # the interval sim.adjoint(nsteps) picks here
    sim.close()
    cells = L * L
    rev_ms = (t_adj - t_fwd) / nsteps
    rev_all = (t_all - t_fwd) / nsteps
    peak, _ = measured_peaks()
    achieved = ADJ_BYTES_PER_LU * cells / (rev_ms * 1e-3) / 1e9
    return {"grid": f"{L}x{L}", "steps": nsteps, "ckpt_every": ckpt, "default_ckpt_every": default_ckpt,
            "ms_forward_per_step": t_fwd / nsteps,
            "ms_reverse_per_step": rev_ms, "mlups_reverse": cells / (rev_ms * 1e-3) / 1e6,
            "mlups_adjoint": cells * nsteps / (t_adj * 1e-3) / 1e6,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_lu": ADJ_BYTES_PER_LU,
                         "what": "reverse sweep incl. forward recomputation, per step"},
            "store_every_step": {"ckpt_every": 1, "ms_reverse_per_step": rev_all,
                                 "cost_ratio": 1 + rev_all / (t_fwd / nsteps), "scratch_gb": scratch_all / 1e9,
                                 "roofline_frac": ADJ_BYTES_PER_LU * cells / (rev_all * 1e-3) / 1e9 / peak}}


def paper_context(experiments=None):
    """What the paper gives about its own runs, beside this run's figures on
    the same grid: its grid and step counts (Sec. 3.1-3.3); it reports no
    runtime, hardware, precision or throughput."""
    ctx = {"grid": "600x150 (Sec. 3.1), periodic x, walls in y",
           "steps": "superheat switched at 20 000 steps; runs of 10 000-50 000 steps, film boiling to 140 000 "
                    "(Sec. 3.2-3.3)",
           "timing": "not reported: the paper gives no runtime, hardware, precision or MLUPS"}
    if experiments:
        sims, steps, s = experiments["simulations"], experiments["steps_per_case"], experiments["s_curves"]
        ctx["here_on_that_grid"] = {"simulations": sims, "steps_each": steps, "seconds": s,
                                    "glups": sims * steps * 600 * 150 / s / 1e9,
                                    "what": "the boiling-curve runs of the experiments block, batched on one GPU"}
    return ctx


def summary(line):
    """The key figures of the line's blocks, compact."""
    r = {"mlups": round(line["value"]), "hbm_frac": round(line["roofline"]["frac"], 4),
         "e2e_mlups": round(line["e2e"]["value"])}
    b = line.get("batched")
    if b:
        r["batched"] = {"speedup_vs_sequential": round(b["speedup"], 2), "ms_per_step": round(b["ms_per_step_batched"], 4),
                        "sims_per_hour": round(b["sims_per_hour_batched"]), "mode": b["launch"]["mode"].split(":")[0],
                        "hbm_frac": round(b["mlups_batched"] * 80e6 / 1e9 / line["roofline"]["peak"], 3)}
    a = line.get("adjoint")
    if a:
        r["adjoint"] = {"cost_vs_forward_256": round(a["cost_ratio"], 2), "rel_err_Gw_vs_fd32": round(a["rel_err_Gw"], 6)}
        if a.get("vs_fp64_reference"):
            f = a["vs_fp64_reference"]
            r["adjoint"].update(rel_err_Gw_vs_fp64=float("%.2e" % f["rel_err_Gw"]),
                                rel_err_Tb_vs_fp64=float("%.2e" % f["rel_err_uniform"]))
        if a.get("large"):
            g = a["large"]
            r["adjoint"].update(reverse_ms_2048=round(g["ms_reverse_per_step"], 4), reverse_hbm_frac_2048=round(g["roofline"]["frac"], 3),
                                cost_vs_forward_2048=round(1 + g["ms_reverse_per_step"] / g["ms_forward_per_step"], 2))
            if g.get("store_every_step"):
                r["adjoint"]["cost_vs_forward_2048_every_step_stored"] = round(g["store_every_step"]["cost_ratio"], 2)
            r["adjoint"]["default_ckpt_2048"] = g.get("default_ckpt_every")
        if a.get("store_every_step"):
            r["adjoint"]["cost_vs_forward_256_every_step_stored"] = round(a["store_every_step"]["cost_ratio"], 2)
        r["adjoint"]["default_ckpt_256"] = a.get("default_ckpt_every")
    e = line.get("experiments")
    if e:
        r["experiments"] = {"sims_per_hour": round(e["sims_per_hour"]),
                            "chf_superheat": {k: v["chf_superheat"] for k, v in e["curves"].items()}}
    c = line.get("cpu_baseline")
    if c:
        r["oracle_mlups"] = round(c["value"], 2)
    return r


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import torch
    import oracle as O
    from paper_1501_03857_gb300 import inputs
    cores = os.cpu_count() or 1
    torch.set_num_threads(cores)
    rows = CPU_BAND_ROWS
    P, f, th = oracle_band(rows)
    for _ in range(args.warmup):
        f, th, _ = O.step(f, th, P)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, th, _ = O.step(f, th, P)
    el = time.perf_counter() - t0
    value = args.steps * L * rows / el / 1e6
    sample = f"FP64 oracle (PyTorch CPU), each step a {L}x{rows} bottom band of the workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample_rows=rows),
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_1501_03857_gb300 import replicas
    rank, world, local = replicas.rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1501_03857_gb300 import lb

    cfg = workload_config()
    rv, rl = lb.coexistence(cfg)
    Tc = lb.critical_temperature(cfg)
    rho0 = workload_rho0(cfg, rv, rl)
    stream = torch.cuda.current_stream()
    sim = lb.Simulation(cfg, superheat=0.1 * Tc, Gw=0.0, rho0=rho0, stream=stream)
    cells = cfg.Lx * cfg.Ly
    WORKLOAD["state_bytes"] = 2 * 10 * cells * 4

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---- device-timed region: K steps, one fused kernel launch each, issued
    # as one lb_step(K) call the way a run is stepped (runs of 32 steps are
    # replayed from a captured graph on the library's private stream, which
    # is event-ordered after and before `stream`, so the events below
    # bracket every launch)
    sim.step(args.warmup)
    barrier()
    clk = ClockSampler(local) if rank == 0 else None
    barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    h0 = time.time()
    t_start.record(stream)
    sim.step(args.steps)
    t_end.record(stream)
    barrier()
    h1 = time.time()
    clocks = clk.stop(h0, h1) if clk else None
    total_ms = t_start.elapsed_time(t_end)
    sim.sync()
    # replicas: every rank ran its own domain; the job took the slowest rank's time
    ms_all = replicas.max_over_ranks(total_ms, dist, device="cuda")
    value = replicas.job_throughput(world, cells * args.steps, ms_all) / 1e6

    # ---- end-to-end through the public API with host buffers
    prof = np.zeros(cfg.Lx, dtype=np.float64)
    try:
        prof_t = torch.from_numpy(prof).pin_memory()
        prof = prof_t.numpy()
    except RuntimeError:
        pass
    e2e_steps = max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_wall_temperature(0.1 * Tc, prof)
        sim.step(1)
        sim.heat_flux()
    barrier()
    e2e_s = replicas.max_over_ranks(time.perf_counter() - t0, dist, device="cuda")
    e2e = {"value": replicas.job_throughput(world, cells * e2e_steps, e2e_s * 1e3) / 1e6, "unit": "MLUPS",
           # per step: the wall profile (Lx FP32) up, the 72-byte accumulator record down
           "h2d_bytes_per_step": cfg.Lx * 4, "d2h_bytes_per_step": 72, "steps": e2e_steps,
           "api": "lb_set_wall_temperature + lb_step(1) + lb_heat_flux per step"}

    if rank == 0:
        peak, src = measured_peaks()
        avg_ms = total_ms / args.steps  # average launch duration over the timed region (launches back to back)
        achieved = BYTES_PER_LU * cells / (avg_ms * 1e-3) / 1e9
        traffic = None
        tp = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tp):
            # DRAM bytes per launch from the committed ncu capture, only while
            # the kernel source is the one that was profiled
            import hashlib
            rec = json.load(open(tp))
            ksrc = os.path.join(ROOT, "paper_1501_03857_gb300", "csrc", "lb_step3.cu")
            sha = hashlib.sha256(open(ksrc, "rb").read()).hexdigest()[:16]
            if rec.get("source_sha256_16") == sha:
                traffic = rec.get("lb_step_dual")
        info = sim.info()
        line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_all / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(WORKLOAD, parallelism=f"replicas{world}", launch=info),
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "traffic": traffic, "peak_source": src,
                             "kernel": "lb_step_dual (paired-FP32 dual-strip fused step)", "bytes_per_lu": BYTES_PER_LU,
                             "avg_kernel_ms": avg_ms},
                "e2e": e2e, "gpu_launches": args.steps, "clocks": clocks}
    # the boiling-curve blocks on every rank: their instances are dealt out
    # to the ranks (the natural replica unit) and gathered back on rank 0
    extras = {}
    if not args.no_batched:
        cal = wettability_calibration(torch, lb)
        extras["batched"] = batched_curve(torch, lb, cal["curve_Gw"], dist=dist)
        extras["batched"]["wettability"] = cal
    if not args.no_experiments:
        extras["experiments"] = paper_experiments(torch, dist)
    if rank == 0:
        line.update(extras)
        if not args.no_adjoint:
            line["adjoint"] = adjoint_window(torch, lb)
            line["adjoint"]["large"] = adjoint_roofline(torch, lb)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        line["paper_context"] = paper_context(line.get("experiments"))
        line["summary"] = summary(line)  # last, so that the end of the line carries the key figures
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched boiling-curve measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-experiments", action="store_true", help="skip the boiling-curve experiments")
    ap.add_argument("--size", type=int, default=4096, help="domain edge (profiling of smaller cases)")
    ap.add_argument("--adjoint-only", type=str, default=None, metavar="L,STEPS,CKPT",
                    help="only the large-domain adjoint measurement, e.g. 2048,8,4 (profiling)")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched 48-instance step with G_w = 0 everywhere (profiling)")
    args = ap.parse_args()
    if args.batched_only:
        import torch
        from paper_1501_03857_gb300 import lb
        print(json.dumps({"batched": batched_curve(torch, lb, [0.0] * len(CURVE_ANGLES))}), flush=True)
        return
    if args.adjoint_only:
        import torch
        from paper_1501_03857_gb300 import lb
        Ls, ns, ck = (int(v) for v in args.adjoint_only.split(","))
        print(json.dumps({"adjoint_large": adjoint_roofline(torch, lb, Ls, ns, ck)}), flush=True)
        return
    global L
    L = args.size
    WORKLOAD["Lx"] = WORKLOAD["Ly"] = L
    if L != 4096:
        WORKLOAD["workload"] = WORKLOAD["workload"].replace("4096x4096", f"{L}x{L}")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
