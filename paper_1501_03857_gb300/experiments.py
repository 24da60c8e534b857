"""The paper's boiling experiments (Sec. 3.2-3.3) on the library's step.

* top_wall_pressure: Fig. 3's protocol. A pool is heated at Delta T = 0.0137
  for 20000 steps, then the wall superheat is set to each case's value; a
  device probe records the pressure at the centre of the top wall every step.
* boiling_curve: Figs. 6-8 and 13. Every (Delta T, G_w) case is one instance
  of one batched launch per step. Cases above the base superheat start from
  the pool at the base superheat and switch at t_switch (Sec. 3.2 raises the
  superheat of its higher cases at t = 20000); cases at or below it run at
  their own superheat from t = 0 (no boiling can be inherited from the base
  run). After t_switch + t_settle the heat flux q(t) (the mean over x of
  q_w of Sec. 3.2) is averaged over t_avg steps: q_bar, its standard
  deviation, and h_c = q_bar / Delta T. The heated wall's vapour coverage
  (the fraction of the first fluid row below the mid density) and the
  number of vapour bubbles in the pool are sampled every sample_every steps.
  Boiling is chaotic: near the top of a curve neighbouring superheats differ
  by less than the run-to-run spread of one window's mean, so the location
  of the maximum moves with any rounding-level change. With several seeds
  (the initial density noise of the pool) every case runs once per seed in
  the same batch and the case statistics are ensemble averages over them.
* classify_curve: the regime of every case of a curve, after Sec. 3.2: no
  boiling forms no vapour at the heated wall and no bubbles; film boiling
  keeps the whole heating surface under a continuous vapour film; the
  remaining (boiling) cases are nucleate up to the largest heat flux
  attainable in nucleate boiling and transition beyond it, where vapour
  patches insulate the liquid and q no longer rises with the superheat
  (Sec. 1 defines transition boiling as lying between the maximum of
  nucleate boiling and the minimum of film boiling). With seed ensembles
  that limit is the lowest superheat no higher case exceeds by more than
  two combined standard errors of the means (nucleate_limit); for single
  runs it is the superheat of the largest mean flux. An ensemble case is
  film (no) boiling when most of its runs are.

Superheats are in lattice units (Delta T = T_b - T_s), as in the paper.
"""

from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import diagnostics, lb, tune

FILM_COVERAGE = 0.95  # wall coverage in every sample: a continuous vapour film


def paper_config(**kw) -> lb.Config:
    """The 600 x 150 pool of Sec. 3.1 (walls in y, liquid below y = 90, the
    paper's EOS and transport parameters)."""
    return replace(lb.Config(), **kw)


def top_wall_pressure(superheats=(0.0137, 0.0165), cfg: lb.Config | None = None, base_superheat: float = 0.0137,
                      t_switch: int = 20000, t_after: int = 20000, window: int = 2000, stream=None) -> dict:
    """Fig. 3: pressure at the centre of the top wall after the switch from
    the base superheat, as means over consecutive windows of `window` steps,
    for each superheat; also the mean wall heat flux after the switch."""
    cfg = cfg or paper_config()
    sim = lb.Simulation(cfg, superheat=base_superheat, stream=stream)
    try:
        sim.step(t_switch)
        blob = sim.save()
        out = {}
        for dT in superheats:
            sim.load(blob)
            sim.set_probes([(cfg.Lx // 2, cfg.Ly - 1)], capacity=t_after)
            sim.set_wall_temperature(dT)
            sim.heat_flux(reset=True)
            sim.step(t_after)
            p = sim.probe_read()["p"][0]
            nwin = len(p) // window
            out[float(dT)] = {"p_top": [float(p[i * window:(i + 1) * window].mean()) for i in range(nwin)],
                              "q_mean": sim.heat_flux()["q_mean"]}
        sim.set_probes([])
    finally:
        sim.close()
    return {"t_switch": t_switch, "window": window, "point": [cfg.Lx // 2, cfg.Ly - 1], "cases": out}


def wall_coverage(rho: np.ndarray, rho_l: float, rho_v: float, row: int = 1) -> float:
    """Fraction of the heated wall's first fluid row that is vapour."""
    return float(np.mean(np.asarray(rho)[row] < 0.5 * (rho_l + rho_v)))


def nucleate_limit(cases) -> float:
    """Superheat of the largest heat flux attainable in nucleate boiling for
    the boiling cases of one curve (dicts with superheat, q_mean and
    optionally q_sem): the lowest superheat whose mean flux no higher case
    exceeds by more than twice the combined standard error (q_sem missing or
    NaN counts as 0, which gives the superheat of the largest mean)."""
    cs = sorted(cases, key=lambda c: c["superheat"])

    def sem(c):
        v = c.get("q_sem", 0.0)
        return 0.0 if v != v else float(v)

    for i, c in enumerate(cs):
        if all(d["q_mean"] <= c["q_mean"] + 2.0 * np.hypot(sem(c), sem(d)) for d in cs[i + 1:]):
            return c["superheat"]
    raise ValueError("no boiling cases")


def classify_curve(cases) -> list:
    """Regime of each case dict (superheat, Gw, q_mean, optionally q_sem,
    coverage_min, coverage_max, bubbles_max) of one or more curves; cases
    are grouped by G_w and the boiling, non-film cases of a group are
    nucleate up to its nucleate_limit and transition beyond it. A seed
    ensemble (film_fraction, none_fraction present) is film or no boiling
    when most of its runs are."""
    labels = []
    for c in cases:
        if "film_fraction" in c:
            film, none = c["film_fraction"] > 0.5, c["none_fraction"] > 0.5
        else:
            film = c["coverage_min"] >= FILM_COVERAGE
            none = c["coverage_max"] == 0.0 and c["bubbles_max"] == 0
        labels.append("film" if film else "none" if none else "boiling")
    limit = {}
    for gw in set(c["Gw"] for c, lab in zip(cases, labels) if lab == "boiling"):
        limit[gw] = nucleate_limit([c for c, lab in zip(cases, labels) if lab == "boiling" and c["Gw"] == gw])
    return [("nucleate" if c["superheat"] <= limit[c["Gw"]] else "transition") if lab == "boiling" else lab
            for c, lab in zip(cases, labels)]


def ensemble(runs: list) -> dict:
    """One case's statistics over the runs of its seeds (dicts with q_mean,
    q_std and the sampled coverage and bubble series): mean flux and its
    standard error over the seeds, mean within-window deviation, coverage
    mean / min / max and bubble count mean / max over every sample of every
    run, and the fractions of runs that kept a film on the wall in every
    sample or formed no vapour at all (film_fraction, none_fraction)."""
    qm = np.array([r["q_mean"] for r in runs], dtype=np.float64)
    cov = np.concatenate([np.asarray(r["coverage"], dtype=np.float64) for r in runs])
    nb = np.concatenate([np.asarray(r["bubbles"]) for r in runs])
    sem = float(qm.std(ddof=1) / np.sqrt(len(qm))) if len(qm) > 1 else float("nan")
    film = [min(r["coverage"]) >= FILM_COVERAGE for r in runs]
    none = [max(r["coverage"]) == 0.0 and max(r["bubbles"]) == 0 for r in runs]
    return {"q_mean": float(qm.mean()), "q_sem": sem, "q_runs": [float(q) for q in qm],
            "q_std": float(np.mean([r["q_std"] for r in runs])),
            "coverage_mean": float(cov.mean()), "coverage_min": float(cov.min()), "coverage_max": float(cov.max()),
            "bubbles_mean": float(nb.mean()), "bubbles_max": int(nb.max()),
            "film_fraction": float(np.mean(film)), "none_fraction": float(np.mean(none))}


def run_cases(runs, cfg: lb.Config, rho_v: float, rho_l: float, base_superheat: float, t_switch: int,
              t_settle: int, t_avg: int, sample_every: int, stream=None) -> list:
    """Run the ((Delta T, G_w), seed) pairs `runs` as the instances of one
    batch (the protocol of boiling_curve) and return, per run, q_mean, q_std
    and the sampled wall coverage and bubble counts."""
    insts = [{"cfg": replace(cfg, seed=sd), "Gw": gw, "superheat": (base_superheat if dT > base_superheat else dT)}
             for (dT, gw), sd in runs]
    batch = lb.Batch(insts, stream=stream)
    tune.tune_batch(batch)  # launch form and shape; the states are restored
    batch.heat_flux(reset=True)
    cov = [[] for _ in runs]
    nbub = [[] for _ in runs]
    try:
        batch.step(t_switch)
        for i, ((dT, gw), _) in enumerate(runs):
            if dT > base_superheat:
                batch.set_wall_temperature(i, dT)
        batch.step(t_settle)
        batch.heat_flux(reset=True)

        def sample(fields):
            for i, rho in enumerate(fields):
                cov[i].append(wall_coverage(rho, rho_l, rho_v))
                nbub[i].append(diagnostics.bubble_count(rho, rho_l, rho_v))

        # every sample_every steps the density fields come back to the host;
        # they are measured while the GPU runs the next steps
        done, pending = 0, None
        while done < t_avg:
            n = min(sample_every, t_avg - done)
            batch.step(n)
            done += n
            if pending is not None:
                sample(pending)
            pending = [batch.fields(i, ("rho",))["rho"] for i in range(len(runs))]
        if pending is not None:
            sample(pending)
        hf = batch.heat_flux()
    finally:
        batch.close()
    return [{"q_mean": float(hf["q_mean"][i]), "q_std": float(hf["q_std"][i]), "coverage": cov[i],
             "bubbles": nbub[i]} for i in range(len(runs))]


def boiling_curve(superheats, Gw_values=(0.0,), cfg: lb.Config | None = None, base_superheat: float = 0.0137,
                  t_switch: int = 20000, t_settle: int = 5000, t_avg: int = 15000, sample_every: int = 500,
                  seeds=None, stream=None, dist=None, runner=None) -> dict:
    """The boiling curve(s) for every (Delta T, G_w) pair in one batch;
    returns per case q_bar, q_std, h_c, the wall coverage (mean, min, max),
    the bubble count (mean, max) and the regime, and per G_w the superheat
    and value of the largest mean heat flux (chf), the nucleate_limit
    superheat and the superheat and value of the largest h_c. `seeds`
    (default: cfg.seed alone) runs every case once per seed of the pool's
    initial noise; the case statistics are then ensemble averages (see
    `ensemble`), with q_sem the standard error of q_bar over the seeds.

    With `dist` (torch.distributed with an initialised group of N ranks,
    one GPU each) the runs are dealt out to the ranks (replicas.shard), each
    rank steps its share as one batch, and the per-run results are gathered
    back in order on every rank (replicas.gather_shards), so every rank
    returns the whole curve. `runner` replaces run_cases (same arguments)."""
    from . import replicas
    cfg = cfg or paper_config()
    seeds = [cfg.seed] if seeds is None else [int(s) for s in seeds]
    rv, rl = lb.coexistence(cfg)
    cases = [(float(dT), float(gw)) for gw in Gw_values for dT in superheats]
    runs = [(c, sd) for c in cases for sd in seeds]
    rank, world = 0, 1
    if dist is not None and dist.is_initialized():
        rank, world = dist.get_rank(), dist.get_world_size()
    mine = replicas.shard(runs, rank, world)
    runner = runner or run_cases
    res = runner(mine, cfg, rv, rl, base_superheat, t_switch, t_settle, t_avg, sample_every, stream) if mine else []
    res = replicas.gather_shards(res, rank, world, dist)
    out = []
    for k, (dT, gw) in enumerate(cases):
        idx = [i for i, (c, _) in enumerate(runs) if c == (dT, gw)]
        st = ensemble([res[i] for i in idx])
        out.append(dict({"superheat": dT, "Gw": gw, "h_c": st["q_mean"] / dT}, **st))
    for c, lab in zip(out, classify_curve(out)):
        c["regime"] = lab
    curves = {}
    for gw in sorted(set(c["Gw"] for c in out)):
        grp = [c for c in out if c["Gw"] == gw]
        top = max(grp, key=lambda c: c["q_mean"])
        best = max(grp, key=lambda c: c["h_c"])
        boil = [c for c in grp if c["regime"] in ("nucleate", "transition")]
        curves[gw] = {"chf_superheat": top["superheat"], "chf": top["q_mean"], "chf_sem": top["q_sem"],
                      "nucleate_limit_superheat": nucleate_limit(boil) if boil else None,
                      "hc_max_superheat": best["superheat"], "hc_max": best["h_c"]}
    return {"t_switch": t_switch, "t_settle": t_settle, "t_avg": t_avg, "base_superheat": base_superheat,
            "seeds": seeds, "cases": out, "curves": curves, "ranks": world, "runs_on_this_rank": len(mine)}


def boiling_history(superheats, Gw_values=(0.0,), cfg: lb.Config | None = None, base_superheat: float = 0.0137,
                    t_switch: int = 20000, t_end: int = 140000, window: int = 5000, sample_every: int = 1000,
                    seeds=(1, 2, 3), stream=None) -> dict:
    """The time course behind the boiling curve: every (Delta T, G_w, seed)
    run of boiling_curve's protocol continued to t_end, with the mean heat
    flux q(t) of each window of `window` steps after the switch and the
    lowest and mean wall vapour coverage of its samples (every
    sample_every steps). Returns per case the window start times, the
    seed-mean flux per window ("q"), each seed's series ("q_runs") and, per
    window, how many seeds kept the heated wall under a film in every sample
    ("film")."""
    cfg = cfg or paper_config()
    rv, rl = lb.coexistence(cfg)
    cases = [(float(dT), float(gw)) for gw in Gw_values for dT in superheats]
    runs = [(c, int(sd)) for c in cases for sd in seeds]
    insts = [{"cfg": replace(cfg, seed=sd), "Gw": gw, "superheat": (base_superheat if dT > base_superheat else dT)}
             for (dT, gw), sd in runs]
    batch = lb.Batch(insts, stream=stream)
    tune.tune_batch(batch)  # launch form and shape; the states are restored
    nwin = (t_end - t_switch) // window
    q = np.zeros((len(runs), nwin))
    cmin = np.zeros((len(runs), nwin))
    try:
        batch.step(t_switch)
        for i, ((dT, gw), _) in enumerate(runs):
            if dT > base_superheat:
                batch.set_wall_temperature(i, dT)
        for w in range(nwin):
            batch.heat_flux(reset=True)
            lo = np.ones(len(runs))
            done = 0
            while done < window:
                n = min(sample_every, window - done)
                batch.step(n)
                done += n
                for i in range(len(runs)):
                    lo[i] = min(lo[i], wall_coverage(batch.fields(i, ("rho",))["rho"], rl, rv))
            q[:, w] = batch.heat_flux()["q_mean"]
            cmin[:, w] = lo
    finally:
        batch.close()
    out = []
    for c in cases:
        idx = [i for i, (cc, _) in enumerate(runs) if cc == c]
        out.append({"superheat": c[0], "Gw": c[1], "q": q[idx].mean(0).tolist(), "q_runs": q[idx].tolist(),
                    "film": (cmin[idx] >= FILM_COVERAGE).sum(0).astype(int).tolist()})
    return {"t_windows": [t_switch + w * window for w in range(nwin)], "window": window, "seeds": list(seeds),
            "cases": out}
