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
* classify_curve: the regime of every case of a curve, after Sec. 3.2: no
  boiling forms no vapour at the heated wall and no bubbles; film boiling
  keeps the whole heating surface under a continuous vapour film; the
  remaining (boiling) cases are nucleate up to the superheat of the
  critical (maximum) heat flux of their curve and transition beyond it,
  where vapour patches insulate the liquid and q falls.

Superheats are in lattice units (Delta T = T_b - T_s), as in the paper.
"""

from __future__ import annotations

from dataclasses import replace

import numpy as np

from . import diagnostics, lb

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


def classify_curve(cases) -> list:
    """Regime of each case dict (superheat, Gw, q_mean, coverage_min,
    coverage_max, bubbles_max) of one or more curves; cases are grouped by
    G_w and each group's critical heat flux is its largest q_mean among the
    boiling, non-film cases."""
    labels = []
    for c in cases:
        if c["coverage_min"] >= FILM_COVERAGE:
            labels.append("film")
        elif c["coverage_max"] == 0.0 and c["bubbles_max"] == 0:
            labels.append("none")
        else:
            labels.append("boiling")
    chf = {}
    for c, lab in zip(cases, labels):
        if lab == "boiling" and (c["Gw"] not in chf or c["q_mean"] > chf[c["Gw"]][1]):
            chf[c["Gw"]] = (c["superheat"], c["q_mean"])
    return [("nucleate" if c["superheat"] <= chf[c["Gw"]][0] else "transition") if lab == "boiling" else lab
            for c, lab in zip(cases, labels)]


def boiling_curve(superheats, Gw_values=(0.0,), cfg: lb.Config | None = None, base_superheat: float = 0.0137,
                  t_switch: int = 20000, t_settle: int = 5000, t_avg: int = 15000, sample_every: int = 500,
                  stream=None) -> dict:
    """The boiling curve(s) for every (Delta T, G_w) pair in one batch;
    returns per case q_bar, q_std, h_c, the wall coverage (mean, min, max),
    the bubble count (mean, max) and the regime, and per G_w the superheat
    and value of the critical heat flux and of the largest h_c."""
    cfg = cfg or paper_config()
    rv, rl = lb.coexistence(cfg)
    cases = [(float(dT), float(gw)) for gw in Gw_values for dT in superheats]
    insts = [{"cfg": cfg, "Gw": gw, "superheat": (base_superheat if dT > base_superheat else dT)}
             for dT, gw in cases]
    batch = lb.Batch(insts, stream=stream)
    cov = [[] for _ in cases]
    nbub = [[] for _ in cases]
    try:
        batch.step(t_switch)
        for i, (dT, gw) in enumerate(cases):
            if dT > base_superheat:
                batch.set_wall_temperature(i, dT)
        batch.step(t_settle)
        batch.heat_flux(reset=True)
        done = 0
        while done < t_avg:
            n = min(sample_every, t_avg - done)
            batch.step(n)
            done += n
            for i in range(len(cases)):
                rho = batch.fields(i, ("rho",))["rho"]
                cov[i].append(wall_coverage(rho, rl, rv))
                nbub[i].append(len(diagnostics.bubbles(rho, rl, rv)))
        hf = batch.heat_flux()
    finally:
        batch.close()
    out = []
    for i, (dT, gw) in enumerate(cases):
        qm, qs = float(hf["q_mean"][i]), float(hf["q_std"][i])
        out.append({"superheat": dT, "Gw": gw, "q_mean": qm, "q_std": qs, "h_c": qm / dT,
                    "coverage_mean": float(np.mean(cov[i])), "coverage_min": float(np.min(cov[i])),
                    "coverage_max": float(np.max(cov[i])), "bubbles_mean": float(np.mean(nbub[i])),
                    "bubbles_max": int(np.max(nbub[i]))})
    for c, lab in zip(out, classify_curve(out)):
        c["regime"] = lab
    curves = {}
    for gw in sorted(set(c["Gw"] for c in out)):
        grp = [c for c in out if c["Gw"] == gw]
        top = max(grp, key=lambda c: c["q_mean"])
        best = max(grp, key=lambda c: c["h_c"])
        curves[gw] = {"chf_superheat": top["superheat"], "chf": top["q_mean"],
                      "hc_max_superheat": best["superheat"], "hc_max": best["h_c"]}
    return {"t_switch": t_switch, "t_settle": t_settle, "t_avg": t_avg, "base_superheat": base_superheat,
            "cases": out, "curves": curves}
