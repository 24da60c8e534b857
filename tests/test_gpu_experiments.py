"""The paper's boiling experiments on the GPU (Sec. 3.2-3.3): the regimes,
critical heat flux and wettability effects its text states
(tests/golden/paper_regimes.txt), and Fig. 3's rising top-wall pressure.
Long boiling runs are chaotic, so these are the paper's qualitative
statements, not values."""

import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden():
    regimes, out = {}, {}
    for line in open(os.path.join(GOLDEN, "paper_regimes.txt")):
        line = line.split("#")[0].split()
        if not line:
            continue
        if line[0] == "regime":
            regimes[float(line[1])] = line[2]
        else:
            out[line[0]] = [float(v) for v in line[1:]]
    return regimes, out


@pytest.fixture(scope="module")
def E():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1501_03857_gb300 import experiments
    return experiments


# Near the top of a curve neighbouring superheats differ by less than the
# spread of one run's window mean, so one realisation's maximum moves with
# any rounding-level change of the step; every case is averaged over six
# seeds of the pool's initial noise (one batch).
SEEDS = (1, 2, 3, 4, 5, 6)


@pytest.fixture(scope="module")
def curve(E):
    dts0 = (0.008, 0.01, 0.0137, 0.0165, 0.019, 0.021, 0.023, 0.025, 0.027, 0.029, 0.032, 0.035)
    r0 = E.boiling_curve(dts0, Gw_values=(0.0,), seeds=SEEDS)
    r1 = E.boiling_curve((0.01, 0.0137, 0.019, 0.021, 0.023, 0.025), Gw_values=(0.105,), seeds=SEEDS)
    for r in (r0, r1):
        for c in r["cases"]:
            print(f"Gw={c['Gw']} dT={c['superheat']} q={c['q_mean']:.4e} sem={c['q_sem']:.1e} "
                  f"runs={['%.4e' % q for q in c['q_runs']]} q_std={c['q_std']:.2e} "
                  f"cov={c['coverage_mean']:.3f}/{c['coverage_min']:.3f}/{c['coverage_max']:.3f} "
                  f"bub={c['bubbles_mean']:.1f}/{c['bubbles_max']} regime={c['regime']}")
    return r0, r1


def test_regimes_match_paper(curve):
    regimes, _ = golden()
    got = {c["superheat"]: c["regime"] for c in curve[0]["cases"]}
    for dT, lab in regimes.items():
        assert got[dT] == lab, (dT, got[dT], lab)


def test_critical_heat_flux_and_hc(curve):
    """CHF inside the superheat range Sec. 3.2 gives: the flux stops rising
    (nucleate limit) within the range, and the largest mean flux over the
    range is within two standard errors of the curve's largest; the largest
    h_c at a lower superheat than the largest mean flux (Sec. 3.2, Fig. 8)."""
    _, g = golden()
    c0 = curve[0]["curves"][0.0]
    lo, hi = g["chf_range"]
    assert lo <= c0["nucleate_limit_superheat"] <= hi
    inside = max((c for c in curve[0]["cases"] if lo <= c["superheat"] <= hi), key=lambda c: c["q_mean"])
    assert inside["q_mean"] >= c0["chf"] - 2.0 * float(np.hypot(inside["q_sem"], c0["chf_sem"]))
    assert c0["hc_max_superheat"] < c0["chf_superheat"]


def test_transition_heat_flux_fluctuates_most(curve):
    """Sec. 3.2, Fig. 6: the transient heat flux of the transition case
    (0.032) fluctuates far more than that of the nucleate (0.0165) and film
    (0.035) cases: its standard deviation over the window is more than
    1.5x and 5x theirs."""
    _, g = golden()
    t, n, f = g["q_fluct"]
    c0 = {c["superheat"]: c for c in curve[0]["cases"]}
    assert c0[t]["q_std"] > 1.5 * c0[n]["q_std"]
    assert c0[t]["q_std"] > 5.0 * c0[f]["q_std"]


def test_wettability_effects(curve):
    """Sec. 3.3, Fig. 13: a larger contact angle lowers the critical heat
    flux, and boiling starts at a lower superheat (G_w = 0.105 boils at
    0.01, G_w = 0 does not); below the crossing of the curves the less
    wettable surface transfers more heat."""
    _, g = golden()
    gw, dT = g["onset_gw"]
    c1 = {c["superheat"]: c for c in curve[1]["cases"]}
    c0 = {c["superheat"]: c for c in curve[0]["cases"]}
    assert curve[1]["curves"][gw]["chf"] < curve[0]["curves"][0.0]["chf"]
    assert c1[dT]["regime"] != "none" and c0[dT]["regime"] == "none"
    assert c1[0.0137]["q_mean"] > c0[0.0137]["q_mean"]
    assert c1[0.025]["q_mean"] < c0[0.025]["q_mean"]


def test_top_wall_pressure_rises(E):
    """Fig. 3: after the switch the pressure at the centre of the top wall
    rises as bubbles reach the vapour above the pool, faster at the higher
    superheat."""
    r = E.top_wall_pressure((0.0137, 0.0165), t_after=10000)["cases"]
    for dT in (0.0137, 0.0165):
        p = r[dT]["p_top"]
        assert p[-1] > p[0]
    assert r[0.0165]["p_top"][-1] > r[0.0137]["p_top"][-1]


def test_film_onset_is_steep_in_wettability(E):
    """Sec. 3.3 puts film boiling at Delta T = 0.029 for G_w = 0.105; here that
    surface stays in transition there (no seed keeps a film at the wall in
    any window to 50 000 steps), while a slightly less wettable one, G_w =
    0.15 (static angle about 66 deg instead of 56.5 deg), is under a film in
    every seed after the switch: the film threshold moves across the
    paper's values within a ~10 deg change of the static angle."""
    r = E.boiling_history((0.029,), Gw_values=(0.105, 0.15), t_end=50000, window=5000, seeds=(1, 2, 3))
    c = {x["Gw"]: x for x in r["cases"]}
    print({gw: (x["film"], ["%.2e" % q for q in x["q"]]) for gw, x in c.items()})
    assert max(c[0.105]["film"]) == 0
    assert min(c[0.15]["film"][-3:]) == 3
    assert max(c[0.15]["q"][-3:]) < 0.3 * min(c[0.105]["q"][-3:])
