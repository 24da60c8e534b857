"""Host logic of the boiling experiments (Sec. 3.2-3.3) on the CPU: the
regime classification of a curve and the wall vapour coverage."""

import numpy as np
import pytest

from paper_1501_03857_gb300 import experiments as E


def case(dT, q, cmin, cmax, nb, gw=0.0):
    return {"superheat": dT, "Gw": gw, "q_mean": q, "coverage_min": cmin, "coverage_max": cmax, "bubbles_max": nb}


def test_classify_curve_uses_each_curves_chf():
    cases = [case(0.008, 1e-4, 0, 0, 0), case(0.0137, 6e-4, 0.02, 0.2, 9), case(0.021, 1.2e-3, 0.4, 0.6, 3),
             case(0.025, 1.3e-3, 0.5, 0.8, 4), case(0.032, 1.2e-3, 0.7, 0.9, 4), case(0.035, 5e-5, 1.0, 1.0, 0),
             # a second curve whose CHF sits at a lower superheat
             case(0.0137, 8e-4, 0.1, 0.3, 9, 0.1), case(0.021, 1.1e-3, 0.5, 0.7, 7, 0.1),
             case(0.025, 1.0e-3, 0.6, 0.8, 7, 0.1)]
    assert E.classify_curve(cases) == ["none", "nucleate", "nucleate", "nucleate", "transition", "film",
                                       "nucleate", "nucleate", "transition"]


def test_film_needs_every_sample_covered():
    # coverage 0.94 at its lowest sample is patches, not a continuous film
    cases = [case(0.02, 1e-3, 0.3, 0.5, 5), case(0.035, 4e-4, 0.94, 1.0, 3)]
    assert E.classify_curve(cases) == ["nucleate", "transition"]
    # vapour at the wall but no detached bubble still counts as boiling
    assert E.classify_curve([case(0.01, 3e-4, 0.0, 0.05, 0)]) == ["nucleate"]


def test_wall_coverage():
    rho = np.full((10, 40), 6.5)
    rho[1, :10] = 0.4
    assert E.wall_coverage(rho, 6.5, 0.38) == 0.25
    assert E.wall_coverage(rho, 6.5, 0.38, row=2) == 0.0


def test_ensemble_statistics():
    """Seed ensembles: the mean of the runs' window means with its standard
    error, the mean within-window deviation, and coverage / bubble extremes
    over every sample of every run."""
    runs = [{"q_mean": 1.0, "q_std": 0.1, "coverage": [0.0, 0.5], "bubbles": [0, 3]},
            {"q_mean": 2.0, "q_std": 0.3, "coverage": [1.0, 1.0], "bubbles": [1, 1]},
            {"q_mean": 3.0, "q_std": 0.2, "coverage": [0.25, 0.25], "bubbles": [2, 0]}]
    st = E.ensemble(runs)
    assert st["q_mean"] == pytest.approx(2.0)
    assert st["q_sem"] == pytest.approx(1.0 / 3.0 ** 0.5)  # sample std 1 over sqrt(3)
    assert st["q_std"] == pytest.approx(0.2)
    assert st["coverage_min"] == 0.0 and st["coverage_max"] == 1.0
    assert st["coverage_mean"] == pytest.approx(0.5)
    assert st["bubbles_max"] == 3 and st["bubbles_mean"] == pytest.approx(7 / 6)
    assert st["film_fraction"] == pytest.approx(1 / 3) and st["none_fraction"] == 0.0
    film2 = runs + [{"q_mean": 0.1, "q_std": 0.0, "coverage": [1.0, 0.99], "bubbles": [0, 0]}]
    e2 = E.ensemble(film2)
    assert e2["film_fraction"] == 0.5
    # majority rule: 2 of 4 runs with a film is not a film case, 3 of 4 is
    c = dict(e2, superheat=0.03, Gw=0.0)
    assert E.classify_curve([c]) == ["nucleate"]
    c3 = dict(E.ensemble(film2 + film2[-1:]), superheat=0.03, Gw=0.0)
    assert E.classify_curve([c3]) == ["film"]
    one = E.ensemble(runs[:1])
    assert one["q_mean"] == 1.0 and one["q_sem"] != one["q_sem"]  # NaN: no spread from one run


def test_nucleate_limit_with_standard_errors():
    """Without errors the limit is the superheat of the largest mean flux;
    with seed standard errors it is the lowest superheat that no higher
    case exceeds by more than twice the combined error."""
    qs = [(0.01, 1.0), (0.02, 3.0), (0.03, 3.3), (0.04, 3.1)]
    cs = [{"superheat": t, "q_mean": q} for t, q in qs]
    assert E.nucleate_limit(cs) == 0.03
    assert E.nucleate_limit([dict(c, q_sem=float("nan")) for c in cs]) == 0.03
    wide = [dict(c, q_sem=0.15) for c in cs]  # 2 x hypot(0.15, 0.15) = 0.42 > 0.3
    assert E.nucleate_limit(wide) == 0.02
    narrow = [dict(c, q_sem=0.05) for c in cs]  # 0.14 < 0.3: 3.3 is significantly above 3.0
    assert E.nucleate_limit(narrow) == 0.03
    assert E.classify_curve([case(t, q, 0.1, 0.5, 3) for t, q in qs]) == ["nucleate"] * 3 + ["transition"]
    assert E.classify_curve([dict(case(t, q, 0.1, 0.5, 3), q_sem=0.15) for t, q in qs]) == \
        ["nucleate"] * 2 + ["transition"] * 2
