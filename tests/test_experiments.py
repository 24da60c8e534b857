"""Host logic of the boiling experiments (Sec. 3.2-3.3) on the CPU: the
regime classification of a curve and the wall vapour coverage."""

import numpy as np

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
