"""The stored oracle ensemble of the time-averaged heat flux is consistent
with its own per-seed values (the file is written by
tests/golden/make_qbar_golden.py from oracle runs only)."""

import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "qbar_boiling_200x100.txt")


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden file not generated")
def test_qbar_golden_summary_matches_its_seeds():
    from test_gpu_statistics import read_golden
    g = read_golden(GOLDEN)
    q = np.array([g["runs"][k] for k in sorted(g["runs"])])
    assert len(q) == g["nseeds"] >= 20
    assert abs(q.mean() / g["mean"] - 1) < 1e-8
    assert abs(q.std(ddof=1) / np.sqrt(len(q)) / g["sem"] - 1) < 1e-6
    assert np.all(q > 0)
