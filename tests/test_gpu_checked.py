"""The checked build (liblbboil_checked.so, compiled with -DLB_CHECKED): its
fused step checks every global and shared-memory address against its buffer,
and the adjoint's reverse kernels every global address, and each flags a
miss as LB_E_BOUNDS instead of faulting. On grids with odd sizes, every
boundary treatment, several launch shapes, batches of uneven instances (one
launch per step and the persistent launch) and adjoints of odd sizes (both
modes) it flags nothing and produces exactly the states of the normal build,
and its gradients within rounding (1e-6 relative)."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# (Lx, Ly, bc, ghost, Gw, isothermal, steps, block_x, seg_rows)
CASES = [(8, 6, 0, 0, 0.0, 0, 5, 64, 0), (33, 17, 0, 0, 0.08, 0, 40, 64, 6), (33, 17, 1, 0, 0.0, 0, 40, 128, 5),
         (33, 17, 2, 0, 0.0, 0, 40, 64, 3), (40, 12, 0, 1, 0.0, 0, 20, 128, 0), (21, 9, 0, 0, 0.0, 1, 20, 64, 2),
         (517, 41, 1, 0, 0.065, 0, 10, 256, 7), (300, 70, 0, 0, 0.105, 0, 10, 128, 0),
         # the smallest grids the library accepts: one column, three rows
         (1, 3, 0, 0, 0.0, 0, 6, 64, 0), (1, 9, 2, 0, 0.0, 0, 6, 64, 2), (2, 3, 1, 0, 0.05, 0, 6, 128, 1),
         (5, 4, 0, 1, 0.0, 0, 6, 64, 1), (3, 5, 2, 0, 0.0, 1, 6, 256, 0),
         # wide enough for interior strips, whose columns do not wrap
         (700, 30, 2, 0, 0.0, 0, 10, 64, 0), (1000, 20, 0, 0, 0.05, 0, 10, 128, 0), (1500, 12, 1, 0, 0.0, 0, 6, 256, 5)]


def random_cases(n=40, seed=7):
    """A seeded sweep of shapes and launch configurations for the index
    checks: Lx 1-300, Ly 3-120, every boundary treatment, the ghost layer,
    the thermal step on and off, block_x 64/128/256, segment rows from 1 to
    past Ly."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        Lx, Ly = int(rng.integers(1, 301)), int(rng.integers(3, 121))
        bc = int(rng.integers(0, 3))
        ghost = int(bc != 2 and rng.random() < 0.25)
        iso = int(rng.random() < 0.2)
        bx = int(rng.choice([64, 128, 256]))
        seg = int(rng.choice([0, int(rng.integers(1, Ly + 20))]))
        out.append((Lx, Ly, bc, ghost, round(float(rng.uniform(0, 0.1)), 3), iso, 3, bx, seg))
    return out


CASES = CASES + random_cases()


def states(tmp_path, lib):
    out = os.path.join(tmp_path, os.path.basename(lib) + ".npz")
    env = dict(os.environ, LBBOIL_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py"), json.dumps(CASES), out],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.load(out)


def test_checked_build_flags_nothing_and_matches(tmp_path):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    lib_dir = os.path.join(ROOT, "paper_1501_03857_gb300", "_lib")
    checked = states(str(tmp_path), os.path.join(lib_dir, "liblbboil_checked.so"))
    normal = states(str(tmp_path), os.path.join(lib_dir, "liblbboil.so"))
    assert sorted(checked.files) == sorted(normal.files)
    worst = 0.0
    for k in normal.files:
        if k.startswith("adj"):
            # J, dJ/dG_w, dJ/dT_b: the checked build's guarded stores can move
            # where the compiler fuses a multiply-add in the reverse kernels,
            # so the gradients agree to rounding, not bit for bit
            a, b = checked[k], normal[k]
            err = float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))
            worst = max(worst, err)
            assert err < 1e-6, (k, err)
        else:
            assert np.array_equal(checked[k], normal[k]), k
    print(f"largest relative difference of the adjoints: {worst:.1e}")
