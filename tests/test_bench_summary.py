"""bench.py's closing summary block on the CPU: built from a line's blocks,
with the blocks that were skipped left out."""

import bench


def test_summary_of_a_full_line():
    line = {"value": 47000.4, "roofline": {"frac": 0.5551, "peak": 6785.9}, "e2e": {"value": 43000.2},
            "batched": {"speedup": 5.87, "ms_per_step_batched": 0.1944, "sims_per_hour_batched": 17733.8,
                        "mlups_batched": 29912.0, "launch": {"mode": "persistent: one cooperative launch per 32 steps"}},
            "adjoint": {"cost_ratio": 3.03, "rel_err_Gw": 1.28e-3,
                        "vs_fp64_reference": {"rel_err_Gw": 2.1e-5, "rel_err_uniform": 3.0e-6},
                        "large": {"ms_reverse_per_step": 0.658, "ms_forward_per_step": 0.106, "roofline": {"frac": 0.188}}},
            "experiments": {"sims_per_hour": 12000.4, "curves": {"0.0": {"chf_superheat": 0.023}}},
            "cpu_baseline": {"value": 5.11}}
    s = bench.summary(line)
    assert s["mlups"] == 47000 and s["batched"]["mode"] == "persistent"
    assert abs(s["batched"]["hbm_frac"] - 29912.0 * 80e6 / 1e9 / 6785.9) < 1e-3
    assert s["adjoint"]["rel_err_Gw_vs_fp64"] == 2.1e-5 and s["adjoint"]["cost_vs_forward_2048"] == round(1 + 0.658 / 0.106, 2)
    assert s["experiments"]["chf_superheat"] == {"0.0": 0.023} and s["oracle_mlups"] == 5.11


def test_summary_without_the_optional_blocks():
    s = bench.summary({"value": 1.0, "roofline": {"frac": 0.5, "peak": 1.0}, "e2e": {"value": 0.9}})
    assert set(s) == {"mlups", "hbm_frac", "e2e_mlups"}
