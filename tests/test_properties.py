"""Property tests of host logic (CPU): the seeded generator against an
independent pure-Python splitmix64, row windows of the pool generator,
dealing cases to ranks and gathering them back, the angle -> G_w inversion,
and the probe ring's size rule. Uses hypothesis where it is installed."""

import numpy as np
import pytest

from paper_1501_03857_gb300 import inputs, replicas

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

MASK = (1 << 64) - 1


def splitmix64_py(seed, n):
    """The published splitmix64 (Steele, Lea and Flood 2014), in Python ints."""
    z = (seed + (n + 1) * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


@settings(max_examples=200, deadline=None)
@given(st.integers(0, MASK), st.lists(st.integers(0, 1 << 40), min_size=1, max_size=16))
def test_splitmix64_matches_definition(seed, counters):
    got = inputs.splitmix64(seed, np.array(counters, dtype=np.uint64))
    assert [int(v) for v in got] == [splitmix64_py(seed, n) for n in counters]


@settings(max_examples=60, deadline=None)
@given(st.integers(8, 90), st.integers(8, 70), st.data())
def test_pool_rows_window_equals_full_field(Lx, Ly, data):
    y0 = data.draw(st.integers(0, Ly - 1))
    y1 = data.draw(st.integers(y0 + 1, Ly))
    seed = data.draw(st.integers(0, 1000))
    full = inputs.pool_density(Lx, Ly, 6.5, 0.38, Ly * 0.4, noise_amp=1e-3, seed=seed)
    part = inputs.pool_density(Lx, Ly, 6.5, 0.38, Ly * 0.4, noise_amp=1e-3, seed=seed, rows=(y0, y1))
    assert np.array_equal(full[y0:y1], part)


@settings(max_examples=200, deadline=None)
@given(st.lists(st.integers(), max_size=40), st.integers(1, 9))
def test_shard_then_gather_restores_order(items, world):
    parts = [replicas.shard(items, r, world) for r in range(world)]
    sizes = sorted(len(p) for p in parts)
    assert sizes[-1] - sizes[0] <= 1 and sum(sizes) == len(items)

    class FakeDist:  # all_gather_object over the in-process parts
        @staticmethod
        def all_gather_object(out, obj):
            out[:] = parts

    assert replicas.gather_shards(parts[0], 0, world, FakeDist) == list(items)


@settings(max_examples=100, deadline=None)
@given(st.lists(st.integers(-2000, 5000), min_size=2, max_size=12, unique=True), st.data())
def test_gw_for_angle_inverts_a_monotone_table(ks, data):
    from paper_1501_03857_gb300 import wetting
    gws = sorted(k * 1e-4 for k in ks)
    angles = [40.0 + 250.0 * (g + 0.2) for g in gws]  # strictly increasing
    k = data.draw(st.integers(0, len(gws) - 1))
    assert abs(float(wetting.gw_for_angle(angles[k], gws, angles)) - gws[k]) < 1e-12


def test_probe_ring_size_rule():
    import ctypes as C
    from paper_1501_03857_gb300 import lb
    n = C.c_size_t()
    assert lb.lib.lb_probe_ring_bytes(3, 1000, C.byref(n)) == 0 and n.value == 256 + 16 * 3 * 1000
    for bad in ((0, 10), (lb.PROBE_MAX + 1, 10), (1, 0), (1, (1 << 26) + 1)):
        assert lb.lib.lb_probe_ring_bytes(bad[0], bad[1], C.byref(n)) == -1
    assert lb.lib.lb_set_probes(None, 0, None, None, None, 0, 0) == -1
