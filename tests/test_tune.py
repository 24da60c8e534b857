"""The launch-shape autotuner's host logic on the CPU, with a fake
simulation and fake CUDA events: it keeps the fastest accepted shape, skips
shapes the library rejects, restores the state it timed from, caches per
problem and fails clearly when no shape is accepted."""

import types

import pytest

from paper_1501_03857_gb300 import tune


class FakeClock:
    now = 0.0


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = FakeClock.now

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


FAKE_TORCH = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=FakeEvent))


class FakeSim:
    """ms per step depends on the launch shape; shapes in `reject` raise
    like the library does for block sizes it does not take."""

    def __init__(self, cost, reject=(), Lx=100, Ly=80):
        self.cfg = types.SimpleNamespace(Lx=Lx, Ly=Ly, bc_y=0, isothermal=False)
        self.torch, self.stream = FAKE_TORCH, None
        self.cost, self.reject = cost, set(reject)
        self.shape, self.t, self.loads = None, 0, 0

    def set_launch(self, bx, seg):
        if (bx, seg) in self.reject:
            raise ValueError("rejected")
        self.shape = (bx, seg)

    def step(self, n):
        self.t += n
        FakeClock.now += n * self.cost[self.shape]

    def save(self):
        return self.t

    def load(self, blob):
        self.t = blob
        self.loads += 1


@pytest.fixture(autouse=True)
def clear_cache():
    tune._CACHE.clear()
    yield
    tune._CACHE.clear()


def test_keeps_fastest_accepted_shape_and_restores_state():
    cost = {(64, 0): 0.5, (128, 0): 0.3, (256, 0): 0.1, (64, 32): 0.4}
    sim = FakeSim(cost, reject={(256, 0)}, Lx=111)
    sim.t = 7
    bx, seg, ms = tune.tune_simulation(sim, candidates=list(cost))
    assert (bx, seg) == (128, 0) and ms == pytest.approx(0.3)
    assert sim.shape == (128, 0) and sim.t == 7 and sim.loads == 1


def test_cached_per_problem():
    cost = {(64, 0): 0.2, (128, 0): 0.3}
    a = FakeSim(cost, Lx=120)
    tune.tune_simulation(a, candidates=list(cost))
    b = FakeSim({(64, 0): 0.9, (128, 0): 0.1}, Lx=120)  # same problem: cached choice
    assert tune.tune_simulation(b, candidates=list(cost))[:2] == (64, 0)
    assert b.loads == 0 and b.shape == (64, 0)
    c = FakeSim({(64, 0): 0.9, (128, 0): 0.1}, Lx=121)  # another problem: timed again
    assert tune.tune_simulation(c, candidates=list(cost))[:2] == (128, 0)


def test_no_accepted_shape_fails_clearly():
    sim = FakeSim({(64, 0): 0.2}, reject={(64, 0)}, Lx=130)
    sim.t = 3
    with pytest.raises(RuntimeError, match="none of the candidate"):
        tune.tune_simulation(sim, candidates=[(64, 0)])
    assert sim.t == 3 and ("sim", 130, 80, 0, False) not in tune._CACHE


class FakeBatch:
    def __init__(self, cost):
        self.cfgs = [types.SimpleNamespace(Lx=200 + 8 * i, Ly=300, bc_y=0) for i in range(3)]
        self.n = len(self.cfgs)
        self.torch, self.stream, self.cost = FAKE_TORCH, None, cost
        self.shape = None
        self.state = {i: ("f%d" % i, "t%d" % i) for i in range(self.n)}

    def set_launch(self, bx, seg):
        self.shape = (bx, seg)

    def step(self, n):
        FakeClock.now += n * self.cost[self.shape]
        self.state = {i: ("stepped", "stepped") for i in range(self.n)}

    def get_state(self, i):
        return self.state[i]

    def set_state(self, i, f, th):
        self.state[i] = (f, th)


class FakePersistentBatch(FakeBatch):
    """A batch with the persistent mode: its cost depends on (bx, seg, tpb)."""

    tpb = 0

    def set_persistent(self, tpb):
        self.tpb = tpb

    def step(self, n):
        FakeClock.now += n * self.cost[self.shape + (self.tpb,)]
        self.state = {i: ("stepped", "stepped") for i in range(self.n)}


def test_batch_keeps_fastest_shape_and_restores_every_instance():
    cost = {(64, 0): 0.4, (64, 32): 0.25, (128, 0): 0.3}
    b = FakeBatch(cost)
    bx, seg, ms, tpb = tune.tune_batch(b, candidates=list(cost))
    assert (bx, seg, tpb) == (64, 32, 0) and ms == pytest.approx(0.25) and b.shape == (64, 32)
    assert b.state == {i: ("f%d" % i, "t%d" % i) for i in range(3)}


def test_batch_picks_the_persistent_mode_when_faster():
    cost = {(64, 0, 0): 0.4, (64, 0, 2): 0.2, (128, 0, 1): 0.3, (64, 32, 0): 0.35}
    b = FakePersistentBatch(cost)
    bx, seg, ms, tpb = tune.tune_batch(b, candidates=list(cost))
    assert (bx, seg, tpb) == (64, 0, 2) and ms == pytest.approx(0.2)
    assert b.shape == (64, 0) and b.tpb == 2
    assert b.state == {i: ("f%d" % i, "t%d" % i) for i in range(3)}
    # the cached choice is applied again, mode included
    b.set_persistent(0)
    assert tune.tune_batch(b, candidates=list(cost))[3] == 2 and b.tpb == 2
