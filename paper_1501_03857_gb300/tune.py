"""Launch-shape autotuner for the fused step.

Times candidate launch shapes (threads per block and rows per segment; for
batches also the mode: one launch per step, or the persistent launch with
about tpb tiles per block) with CUDA events on the simulation's stream over
a few steps and keeps the fastest. Results are cached per problem signature (grid sizes, boundary
condition) for the life of the process. The state is saved before tuning and
restored afterwards, so tuning does not advance the simulation.
"""

from __future__ import annotations

from typing import Dict, Iterable, Optional, Tuple

_CACHE: Dict[tuple, tuple] = {}

SIM_CANDIDATES = tuple((bx, seg) for bx in (64, 128, 256) for seg in (0, 32, 64, 128, 256))
# (block_x, seg_rows, tiles per block of the persistent launch; 0: one launch per step)
BATCH_CANDIDATES = (tuple((bx, seg, 0) for bx in (64, 128) for seg in (0, 16, 32, 64, 128))
                    + tuple((bx, 0, tpb) for bx in (64, 128) for tpb in (1, 2)))


def _time(torch, stream, fn, steps: int) -> float:
    fn(2)  # warm-up for this shape
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn(steps)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune_simulation(sim, candidates: Optional[Iterable[Tuple[int, int]]] = None, steps: int = 8):
    """Pick the fastest (block_x, seg_rows) of the default kernel for `sim`
    and apply it. Returns (block_x, seg_rows, ms_per_step)."""
    c = sim.cfg
    key = ("sim", c.Lx, c.Ly, c.bc_y, c.isothermal)
    if key not in _CACHE:
        blob = sim.save()
        best = None
        for bx, seg in (candidates or SIM_CANDIDATES):
            try:
                sim.set_launch(bx, seg)
            except Exception:
                continue
            ms = _time(sim.torch, sim.stream, sim.step, steps)
            if best is None or ms < best[2]:
                best = (bx, seg, ms)
        sim.load(blob)
        if best is None:
            raise RuntimeError("the simulation accepted none of the candidate launch shapes")
        _CACHE[key] = best
    bx, seg, ms = _CACHE[key]
    sim.set_launch(bx, seg)
    return bx, seg, ms


def _apply_batch(batch, bx, seg, tpb):
    if tpb or hasattr(batch, "set_persistent"):
        batch.set_persistent(tpb)
    batch.set_launch(bx, seg)


def time_batch_candidates(batch, candidates: Optional[Iterable[tuple]] = None, steps: int = 32) -> dict:
    """ms per step of every accepted candidate (block_x, seg_rows[,
    tiles_per_block]) of `batch`, keyed by the (block_x, seg_rows,
    tiles_per_block) triple; the instances' states are restored."""
    saved = [batch.get_state(i) for i in range(batch.n)]
    out = {}
    for cand in (candidates or BATCH_CANDIDATES):
        bx, seg, tpb = (tuple(cand) + (0,))[:3]
        try:
            _apply_batch(batch, bx, seg, tpb)
        except Exception:
            continue
        out[(bx, seg, tpb)] = _time(batch.torch, batch.stream, batch.step, steps)
    for i, (f, th) in enumerate(saved):
        batch.set_state(i, f, th)
    return out


def tune_batch(batch, candidates: Optional[Iterable[tuple]] = None, steps: int = 32):
    """Pick the fastest (block_x, seg_rows[, tiles_per_block]) shared by all
    instances of `batch` and apply it (tiles_per_block 0 or absent: one
    launch per step; >= 1: the persistent launch). Returns (block_x,
    seg_rows, ms_per_step, tiles_per_block). The instances' states are
    restored; their heat-flux accumulators keep the samples of the timing
    steps (reset them after tuning if that matters)."""
    key = ("batch",) + tuple((c.Lx, c.Ly, c.bc_y) for c in batch.cfgs)
    if key not in _CACHE:
        times = time_batch_candidates(batch, candidates, steps)
        if not times:
            raise RuntimeError("the batch accepted none of the candidate launch shapes")
        (bx, seg, tpb), ms = min(times.items(), key=lambda kv: kv[1])
        _CACHE[key] = (bx, seg, ms, tpb)
    bx, seg, ms, tpb = _CACHE[key]
    _apply_batch(batch, bx, seg, tpb)
    return bx, seg, ms, tpb
