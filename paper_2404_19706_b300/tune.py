"""Autotuner for the render path's launch configuration (rtg_tuning).

Section 3.1 rasterises by screen tiles but leaves the tile shape, the work schedule and the
sort's arrangement free.  None of these changes a rendered value (rtg.h, rtg_tuning), so the
tuner may pick any of them by speed alone.  It still checks that claim on the workload
itself: every candidate's render must equal the first candidate's bit for bit, or tuning
stops with an error.

Search, in stages (each stage keeps the previous stages' best values):
  1. render tile x record batch x schedule (CTA per tile, or persistent warps at 2, 4 or
     8 CTAs per SM), with 8-bit digits and ranking for buckets of at most 256 keys;
  2. sort digit width x ranking cutoff.
Each candidate is captured in a CUDA graph and timed by replaying it between CUDA events
on the capture stream.  With a flush buffer (larger than L2), the buffer is written before
every replay and each replay is timed alone, so candidates are ranked under the same
cold-L2 conditions as a benchmark that flushes between steps; the score is the median over
the replays.  A candidate whose forward overflows the pair capacity (RTG_ERR_WORKSPACE) is
skipped.
"""

from __future__ import annotations

import dataclasses
import statistics
from typing import Callable, Dict, List, Optional, Sequence

import torch

from . import api
from .api import Tuning

TILES = [(16, 16), (16, 8), (8, 16), (8, 8), (32, 8)]
BATCHES = [32, 64]
SCHEDULES = [(0, 4), (1, 2), (1, 4), (1, 8)]  # (schedule, persistent CTAs per SM)
SORTS = [(8, 0), (8, 256), (8, 512), (4, 0), (4, 256)]  # (digit bits, ranking cutoff)


STAGE1_SORT = (8, 256)  # sort used while the tile shape and schedule are searched


def stage1(base: Tuning = Tuning()) -> List[Tuning]:
    """Tile x batch x schedule, with the ranking sort for short buckets: smaller tiles make
    shorter buckets, and ranking them is what makes those tiles pay, so searching the tile
    shapes under the plain radix sort would rank them too low."""
    out = []
    base = dataclasses.replace(base, sort_digit_bits=STAGE1_SORT[0], sort_rank_max=STAGE1_SORT[1])
    for (tw, th) in TILES:
        for b in BATCHES:
            for (sch, ctas) in SCHEDULES:
                out.append(dataclasses.replace(base, tile_w=tw, tile_h=th, batch=b, schedule=sch,
                                               persist_ctas_per_sm=ctas))
    return out


def stage2(base: Tuning) -> List[Tuning]:
    return [dataclasses.replace(base, sort_digit_bits=bits, sort_rank_max=cut) for (bits, cut) in SORTS]


@dataclasses.dataclass
class TuneResult:
    best: Tuning
    best_ms: float
    default_ms: float
    table: List[dict]  # one row per candidate: tuning, median ms per step (None if skipped), note

    def summary(self) -> dict:
        timed = [r for r in self.table if r["ms"] is not None]
        return {"best": self.best.as_dict(), "best_ms_per_step": round(self.best_ms, 5),
                "default_ms_per_step": round(self.default_ms, 5), "candidates": len(self.table),
                "timed": len(timed), "skipped": len(self.table) - len(timed)}


class Autotuner:
    """Times ``step`` (one iteration on fixed buffers, launched on the current stream) under
    each candidate tuning of ``ctx``.

    check: optional callable returning a list of tensors that must be bit-identical under
        every candidate (e.g. a forward-only render); run once per candidate before timing.
    restore: optional callable run after every candidate (e.g. to put back parameters that
        the step's optimiser moved), so every candidate sees the same workload.
    """

    def __init__(self, ctx, step: Callable[[], object], check: Optional[Callable[[], Sequence]] = None,
                 restore: Optional[Callable[[], None]] = None, warmup: int = 3, iters: int = 15, repeats: int = 3,
                 flush: Optional[torch.Tensor] = None):
        # ctx: a Context, or a sequence of Contexts that the step uses together (each gets
        # every candidate tuning)
        self.ctxs = list(ctx) if isinstance(ctx, (list, tuple)) else [ctx]
        self.step, self.check, self.restore = step, check, restore
        self.warmup, self.iters, self.repeats = warmup, iters, repeats
        self.flush = flush
        self._ref = None

    def _status_ok(self) -> bool:
        bad = [c for c in self.ctxs if api.get_status(c) != 0]
        for c in bad:
            api.reset_status(c)
        return not bad

    def _verify(self, t: Tuning) -> Optional[str]:
        for c in self.ctxs:
            api.reset_status(c)
        if self.check is not None:  # before the step moves any parameter
            out = [x.clone() for x in self.check()]
            torch.cuda.synchronize()
            if not self._status_ok():
                return "pair capacity exceeded"
            if self._ref is None:
                self._ref = out
            else:
                for a, b in zip(self._ref, out):
                    if not torch.equal(a, b):
                        raise AssertionError(f"tuning {t} changed a rendered value")
        self.step()  # eager once (also the first use of this configuration)
        torch.cuda.synchronize()
        if not self._status_ok():
            return "pair capacity exceeded"
        return None

    def time(self, t: Tuning) -> Optional[float]:
        """Median ms per step of ``t``: over iters x repeats single replays with the flush buffer
        written before each, else over ``repeats`` timed runs of ``iters`` back-to-back replays."""
        for c in self.ctxs:
            c.set_tuning(t)
        note = self._verify(t)
        if note is not None:
            if self.restore is not None:
                self.restore()
            return None
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.step()
        stream = torch.cuda.current_stream()
        for _ in range(self.warmup):
            graph.replay()
        samples = []
        if self.flush is not None:  # cold L2 before every replay, each replay timed alone
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(self.iters * self.repeats)]
            torch.cuda.synchronize()
            for a, b in ev:
                self.flush.zero_()
                a.record(stream)
                graph.replay()
                b.record(stream)
            torch.cuda.synchronize()
            samples = [a.elapsed_time(b) for a, b in ev]
        for _ in range(self.repeats if self.flush is None else 0):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            for _ in range(self.iters):
                graph.replay()
            b.record(stream)
            b.synchronize()
            samples.append(a.elapsed_time(b) / self.iters)
        del graph
        if self.restore is not None:
            self.restore()
        return statistics.median(samples)

    def run(self, start: Tuning = Tuning()) -> TuneResult:
        table: List[Dict] = []

        def measure(cands: Sequence[Tuning]) -> Tuning:
            best, best_ms = None, float("inf")
            for t in cands:
                ms = self.time(t)
                table.append({"tuning": t.as_dict(), "ms": None if ms is None else round(ms, 5),
                              "note": "" if ms is not None else "skipped: pair capacity exceeded"})
                if ms is not None and ms < best_ms:
                    best, best_ms = t, ms
            if best is None:
                raise RuntimeError("no candidate tuning ran within the pair capacity")
            return best

        default_ms = self.time(start)
        if default_ms is None:
            raise RuntimeError("the starting tuning exceeds the pair capacity")
        table.append({"tuning": start.as_dict(), "ms": round(default_ms, 5), "note": "start"})
        b1 = measure(stage1(start))
        best = measure(stage2(b1))
        best_ms = min(r["ms"] for r in table if r["ms"] is not None and r["tuning"] == best.as_dict())
        for c in self.ctxs:
            c.set_tuning(best)
        return TuneResult(best=best, best_ms=best_ms, default_ms=default_ms, table=table)


def autotune(ctx, step: Callable[[], object], check: Optional[Callable[[], Sequence]] = None,
             restore: Optional[Callable[[], None]] = None, **kw) -> TuneResult:
    """Runs the staged search and leaves ``ctx`` set to the fastest tuning."""
    return Autotuner(ctx, step, check, restore, **kw).run()
