"""Batch autotuner logic on the CPU: a fake context/batch whose step time depends on the
candidate checks that the fastest candidate is chosen, that failing candidates are skipped,
and that the sample is spread over the job list."""
import time

import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, tune


class FakeContext:
    created = []

    def __init__(self, image, labels0, stream=None, cell_edge=0, tile=None, **kw):
        if tile == (64, 64):
            raise seg.SegError.__new__(seg.SegError)
        self.cost = {(16, 16): 3e-3, (32, 32): 1e-3, (32, 64): 2e-3}.get(tuple(tile), 4e-3) * (cell_edge / 3)
        FakeContext.created.append((image.shape, cell_edge, tuple(tile)))

    def close(self):
        pass


class FakeBatch:
    def __init__(self, stream=None):
        self.members = []

    def add(self, c):
        self.members.append(c)

    def step(self, iters=1):
        time.sleep(iters * max(c.cost for c in self.members))

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(seg, "Context", FakeContext)
    monkeypatch.setattr(seg, "Batch", FakeBatch)
    FakeContext.created = []


def _jobs(n):
    return [(np.zeros((8 + i, 8), np.float32), np.zeros((8 + i, 8), np.int32), {"cutoff": 3.0}) for i in range(n)]


def test_picks_fastest_and_skips_failures(fake):
    cands = [(1, (16, 16)), (1, (32, 32)), (1, (64, 64)), (2, (32, 32)), (1, (32, 64))]
    best, table = tune.autotune_batch(_jobs(10), iters=2, sample=4, candidates=cands)
    assert best == {"cell_multiple": 1, "tile": (32, 32)}
    assert [t[:2] for t in table] == [(m, t) for m, t in cands]
    assert table[2][2] == float("inf")                       # the failing candidate
    assert all(t[2] < float("inf") for i, t in enumerate(table) if i != 2)


def test_sample_spread_and_cell_edges(fake):
    tune.autotune_batch(_jobs(12), iters=1, sample=4, candidates=[(2, (32, 32))])
    shapes = [s for s, _, _ in FakeContext.created]
    assert shapes == [(8, 8), (11, 8), (14, 8), (17, 8)]     # every third job
    assert {e for _, e, _ in FakeContext.created} == {6}    # 2 x ceil(cutoff)
