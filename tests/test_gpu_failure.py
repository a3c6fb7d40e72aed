"""Failure detection without a GPU fault: a tile whose label copy is never issued (a test-only
injection; nothing completes the barrier the tile waits on) makes the bounded device wait run
out. The iteration reports SEG_ETIMEOUT within seconds, the device stays usable, and in a batch
only the injected job is affected."""
import time

import numpy as np
import pytest

from paper_1403_0240_gb300 import seg, synth

pytestmark = pytest.mark.gpu


def _job():
    return synth.disks(96, 128, seed=3)        # 12 extraction tiles


def test_unpublished_tile_times_out_and_reports():
    w = _job()
    ctx = seg.Context.from_workload(w)
    ctx.step(1)
    ctx.inject(seg.SEG_INJECT_WITHHELD_COPY)
    t0 = time.time()
    with pytest.raises(seg.SegError) as e:
        ctx.step(1)
    elapsed = time.time() - t0
    assert e.value.code == seg.SEG_ETIMEOUT
    assert elapsed < 30.0
    with pytest.raises(seg.SegError):
        ctx.step(1)                              # the context stays poisoned
    ctx.close()
    # the device is usable: a fresh context runs normally
    c2 = seg.Context.from_workload(w)
    st = c2.step(3)
    assert st["error"] == 0 and st["n_particles"] > 0
    c2.close()


def test_injected_job_does_not_disturb_its_batch():
    w_bad, w_ok = _job(), synth.disks(80, 72, seed=4)
    ref = seg.Context.from_workload(w_ok)
    ref.step(4)
    ref_labels = ref.labels().copy()
    ref.close()
    bad, ok = seg.Context.from_workload(w_bad), seg.Context.from_workload(w_ok)
    batch = seg.Batch()
    batch.add(bad)
    batch.add(ok)
    batch.step(2)
    bad.inject(seg.SEG_INJECT_WITHHELD_COPY)
    with pytest.raises(seg.SegError) as e:
        batch.step(2)
    assert e.value.code == seg.SEG_ETIMEOUT
    assert np.array_equal(ok.labels(), ref_labels)
    batch.remove(bad)
    batch.close()
    bad.close()
    ok.close()
