"""The C-ABI library builds, loads and exports every entry point include/seg.h declares.

No compute call is made here (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_1403_0240_gb300 import build, seg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libseg():
    build.build()
    return seg.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "seg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seg_\w+)\s*\(", text)))


def test_header_symbols_exported(libseg):
    names = _declared()
    assert len(names) >= 19
    bound = {n for n, _, _ in seg.SIGNATURES}
    for n in names:
        assert hasattr(libseg, n), f"{n} declared but not exported"
        assert n in bound, f"{n} not bound in the Python layer"


def test_struct_layouts():
    # seg_params: 2 x int32, 3 x int64, 2 x int32, 3 x double, 5 x int32, 3 x int32 tile, topology,
    # max_labels, regulariser, reserved int32, curv_radius double
    assert C.sizeof(seg.Params) == 120
    assert C.sizeof(seg.Status) == 72
    assert C.sizeof(seg.State) == 32
    assert C.sizeof(seg.ParticleBuffers) == 9 * C.sizeof(C.c_void_p)


def test_strerror_and_validation_without_gpu(libseg):
    assert libseg.seg_strerror(seg.SEG_EINVAL) == b"invalid argument"
    assert libseg.seg_strerror(seg.SEG_ETIMEOUT).startswith(b"bounded")
    import numpy as np
    p = seg.make_params(np.zeros((4, 5), np.float32), cutoff=3.0)
    out = C.c_size_t(0)
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_OK and out.value > 0
    p.cutoff = -1.0
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_EINVAL
    p.cutoff = 3.0
    p.connectivity = 6
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_EINVAL
    p.connectivity = 4
    for tile, code in [((0, 16, 16), seg.SEG_OK), ((1, 64, 128), seg.SEG_OK), ((2, 16, 16), seg.SEG_EINVAL),
                       ((0, -1, 16), seg.SEG_EINVAL), ((0, 16, 1025), seg.SEG_EINVAL)]:
        p.tile[0], p.tile[1], p.tile[2] = tile
        assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == code, tile
    p.tile[0] = p.tile[1] = p.tile[2] = 0
    p.reserved = 1
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_EINVAL
    p.reserved = 0
    # the curvature regulariser needs a ball radius in [1, 16]
    for reg, radius, code in [(seg.SEG_REG_CURVATURE, 4.0, seg.SEG_OK), (seg.SEG_REG_CURVATURE, 0.5, seg.SEG_EINVAL),
                              (seg.SEG_REG_CURVATURE, 17.0, seg.SEG_EINVAL), (seg.SEG_REG_LENGTH, 0.0, seg.SEG_OK),
                              (2, 4.0, seg.SEG_EINVAL), (-1, 4.0, seg.SEG_EINVAL)]:
        p.regulariser, p.curv_radius = reg, radius
        assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == code, (reg, radius)
    p.regulariser, p.curv_radius = seg.SEG_REG_LENGTH, 0.0
    for topology, code in [(seg.SEG_TOPO_STRICT, seg.SEG_OK), (seg.SEG_TOPO_VANISH, seg.SEG_OK),
                           (seg.SEG_TOPO_SPLIT, seg.SEG_OK), (seg.SEG_TOPO_VANISH | seg.SEG_TOPO_SPLIT, seg.SEG_OK),
                           (seg.SEG_TOPO_FUSE, seg.SEG_OK), (7, seg.SEG_OK), (8, seg.SEG_EINVAL),
                           (-1, seg.SEG_EINVAL)]:
        p.topology = topology
        assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == code, topology
    # with splits the label tables (and the relabelling arrays) grow to the capacity
    p.topology = seg.SEG_TOPO_STRICT
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_OK
    strict = out.value
    p.topology = seg.SEG_TOPO_SPLIT
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_OK and out.value > strict
    p.max_labels = 1                               # below the initial count
    assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == seg.SEG_EINVAL
    p.max_labels = 0
    p.topology = seg.SEG_TOPO_STRICT
    # fusion: piecewise constant with exact statistics only
    p.topology = seg.SEG_TOPO_FUSE
    for model, stats, code in [(seg.MODELS["pc"], seg.STATS_MODES["exact"], seg.SEG_OK),
                               (seg.MODELS["ps"], seg.STATS_MODES["exact"], seg.SEG_EINVAL),
                               (seg.MODELS["pc"], seg.STATS_MODES["f64"], seg.SEG_EINVAL)]:
        model0, stats0, radius0 = p.model, p.stats_mode, p.ps_radius
        p.model, p.stats_mode, p.ps_radius = model, stats, 4.0
        assert libseg.seg_estimate_bytes(C.byref(p), 2, C.byref(out)) == code, (model, stats)
        p.model, p.stats_mode, p.ps_radius = model0, stats0, radius0
    p.topology = seg.SEG_TOPO_STRICT


def test_model_and_stats_mode_validation_without_gpu(libseg):
    import numpy as np
    out = C.c_size_t(0)
    p = seg.make_params(np.zeros((64, 48), np.float32), model="pc", cutoff=3.0)
    assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == seg.SEG_OK
    pc_bytes = out.value
    # the deconvolving model needs no local-mean radius; it adds its FP64 fields (T, R, G)
    # and the PSF tables
    p.model = seg.SEG_PC_DECONV
    assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == seg.SEG_OK
    assert out.value >= pc_bytes + 3 * 64 * 48 * 8
    p.model = 4
    assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == seg.SEG_EINVAL
    p.model = seg.SEG_PS                     # piecewise smooth needs R >= 1
    assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == seg.SEG_EINVAL
    p.model = seg.SEG_PC
    for mode, code in [(seg.SEG_STATS_EXACT, seg.SEG_OK), (seg.SEG_STATS_F64, seg.SEG_OK),
                       (seg.SEG_STATS_KAHAN32, seg.SEG_OK), (3, seg.SEG_EINVAL), (-1, seg.SEG_EINVAL)]:
        p.stats_mode = mode
        assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == code, mode


def test_option_edge_values_without_gpu(libseg):
    import math

    import numpy as np
    out = C.c_size_t(0)
    p = seg.make_params(np.zeros((6, 10, 12), np.uint16), model="pc", cutoff=2.0)
    # fusion on a 3D uint16 piecewise-constant job with exact sums is allowed
    p.topology = seg.SEG_TOPO_FUSE
    assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == seg.SEG_OK
    p.topology = seg.SEG_TOPO_SPLIT
    for cap, code in [(3, seg.SEG_OK), (1 << 24, seg.SEG_OK), ((1 << 24) + 1, seg.SEG_EINVAL), (-1, seg.SEG_EINVAL)]:
        p.max_labels = cap
        assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == code, cap
    p.max_labels, p.topology = 0, 0
    p.regulariser = seg.SEG_REG_CURVATURE
    for r, code in [(1.0, seg.SEG_OK), (16.0, seg.SEG_OK), (math.nan, seg.SEG_EINVAL), (math.inf, seg.SEG_EINVAL)]:
        p.curv_radius = r
        assert libseg.seg_estimate_bytes(C.byref(p), 3, C.byref(out)) == code, r
