"""Python binding of libseg (include/seg.h): argument marshalling only.

Every step of the segmentation runs in the CUDA library; this module converts numpy
arrays or torch tensors into the pointers and sizes of the C-ABI and back. It fails
loudly when the library has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

SEG_OK, SEG_EINVAL, SEG_ENOMEM, SEG_ECUDA, SEG_ETIMEOUT, SEG_ESTATE = 0, -1, -2, -3, -4, -5
SEG_F32, SEG_U16 = 0, 1
SEG_PC, SEG_PS, SEG_PS_POISSON, SEG_PC_DECONV = 0, 1, 2, 3
SEG_PSF_MAX_RADIUS = 512
MODELS = {"pc": SEG_PC, "ps": SEG_PS, "psp": SEG_PS_POISSON, "pcd": SEG_PC_DECONV}
SEG_SOBOLEV, SEG_L2, SEG_SOBOLEV_GLOBAL = 0, 1, 2
SEG_STATS_EXACT, SEG_STATS_F64, SEG_STATS_KAHAN32 = 0, 1, 2
SEG_TOPO_STRICT, SEG_TOPO_VANISH, SEG_TOPO_SPLIT, SEG_TOPO_FUSE = 0, 1, 2, 4
TOPOLOGY = {"strict": 0, "vanish": 1, "split": 2, "vanish+split": 3, "fuse": 4, "vanish+fuse": 5, "split+fuse": 6,
            "vanish+split+fuse": 7}
SEG_REG_LENGTH, SEG_REG_CURVATURE = 0, 1
STATS_MODES = {"exact": SEG_STATS_EXACT, "f64": SEG_STATS_F64, "kahan32": SEG_STATS_KAHAN32}
SEG_INJECT_NONE, SEG_INJECT_WITHHELD_COPY = 0, 1


class Params(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dtype", C.c_int32), ("shape", C.c_int64 * 3),
                ("model", C.c_int32), ("connectivity", C.c_int32),
                ("lam", C.c_double), ("cutoff", C.c_double), ("ps_radius", C.c_double),
                ("gradient", C.c_int32), ("osc_window", C.c_int32), ("stats_mode", C.c_int32),
                ("validate", C.c_int32), ("cell_edge", C.c_int32), ("tile", C.c_int32 * 3),
                ("topology", C.c_int32), ("max_labels", C.c_int32), ("regulariser", C.c_int32),
                ("reserved", C.c_int32), ("curv_radius", C.c_double)]


class TuneEntry(C.Structure):
    _fields_ = [("cell_edge", C.c_int32), ("tile", C.c_int32 * 3), ("ms_per_iter", C.c_float),
                ("status", C.c_int32)]


class Status(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("n_particles", C.c_int64), ("n_candidates", C.c_int64),
                ("n_accepted", C.c_int64), ("n_osc", C.c_int64), ("n_fixup", C.c_int64),
                ("mode_used", C.c_int32), ("converged", C.c_int32), ("mis_rounds", C.c_int32),
                ("error", C.c_int32), ("particles_total", C.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class State(C.Structure):
    _fields_ = [("t", C.c_int64), ("best_A", C.c_int64), ("t_best", C.c_int64),
                ("mode", C.c_int32), ("converged", C.c_int32)]


class ParticleBuffers(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("idx", "l", "c", "dE", "eE", "g", "eg", "key", "flags")]


# every function the header declares: (name, restype, argtypes)
_P, _V = C.POINTER, C.c_void_p
SIGNATURES = [
    ("seg_estimate_bytes", C.c_int, [_P(Params), C.c_int32, _P(C.c_size_t)]),
    ("seg_autotune", C.c_int, [_P(Params), _V, _V, C.c_int32, _V, _P(Params), _P(TuneEntry), C.c_int32,
                               _P(C.c_int32)]),
    ("seg_init", C.c_int, [_P(Params), _V, _V, _V, _P(_V)]),
    ("seg_set_psf", C.c_int, [_V, _P(C.c_double), C.c_int32]),
    ("seg_step", C.c_int, [_V, C.c_int32, _P(Status)]),
    ("seg_step_async", C.c_int, [_V, C.c_int32]),
    ("seg_poll", C.c_int, [_V, _P(Status)]),
    ("seg_profile", C.c_int, [_V, C.c_int32]),
    ("seg_stage_times", C.c_int, [_V, _P(C.c_float), C.c_int32]),
    ("seg_labels", C.c_int, [_V, _V, C.c_size_t]),
    ("seg_particles", C.c_int, [_V, _P(ParticleBuffers), C.c_int64, _P(C.c_int64)]),
    ("seg_stats", C.c_int, [_V, _V, _V, _V, C.c_int32]),
    ("seg_get_state", C.c_int, [_V, _P(State)]),
    ("seg_set_state", C.c_int, [_V, _P(State)]),
    ("seg_info", C.c_int, [_V, _P(C.c_int32), _V]),
    ("seg_destroy", None, [_V]),
    ("seg_batch_create", C.c_int, [_V, _P(_V)]),
    ("seg_batch_add", C.c_int, [_V, _V]),
    ("seg_batch_remove", C.c_int, [_V, _V]),
    ("seg_batch_size", C.c_int, [_V]),
    ("seg_batch_step", C.c_int, [_V, C.c_int32, _V, C.c_int32]),
    ("seg_batch_step_async", C.c_int, [_V, C.c_int32]),
    ("seg_batch_profile", C.c_int, [_V, C.c_int32]),
    ("seg_batch_stage_times", C.c_int, [_V, _P(C.c_float), C.c_int32]),
    ("seg_kernel_launches", C.c_int, [_P(C.c_uint64)]),
    ("seg_batch_poll", C.c_int, [_V, _V, C.c_int32]),
    ("seg_batch_destroy", None, [_V]),
    ("seg_region_stats_noalloc", C.c_int, [C.c_int32, C.c_int64, _V, _V, C.c_int32, _V, _V, _V, _V]),
    ("seg_debug_simple", C.c_int, [C.c_int32, _V, C.c_int32, _V]),
    ("seg_debug_inject", C.c_int, [_V, C.c_int32]),
    ("seg_strerror", C.c_char_p, [C.c_int]),
    ("seg_last_cuda_error", C.c_char_p, []),
]

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libseg.so from the package's build directory (built by __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libseg is not built ({path} missing): run __graft_entry__.build()")
            L = C.CDLL(path)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class SegError(RuntimeError):
    def __init__(self, code: int, what: str):
        L = lib()
        msg = f"{what}: {L.seg_strerror(code).decode()} ({code})"
        cu = L.seg_last_cuda_error().decode()
        if cu:
            msg += f" [{cu}]"
        super().__init__(msg)
        self.code = code


def _check(code: int, what: str):
    if code != SEG_OK:
        raise SegError(code, what)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keepalive) of a numpy array or a torch tensor (host or CUDA)."""
    if _is_torch(x):
        if not x.is_contiguous():
            x = x.contiguous()
        return C.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x)
    return a.ctypes.data_as(C.c_void_p), a


def _dtype_code(x) -> int:
    name = str(x.dtype)
    if name.endswith("float32"):
        return SEG_F32
    if name.endswith("uint16"):
        return SEG_U16
    raise ValueError(f"image dtype {x.dtype} not supported (float32 or uint16)")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def make_params(image, model="pc", connectivity=None, lam=0.0, cutoff=3.0, ps_radius=0.0,
                gradient="sobolev", osc_window=0, validate=False, cell_edge=0, tile=None, stats="exact",
                topology=0, max_labels=0, curv_radius=0.0) -> Params:
    shape = tuple(int(s) for s in image.shape)
    p = Params()
    p.ndim = len(shape)
    p.dtype = _dtype_code(image)
    p.shape[0], p.shape[1], p.shape[2] = (1,) + shape if len(shape) == 2 else shape
    p.model = model if isinstance(model, int) else MODELS[model]
    p.connectivity = connectivity or (4 if len(shape) == 2 else 6)
    p.lam = float(lam)
    p.cutoff = float(cutoff)
    p.ps_radius = float(ps_radius)
    p.gradient = gradient if isinstance(gradient, int) else {"sobolev": SEG_SOBOLEV, "l2": SEG_L2,
                                                                  "sobolev_global": SEG_SOBOLEV_GLOBAL}[gradient]
    p.osc_window = int(osc_window)
    p.stats_mode = stats if isinstance(stats, int) else STATS_MODES[stats]
    p.topology = topology if isinstance(topology, int) else TOPOLOGY[topology]
    p.max_labels = int(max_labels)
    # curvature regulariser (SEG_REG_CURVATURE) when a ball radius is given, else the length prior
    p.regulariser = SEG_REG_CURVATURE if curv_radius > 0 else SEG_REG_LENGTH
    p.curv_radius = float(curv_radius)
    p.validate = int(bool(validate))
    p.cell_edge = int(cell_edge)
    if tile is not None:
        t = [int(v) for v in tile]
        t = [0] * (3 - len(t)) + t          # (y, x) in 2D
        p.tile[0], p.tile[1], p.tile[2] = t
    return p


def autotune(image, labels0, iters: int = 10, stream=None, **kw):
    """Time the cell-edge x tile-shape candidates of seg_autotune on this job; returns
    (best keyword arguments for Context, [(cell_edge, tile, ms_per_iter, status), ...])."""
    params = make_params(image, **kw)
    ip, ikeep = _ptr(image)
    lp, lkeep = _ptr(labels0 if _is_torch(labels0) else np.asarray(labels0, dtype=np.int32))
    best = Params()
    entries = (TuneEntry * 16)()
    n = C.c_int32(0)
    _check(lib().seg_autotune(C.byref(params), ip, lp, int(iters), _stream_handle(stream), C.byref(best), entries, 16,
                              C.byref(n)), "seg_autotune")
    table = [(int(e.cell_edge), tuple(int(v) for v in e.tile), float(e.ms_per_iter), int(e.status))
             for e in entries[:n.value]]
    out = dict(kw)
    out["cell_edge"] = int(best.cell_edge)
    out["tile"] = tuple(int(v) for v in best.tile)
    return out, table


def estimate_bytes(params: Params, nlabels: int) -> int:
    out = C.c_size_t(0)
    _check(lib().seg_estimate_bytes(C.byref(params), int(nlabels), C.byref(out)), "seg_estimate_bytes")
    return int(out.value)


class Context:
    """One segmentation job resident on the GPU (seg_init ... seg_destroy)."""

    def __init__(self, image, labels0, model="pc", connectivity=None, lam=0.0, cutoff=3.0, ps_radius=0.0,
                 gradient="sobolev", osc_window=0, validate=False, cell_edge=0, tile=None, stream=None,
                 psf=None, stats="exact", topology=0, max_labels=0, curv_radius=0.0):
        self.params = make_params(image, model, connectivity, lam, cutoff, ps_radius, gradient, osc_window,
                                  validate, cell_edge, tile, stats, topology, max_labels, curv_radius)
        self.shape = tuple(int(s) for s in image.shape)
        ip, ikeep = _ptr(image)
        lp, lkeep = _ptr(labels0 if _is_torch(labels0) else np.asarray(labels0, dtype=np.int32))
        if _is_torch(labels0) and str(labels0.dtype) != "torch.int32":
            raise ValueError("labels0 must be int32")
        h = C.c_void_p()
        _check(lib().seg_init(C.byref(self.params), ip, lp, _stream_handle(stream), C.byref(h)), "seg_init")
        self._h = h
        self.npix = int(np.prod(self.shape))
        if psf is not None:
            try:
                self.set_psf(psf)
            except Exception:
                self.close()
                raise

    def set_psf(self, psf):
        """Deconvolving model: the symmetric 1D PSF profile, 2r+1 taps (seg_set_psf)."""
        k = np.ascontiguousarray(psf, dtype=np.float64).reshape(-1)
        if k.size % 2 != 1:
            raise ValueError("the PSF profile needs an odd number of taps")
        _check(lib().seg_set_psf(self.handle, k.ctypes.data_as(C.POINTER(C.c_double)), (k.size - 1) // 2),
               "seg_set_psf")

    @classmethod
    def from_workload(cls, w, **kw) -> "Context":
        args = dict(model=w.model, connectivity=w.connectivity, lam=w.lam, cutoff=w.cutoff,
                    ps_radius=w.ps_radius, psf=getattr(w, "psf", None))
        args.update(kw)
        return cls(w.image, w.labels0, **args)

    @property
    def nlabels(self) -> int:
        """Labels in use (grows when regions split, SEG_TOPO_SPLIT)."""
        nl = C.c_int32(0)
        _check(lib().seg_info(self.handle, C.byref(nl), None), "seg_info")
        return int(nl.value)

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("context destroyed")
        return self._h

    def step(self, iters: int = 1) -> dict:
        st = Status()
        _check(lib().seg_step(self.handle, int(iters), C.byref(st)), "seg_step")
        return st.as_dict()

    def step_async(self, iters: int = 1):
        _check(lib().seg_step_async(self.handle, int(iters)), "seg_step_async")

    def poll(self) -> dict:
        st = Status()
        _check(lib().seg_poll(self.handle, C.byref(st)), "seg_poll")
        return st.as_dict()

    STAGES = ("psf", "extract", "sobolev", "select", "lists", "fixup", "rounds", "moves", "finish")

    def inject(self, what: int):
        """Test-only fault injection (seg_debug_inject)."""
        _check(lib().seg_debug_inject(self.handle, int(what)), "seg_debug_inject")

    def profile(self, on: bool = True):
        _check(lib().seg_profile(self.handle, int(bool(on))), "seg_profile")

    def stage_times(self) -> dict:
        ms = (C.c_float * len(self.STAGES))()
        _check(lib().seg_stage_times(self.handle, ms, len(self.STAGES)), "seg_stage_times")
        return {k: float(ms[i]) for i, k in enumerate(self.STAGES)}

    def labels(self, out=None):
        if out is None:
            out = np.empty(self.shape, np.int32)
        p, keep = _ptr(out)
        _check(lib().seg_labels(self.handle, p, self.npix), "seg_labels")
        return out

    def particles(self) -> dict:
        n = C.c_int64(0)
        b = ParticleBuffers()
        _check(lib().seg_particles(self.handle, C.byref(b), 0, C.byref(n)), "seg_particles")
        N = int(n.value)
        out = {"idx": np.empty(N, np.uint32), "l": np.empty(N, np.int32), "c": np.empty(N, np.int32),
               "dE": np.empty(N, np.float32), "eE": np.empty(N, np.float32), "g": np.empty(N, np.float32),
               "eg": np.empty(N, np.float32), "key": np.empty(N, np.float64), "flags": np.empty(N, np.uint8)}
        for k, a in out.items():
            setattr(b, k, a.ctypes.data_as(C.c_void_p))
        _check(lib().seg_particles(self.handle, C.byref(b), N, C.byref(n)), "seg_particles")
        return out

    def stats(self, max_labels: int | None = None):
        M = self.nlabels if max_labels is None else int(max_labels)
        n, S, Q = np.zeros(M, np.int64), np.zeros(M, np.float64), np.zeros(M, np.float64)
        _check(lib().seg_stats(self.handle, n.ctypes.data_as(C.c_void_p), S.ctypes.data_as(C.c_void_p),
                               Q.ctypes.data_as(C.c_void_p), M), "seg_stats")
        return n, S, Q

    def get_state(self) -> dict:
        s = State()
        _check(lib().seg_get_state(self.handle, C.byref(s)), "seg_get_state")
        return {k: int(getattr(s, k)) for k, _ in State._fields_}

    def set_state(self, state: dict):
        s = State(**{k: int(state[k]) for k, _ in State._fields_})
        _check(lib().seg_set_state(self.handle, C.byref(s)), "seg_set_state")

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().seg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Contexts stepped together: one launch per stage for all of them."""

    def __init__(self, stream=None):
        h = C.c_void_p()
        _check(lib().seg_batch_create(_stream_handle(stream), C.byref(h)), "seg_batch_create")
        self._h = h
        self.members: list[Context] = []

    def add(self, ctx: Context):
        _check(lib().seg_batch_add(self._h, ctx.handle), "seg_batch_add")
        self.members.append(ctx)

    def remove(self, ctx: Context):
        _check(lib().seg_batch_remove(self._h, ctx.handle), "seg_batch_remove")
        self.members.remove(ctx)

    def __len__(self):
        return int(lib().seg_batch_size(self._h))

    def step(self, iters: int = 1) -> list[dict]:
        n = len(self.members)
        st = (Status * max(n, 1))()
        _check(lib().seg_batch_step(self._h, int(iters), C.cast(st, C.c_void_p), n), "seg_batch_step")
        return [st[i].as_dict() for i in range(n)]

    def step_async(self, iters: int = 1):
        _check(lib().seg_batch_step_async(self._h, int(iters)), "seg_batch_step_async")

    def poll(self) -> list[dict]:
        n = len(self.members)
        st = (Status * max(n, 1))()
        _check(lib().seg_batch_poll(self._h, C.cast(st, C.c_void_p), n), "seg_batch_poll")
        return [st[i].as_dict() for i in range(n)]

    def profile(self, on: bool = True):
        _check(lib().seg_batch_profile(self._h, int(bool(on))), "seg_batch_profile")

    def stage_times(self) -> dict:
        ms = (C.c_float * len(Context.STAGES))()
        _check(lib().seg_batch_stage_times(self._h, ms, len(Context.STAGES)), "seg_batch_stage_times")
        return {k: float(ms[i]) for i, k in enumerate(Context.STAGES)}

    def close(self):
        if getattr(self, "_h", None) is not None:
            lib().seg_batch_destroy(self._h)
            self._h = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    """Kernels libseg has launched in this process (graph replays count each of their kernels)."""
    out = C.c_uint64(0)
    _check(lib().seg_kernel_launches(C.byref(out)), "seg_kernel_launches")
    return int(out.value)


def debug_simple(ndim: int, masks) -> np.ndarray:
    m = np.ascontiguousarray(masks, dtype=np.uint32)
    out = np.zeros(m.size, np.uint8)
    _check(lib().seg_debug_simple(int(ndim), m.ctypes.data_as(C.c_void_p), m.size,
                                  out.ctypes.data_as(C.c_void_p)), "seg_debug_simple")
    return out


def region_stats_noalloc(image, labels, nlabels: int, n=None, S=None, Q=None, stream=None):
    """Exact region statistics through the allocation-free entry point.

    image (float32 or uint16) and labels (int32, as many elements as image) are CUDA tensors
    on one device; n, S, Q (int64 / float64 CUDA tensors of nlabels elements on that device)
    are allocated here by torch when not given, since the library allocates nothing. The work
    is ordered on `stream`, by default the current torch stream of the image's device.
    Returns (n, S, Q)."""
    import torch
    if not (torch.is_tensor(image) and torch.is_tensor(labels) and image.is_cuda and labels.is_cuda):
        raise ValueError("image and labels must be CUDA tensors")
    dev = image.device
    if labels.device != dev:
        raise ValueError("image and labels must be on one device")
    if labels.dtype != torch.int32:
        raise ValueError(f"labels must be int32, not {labels.dtype}")
    if labels.numel() != image.numel():
        raise ValueError(f"labels has {labels.numel()} elements, the image {image.numel()}")
    _dtype_code(image)
    want = {"n": torch.int64, "S": torch.float64, "Q": torch.float64}
    outs = {"n": n, "S": S, "Q": Q}
    for k, t in outs.items():
        if t is None:
            outs[k] = torch.empty(nlabels, dtype=want[k], device=dev)
        elif not (torch.is_tensor(t) and t.device == dev and t.dtype == want[k] and t.numel() == nlabels
                  and t.is_contiguous()):
            raise ValueError(f"{k} must be a contiguous {want[k]} tensor of {nlabels} elements on {dev}")
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    ip, ikeep = _ptr(image)
    lp, lkeep = _ptr(labels)
    code = lib().seg_region_stats_noalloc(_dtype_code(image), int(image.numel()), ip, lp, int(nlabels),
                                          C.c_void_p(outs["n"].data_ptr()), C.c_void_p(outs["S"].data_ptr()),
                                          C.c_void_p(outs["Q"].data_ptr()), _stream_handle(stream))
    del ikeep, lkeep                              # the call has returned: the copies may go
    _check(code, "seg_region_stats_noalloc")
    return outs["n"], outs["S"], outs["Q"]
