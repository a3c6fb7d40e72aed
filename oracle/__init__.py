"""CPU oracle of particle region competition with Sobolev gradients (arXiv:1403.0240).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use this package; the product path never does. It wraps the
plain single-threaded FP64 C implementation in ``rc_oracle.c`` (see its header for the
readings of the paper and for which test pins each function).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "rc_oracle.c")]
_HDR = os.path.join(_HERE, "rc_oracle.h")
_lock = threading.Lock()
_lib = None

F32, U16 = 0, 1
PC, PS, PSP, PCD = 0, 1, 2, 3
SOBOLEV, L2, SOBOLEV_GLOBAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no fused multiply-add)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + [_HDR])
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Params(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("dtype", C.c_int32),
                ("D", C.c_int64), ("H", C.c_int64), ("W", C.c_int64),
                ("model", C.c_int32), ("conn", C.c_int32),
                ("lam", C.c_double), ("cutoff", C.c_double), ("ps_radius", C.c_double),
                ("gradient", C.c_int32), ("osc_window", C.c_int32),
                ("nlabels", C.c_int32), ("pad_", C.c_int32), ("mu_floor", C.c_double),
                ("psf_r", C.c_int32), ("topology", C.c_int32), ("psf", C.c_void_p),
                ("regulariser", C.c_int32), ("pad2_", C.c_int32), ("curv_radius", C.c_double)]


class State(C.Structure):
    _fields_ = [("mode", C.c_int32), ("converged", C.c_int32), ("t", C.c_int64),
                ("best_A", C.c_int64), ("t_best", C.c_int64), ("nlabels", C.c_int32), ("pad_", C.c_int32)]


class Dump(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("idx", "l", "c", "dE", "g", "dE_terms", "g_terms")]


class Status(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("n_candidates", C.c_int64),
                ("n_accepted", C.c_int64), ("n_osc", C.c_int64),
                ("mode_used", C.c_int32), ("converged", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            vp = C.c_void_p
            L.orc_kernel_eq5.restype = C.c_double
            L.orc_kernel_eq5.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_extract.restype = C.c_int64
            L.orc_extract.argtypes = [P(Params), vp, vp, vp, vp, C.c_int64]
            L.orc_exact_sum_f32.restype = C.c_double
            L.orc_exact_sum_f32.argtypes = [vp, C.c_int64, C.c_int]
            L.orc_stats.restype = None
            L.orc_stats.argtypes = [P(Params), vp, vp, vp, vp, vp]
            L.orc_energy.restype = None
            L.orc_energy.argtypes = [P(Params), vp, vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp]
            L.orc_delta_perimeter.restype = C.c_int64
            L.orc_delta_perimeter.argtypes = [P(Params), vp, C.c_uint32, C.c_int32, C.c_int32]
            L.orc_ball_balance.restype = C.c_int64
            L.orc_ball_balance.argtypes = [P(Params), vp, C.c_uint32, C.c_int32, C.c_int32]
            L.orc_curvature_weight.restype = C.c_double
            L.orc_curvature_weight.argtypes = [P(Params)]
            L.orc_fuse_pairs.restype = C.c_int64
            L.orc_fuse_pairs.argtypes = [P(Params), vp, vp, vp, vp, C.c_int64]
            L.orc_fuse_energy.restype = C.c_double
            L.orc_fuse_energy.argtypes = [P(Params), vp, vp, C.c_int32, C.c_int32, C.c_int64]
            L.orc_fuse.restype = C.c_int64
            L.orc_fuse.argtypes = [P(Params), vp, vp]
            L.orc_sobolev.restype = None
            L.orc_sobolev.argtypes = [P(Params), C.c_int64, vp, vp, vp, vp, C.c_int, vp, vp, vp, vp, vp, vp]
            L.orc_simple_2d.restype = C.c_int
            L.orc_simple_2d.argtypes = [vp]
            L.orc_simple_3d.restype = C.c_int
            L.orc_simple_3d.argtypes = [vp]
            L.orc_admissible.restype = C.c_int
            L.orc_admissible.argtypes = [P(Params), vp, C.c_uint32, C.c_int32, C.c_int32]
            L.orc_relabel.restype = C.c_int32
            L.orc_relabel.argtypes = [P(Params), vp, C.c_int32]
            L.orc_select.restype = C.c_int64
            L.orc_select.argtypes = [P(Params), vp, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
            L.orc_psf_correlate.restype = None
            L.orc_psf_correlate.argtypes = [P(Params), vp, vp]
            L.orc_deconv_fields.restype = None
            L.orc_deconv_fields.argtypes = [P(Params), vp, vp, vp, vp, vp, vp, vp]
            L.orc_psf_norm2.restype = C.c_double
            L.orc_psf_norm2.argtypes = [P(Params), C.c_int64, C.c_int64, C.c_int64]
            L.orc_log.restype = C.c_double
            L.orc_log.argtypes = [C.c_double]
            L.orc_perimeter.restype = C.c_int64
            L.orc_perimeter.argtypes = [P(Params), vp]
            L.orc_state_init.restype = None
            L.orc_state_init.argtypes = [P(Params), P(State)]
            L.orc_advance_mode.restype = None
            L.orc_advance_mode.argtypes = [P(Params), P(State), C.c_int32, C.c_int64]
            L.orc_iterate.restype = C.c_int
            L.orc_iterate.argtypes = [P(Params), vp, vp, P(State), P(Status), C.c_int64, P(Dump)]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_params(image: np.ndarray, labels: np.ndarray, model: str | int = "pc", connectivity: int | None = None,
                lam: float = 0.0, cutoff: float = 3.0, ps_radius: float = 0.0,
                gradient: str | int = "sobolev", osc_window: int = 0, nlabels: int | None = None,
                psf: np.ndarray | None = None, topology: int = 0, curv_radius: float = 0.0) -> Params:
    shape = image.shape
    if image.ndim == 2:
        D, H, W = 1, shape[0], shape[1]
    else:
        D, H, W = shape
    p = Params()
    p.ndim = image.ndim
    p.dtype = F32 if image.dtype == np.float32 else U16
    p.D, p.H, p.W = D, H, W
    p.model = model if isinstance(model, int) else {"pc": PC, "ps": PS, "psp": PSP, "pcd": PCD}[model]
    p.conn = connectivity or (4 if image.ndim == 2 else 6)
    p.lam = float(lam)
    p.cutoff = float(cutoff)
    p.ps_radius = float(ps_radius)
    p.gradient = gradient if isinstance(gradient, int) else {"sobolev": SOBOLEV, "l2": L2,
                                                             "sobolev_global": SOBOLEV_GLOBAL}[gradient]
    p.osc_window = int(osc_window)
    p.nlabels = int(nlabels if nlabels is not None else int(labels.max()) + 1)
    # Poisson model: local means are floored at 2^-20 of the largest intensity (at least 2^-20)
    p.mu_floor = math.ldexp(max(1.0, float(np.abs(image).max()) if image.size else 1.0), -20)
    set_psf(p, psf)
    p.topology = int(topology)
    # curvature regulariser when a ball radius is given, else the length prior
    p.regulariser = 1 if curv_radius > 0 else 0
    p.curv_radius = float(curv_radius)
    return p


def set_psf(p: Params, psf: np.ndarray | None):
    """Attach the 2r+1 taps of the deconvolving model's PSF profile (kept alive on p)."""
    if psf is None:
        p.psf_r, p.psf = 0, None
        p._psf = None
        return
    k = np.ascontiguousarray(psf, dtype=np.float64).reshape(-1)
    if k.size % 2 != 1:
        raise ValueError("the PSF profile needs an odd number of taps")
    p._psf = k
    p.psf_r = (k.size - 1) // 2
    p.psf = k.ctypes.data


def psf_correlate(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    lib().orc_psf_correlate(C.byref(p), _ptr(f), _ptr(out))
    return out


def deconv_fields(p: Params, I: np.ndarray, L: np.ndarray, n=None, S=None):
    """(J, R, G) of the deconvolving model for labels L (theta = region means)."""
    I = np.ascontiguousarray(I)
    L = np.ascontiguousarray(L, dtype=np.int32)
    if n is None:
        n, S, _ = stats(p, I, L)
    J, R, G = (np.zeros(L.shape, np.float64) for _ in range(3))
    lib().orc_deconv_fields(C.byref(p), _ptr(I), _ptr(L), _ptr(np.ascontiguousarray(n, np.int64)),
                            _ptr(np.ascontiguousarray(S, np.float64)), _ptr(J), _ptr(R), _ptr(G))
    return J, R, G


def psf_norm2(p: Params, z: int, y: int, x: int) -> float:
    return lib().orc_psf_norm2(C.byref(p), z, y, x)


def log(x: float) -> float:
    return lib().orc_log(x)


def kernel_eq5(r: float, E: float, eps: float = 1.0 / 24.0) -> float:
    return lib().orc_kernel_eq5(r, E, eps)


def extract(p: Params, L: np.ndarray):
    L = np.ascontiguousarray(L, dtype=np.int32)
    n = lib().orc_extract(C.byref(p), _ptr(L), None, None, None, 0)
    idx = np.zeros(n, np.uint32)
    l = np.zeros(n, np.int32)
    c = np.zeros(n, np.int32)
    lib().orc_extract(C.byref(p), _ptr(L), _ptr(idx), _ptr(l), _ptr(c), n)
    return idx, l, c


def exact_sum_f32(v: np.ndarray, squares: bool = False) -> float:
    v = np.ascontiguousarray(v, dtype=np.float32).reshape(-1)
    return lib().orc_exact_sum_f32(_ptr(v), v.size, int(squares))


def stats(p: Params, I: np.ndarray, L: np.ndarray):
    I = np.ascontiguousarray(I)
    L = np.ascontiguousarray(L, dtype=np.int32)
    M = p.nlabels
    n = np.zeros(M, np.int64)
    S = np.zeros(M, np.float64)
    Q = np.zeros(M, np.float64)
    lib().orc_stats(C.byref(p), _ptr(I), _ptr(L), _ptr(n), _ptr(S), _ptr(Q))
    return n, S, Q


def energy(p: Params, I: np.ndarray, L: np.ndarray, idx, l, c, n=None, S=None, with_terms: bool = False):
    """dE of every particle; with_terms also returns each dE's sum of term magnitudes."""
    I = np.ascontiguousarray(I)
    L = np.ascontiguousarray(L, dtype=np.int32)
    if n is None:
        n, S, _ = stats(p, I, L)
    idx = np.ascontiguousarray(idx, np.uint32)
    l = np.ascontiguousarray(l, np.int32)
    c = np.ascontiguousarray(c, np.int32)
    dE = np.zeros(idx.size, np.float64)
    sc = np.zeros(idx.size, np.float64)
    lib().orc_energy(C.byref(p), _ptr(I), _ptr(L), _ptr(np.ascontiguousarray(n, np.int64)),
                     _ptr(np.ascontiguousarray(S, np.float64)), idx.size, _ptr(idx), _ptr(l), _ptr(c), _ptr(dE),
                     _ptr(sc))
    return (dE, sc) if with_terms else dE


def delta_perimeter(p: Params, L: np.ndarray, x: int, l: int, c: int) -> int:
    L = np.ascontiguousarray(L, dtype=np.int32)
    return lib().orc_delta_perimeter(C.byref(p), _ptr(L), x, l, c)


def ball_balance(p: Params, L: np.ndarray, x: int, l: int, c: int) -> int:
    """Curvature regulariser: pixels of label l minus pixels of label c in the ball of radius
    p.curv_radius around pixel x."""
    L = np.ascontiguousarray(L, dtype=np.int32)
    return lib().orc_ball_balance(C.byref(p), _ptr(L), x, l, c)


def fuse_pairs(p: Params, L: np.ndarray):
    """Touching foreground label pairs (a < b) and their shared boundary pair counts B."""
    L = np.ascontiguousarray(L, dtype=np.int32)
    n = lib().orc_fuse_pairs(C.byref(p), _ptr(L), None, None, None, 0)
    a, b, B = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int64)
    lib().orc_fuse_pairs(C.byref(p), _ptr(L), _ptr(a), _ptr(b), _ptr(B), n)
    return a, b, B


def fuse_energy(p: Params, n, S, a: int, b: int, B: int) -> float:
    n = np.ascontiguousarray(n, np.int64)
    S = np.ascontiguousarray(S, np.float64)
    return lib().orc_fuse_energy(C.byref(p), _ptr(n), _ptr(S), a, b, B)


def fuse(p: Params, I: np.ndarray, L: np.ndarray) -> tuple[np.ndarray, int]:
    """One fusion pass (the label count of p must cover L); returns (new labels, fusions)."""
    L = np.ascontiguousarray(L, dtype=np.int32).copy()
    nf = lib().orc_fuse(C.byref(p), _ptr(np.ascontiguousarray(I)), _ptr(L))
    return L, int(nf)


def curvature_weight(p: Params) -> float:
    return lib().orc_curvature_weight(C.byref(p))


def perimeter(p: Params, L: np.ndarray) -> int:
    """|Gamma|: connectivity-adjacent pixel pairs with different labels."""
    L = np.ascontiguousarray(L, dtype=np.int32)
    return int(lib().orc_perimeter(C.byref(p), _ptr(L)))


def sobolev(p: Params, idx, l, c, dE, all_pairs: bool = False, with_terms: bool = False):
    """(g, A, B, |Q|, |Q'|) of Eq. 6; with_terms also returns each g's sum of term magnitudes."""
    idx = np.ascontiguousarray(idx, np.uint32)
    l = np.ascontiguousarray(l, np.int32)
    c = np.ascontiguousarray(c, np.int32)
    dE = np.ascontiguousarray(dE, np.float64)
    N = idx.size
    g, A, B = (np.zeros(N, np.float64) for _ in range(3))
    nQ, nQp = np.zeros(N, np.int32), np.zeros(N, np.int32)
    terms = np.zeros(N, np.float64)
    lib().orc_sobolev(C.byref(p), N, _ptr(idx), _ptr(l), _ptr(c), _ptr(dE), int(all_pairs),
                      _ptr(g), _ptr(A), _ptr(B), _ptr(nQ), _ptr(nQp), _ptr(terms))
    return (g, A, B, nQ, nQp, terms) if with_terms else (g, A, B, nQ, nQp)


def simple_2d(nb9) -> bool:
    a = np.ascontiguousarray(np.asarray(nb9, np.uint8).reshape(9))
    return bool(lib().orc_simple_2d(_ptr(a)))


def simple_3d(nb27) -> bool:
    a = np.ascontiguousarray(np.asarray(nb27, np.uint8).reshape(27))
    return bool(lib().orc_simple_3d(_ptr(a)))


def admissible(p: Params, L: np.ndarray, x: int, l: int, c: int) -> bool:
    L = np.ascontiguousarray(L, dtype=np.int32)
    return bool(lib().orc_admissible(C.byref(p), _ptr(L), x, l, c))


def relabel(p: Params, L: np.ndarray, nlabels: int):
    """(labels, count) after giving split components new labels (topology 2)."""
    L = np.ascontiguousarray(L, dtype=np.int32).copy()
    n = lib().orc_relabel(C.byref(p), _ptr(L), int(nlabels))
    return L, int(n)


def select(p: Params, L: np.ndarray, idx, l, c, g):
    L = np.ascontiguousarray(L, dtype=np.int32)
    idx = np.ascontiguousarray(idx, np.uint32)
    l = np.ascontiguousarray(l, np.int32)
    c = np.ascontiguousarray(c, np.int32)
    g = np.ascontiguousarray(g, np.float64)
    N = idx.size
    acc_idx = np.zeros(max(N, 1), np.uint32)
    acc_c = np.zeros(max(N, 1), np.int32)
    ncand = C.c_int64(0)
    na = lib().orc_select(C.byref(p), _ptr(L), N, _ptr(idx), _ptr(l), _ptr(c), _ptr(g),
                          _ptr(acc_idx), _ptr(acc_c), C.byref(ncand))
    return acc_idx[:na].copy(), acc_c[:na].copy(), int(ncand.value)


def mode_sequence(osc_window: int, accepted, gradient: int = SOBOLEV):
    """Drive the mode and convergence rule with a given accepted-move count per iteration;
    returns (mode used, converged after) per iteration."""
    p = Params()
    p.gradient = gradient
    p.osc_window = int(osc_window)
    st = State()
    lib().orc_state_init(C.byref(p), C.byref(st))
    out = []
    for na in accepted:
        used = int(st.mode)
        if st.converged:
            st.t += 1
            out.append((used, 1))
            continue
        lib().orc_advance_mode(C.byref(p), C.byref(st), used, int(na))
        out.append((used, int(st.converged)))
    return out


class Run:
    """Iterates the oracle on its own copy of the label image."""

    def __init__(self, p: Params, image: np.ndarray, labels0: np.ndarray):
        self.p = p
        self.I = np.ascontiguousarray(image)
        self.L = np.ascontiguousarray(labels0, dtype=np.int32).copy()
        self.st = State()
        lib().orc_state_init(C.byref(p), C.byref(self.st))

    def step(self, dump: bool = False):
        s = Status()
        if not dump:
            lib().orc_iterate(C.byref(self.p), _ptr(self.I), _ptr(self.L), C.byref(self.st), C.byref(s), 0, None)
            return s.as_dict(), None
        L_before = self.L.copy()
        N = lib().orc_extract(C.byref(self.p), _ptr(L_before), None, None, None, 0)
        out = {"idx": np.zeros(N, np.uint32), "l": np.zeros(N, np.int32), "c": np.zeros(N, np.int32)}
        for k in ("dE", "g", "dE_terms", "g_terms"):
            out[k] = np.zeros(N, np.float64)
        d = Dump(**{k: out[k].ctypes.data_as(C.c_void_p) for k in out})
        lib().orc_iterate(C.byref(self.p), _ptr(self.I), _ptr(self.L), C.byref(self.st), C.byref(s), N,
                          C.byref(d))
        out["labels_before"] = L_before
        return s.as_dict(), out

    def state(self) -> dict:
        return {k: int(getattr(self.st, k)) for k, _ in State._fields_ if k != "pad_"}
