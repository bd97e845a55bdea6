"""ctypes wrapper around the sequential C oracle (``cd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline leg are its only callers.  It shares no code with the
CUDA library and never imports it.

Every function takes a symmetric CSR (``row_ptr`` int64[n+1], ``col`` int32,
``w`` integer or None for unit weights; a self-loop is stored once in its row)
as numpy arrays or torch CPU tensors.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cd_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

# stats layout (enum in cd_oracle.c)
STATS = ["levels", "sweeps", "moves", "colors0", "converged", "entries",
         "candidates", "decisions", "iters", "ncomm", "sweeps0", "entries0",
         "candidates0"]

MAX_SWEEPS = 256
MAX_LEVELS = 64
MAX_PLP_ITERS = 1000


def _compile(out: str, extra, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", *extra,
                               "-o", tmp, _SRC])
        os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable: no -march), and its
    OpenMP build beside it (same source, -fopenmp)."""
    _compile(_OUT_OMP, ["-fopenmp"], force)
    return _compile(_OUT, [], force)


def lib(threads: int = 1):
    """The sequential oracle (threads == 1) or its OpenMP build set to
    `threads` threads (0: the OpenMP default, all cores)."""
    omp = threads != 1
    with _lock:
        L = _libs.get(omp)
        if L is None:
            build()
            L = ctypes.CDLL(_OUT_OMP if omp else _OUT)
            P = ctypes.c_void_p
            i64, i32, dbl, u64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint64
            L.or_modularity.argtypes = [i64, P, P, P, P, P, P]
            L.or_gain.argtypes = [i64, P, P, P, P, i32, i32, i64, i64, P]
            L.or_color.argtypes = [i64, P, P, P, u64, P]
            L.or_color.restype = i32
            L.or_color_jp.argtypes = [i64, P, P, P, u64, P]
            L.or_color_jp.restype = i32
            L.or_move_phase.argtypes = [i64, P, P, P, u64, i32, ctypes.c_int, P, P]
            L.or_plm.argtypes = [i64, P, P, P, ctypes.c_int, u64, i32, i32, ctypes.c_int, i64, i64, P, P, P]
            L.or_plp.argtypes = [i64, P, P, P, u64, dbl, i32, ctypes.c_int, ctypes.c_int, P, P, P]
            L.or_combine.argtypes = [i64, ctypes.c_int, P, P]
            L.or_combine.restype = i64
            L.or_coarsen.argtypes = [i64, P, P, P, P, P, P, P, P]
            L.or_coarsen.restype = i64
            L.or_epp.argtypes = [i64, P, P, P, ctypes.c_int, ctypes.c_int, u64, i32, i32,
                                 dbl, i32, i64, i64, P, P, P, P, P]
            L.or_positive_moves.argtypes = [i64, P, P, P, P, i64, i64, P]
            L.or_epp_general.argtypes = [i64, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         u64, i32, i32, dbl, i32, i64, i64, P, P, P]
            L.or_positive_moves.restype = i64
            L.or_set_threads.argtypes = [ctypes.c_int]
            L.or_set_threads.restype = ctypes.c_int
            _libs[omp] = L
        if omp:
            L.or_set_threads(int(threads) if threads > 0 else (os.cpu_count() or 1))
    return L


def threads_used(threads: int) -> int:
    """Threads a parallel colour class of the given build runs on."""
    return 1 if threads == 1 else int(lib(threads).or_set_threads(0))


def _np(x, dtype):
    if x is None:
        return None
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _CSR:
    def __init__(self, row_ptr, col, w):
        self.rp = _np(row_ptr, np.int64)
        self.col = _np(col, np.int32)
        self.w = _np(w, np.int64)
        self.n = len(self.rp) - 1
        if len(self.col) == 0:   # keep a valid pointer
            self.col = np.zeros(1, np.int32)
            if self.w is not None:
                self.w = np.zeros(1, np.int64)

    def args(self):
        return (self.n, _ptr(self.rp), _ptr(self.col), _ptr(self.w))


def _i128(hi, lo):
    return (int(hi) << 64) | (int(lo) & ((1 << 64) - 1))


@dataclass
class Result:
    labels: np.ndarray
    modularity: float
    stats: dict


def _stats(a):
    return {k: int(v) for k, v in zip(STATS, a)}


def modularity(row_ptr, col, w, labels):
    """(mod, N, D): mod = N / D with N, D exact Python ints (Eq. 1 over 4W^2)."""
    g = _CSR(row_ptr, col, w)
    z = _np(labels, np.int32)
    out = ctypes.c_double()
    nd = np.zeros(4, np.int64)
    if lib().or_modularity(*g.args(), _ptr(z), ctypes.byref(out), _ptr(nd)):
        raise MemoryError
    return out.value, _i128(nd[0], nd[1]), _i128(nd[2], nd[3])


def gain(row_ptr, col, w, labels, u, D, resolution=(1, 1)):
    """Exact gain numerator g = 2W^2 q * Delta Q_gamma(u, labels[u] -> D) for
    the resolution gamma = p/q given as resolution = (p, q); (1, 1) is
    modularity, where g = 2W^2 * Delta mod."""
    g = _CSR(row_ptr, col, w)
    z = _np(labels, np.int32)
    out = np.zeros(2, np.int64)
    p, q = resolution
    if lib().or_gain(*g.args(), _ptr(z), int(u), int(D), int(p), int(q), _ptr(out)) == -2:
        raise ValueError("resolution must be p >= 0, q >= 1, max(p, q) (2W)^2 < 2^126")
    return _i128(out[0], out[1])


def color(row_ptr, col, w, seed):
    """(number of colours, colour per vertex) of the schedule's colouring."""
    g = _CSR(row_ptr, col, w)
    c = np.zeros(max(g.n, 1), np.int32)
    k = lib().or_color(*g.args(), seed, _ptr(c))
    return k, c[:g.n]


def color_jp(row_ptr, col, w, seed):
    """The same colouring computed by Jones-Plassmann rounds (small graphs)."""
    g = _CSR(row_ptr, col, w)
    c = np.zeros(max(g.n, 1), np.int32)
    k = lib().or_color_jp(*g.args(), seed, _ptr(c))
    return k, c[:g.n]


def move_phase(row_ptr, col, w, seed, labels=None, max_sweeps=MAX_SWEEPS, rev=False):
    g = _CSR(row_ptr, col, w)
    z = np.arange(g.n, dtype=np.int32) if labels is None else _np(labels, np.int32).copy()
    st = np.zeros(len(STATS), np.int64)
    lib().or_move_phase(*g.args(), seed, max_sweeps, int(rev), _ptr(z), _ptr(st))
    return z, _stats(st)


def plm(row_ptr, col, w, refine=False, seed=1, max_sweeps=MAX_SWEEPS,
        max_levels=MAX_LEVELS, rev=False, resolution=(1, 1), threads=1) -> Result:
    """PLM / PLMR.  resolution = (p, q): the moves maximise the objective with
    gamma = p/q scaling the volume term (Sec. III-B); the returned modularity
    is always the standard one (gamma = 1).  threads != 1 runs the OpenMP
    build (identical results)."""
    g = _CSR(row_ptr, col, w)
    z = np.zeros(max(g.n, 1), np.int32)
    mod = ctypes.c_double()
    st = np.zeros(len(STATS), np.int64)
    p, q = resolution
    rc = lib(threads).or_plm(*g.args(), int(refine), seed, max_sweeps, max_levels, int(rev), int(p), int(q),
                      _ptr(z), ctypes.byref(mod), _ptr(st))
    if rc == -2:
        raise ValueError("resolution must be p >= 0, q >= 1, max(p, q) (2W)^2 < 2^126")
    if rc:
        raise MemoryError
    return Result(z[:g.n], mod.value, _stats(st))


def plp(row_ptr, col, w, seed=1, theta=None, max_iter=MAX_PLP_ITERS,
        use_active=True, rev=False, threads=1) -> Result:
    g = _CSR(row_ptr, col, w)
    if theta is None:
        theta = g.n * 1e-5
    z = np.zeros(max(g.n, 1), np.int32)
    mod = ctypes.c_double()
    st = np.zeros(len(STATS), np.int64)
    if lib(threads).or_plp(*g.args(), seed, float(theta), max_iter, int(use_active), int(rev),
                    _ptr(z), ctypes.byref(mod), _ptr(st)):
        raise MemoryError
    return Result(z[:g.n], mod.value, _stats(st))


def combine(labels_list):
    """Exact core communities of several labellings (Eq. 2), dense ids."""
    L = np.ascontiguousarray(np.stack([_np(z, np.int32) for z in labels_list]))
    n = L.shape[1]
    core = np.zeros(max(n, 1), np.int32)
    k = lib().or_combine(n, L.shape[0], _ptr(L), _ptr(core))
    return int(k), core[:n]


def coarsen(row_ptr, col, w, labels):
    """(coarse row_ptr, col, w int64, pi) in input-CSR form."""
    g = _CSR(row_ptr, col, w)
    z = _np(labels, np.int32)
    nnz = len(g.col)
    rp = np.zeros(g.n + 1, np.int64)
    c = np.zeros(nnz + g.n + 1, np.int32)
    ww = np.zeros(nnz + g.n + 1, np.int64)
    pi = np.zeros(max(g.n, 1), np.int32)
    k = lib().or_coarsen(*g.args(), _ptr(z), _ptr(rp), _ptr(c), _ptr(ww), _ptr(pi))
    rp = rp[:k + 1]
    return rp, c[:rp[-1]], ww[:rp[-1]], pi[:g.n]


def epp(row_ptr, col, w, b=4, final_refine=True, seed=1, theta=None,
        max_sweeps=MAX_SWEEPS, max_levels=MAX_LEVELS, max_iter=MAX_PLP_ITERS,
        want_parts=False, threads=1, resolution=(1, 1)):
    g = _CSR(row_ptr, col, w)
    if theta is None:
        theta = g.n * 1e-5
    z = np.zeros(max(g.n, 1), np.int32)
    base = np.zeros(max(b * g.n, 1), np.int32) if want_parts else None
    core = np.zeros(max(g.n, 1), np.int32) if want_parts else None
    mod = ctypes.c_double()
    st = np.zeros(len(STATS), np.int64)
    p, q = resolution
    rc = lib(threads).or_epp(*g.args(), b, int(final_refine), seed, max_sweeps, max_levels,
                             float(theta), max_iter, int(p), int(q), _ptr(z), _ptr(base), _ptr(core),
                             ctypes.byref(mod), _ptr(st))
    if rc == -2:
        raise ValueError("resolution must be p >= 0, q >= 1, max(p, q) (2W)^2 < 2^126")
    if rc:
        raise MemoryError
    r = Result(z[:g.n], mod.value, _stats(st))
    if want_parts:
        return r, base[:b * g.n].reshape(b, g.n), core[:g.n]
    return r


BASE_PLP, BASE_PLM, BASE_PLMR = 0, 1, 2


def epp_general(row_ptr, col, w, b=4, base=BASE_PLP, final_refine=True, rounds=1, seed=1, theta=None,
                max_sweeps=MAX_SWEEPS, max_levels=MAX_LEVELS, max_iter=MAX_PLP_ITERS, resolution=(1, 1),
                threads=1) -> Result:
    """EPP(b, Base, Final) with up to `rounds` ensemble rounds (Section
    III-D; see or_epp_general).  stats["levels"] is the number of core
    graphs taken."""
    g = _CSR(row_ptr, col, w)
    if theta is None:
        theta = g.n * 1e-5
    z = np.zeros(max(g.n, 1), np.int32)
    mod = ctypes.c_double()
    st = np.zeros(len(STATS), np.int64)
    p, q = resolution
    rc = lib(threads).or_epp_general(*g.args(), int(b), int(base), int(final_refine), int(rounds), seed,
                                     max_sweeps, max_levels, float(theta), max_iter, int(p), int(q),
                                     _ptr(z), ctypes.byref(mod), _ptr(st))
    if rc == -2:
        raise ValueError("b >= 1, base in {0, 1, 2}, 1 <= rounds <= 64, valid resolution")
    if rc:
        raise MemoryError
    return Result(z[:g.n], mod.value, _stats(st))


def positive_moves(row_ptr, col, w, labels, resolution=(1, 1)):
    """Vertices with a positive-gain move under ``labels`` for the resolution
    gamma = p/q, resolution = (p, q) (0 at convergence)."""
    g = _CSR(row_ptr, col, w)
    z = _np(labels, np.int32)
    mg = np.zeros(2, np.int64)
    p, q = resolution
    k = int(lib().or_positive_moves(*g.args(), _ptr(z), int(p), int(q), _ptr(mg)))
    if k == -2:
        raise ValueError("resolution must be p >= 0, q >= 1, max(p, q) (2W)^2 < 2^126")
    return k
