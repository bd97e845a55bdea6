"""Python binding of the C ABI in include/cd.h (argument marshalling only).

Functions keep the C names (``cd_graph_create``, ``cd_plp``, ``cd_plm``,
``cd_epp``, ``cd_modularity``, ``cd_run_batch``, ``cd_server_submit``, ...).  Arrays may be torch tensors (CPU or CUDA)
or numpy arrays; CUDA tensors are passed as device pointers, everything else
as host pointers.  PyTorch supplies device memory and the CUDA stream; all
computation happens in libcdgpu.so.  If the library is not built, every call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ECUDA, CD_ENOTCONV, CD_EBUSY, CD_ETIMEOUT = range(7)
CD_MEM_HOST, CD_MEM_DEVICE = 0, 1
CD_ALGO_PLP, CD_ALGO_PLM, CD_ALGO_EPP = 0, 1, 2


class CDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "CD_OK", 1: "CD_EINVAL", 2: "CD_ENOMEM", 3: "CD_ECUDA", 4: "CD_ENOTCONV",
           5: "CD_EBUSY", 6: "CD_ETIMEOUT"}


class cd_opts(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("max_sweeps", ctypes.c_int32),
                ("max_levels", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("team_quantum", ctypes.c_int64),
                ("team_min", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("bin_max", ctypes.c_int32 * 5), ("res_num", ctypes.c_int64), ("res_den", ctypes.c_int64),
                ("schedule", ctypes.c_int32), ("int_path", ctypes.c_int32), ("scratch_budget", ctypes.c_int64)]


class cd_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("colors0", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("ncomm", ctypes.c_int32),
                ("sweeps", ctypes.c_int64), ("moves", ctypes.c_int64),
                ("iters", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("decisions", ctypes.c_int64),
                ("ms_color", ctypes.c_double), ("ms_move", ctypes.c_double),
                ("ms_coarsen", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("k_launches", ctypes.c_int64), ("k_ms", ctypes.c_double),
                ("k_bytes", ctypes.c_double), ("stage_items_ms", ctypes.c_double),
                ("stage_sort_ms", ctypes.c_double), ("stage_recheck_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class cd_task(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("refine", ctypes.c_int32), ("ensemble", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("theta", ctypes.c_double)]


def make_task(algo: int, refine: bool = False, ensemble: int = 1, theta: float = -1.0) -> cd_task:
    return cd_task(int(algo), int(refine), int(ensemble), 0, float(theta))


_lock = threading.Lock()
_lib = None

SYMBOLS = ["cd_opts_default", "cd_status_str", "cd_last_error", "cd_graph_create",
           "cd_graph_destroy", "cd_graph_info", "cd_modularity", "cd_plp", "cd_plm",
           "cd_epp", "cd_color", "cd_coarsen", "cd_graph_export", "cd_debug_fail_alloc",
           "cd_launch_count", "cd_modularity_static", "cd_run_batch", "cd_plm_batch",
           "cd_server_create", "cd_server_submit", "cd_server_poll", "cd_server_info",
           "cd_server_destroy", "cd_tune", "cd_debug_plan_launch", "cd_debug_class_trace", "cd_epp_general",
           "cd_memory_stats"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libcdgpu.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path} (run paper_1304_4453_gb300.build.build())")
            L = ctypes.CDLL(path)
            P, i64, i32, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
            L.cd_status_str.restype = ctypes.c_char_p
            L.cd_last_error.restype = ctypes.c_char_p
            L.cd_opts_default.argtypes = [P]
            L.cd_graph_create.argtypes = [i64, P, P, P, c_int, P, P]
            L.cd_graph_destroy.argtypes = [P]
            L.cd_graph_info.argtypes = [P, P, P, P]
            L.cd_modularity.argtypes = [P, P, c_int, P]
            L.cd_plp.argtypes = [P, P, ctypes.c_double, P, c_int, P, P]
            L.cd_plm.argtypes = [P, c_int, P, P, c_int, P, P]
            L.cd_epp.argtypes = [P, c_int, c_int, P, P, c_int, P, P]
            L.cd_epp_general.argtypes = [P, c_int, c_int, c_int, c_int, P, P, c_int, P, P]
            L.cd_memory_stats.argtypes = [P, P, P, c_int]
            L.cd_color.argtypes = [P, ctypes.c_uint64, P, c_int, P]
            L.cd_coarsen.argtypes = [P, P, c_int, P]
            L.cd_graph_export.argtypes = [P, P, P, P, c_int, P]
            L.cd_debug_fail_alloc.argtypes = [c_int]
            L.cd_debug_fail_alloc.restype = None
            L.cd_debug_plan_launch.argtypes = [P, c_int, i64, ctypes.c_int32, c_int, P, P, P, P]
            L.cd_debug_class_trace.argtypes = [P, i64, P]
            L.cd_modularity_static.argtypes = [i64, P, P, P, P, P, P]
            L.cd_run_batch.argtypes = [P, c_int, P, P, P, c_int, P, P, P]
            L.cd_plm_batch.argtypes = [P, c_int, c_int, P, P, c_int, P, P]
            L.cd_server_create.argtypes = [ctypes.c_size_t, c_int, c_int, P, P]
            L.cd_server_submit.argtypes = [P, P, P, P, P]
            L.cd_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.c_double, P, c_int, P, P, P]
            L.cd_server_info.argtypes = [P, P, P, P]
            L.cd_server_destroy.argtypes = [P]
            L.cd_tune.argtypes = [P, c_int, P, P, c_int, P, P, P]
            L.cd_launch_count.argtypes = []
            L.cd_launch_count.restype = ctypes.c_uint64
            for name in SYMBOLS:
                if name not in ("cd_status_str", "cd_last_error", "cd_opts_default", "cd_debug_fail_alloc",
                                "cd_launch_count"):
                    getattr(L, name).restype = c_int
            _lib = L
    return _lib


def _check(st: int, allow_notconv: bool = True) -> int:
    if st == CD_OK or (allow_notconv and st == CD_ENOTCONV):
        return st
    raise CDError(st, lib().cd_last_error().decode(errors="replace"))


def _arr(x, dtype):
    """(pointer, mem flag, keepalive) for a tensor / array / None."""
    if x is None:
        return None, CD_MEM_HOST, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            tdt = {np.int32: torch.int32, np.int64: torch.int64, np.float64: torch.float64}[dtype]
            if x.dtype != tdt or not x.is_contiguous():
                x = x.to(tdt).contiguous()
            return ctypes.c_void_p(x.data_ptr()), (CD_MEM_DEVICE if x.is_cuda else CD_MEM_HOST), x
    except ImportError:
        pass
    a = np.ascontiguousarray(np.asarray(x), dtype=dtype)
    return a.ctypes.data_as(ctypes.c_void_p), CD_MEM_HOST, a


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


RACY_ROUNDS = 128


def default_opts(seed: int = 1, max_sweeps: int = 256, max_levels: int = 64,
                 max_iters: int = 1000, profile: bool = False, team_quantum: int = 0,
                 team_min: int = 0, bin_max=None, resolution=(1, 1), racy=False,
                 scratch_budget: int = 0, int_path: int = 0) -> cd_opts:
    """Options; resolution = (p, q) is gamma = p / q of the PLM move gain;
    racy selects the paper's nondeterministic schedule (no colouring): True
    for RACY_ROUNDS hash rounds per sweep, or an int for that many."""
    o = cd_opts()
    lib().cd_opts_default(ctypes.byref(o))
    o.seed, o.max_sweeps, o.max_levels, o.max_iters, o.profile = seed, max_sweeps, max_levels, max_iters, int(profile)
    o.res_num, o.res_den = int(resolution[0]), int(resolution[1])
    o.schedule = (RACY_ROUNDS if racy is True else int(racy)) if racy else 0
    o.scratch_budget = int(scratch_budget)
    o.int_path = int(int_path)
    if team_quantum:
        o.team_quantum = team_quantum
    if team_min:
        o.team_min = team_min
    if bin_max is not None:
        for i, v in enumerate(bin_max):
            o.bin_max[i] = int(v)
    return o


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------

CD_BORROW = 2


def cd_graph_create(row_ptr, col, w=None, stream=None, borrow=False):
    """Returns an opaque handle (ctypes pointer).  All three arrays must live
    in the same memory (host or one CUDA device).  borrow=True (device arrays
    of the right dtypes only): the handle reads them in place; the caller
    keeps them alive and unchanged until the handle is destroyed."""
    rp, m1, k1 = _arr(row_ptr, np.int64)
    cp, m2, k2 = _arr(col, np.int32)
    wp, m3, k3 = _arr(w, np.int32)
    n = (k1.numel() if hasattr(k1, "numel") else len(k1)) - 1
    if w is not None and m3 != m1 or m2 != m1:
        raise CDError(CD_EINVAL, "row_ptr, col and w must live in the same memory")
    mem = m1
    if borrow:
        if m1 != CD_MEM_DEVICE or k1 is not row_ptr or k2 is not col or (w is not None and k3 is not w):
            raise CDError(CD_EINVAL, "borrow needs contiguous CUDA tensors of dtypes int64, int32, int32")
        mem = CD_BORROW
    h = ctypes.c_void_p()
    _check(lib().cd_graph_create(n, rp, cp, wp, mem, _stream(stream), ctypes.byref(h)), False)
    return h


def cd_graph_destroy(h):
    _check(lib().cd_graph_destroy(h), False)


def cd_graph_info(h):
    n, m, W = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cd_graph_info(h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(W)), False)
    return n.value, m.value, W.value


def cd_modularity(h, labels) -> float:
    lp, mem, keep = _arr(labels, np.int32)
    out = ctypes.c_double()
    _check(lib().cd_modularity(h, lp, mem, ctypes.byref(out)), False)
    return out.value


def _run(fn, h, args, labels_out):
    lp, mem, keep = _arr(labels_out, np.int32)
    mod = ctypes.c_double()
    st = cd_stats()
    status = fn(h, *args(lp, mem, ctypes.byref(mod), ctypes.byref(st)))
    _check(status)
    return mod.value, st.as_dict(), status


def cd_plp(h, labels_out, opts=None, theta: float = -1.0):
    o = opts or default_opts()
    return _run(lib().cd_plp, h, lambda lp, mem, mp, sp: (ctypes.byref(o), theta, lp, mem, mp, sp), labels_out)


def cd_plm(h, labels_out, refine: bool = False, opts=None):
    o = opts or default_opts()
    return _run(lib().cd_plm, h, lambda lp, mem, mp, sp: (int(refine), ctypes.byref(o), lp, mem, mp, sp),
                labels_out)


def cd_epp(h, labels_out, ensemble_size: int = 4, final_refine: bool = True, opts=None):
    o = opts or default_opts()
    return _run(lib().cd_epp, h,
                lambda lp, mem, mp, sp: (int(ensemble_size), int(final_refine), ctypes.byref(o), lp, mem, mp, sp),
                labels_out)


def cd_memory_stats(reset_high: bool = False):
    """(used, used_high, reserved) bytes of the library's device pool."""
    u, hgh, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().cd_memory_stats(ctypes.byref(u), ctypes.byref(hgh), ctypes.byref(r), int(reset_high)), False)
    return u.value, hgh.value, r.value


CD_BASE_PLP, CD_BASE_PLM, CD_BASE_PLMR = 0, 1, 2


def cd_epp_general(h, labels_out, ensemble_size: int = 4, base: int = CD_BASE_PLP, final_refine: bool = True,
                   rounds: int = 1, opts=None):
    o = opts or default_opts()
    return _run(lib().cd_epp_general, h,
                lambda lp, mem, mp, sp: (int(ensemble_size), int(base), int(final_refine), int(rounds),
                                         ctypes.byref(o), lp, mem, mp, sp),
                labels_out)


def cd_color(h, colors_out, seed: int = 1) -> int:
    cp, mem, keep = _arr(colors_out, np.int32)
    k = ctypes.c_int32()
    _check(lib().cd_color(h, seed, cp, mem, ctypes.byref(k)), False)
    return k.value


def cd_coarsen(h, labels):
    lp, mem, keep = _arr(labels, np.int32)
    out = ctypes.c_void_p()
    _check(lib().cd_coarsen(h, lp, mem, ctypes.byref(out)), False)
    return out


def cd_graph_export(h):
    """(row_ptr int64, col int32, w int64) numpy arrays in input form."""
    n, _, _ = cd_graph_info(h)
    nnz = ctypes.c_int64()
    _check(lib().cd_graph_export(h, None, None, None, CD_MEM_HOST, ctypes.byref(nnz)), False)
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(nnz.value, 1), np.int32)
    w = np.zeros(max(nnz.value, 1), np.int64)
    _check(lib().cd_graph_export(h, rp.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p),
                                 w.ctypes.data_as(ctypes.c_void_p), CD_MEM_HOST, ctypes.byref(nnz)), False)
    return rp, col[:nnz.value], w[:nnz.value]


def cd_debug_fail_alloc(k: int):
    lib().cd_debug_fail_alloc(int(k))


TRACE_FIELDS = ("phase", "sweep", "cls", "vertices", "entries", "hub_chunks", "hub_slices", "big_hubs", "ns",
                "items_end_ns", "decide_end_ns", "finisher_end_ns", "first_item_ns", "max_group_ns", "max_block_ns",
                "max_chunk_ns", "max_slice_wait_ns", "max_slice_ns", "moves_or_candidates")


def cd_debug_class_trace() -> np.ndarray:
    """Rows (one per class step, fields TRACE_FIELDS) of the move phases run
    with profile=2 since the last call; the library's trace is cleared."""
    cnt = ctypes.c_int64()
    _check(lib().cd_debug_class_trace(None, 0, ctypes.byref(cnt)), False)
    out = np.zeros((max(cnt.value, 1), len(TRACE_FIELDS)), np.int64)
    _check(lib().cd_debug_class_trace(out.ctypes.data, cnt.value, ctypes.byref(cnt)), False)
    return out[:cnt.value]


def cd_debug_plan_launch(work, team_quantum: int, team_min: int, grid_max: int):
    """The batch engine's launch planner on bare phase sizes (host only).
    Returns (grid, tiers, order): tiers as dicts of begin, blocks, team_size,
    team0, first, count; order lists the runs in tier order."""
    w = np.ascontiguousarray(np.asarray(work, dtype=np.int64))
    grid = ctypes.c_int32()
    nt = ctypes.c_int32()
    tiers = np.zeros(16 * 6, np.int32)
    order = np.zeros(len(w), np.int32)
    _check(lib().cd_debug_plan_launch(w.ctypes.data, len(w), int(team_quantum), int(team_min), int(grid_max),
                                      ctypes.byref(grid), ctypes.byref(nt), tiers.ctypes.data, order.ctypes.data),
           False)
    keys = ("begin", "blocks", "team_size", "team0", "first", "count")
    return grid.value, [dict(zip(keys, tiers[6 * i:6 * i + 6].tolist())) for i in range(nt.value)], order.tolist()


def cd_modularity_static(row_ptr, col, w, labels, stream=None) -> float:
    """Modularity through the allocation-free entry point: every array must be
    a CUDA tensor (the caller's device CSR and labels)."""
    rp, m1, k1 = _arr(row_ptr, np.int64)
    cp, m2, k2 = _arr(col, np.int32)
    wp, m3, k3 = _arr(w, np.int32)
    lp, m4, k4 = _arr(labels, np.int32)
    if CD_MEM_HOST in (m1, m2, m4) or (w is not None and m3 == CD_MEM_HOST):
        raise CDError(CD_EINVAL, "cd_modularity_static takes device arrays only")
    n = k1.numel() - 1
    out = ctypes.c_double()
    _check(lib().cd_modularity_static(n, rp, cp, wp, lp, _stream(stream), ctypes.byref(out)), False)
    return out.value


def _batch_args(handles, labels_list):
    if len(handles) != len(labels_list):
        raise CDError(CD_EINVAL, "one labels buffer per graph")
    count = len(handles)
    hs = (ctypes.c_void_p * max(count, 1))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    ptrs, mems, keep = [], set(), []
    for lab in labels_list:
        lp, mem, k = _arr(lab, np.int32)
        ptrs.append(lp.value if lp is not None else None)
        mems.add(mem)
        keep.append(k)
    if len(mems) > 1:
        raise CDError(CD_EINVAL, "labels must all live in the same memory")
    lps = (ctypes.c_void_p * max(count, 1))(*ptrs)
    return count, hs, lps, (mems.pop() if mems else CD_MEM_DEVICE), keep


def cd_run_batch(handles, task: cd_task, labels_list, opts=None, stream=None):
    """Runs ``task`` on every graph together.  Returns (mods, stats, status)."""
    o = opts or default_opts()
    count, hs, lps, mem, keep = _batch_args(handles, labels_list)
    mods = (ctypes.c_double * max(count, 1))()
    sts = (cd_stats * max(count, 1))()
    status = lib().cd_run_batch(hs, count, ctypes.byref(task), ctypes.byref(o), lps, mem, mods, sts,
                                _stream(stream))
    _check(status)
    return [mods[i] for i in range(count)], [sts[i].as_dict() for i in range(count)], status


def cd_plm_batch(handles, labels_list, refine: bool = False, opts=None):
    o = opts or default_opts()
    count, hs, lps, mem, keep = _batch_args(handles, labels_list)
    mods = (ctypes.c_double * max(count, 1))()
    sts = (cd_stats * max(count, 1))()
    status = lib().cd_plm_batch(hs, count, int(refine), ctypes.byref(o), lps, mem, mods, sts)
    _check(status)
    return [mods[i] for i in range(count)], [sts[i].as_dict() for i in range(count)], status


def cd_tune(handles, task: cd_task, opts=None, max_trials: int = 12, stream=None):
    """Returns (best cd_opts, its run time in ms)."""
    o = opts or default_opts()
    count = len(handles)
    hs = (ctypes.c_void_p * max(count, 1))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    best = cd_opts()
    ms = ctypes.c_double()
    _check(lib().cd_tune(hs, count, ctypes.byref(task), ctypes.byref(o), int(max_trials), ctypes.byref(best),
                         ctypes.byref(ms), _stream(stream)), False)
    return best, ms.value


def cd_server_create(device_mem_budget: int = 0, max_slots: int = 64, max_queue: int = 4096, stream=None):
    h = ctypes.c_void_p()
    st = _stream(stream) if stream is not None else ctypes.c_void_p(0)
    _check(lib().cd_server_create(int(device_mem_budget), int(max_slots), int(max_queue), st, ctypes.byref(h)),
           False)
    return h


def cd_server_submit(server, h, task: cd_task, opts=None) -> int:
    o = opts or default_opts()
    t = ctypes.c_uint64()
    _check(lib().cd_server_submit(server, h, ctypes.byref(task), ctypes.byref(o), ctypes.byref(t)), False)
    return t.value


def cd_server_poll(server, ticket: int, labels_out=None, timeout_ms: float = 0.0):
    """None while the run is queued or running, else (status, mod, latency_ms, stats)."""
    lp, mem, keep = _arr(labels_out, np.int32)
    mod, lat, st = ctypes.c_double(), ctypes.c_double(), cd_stats()
    status = lib().cd_server_poll(server, ctypes.c_uint64(ticket), float(timeout_ms), lp, mem, ctypes.byref(mod),
                                  ctypes.byref(lat), ctypes.byref(st))
    if status == CD_EBUSY:
        return None
    _check(status)
    return status, mod.value, lat.value, st.as_dict()


def cd_server_info(server):
    q, r, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().cd_server_info(server, ctypes.byref(q), ctypes.byref(r), ctypes.byref(f)), False)
    return q.value, r.value, f.value


def cd_server_destroy(server):
    _check(lib().cd_server_destroy(server), False)


def cd_launch_count() -> int:
    return int(lib().cd_launch_count())


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

@dataclass
class Result:
    labels: object
    modularity: float
    stats: dict
    status: int


class Graph:
    """Owns a cd_graph handle.  Results come back as torch tensors on the
    device of ``device`` (default cuda:0)."""

    def __init__(self, row_ptr, col, w=None, stream=None, borrow=False):
        self.h = cd_graph_create(row_ptr, col, w, stream, borrow)
        # a borrowed CSR must outlive the handle
        self._borrowed = (row_ptr, col, w) if borrow else None
        self.n, self.m, self.W = cd_graph_info(self.h)

    @classmethod
    def from_synth(cls, g, device=None, stream=None):
        if device is not None:
            g = g.to(device)
        return cls(g.row_ptr, g.col, g.w, stream)

    def close(self):
        if self.h is not None:
            cd_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, out):
        if out is not None:
            return out
        import torch
        return torch.empty(max(self.n, 1), dtype=torch.int32, device="cuda")[:self.n]

    def plm(self, refine=False, out=None, **kw) -> Result:
        out = self._out(out)
        mod, st, status = cd_plm(self.h, out, refine, default_opts(**kw))
        return Result(out, mod, st, status)

    def plp(self, out=None, theta=-1.0, **kw) -> Result:
        out = self._out(out)
        mod, st, status = cd_plp(self.h, out, default_opts(**kw), theta)
        return Result(out, mod, st, status)

    def epp(self, b=4, final_refine=True, out=None, **kw) -> Result:
        out = self._out(out)
        mod, st, status = cd_epp(self.h, out, b, final_refine, default_opts(**kw))
        return Result(out, mod, st, status)

    def epp_general(self, b=4, base=CD_BASE_PLP, final_refine=True, rounds=1, out=None, **kw) -> Result:
        out = self._out(out)
        mod, st, status = cd_epp_general(self.h, out, b, base, final_refine, rounds, default_opts(**kw))
        return Result(out, mod, st, status)

    def modularity(self, labels) -> float:
        return cd_modularity(self.h, labels)


def run_batch(graphs, algo: int = CD_ALGO_PLM, refine: bool = False, ensemble: int = 1, theta: float = -1.0,
              outs=None, stream=None, **kw):
    """Runs one task on many ``Graph`` objects in one batched call; returns a
    list of ``Result`` (labels as CUDA tensors unless ``outs`` is given)."""
    outs = outs if outs is not None else [g._out(None) for g in graphs]
    mods, sts, status = cd_run_batch([g.h for g in graphs], make_task(algo, refine, ensemble, theta), outs,
                                     default_opts(**kw), stream)
    return [Result(o, m, s, status) for o, m, s in zip(outs, mods, sts)]


class Server:
    """Continuous-batching server (cd_server_*).  Submitted graphs must stay
    alive until their result is taken."""

    def __init__(self, device_mem_budget: int = 0, max_slots: int = 64, max_queue: int = 4096, stream=None):
        self.h = cd_server_create(device_mem_budget, max_slots, max_queue, stream)

    def submit(self, graph: "Graph", algo: int = CD_ALGO_PLM, refine: bool = False, ensemble: int = 1,
               theta: float = -1.0, **kw) -> int:
        return cd_server_submit(self.h, graph.h, make_task(algo, refine, ensemble, theta), default_opts(**kw))

    def poll(self, ticket: int, out=None, timeout_ms: float = 0.0):
        return cd_server_poll(self.h, ticket, out, timeout_ms)

    def info(self):
        return cd_server_info(self.h)

    def close(self):
        if self.h is not None:
            cd_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
