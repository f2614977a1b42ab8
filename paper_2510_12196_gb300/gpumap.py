"""ctypes binding of the CUDA mapping library ``libgpumap.so``.

Function names match the C ABI in ``include/gpumap.h``; this module only
marshals arguments (numpy arrays for host data, torch CUDA tensors or raw
device pointers for device data) and turns non-OK statuses into
``MapError``.  Every step of the mapping path runs in the library's kernels.
There is no CPU fallback: without the built library (and a CUDA device) every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

_lib = None


class MapError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


STATUS = {0: "MAP_OK", 1: "MAP_E_INVALID", 2: "MAP_E_OOM", 3: "MAP_E_CUDA", 4: "MAP_E_OVERFLOW",
          5: "MAP_E_TIMEOUT", 6: "MAP_E_STATE", 7: "MAP_E_INTERNAL"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class MapConfig(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("patience", C.c_int32), ("weak_max", C.c_int32),
                ("phi_num", C.c_int32), ("phi_den", C.c_int32), ("sigma_gap", C.c_int32),
                ("coarsest_factor", C.c_int32), ("cluster_iters", C.c_int32),
                ("cluster_cap_div", C.c_int32), ("max_levels", C.c_int32),
                ("stall_num", C.c_int32), ("stall_den", C.c_int32),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p),
                ("launch_mode", C.c_int32), ("engine_max_n", C.c_int32),
                ("grid_engine_max_n", C.c_int32), ("coarsener", C.c_int32),
                ("match_rounds", C.c_int32), ("initial", C.c_int32), ("lp_relax_num", C.c_int32),
                ("lp_relax_den", C.c_int32), ("reb_objective", C.c_int32), ("mid_deg", C.c_int32),
                ("split_deg", C.c_int32)]


class MapStats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n", C.c_int32 * 65), ("m_dir", C.c_int64 * 65),
                ("J", C.c_int64 * 65), ("iters", C.c_int32 * 65), ("ms_coarsen", C.c_double),
                ("ms_initial", C.c_double), ("ms_refine", C.c_double), ("ms_project", C.c_double),
                ("device_bytes", C.c_int64), ("device_bytes_peak", C.c_int64),
                ("ms_refine_level", C.c_double * 65), ("mid_deg", C.c_int32 * 65), ("split_deg", C.c_int32 * 65),
                ("tuned", C.c_int32 * 65), ("ms_tune", C.c_double), ("lp_iters", C.c_int32 * 65),
                ("weak_iters", C.c_int32 * 65), ("strong_iters", C.c_int32 * 65)]


class MapHmStats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("workers", C.c_int32), ("calls", C.c_int64 * 16),
                ("first_eps", C.c_double * 16), ("ms_partition", C.c_double), ("ms_build", C.c_double),
                ("ms_total", C.c_double), ("ms_level", C.c_double * 16), ("ms_create", C.c_double),
                ("ms_run", C.c_double), ("ms_destroy", C.c_double)]


_P = C.c_void_p
_SIGS = {
    "map_config_default": (None, [_P]),
    "map_status_string": (C.c_char_p, [C.c_int]),
    "map_create": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P, C.c_int32, C.c_double, _P, _P, C.c_int32, _P]),
    "map_destroy": (None, [_P]),
    "map_last_error": (C.c_char_p, [_P]),
    "map_sync": (C.c_int, [_P]),
    "map_info": (C.c_int, [_P, _P, _P, _P]),
    "map_set_mapping": (C.c_int, [_P, C.c_int32, _P]),
    "map_get_mapping": (C.c_int, [_P, C.c_int32, _P]),
    "map_objective": (C.c_int, [_P, C.c_int32, _P, _P]),
    "map_block_weights": (C.c_int, [_P, C.c_int32, _P]),
    "map_lp_step": (C.c_int, [_P, C.c_int32, _P]),
    "map_get_lp_state": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "map_set_lock": (C.c_int, [_P, C.c_int32, _P]),
    "map_rebalance_step": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, _P]),
    "map_refine": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P]),
    "map_get_refine_trace": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "map_coarsen": (C.c_int, [_P, _P]),
    "map_level_info": (C.c_int, [_P, C.c_int32, _P, _P]),
    "map_get_level_graph": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "map_initial": (C.c_int, [_P]),
    "map_project": (C.c_int, [_P, C.c_int32]),
    "map_run": (C.c_int, [_P, _P, _P]),
    "map_stats": (C.c_int, [_P, _P]),
    "map_run_hm": (C.c_int, [_P, C.c_int32, _P, _P]),
    "map_hm_stats": (C.c_int, [_P, C.c_int32, _P]),
    "map_profile_enable": (C.c_int, [_P, C.c_int32]),
    "map_profile_read": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P]),
    "map_launch_count": (C.c_longlong, []),
    "map_objective_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P, _P, _P, C.c_int32, _P, _P]),
    "map_selftest_barrier_timeout": (C.c_int, [_P]),
    "map_batch_opts_default": (None, [_P]),
    "map_batch_create": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "map_batch_launch": (C.c_int, [_P]),
    "map_batch_results": (C.c_int, [_P, _P, _P, _P]),
    "map_batch_schedule": (C.c_int, [_P, _P, _P, _P, _P]),
    "map_batch_last_error": (C.c_char_p, [_P]),
    "map_batch_destroy": (None, [_P]),
    "map_server_opts_default": (None, [_P]),
    "map_job_estimate_bytes": (C.c_int64, [C.c_int32, C.c_int64, _P, C.c_int32]),
    "map_server_create": (C.c_int, [_P, _P]),
    "map_server_submit": (C.c_int, [_P, _P, _P]),
    "map_server_wait": (C.c_int, [_P, C.c_uint64, C.c_double, _P]),
    "map_server_poll": (C.c_int, [_P, C.c_uint64, _P]),
    "map_server_stats": (C.c_int, [_P, _P]),
    "map_server_last_error": (C.c_char_p, [_P]),
    "map_server_destroy": (None, [_P]),
}


def library_path() -> str:
    return _build.OUT


def lib(build_if_missing: bool = True):
    """Loads libgpumap.so (building it in-tree first if needed)."""
    global _lib
    if _lib is None:
        path = _build.OUT
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a) -> int:
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


def _check(ctx, st: int, where: str):
    if st != 0:
        msg = lib().map_last_error(ctx)
        raise MapError(st, where, msg.decode() if msg else "")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def map_config_default(seed: Optional[int] = None) -> MapConfig:
    cfg = MapConfig()
    lib().map_config_default(C.byref(cfg))
    if seed is not None:
        cfg.seed = seed
    return cfg


def torch_allocator(cfg: MapConfig) -> tuple:
    """Routes the context's device allocations through torch's caching
    allocator.  Returns the callback objects, which must outlive the context."""
    import torch

    dev = torch.cuda.current_device()

    def _alloc(nbytes, user, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
        except Exception:
            return None

    def _free(ptr, nbytes, user, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    cfg.alloc, cfg.free = a, f
    return (a, f)


def map_create(xadj, adjncy, adjwgt, vwgt, n: int, hier: Sequence[int], dist: Sequence[int], eps: float,
               cfg: Optional[MapConfig] = None, stream=None, inputs_on_device: bool = False):
    h = np.ascontiguousarray(hier, dtype=np.int32)
    d = np.ascontiguousarray(dist, dtype=np.int32)
    out = C.c_void_p()
    st = lib().map_create(_ptr(xadj), _ptr(adjncy), _ptr(adjwgt), _ptr(vwgt), int(n), _ptr(h), _ptr(d), len(h),
                          float(eps), C.byref(cfg) if cfg is not None else None, _stream_handle(stream),
                          int(bool(inputs_on_device)), C.byref(out))
    if st != 0:
        msg = lib().map_last_error(None)
        raise MapError(st, "map_create", msg.decode() if msg else "")
    return out.value


def map_destroy(ctx) -> None:
    lib().map_destroy(ctx)


def map_last_error(ctx) -> str:
    m = lib().map_last_error(ctx)
    return m.decode() if m else ""


def map_sync(ctx) -> None:
    _check(ctx, lib().map_sync(ctx), "map_sync")


def map_info(ctx):
    k, lm, tw = C.c_int32(), C.c_int64(), C.c_int64()
    _check(ctx, lib().map_info(ctx, C.byref(k), C.byref(lm), C.byref(tw)), "map_info")
    return k.value, lm.value, tw.value


def map_level_info(ctx, level: int = 0):
    n, m = C.c_int32(), C.c_int64()
    _check(ctx, lib().map_level_info(ctx, level, C.byref(n), C.byref(m)), "map_level_info")
    return n.value, m.value


def map_set_mapping(ctx, level: int, pi) -> None:
    pi = np.ascontiguousarray(pi, dtype=np.int32)
    _check(ctx, lib().map_set_mapping(ctx, level, _ptr(pi)), "map_set_mapping")


def map_get_mapping(ctx, level: int = 0) -> np.ndarray:
    n, _ = map_level_info(ctx, level)
    pi = np.zeros(n, np.int32)
    _check(ctx, lib().map_get_mapping(ctx, level, _ptr(pi)), "map_get_mapping")
    return pi


def map_objective(ctx, level: int = 0):
    J, mw = C.c_int64(), C.c_int64()
    _check(ctx, lib().map_objective(ctx, level, C.byref(J), C.byref(mw)), "map_objective")
    return J.value, mw.value


def map_block_weights(ctx, level: int = 0) -> np.ndarray:
    k, _, _ = map_info(ctx)
    W = np.zeros(k, np.int64)
    _check(ctx, lib().map_block_weights(ctx, level, _ptr(W)), "map_block_weights")
    return W


def map_lp_step(ctx, level: int = 0) -> int:
    mv = C.c_int32()
    _check(ctx, lib().map_lp_step(ctx, level, C.byref(mv)), "map_lp_step")
    return mv.value


def map_get_lp_state(ctx, level: int = 0):
    n, _ = map_level_info(ctx, level)
    pp = np.zeros(n, np.int32)
    g = np.zeros(n, np.int64)
    inx = np.zeros(n, np.uint8)
    mv = np.zeros(n, np.uint8)
    _check(ctx, lib().map_get_lp_state(ctx, level, _ptr(pp), _ptr(g), _ptr(inx), _ptr(mv)), "map_get_lp_state")
    return pp, g, inx, mv


def map_set_lock(ctx, level: int, lock) -> None:
    lock = np.ascontiguousarray(lock, dtype=np.uint8)
    _check(ctx, lib().map_set_lock(ctx, level, _ptr(lock)), "map_set_lock")


def map_rebalance_step(ctx, level: int, strong: bool, t: int = 1) -> int:
    mv = C.c_int32()
    _check(ctx, lib().map_rebalance_step(ctx, level, int(bool(strong)), int(t), C.byref(mv)), "map_rebalance_step")
    return mv.value


def map_refine(ctx, level: int = 0, rounds: int = -1):
    J, mw, it = C.c_int64(), C.c_int64(), C.c_int32()
    _check(ctx, lib().map_refine(ctx, level, rounds, C.byref(J), C.byref(mw), C.byref(it)), "map_refine")
    return J.value, mw.value, it.value


def map_get_refine_trace(ctx, cap: int = 4096):
    kind = np.zeros(cap, np.int32)
    J = np.zeros(cap, np.int64)
    W = np.zeros(cap, np.int64)
    cnt = C.c_int32()
    _check(ctx, lib().map_get_refine_trace(ctx, cap, _ptr(kind), _ptr(J), _ptr(W), C.byref(cnt)),
           "map_get_refine_trace")
    m = min(cnt.value, cap)
    return kind[:m], J[:m], W[:m], cnt.value


def map_coarsen(ctx) -> int:
    lv = C.c_int32()
    _check(ctx, lib().map_coarsen(ctx, C.byref(lv)), "map_coarsen")
    return lv.value


def map_get_level_graph(ctx, level: int, with_M: bool = True):
    n, m = map_level_info(ctx, level)
    xadj = np.zeros(n + 1, np.int64)
    adj = np.zeros(max(m, 1), np.int32)
    w = np.zeros(max(m, 1), np.int32)
    vw = np.zeros(n, np.int32)
    M = np.zeros(n, np.int32) if with_M else None
    _check(ctx, lib().map_get_level_graph(ctx, level, _ptr(xadj), _ptr(adj), _ptr(w), _ptr(vw), _ptr(M)),
           "map_get_level_graph")
    return xadj, adj[:m], w[:m], vw, M


def map_initial(ctx) -> None:
    _check(ctx, lib().map_initial(ctx), "map_initial")


def map_project(ctx, level: int) -> None:
    _check(ctx, lib().map_project(ctx, level), "map_project")


def map_run(ctx, out_pi=None):
    J = C.c_int64()
    _check(ctx, lib().map_run(ctx, _ptr(out_pi), C.byref(J)), "map_run")
    return J.value


def map_run_hm(ctx, out_pi=None, workers: int = 0):
    """Hierarchical multisection (GPU-HM) of the context's input graph; returns J."""
    J = C.c_int64()
    _check(ctx, lib().map_run_hm(ctx, int(workers), _ptr(out_pi), C.byref(J)), "map_run_hm")
    return J.value


def map_hm_stats(ctx, which: int = 0) -> MapHmStats:
    """which = 0: the last map_run_hm; 1: the last multisection initial mapping."""
    s = MapHmStats()
    _check(ctx, lib().map_hm_stats(ctx, int(which), C.byref(s)), "map_hm_stats")
    return s


def map_stats(ctx) -> MapStats:
    s = MapStats()
    _check(ctx, lib().map_stats(ctx, C.byref(s)), "map_stats")
    return s


KERNEL_CLASSES = {0: "lp_gain", 1: "lp_after", 2: "eval_J", 3: "cluster", 4: "radix_sort", 5: "eval_J_close",
                  6: "match_prefer", 7: "cluster_mid", 8: "cluster_high", 9: "eval_J_mid", 10: "eval_J_high",
                  11: "lp_gain_mid", 12: "lp_gain_high"}
# the kernel each profiled class times
KERNEL_OF_CLASS = {"lp_gain": "k_lp_gain_tile", "lp_after": "k_lp_after_low", "eval_J": "k_eval_tile",
                   "cluster": "k_cluster_tile", "radix_sort": "radix-sort passes (k_sort_hist + k_sort_scatter)",
                   "eval_J_close": "k_eval_tile (controller only)", "match_prefer": "k_match_prefer",
                   "cluster_mid": "k_cluster_mid", "cluster_high": "k_cluster_high", "eval_J_mid": "k_eval_mid",
                   "eval_J_high": "k_eval_high", "lp_gain_mid": "k_lp_gain_mid", "lp_gain_high": "k_lp_gain_high"}


def map_profile_enable(ctx, enable: bool = True) -> None:
    _check(ctx, lib().map_profile_enable(ctx, int(bool(enable))), "map_profile_enable")


def map_profile_read(ctx, which: int, level: int = -1):
    """(launches, total ms, algorithmic bytes) of one kernel class since the last
    read, on one hierarchy level (-1: all levels)."""
    l, ms, by = C.c_int64(), C.c_double(), C.c_int64()
    _check(ctx, lib().map_profile_read(ctx, which, level, C.byref(l), C.byref(ms), C.byref(by)),
           "map_profile_read")
    return l.value, ms.value, by.value


def map_launch_count() -> int:
    return int(lib().map_launch_count())


def map_objective_noalloc(xadj, adjncy, adjwgt, vwgt, n: int, pi, hier, dist, out, stream=None) -> None:
    """J and max block weight into the device int64[2] ``out`` without any
    device allocation (all graph / mapping / output arguments are device
    tensors or pointers; see include/gpumap.h)."""
    h = np.ascontiguousarray(hier, dtype=np.int32)
    d = np.ascontiguousarray(dist, dtype=np.int32)
    st = lib().map_objective_noalloc(_ptr(xadj), _ptr(adjncy), _ptr(adjwgt), _ptr(vwgt), int(n), _ptr(pi),
                                     _ptr(h), _ptr(d), len(h), _ptr(out), _stream_handle(stream))
    if st != 0:
        msg = lib().map_last_error(None)
        raise MapError(st, "map_objective_noalloc", msg.decode() if msg else "")


def map_selftest_barrier_timeout(stream=None) -> int:
    """Status of the bounded grid-barrier self-test (MAP_E_TIMEOUT = 5 is the pass)."""
    return int(lib().map_selftest_barrier_timeout(_stream_handle(stream)))


class MapBatchOpts(C.Structure):
    _fields_ = [("level", C.c_int32), ("rounds", C.c_int32), ("autotune", C.c_int32),
                ("cluster", C.c_int32), ("tile_entries", C.c_int32)]


def map_batch_opts_default(**over) -> MapBatchOpts:
    o = MapBatchOpts()
    lib().map_batch_opts_default(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def _check_batch(b, st: int, where: str):
    if st != 0:
        msg = lib().map_batch_last_error(b)
        raise MapError(st, where, msg.decode() if msg else "")


def map_batch_create(ctxs, opts: Optional[MapBatchOpts] = None, stream=None):
    """One batch over the contexts ``ctxs`` (see include/gpumap.h)."""
    arr = (C.c_void_p * len(ctxs))(*[C.cast(c, C.c_void_p) for c in ctxs])
    out = C.c_void_p()
    st = lib().map_batch_create(arr, len(ctxs), C.byref(opts) if opts is not None else None,
                                _stream_handle(stream), C.byref(out))
    _check_batch(None, st, "map_batch_create")
    return out


def map_batch_launch(b) -> None:
    _check_batch(b, lib().map_batch_launch(b), "map_batch_launch")


def map_batch_results(b, njobs: int):
    J = np.zeros(njobs, np.int64)
    mw = np.zeros(njobs, np.int64)
    it = np.zeros(njobs, np.int32)
    _check_batch(b, lib().map_batch_results(b, J.ctypes.data, mw.ctypes.data, it.ctypes.data), "map_batch_results")
    return J, mw, it


def map_batch_schedule(b):
    """(CTAs per job, staged entries per warp tile, clusters, autotune ms)."""
    c, te, ncl, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
    _check_batch(b, lib().map_batch_schedule(b, C.byref(c), C.byref(te), C.byref(ncl), C.byref(ms)),
                 "map_batch_schedule")
    return c.value, te.value, ncl.value, ms.value


def map_batch_destroy(b) -> None:
    lib().map_batch_destroy(b)


class MapJob(C.Structure):
    _fields_ = [("xadj", C.c_void_p), ("adjncy", C.c_void_p), ("adjwgt", C.c_void_p), ("vwgt", C.c_void_p),
                ("n", C.c_int32), ("hier", C.c_void_p), ("dist", C.c_void_p), ("levels", C.c_int32),
                ("eps", C.c_double), ("cfg", C.c_void_p), ("out_pi", C.c_void_p), ("user", C.c_void_p)]


class MapJobResult(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int), ("levels", C.c_int32), ("J", C.c_int64),
                ("device_bytes_est", C.c_int64), ("device_bytes_peak", C.c_int64),
                ("t_submit_ms", C.c_double), ("t_start_ms", C.c_double), ("t_done_ms", C.c_double),
                ("user", C.c_void_p), ("error", C.c_char * 256)]


JOB_RUNNER = C.CFUNCTYPE(C.c_int32, C.POINTER(MapJob), C.c_void_p, C.c_void_p, C.POINTER(MapJobResult))


class MapServerOpts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("lookahead", C.c_int32), ("mem_budget", C.c_int64),
                ("runner", JOB_RUNNER), ("runner_user", C.c_void_p), ("batch_lanes", C.c_int32),
                ("whole_gpu_levels", C.c_int32)]


class MapServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("queued", C.c_int64), ("running", C.c_int64), ("bytes_in_flight", C.c_int64),
                ("peak_bytes_in_flight", C.c_int64), ("mem_budget", C.c_int64), ("peak_running", C.c_int32),
                ("uptime_ms", C.c_double), ("engine_launches", C.c_int64), ("engine_jobs", C.c_int64),
                ("peak_batch", C.c_int32)]


def map_job_estimate_bytes(n: int, m_dir: int, hier) -> int:
    h = np.ascontiguousarray(hier, dtype=np.int32)
    return int(lib().map_job_estimate_bytes(int(n), int(m_dir), h.ctypes.data, len(h)))


class MapServer:
    """Request loop over the C server (see include/gpumap.h).  Keeps every
    submitted job's host arrays alive until its result is collected."""

    def __init__(self, slots: int = 8, lookahead: int = 8, mem_budget: int = 0, runner=None,
                 batch_lanes: int = 0, whole_gpu_levels: int = 0):
        o = MapServerOpts()
        lib().map_server_opts_default(C.byref(o))
        o.slots, o.lookahead, o.mem_budget = slots, lookahead, mem_budget
        o.batch_lanes, o.whole_gpu_levels = batch_lanes, whole_gpu_levels
        self._runner = JOB_RUNNER(runner) if runner is not None else None
        if self._runner is not None:
            o.runner = self._runner
        out = C.c_void_p()
        st = lib().map_server_create(C.byref(o), C.byref(out))
        if st != 0:
            msg = lib().map_server_last_error(None)
            raise MapError(st, "map_server_create", msg.decode() if msg else "")
        self.h = out
        self._keep = {}

    def _check(self, st, where):
        if st != 0:
            msg = lib().map_server_last_error(self.h)
            raise MapError(st, where, msg.decode() if msg else "")

    def submit(self, graph, hier, dist, eps=0.03, cfg: Optional[MapConfig] = None, out_pi=None, user: int = 0):
        """Queues one job on host arrays; returns its ticket."""
        arrs = [np.ascontiguousarray(graph.xadj, np.int64), np.ascontiguousarray(graph.adj, np.int32),
                np.ascontiguousarray(graph.adjw, np.int32), np.ascontiguousarray(graph.vw, np.int32)]
        h = np.ascontiguousarray(hier, dtype=np.int32)
        d = np.ascontiguousarray(dist, dtype=np.int32)
        if out_pi is None:
            out_pi = np.zeros(graph.n, np.int32)
        j = MapJob()
        j.xadj, j.adjncy, j.adjwgt, j.vwgt = [a.ctypes.data for a in arrs]
        j.n, j.hier, j.dist, j.levels, j.eps = graph.n, h.ctypes.data, d.ctypes.data, len(h), float(eps)
        j.cfg = C.cast(C.pointer(cfg), C.c_void_p) if cfg is not None else None
        j.out_pi = out_pi.ctypes.data
        j.user = user
        t = C.c_uint64()
        self._check(lib().map_server_submit(self.h, C.byref(j), C.byref(t)), "map_server_submit")
        self._keep[t.value] = (arrs, h, d, cfg, out_pi, j)
        return t.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        """(result, mapping) of a job; MapError with status MAP_E_TIMEOUT (5) if not done in time."""
        r = MapJobResult()
        self._check(lib().map_server_wait(self.h, ticket, float(timeout_ms), C.byref(r)), "map_server_wait")
        keep = self._keep.pop(ticket)
        return r, keep[4]

    def poll(self, ticket: int) -> bool:
        d = C.c_int32()
        self._check(lib().map_server_poll(self.h, ticket, C.byref(d)), "map_server_poll")
        return bool(d.value)

    def stats(self) -> MapServerStats:
        s = MapServerStats()
        self._check(lib().map_server_stats(self.h, C.byref(s)), "map_server_stats")
        return s

    def close(self):
        if self.h:
            lib().map_server_destroy(self.h)
            self.h = None
            self._keep.clear()


class Mapper:
    """Owns one context; convenience wrapper over the functions above."""

    def __init__(self, graph, hier, dist, eps=0.03, seed=None, cfg=None, stream=None, device_inputs=None,
                 torch_alloc=False):
        self._keep = None
        cfg = cfg or map_config_default(seed)
        if torch_alloc:
            self._keep = torch_allocator(cfg)
        if device_inputs is not None:
            xadj, adj, w, vw = device_inputs
            self.ctx = map_create(xadj, adj, w, vw, graph.n, hier, dist, eps, cfg, stream, True)
        else:
            self.ctx = map_create(graph.xadj, graph.adj if graph.m_dir else None, graph.adjw if graph.m_dir else None,
                                  graph.vw, graph.n, hier, dist, eps, cfg, stream, False)
        self.n = graph.n

    def close(self):
        if self.ctx:
            map_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
