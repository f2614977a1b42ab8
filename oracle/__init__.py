"""ctypes wrapper around the plain-C CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls anything here, and this module imports nothing from the CUDA
package.  Inputs are plain numpy arrays (CSR as described in ``oracle.h``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("patience", C.c_int32), ("weak_max", C.c_int32),
                ("phi_num", C.c_int32), ("phi_den", C.c_int32), ("sigma_gap", C.c_int32),
                ("coarsest_factor", C.c_int32), ("cluster_iters", C.c_int32),
                ("cluster_cap_div", C.c_int32), ("max_levels", C.c_int32),
                ("stall_num", C.c_int32), ("stall_den", C.c_int32),
                ("coarsener", C.c_int32), ("match_rounds", C.c_int32), ("initial", C.c_int32),
                ("lp_relax_num", C.c_int32), ("lp_relax_den", C.c_int32), ("reb_objective", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("n", C.c_int32 * 65), ("m_dir", C.c_int64 * 65),
                ("J", C.c_int64 * 65), ("iters", C.c_int32 * 65)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(_LIB)
        _lib.orc_dist.restype = C.c_int64
        _lib.orc_num_pes.restype = C.c_int64
        _lib.orc_lmax.restype = C.c_int64
        _lib.orc_lmax.argtypes = [C.c_int64, C.c_int64, C.c_double]
        _lib.orc_objective.restype = C.c_int64
        _lib.orc_gain.restype = C.c_int64
        _lib.orc_contract.restype = C.c_int64
        _lib.orc_map_run.restype = C.c_int64
        _lib.orc_hash.restype = C.c_uint64
        _lib.orc_hash.argtypes = [C.c_uint64, C.c_uint64]
        _lib.orc_adaptive_eps.restype = C.c_double
        _lib.orc_adaptive_eps.argtypes = [C.c_double, C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.c_int32]
        _lib.orc_hm_run.restype = C.c_int64
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


def default_params(seed: int = 0x5EED0000) -> Params:
    p = Params()
    lib().orc_default_params(C.byref(p))
    p.seed = seed
    return p


def _topo(hier: Sequence[int], dist: Sequence[int]):
    h, d = _i32(hier), _i32(dist)
    return h, d, C.c_int32(len(h))


def hash64(seed: int, x: int) -> int:
    return int(lib().orc_hash(C.c_uint64(seed), C.c_uint64(x)))


def dist(hier, dist_, p: int, q: int) -> int:
    h, d, l = _topo(hier, dist_)
    return int(lib().orc_dist(_p(h), _p(d), l, C.c_int64(p), C.c_int64(q)))


def num_pes(hier) -> int:
    h = _i32(hier)
    return int(lib().orc_num_pes(_p(h), C.c_int32(len(h))))


def lmax(total_weight: int, k: int, eps: float) -> int:
    return int(lib().orc_lmax(total_weight, k, eps))


def objective(g, hier, dist_, pi) -> Tuple[int, int, np.ndarray]:
    """(J, max block weight, block weights[k])."""
    h, d, l = _topo(hier, dist_)
    k = num_pes(hier)
    W = np.zeros(k, dtype=np.int64)
    mx = C.c_int64(0)
    pi = _i32(pi)
    J = lib().orc_objective(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw),
                            _p(h), _p(d), l, _p(pi), _p(W), C.byref(mx))
    return int(J), int(mx.value), W


def gain(g, hier, dist_, pi, v: int, q: int) -> int:
    h, d, l = _topo(hier, dist_)
    pi = _i32(pi)
    return int(lib().orc_gain(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(h), _p(d), l,
                              _p(pi), C.c_int32(v), C.c_int32(q)))


def lp_step(g, hier, dist_, pi, lock, relax=(0, 1)):
    """One Alg. 4 step.  Returns (new pi, new lock, pi', g, inX, moved, |M|).
    relax = (num, den) > (0, .): the relaxed filter -G < floor(num conn(v, P(v)) / den)."""
    h, d, l = _topo(hier, dist_)
    pi = _i32(pi).copy()
    lock = np.ascontiguousarray(lock, dtype=np.uint8).copy()
    pp = np.zeros(g.n, np.int32)
    gn = np.zeros(g.n, np.int64)
    inx = np.zeros(g.n, np.uint8)
    mv = np.zeros(g.n, np.uint8)
    cnt = lib().orc_lp_step_relaxed(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(h), _p(d), l,
                                    _p(pi), _p(lock), _p(pp), _p(gn), _p(inx), _p(mv), C.c_int32(relax[0]),
                                    C.c_int32(relax[1]))
    return pi, lock, pp, gn, inx, mv, int(cnt)


def rebalance(g, hier, dist_, lmax_: int, strong: bool, pi, sigma_gap: int = 100,
              seed: int = 0x5EED0000, level: int = 0, t: int = 1, objective: int = 0):
    """One weak / strong rebalancing step (objective 0: cut gains, 1: Eq. 1's
    J gains).  Returns (new pi, dest, moved, count)."""
    h, d, l = _topo(hier, dist_)
    pi = _i32(pi).copy()
    dest = np.zeros(g.n, np.int32)
    mv = np.zeros(g.n, np.uint8)
    cnt = lib().orc_rebalance_obj(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw),
                                  _p(h), _p(d), l, C.c_int64(lmax_), C.c_int32(int(strong)),
                                  C.c_int32(sigma_gap), C.c_uint64(seed), C.c_int32(level), C.c_int32(t),
                                  _p(pi), _p(dest), _p(mv), C.c_int32(objective))
    return pi, dest, mv, int(cnt)


def refine(g, hier, dist_, lmax_: int, pi, rounds: int = -1, params: Optional[Params] = None,
           level: int = 0, trace_cap: int = 4096):
    """Alg. 6.  Returns (best pi, J, max block weight, iterations, kinds, Js, maxws)."""
    h, d, l = _topo(hier, dist_)
    prm = params or default_params()
    pi = _i32(pi).copy()
    J = C.c_int64(0)
    mx = C.c_int64(0)
    kinds = np.full(trace_cap, -1, np.int32)
    Js = np.zeros(trace_cap, np.int64)
    Ws = np.zeros(trace_cap, np.int64)
    it = lib().orc_refine(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), _p(h), _p(d), l,
                          C.c_int64(lmax_), C.byref(prm), C.c_int32(level), C.c_int32(rounds),
                          _p(pi), C.byref(J), C.byref(mx), _p(kinds), _p(Js), _p(Ws),
                          C.c_int32(trace_cap))
    it = int(it)
    m = min(it, trace_cap)
    return pi, int(J.value), int(mx.value), it, kinds[:m], Js[:m], Ws[:m]


def cluster(g, wcap: int, params: Optional[Params] = None, level: int = 0):
    """LP clustering of one level.  Returns (M, n_c)."""
    prm = params or default_params()
    M = np.zeros(g.n, np.int32)
    nc = lib().orc_cluster(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw),
                           C.c_int64(wcap), C.byref(prm), C.c_int32(level), _p(M))
    return M, int(nc)


def match(g, lmax_: int, params: Optional[Params] = None, level: int = 0):
    """Two-hop matching of one level.  Returns (M, n_c, mate, stage counts:
    heavy-edge, leaf, twin, relative, isolated matched vertices, heavy-edge rounds)."""
    prm = params or default_params()
    M = np.zeros(g.n, np.int32)
    mate = np.zeros(g.n, np.int32)
    st = np.zeros(6, np.int32)
    nc = lib().orc_match(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), C.c_int64(lmax_),
                         C.byref(prm), C.c_int32(level), _p(mate), _p(M), _p(st))
    return M, int(nc), mate, st


def contract(g, M, nc: int):
    """Coarse CSR (xadj, adj, adjw, vw)."""
    M = _i32(M)
    xc = np.zeros(nc + 1, np.int64)
    cap = max(1, g.m_dir)
    ac = np.zeros(cap, np.int32)
    wc = np.zeros(cap, np.int32)
    vc = np.zeros(max(nc, 1), np.int32)
    mc = lib().orc_contract(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), _p(M),
                            C.c_int32(nc), _p(xc), _p(ac), _p(wc), _p(vc))
    mc = int(mc)
    return xc, ac[:mc].copy(), wc[:mc].copy(), vc[:nc].copy()


def initial(g, k: int):
    pi = np.zeros(g.n, np.int32)
    lib().orc_initial(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.vw), C.c_int64(k), _p(pi))
    return pi


def project(M, pi_coarse):
    M = _i32(M)
    pc = _i32(pi_coarse)
    pi = np.zeros(M.size, np.int32)
    lib().orc_project(C.c_int32(M.size), _p(M), _p(pc), _p(pi))
    return pi


def map_run(g, hier, dist_, eps: float, params: Optional[Params] = None):
    """Full pipeline.  Returns (pi, J, Stats)."""
    h, d, l = _topo(hier, dist_)
    prm = params or default_params()
    pi = np.zeros(g.n, np.int32)
    st = Stats()
    J = lib().orc_map_run(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), _p(h), _p(d), l,
                          C.c_double(eps), C.byref(prm), _p(pi), C.byref(st))
    return pi, int(J), st


class HmStats(C.Structure):
    _fields_ = [("calls", C.c_int64 * 16), ("first_eps", C.c_double * 16)]


def adaptive_eps(eps: float, cV: int, cVp: int, k: int, kp: int, d: int) -> float:
    """Eq. 2: ((1 + eps) k' c(V) / (k c(V')))^(1/d) - 1."""
    return float(lib().orc_adaptive_eps(eps, cV, cVp, k, kp, d))


def build_subgraph(g, part, b: int):
    """Alg. 2: the subgraph induced by block b.  Returns ((n', xadj, adj, adjw, vw), M, m', w')."""
    part = _i32(part)
    xs = np.zeros(g.n + 1, np.int64)
    cap = max(1, g.m_dir)
    as_ = np.zeros(cap, np.int32)
    ws = np.zeros(cap, np.int32)
    vs = np.zeros(max(1, g.n), np.int32)
    M = np.zeros(max(1, g.n), np.int32)
    mo = C.c_int64(0)
    wo = C.c_int64(0)
    ns = lib().orc_build_subgraph(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), _p(part),
                                  C.c_int32(b), _p(xs), _p(as_), _p(ws), _p(vs), _p(M), C.byref(mo), C.byref(wo))
    ns = int(ns)
    ms = int(xs[ns])
    sub = (ns, xs[:ns + 1].copy(), as_[:ms].copy(), ws[:ms].copy(), vs[:ns].copy())
    return sub, M[:g.n].copy(), int(mo.value), int(wo.value)


def hm_run(g, hier, dist_, eps: float, params: Optional[Params] = None):
    """Hierarchical multisection (Alg. 3).  Returns (pi, J, HmStats)."""
    h, d, l = _topo(hier, dist_)
    prm = params or default_params()
    pi = np.zeros(g.n, np.int32)
    st = HmStats()
    J = lib().orc_hm_run(C.c_int32(g.n), _p(g.xadj), _p(g.adj), _p(g.adjw), _p(g.vw), _p(h), _p(d), l,
                         C.c_double(eps), C.byref(prm), _p(pi), C.byref(st))
    return pi, int(J), st
