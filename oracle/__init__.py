"""CPU oracle for deep multilevel graph partitioning -- TEST INFRASTRUCTURE.

A plain, slow, single-threaded C implementation (kmpo_*.c) of what the method
computes, plus this ctypes marshalling layer.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the CUDA product path
never does.  See kmpo.h for the paper passages each function follows.
"""
from __future__ import annotations

import ctypes
import glob
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
_LIB = None


def build() -> str:
    srcs = sorted(glob.glob(os.path.join(HERE, "kmpo_*.c")))
    deps = srcs + [os.path.join(HERE, "kmpo.h")]
    if not os.path.exists(LIB_PATH) or any(os.path.getmtime(s) > os.path.getmtime(LIB_PATH)
                                           for s in deps):
        subprocess.check_call(["gcc", "-O3", "-fPIC", "-shared", "-o", LIB_PATH + ".tmp", *srcs,
                               "-lm"])
        os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


class Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "C", "lp_rounds", "refine_rounds", "subrounds", "two_hop", "conv_num", "conv_den",
        "ip_C", "ip_lp_rounds", "rep_random", "rep_bfs", "rep_ggg", "fm_passes", "fm_stop",
        "learned", "lrep_random", "lrep_bfs", "lrep_ggg", "replicas", "async_lp", "sample_subrounds", "adaptive",
        "sample_nodes")]


class OGraph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("xadj", ctypes.POINTER(ctypes.c_int64)),
                ("adj", ctypes.POINTER(ctypes.c_int32)), ("vw", ctypes.POINTER(ctypes.c_int32)),
                ("ew", ctypes.POINTER(ctypes.c_int32))]


class LPStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("moved", ctypes.c_int64 * 16),
                ("scanned", ctypes.c_int64 * 16)]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("level_n", ctypes.c_int32 * 64),
                ("level_m", ctypes.c_int64 * 64), ("lp_scanned", ctypes.c_int64),
                ("refine_scanned", ctypes.c_int64), ("cut", ctypes.c_int64),
                ("feasible", ctypes.c_int32), ("t_coarsen", ctypes.c_double),
                ("t_ip", ctypes.c_double), ("t_refine", ctypes.c_double),
                ("t_total", ctypes.c_double), ("level_kp", ctypes.c_int32 * 64),
                ("level_U", ctypes.c_int64 * 64), ("level_k", ctypes.c_int32 * 64),
                ("clustered", ctypes.c_int32), ("t_contract", ctypes.c_double),
                ("t_balance", ctypes.c_double)]


def lib():
    global _LIB
    if _LIB is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "kmpo_config_default": (None, [P]),
            "kmpo_key": (u64, [u64, i32, P]),
            "kmpo_step": (u64, [u64, u64]),
            "kmpo_perm32": (ctypes.c_uint32, [u64, i32]),
            "kmpo_subround": (i32, [u64, i32, i32]),
            "kmpo_cut": (i64, [i32, P, P, P, P]),
            "kmpo_cluster": (i32, [i32, P, P, P, P, i32, i32, u64, i32, P, i32, i32, P, P, P]),
            "kmpo_contract": (i32, [i32, P, P, P, P, P, P, P]),
            "kmpo_graph_free": (None, [P]),
            "kmpo_refine": (i64, [i32, P, P, P, P, i32, P, i32, u64, P, P, P]),
            "kmpo_balance": (i64, [i32, P, P, P, P, i32, P, P]),
            "kmpo_bipartition": (i64, [i32, P, P, P, P, i32, i32, i32, i32, u64, P, P]),
            "kmpo_fm": (i64, [i32, P, P, P, P, i32, i32, P, P]),
            "kmpo_initial": (None, [i32, i32, P, P, P, P, i32, u64, P]),
            "kmpo_eps_prime": (dbl, [dbl, i64, i32, i64, i32]),
            "kmpo_split_caps": (None, [dbl, i64, i32, i64, i32, P, P, P, P]),
            "kmpo_block_cap": (i32, [dbl, i64, i32, i32, i32]),
            "kmpo_partition": (i32, [i32, P, P, P, P, i32, dbl, u64, P, P, P]),
            "kmpo_bipartition_blocks": (i32, [i32, P, P, P, P, i32, P, dbl, i64, i32, u64, P, P, P]),
            "kmpo_brute_bisection": (i64, [i32, P, P, P, P, i64, i64, P]),
            "kmpo_adaptive_keep": (i32, [i32, P, i64]),
            "kmpo_async_cluster": (i32, [i32, P, P, P, P, i32, i32, u64, P]),
            "kmpo_mpnn_num_params": (i32, []),
            "kmpo_mpnn_features": (None, [i32, P, P, P, P, u64, P]),
            "kmpo_mpnn_forward": (None, [i32, P, P, P, P, P, P, P]),
            "kmpo_mpnn_loss": (dbl, [i32, P, P, P]),
            "kmpo_mpnn_backward": (None, [i32, P, P, P, P, P, P, P]),
            "kmpo_mpnn_propose": (None, [i32, P, P, i32, P]),
            "kmpo_mpnn_scores_f32": (None, [i32, P, P, P, P, u64, P, P]),
            "kmpo_mpnn_score_key": (ctypes.c_uint32, [ctypes.c_float]),
            "kmpo_set_proposer": (None, [P]),
            "kmpo_learned_initial": (None, [i32, P, P, P, P, i32, u64, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def config(**kw) -> Config:
    c = Config()
    lib().kmpo_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _p(a):
    return None if a is None else a.ctypes.data


def _g(g):
    xadj = np.ascontiguousarray(g.xadj, np.int64)
    adj = np.ascontiguousarray(g.adjncy, np.int32)
    vw = None if g.vwgt is None else np.ascontiguousarray(g.vwgt, np.int32)
    ew = None if g.adjwgt is None else np.ascontiguousarray(g.adjwgt, np.int32)
    return g.n, xadj, adj, vw, ew


def key(seed: int, words) -> int:
    w = np.asarray(list(words), np.uint64)
    return int(lib().kmpo_key(seed, len(w), w.ctypes.data if len(w) else None))


def step(x: int, w: int) -> int:
    return int(lib().kmpo_step(x, w))


def cut(g, part) -> int:
    n, xadj, adj, vw, ew = _g(g)
    part = np.ascontiguousarray(part, np.int32)
    return int(lib().kmpo_cut(n, _p(xadj), _p(adj), _p(ew), _p(part)))


def cluster(g, U, rounds, seed, level, cfg=None, isolated=True, two_hop=None, stats=False):
    """LP clustering of one level; returns labels (and fav, LP stats)."""
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    label = np.zeros(n, np.int32)
    fav = np.zeros(n, np.int32)
    st = LPStats()
    th = cfg.two_hop if two_hop is None else int(two_hop)
    lib().kmpo_cluster(n, _p(xadj), _p(adj), _p(vw), _p(ew), int(U), int(rounds), seed, int(level),
                       ctypes.byref(cfg), int(isolated), th, _p(label), _p(fav), ctypes.byref(st))
    if stats:
        return label, fav, st
    return label


def contract(g, label):
    """Returns (coarse Graph, map)."""
    from paper_2105_02022_gb300.graphgen import Graph

    n, xadj, adj, vw, ew = _g(g)
    label = np.ascontiguousarray(label, np.int32)
    mp = np.zeros(n, np.int32)
    og = OGraph()
    nn = lib().kmpo_contract(n, _p(xadj), _p(adj), _p(vw), _p(ew), _p(label), _p(mp),
                             ctypes.byref(og))
    m = int(og.xadj[nn]) if nn >= 0 else 0
    cx = np.ctypeslib.as_array(og.xadj, shape=(nn + 1,)).copy()
    ca = np.ctypeslib.as_array(og.adj, shape=(max(m, 1),))[:m].copy()
    cw = np.ctypeslib.as_array(og.ew, shape=(max(m, 1),))[:m].copy()
    cv = np.ctypeslib.as_array(og.vw, shape=(max(nn, 1),))[:nn].copy()
    lib().kmpo_graph_free(ctypes.byref(og))
    return Graph(nn, cx, ca, cv, cw, "coarse"), mp


def refine(g, k, caps, rounds, seed, part, cfg=None, stats=False):
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    part = np.array(part, np.int32, copy=True)
    caps = np.ascontiguousarray(caps, np.int32)
    st = LPStats()
    c = lib().kmpo_refine(n, _p(xadj), _p(adj), _p(vw), _p(ew), k, _p(caps), rounds, seed,
                          ctypes.byref(cfg), _p(part), ctypes.byref(st))
    if stats:
        return part, int(c), st
    return part, int(c)


def balance(g, k, caps, part):
    n, xadj, adj, vw, ew = _g(g)
    part = np.array(part, np.int32, copy=True)
    caps = np.ascontiguousarray(caps, np.int32)
    mv = lib().kmpo_balance(n, _p(xadj), _p(adj), _p(vw), _p(ew), k, _p(caps), _p(part))
    return part, int(mv)


def bipartition(g, L0, L1, target0, target1, itemkey, cfg=None):
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    side = np.zeros(n, np.int32)
    c = lib().kmpo_bipartition(n, _p(xadj), _p(adj), _p(vw), _p(ew), L0, L1, target0, target1,
                               itemkey, ctypes.byref(cfg), _p(side))
    return side, int(c)


def fm(g, L0, L1, side, cfg=None):
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    side = np.array(side, np.int32, copy=True)
    c = lib().kmpo_fm(n, _p(xadj), _p(adj), _p(vw), _p(ew), L0, L1, ctypes.byref(cfg), _p(side))
    return side, int(c)


def initial(algo, g, target0, key_):
    n, xadj, adj, vw, ew = _g(g)
    side = np.zeros(n, np.int32)
    lib().kmpo_initial(algo, n, _p(xadj), _p(adj), _p(vw), _p(ew), target0, key_, _p(side))
    return side


def eps_prime(eps, cV, k, cB, fB) -> float:
    return float(lib().kmpo_eps_prime(eps, cV, k, cB, fB))


def split_caps(eps, cV, k, cB, fB):
    """Returns (target0, target1, L0, L1)."""
    t0, t1, L0, L1 = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    lib().kmpo_split_caps(eps, cV, k, cB, fB, ctypes.byref(t0), ctypes.byref(t1), ctypes.byref(L0),
                          ctypes.byref(L1))
    return t0.value, t1.value, L0.value, L1.value


def block_cap(eps, cV, k, fb, maxc) -> int:
    return int(lib().kmpo_block_cap(eps, cV, k, fb, maxc))


def partition(g, k, eps, seed, cfg=None):
    """Full deep multilevel partition; returns (part, status, Stats)."""
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    part = np.zeros(n, np.int32)
    st = Stats()
    rc = lib().kmpo_partition(n, _p(xadj), _p(adj), _p(vw), _p(ew), k, eps, seed,
                              ctypes.byref(cfg), _p(part), ctypes.byref(st))
    return part, int(rc), st


def bipartition_blocks(g, nblocks, f, eps, cV, k, roundkey, part, cfg=None):
    """One split round of Algorithm 2; returns (new part, new f)."""
    cfg = cfg or config()
    n, xadj, adj, vw, ew = _g(g)
    part = np.array(part, np.int32, copy=True)
    f = np.ascontiguousarray(f, np.int32)
    fo = np.zeros(2 * nblocks + 2, np.int32)
    nb = lib().kmpo_bipartition_blocks(n, _p(xadj), _p(adj), _p(vw), _p(ew), nblocks, _p(f), eps, cV, k,
                                       roundkey, ctypes.byref(cfg), _p(part), _p(fo))
    return part, fo[:nb].copy()


def adaptive_keep(cuts, best) -> bool:
    c = np.ascontiguousarray(cuts, np.int64)
    return bool(lib().kmpo_adaptive_keep(len(c), _p(c) if len(c) else None, int(best)))


def brute_bisection(g, L0, L1):
    n, xadj, adj, vw, ew = _g(g)
    side = np.zeros(n, np.int32)
    c = lib().kmpo_brute_bisection(n, _p(xadj), _p(adj), _p(vw), _p(ew), L0, L1, _p(side))
    return int(c), side


MPNN_F, MPNN_H = 8, 64


def mpnn_num_params() -> int:
    return int(lib().kmpo_mpnn_num_params())


def mpnn_features(g, key_):
    n, xadj, adj, vw, ew = _g(g)
    X = np.zeros((n, MPNN_F), np.float64)
    lib().kmpo_mpnn_features(n, _p(xadj), _p(adj), _p(vw), _p(ew), key_, _p(X))
    return X


def mpnn_forward(g, X, P):
    n, xadj, adj, vw, ew = _g(g)
    X = np.ascontiguousarray(X, np.float64)
    P = np.ascontiguousarray(P, np.float64)
    S = np.zeros(n, np.float64)
    lib().kmpo_mpnn_forward(n, _p(xadj), _p(adj), _p(ew), _p(X), _p(P), _p(S), None)
    return S


def mpnn_loss(S, side):
    S = np.ascontiguousarray(S, np.float64)
    side = np.ascontiguousarray(side, np.int32)
    gS = np.zeros(len(S), np.float64)
    L = lib().kmpo_mpnn_loss(len(S), _p(S), _p(side), _p(gS))
    return float(L), gS


def mpnn_backward(g, X, P, gS):
    n, xadj, adj, vw, ew = _g(g)
    X = np.ascontiguousarray(X, np.float64)
    P = np.ascontiguousarray(P, np.float64)
    gS = np.ascontiguousarray(gS, np.float64)
    gP = np.zeros(mpnn_num_params(), np.float64)
    lib().kmpo_mpnn_backward(n, _p(xadj), _p(adj), _p(ew), _p(X), _p(P), _p(gS), _p(gP))
    return gP


def mpnn_propose(g, S, target0):
    n = g.n
    vw = None if g.vwgt is None else np.ascontiguousarray(g.vwgt, np.int32)
    S = np.ascontiguousarray(S, np.float64)
    side = np.zeros(n, np.int32)
    lib().kmpo_mpnn_propose(n, _p(vw), _p(S), int(target0), _p(side))
    return side


def mpnn_scores_f32(g, key_, W):
    """Scores in the kernel's precision; W: parameters as float32 values."""
    n, xadj, adj, vw, ew = _g(g)
    W = np.ascontiguousarray(W, np.float32)
    S = np.zeros(max(n, 1), np.float32)
    lib().kmpo_mpnn_scores_f32(n, _p(xadj), _p(adj), _p(vw), _p(ew), key_, _p(W), _p(S))
    return S[:n]


def mpnn_score_key(s) -> int:
    return int(lib().kmpo_mpnn_score_key(ctypes.c_float(float(s))))


def set_proposer(W):
    """Proposer of learned mode (None clears); W: float32 parameters."""
    if W is None:
        lib().kmpo_set_proposer(None)
        return
    W = np.ascontiguousarray(W, np.float32)
    assert W.size == mpnn_num_params()
    lib().kmpo_set_proposer(_p(W))


def learned_initial(g, target0, key_, W):
    n, xadj, adj, vw, ew = _g(g)
    W = np.ascontiguousarray(W, np.float32)
    side = np.zeros(max(n, 1), np.int32)
    lib().kmpo_learned_initial(n, _p(xadj), _p(adj), _p(vw), _p(ew), int(target0), key_, _p(W), _p(side))
    return side[:n]


def async_cluster(g, U, rounds, seed=1):
    n, xadj, adj, vw, ew = _g(g)
    label = np.zeros(n, np.int32)
    nc = lib().kmpo_async_cluster(n, _p(xadj), _p(adj), _p(vw), _p(ew), U, rounds, seed, _p(label))
    return label, int(nc)
