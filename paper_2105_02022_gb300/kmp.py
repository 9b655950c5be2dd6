"""Thin Python binding of libkmp's C ABI (include/kmp.h): argument marshalling
only.  Device memory and streams come from PyTorch; every step of the method
runs in the library's CUDA kernels.  Importing this module does not build
anything: when libkmp.so is missing, load() raises, so a missing extension
fails loudly instead of falling back to any CPU code."""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _build

KMP_OK = 0
KMP_ERR_ARG = -1
KMP_ERR_NOMEM = -2
KMP_ERR_CUDA = -3
KMP_ERR_TIMEOUT = -4
KMP_ERR_INFEASIBLE = -5
KMP_ERR_UNSUPPORTED = -6

_LIB = None


class KmpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kmp error {code}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "C", "lp_rounds", "refine_rounds", "subrounds", "two_hop", "conv_num", "conv_den",
        "ip_C", "ip_lp_rounds", "rep_random", "rep_bfs", "rep_ggg", "fm_passes", "fm_stop",
        "learned", "lrep_random", "lrep_bfs", "lrep_ggg", "replicas", "adaptive")]


class Stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("level_n", ctypes.c_int32 * 64),
                ("level_m", ctypes.c_int64 * 64), ("lp_scanned", ctypes.c_int64),
                ("refine_scanned", ctypes.c_int64), ("lp_rounds_run", ctypes.c_int64),
                ("cut", ctypes.c_int64), ("feasible", ctypes.c_int32), ("ip_items", ctypes.c_int32),
                ("ms_lp", ctypes.c_float), ("ms_cluster_other", ctypes.c_float),
                ("ms_contract", ctypes.c_float), ("ms_ip", ctypes.c_float),
                ("ms_balance", ctypes.c_float), ("ms_refine", ctypes.c_float),
                ("ms_project", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("ms_lp_level0", ctypes.c_float), ("lp_scanned_level0", ctypes.c_int64),
                ("lp_rounds_level0", ctypes.c_int32), ("gpu_launches", ctypes.c_int32),
                ("clustered", ctypes.c_int32), ("level_kp", ctypes.c_int32 * 64),
                ("level_U", ctypes.c_int64 * 64), ("level_k", ctypes.c_int32 * 64),
                ("bal_over_blocks", ctypes.c_int64), ("bal_moves", ctypes.c_int64),
                ("bal_spec_moves", ctypes.c_int64), ("bal_exact_batches", ctypes.c_int64),
                ("bal_exact_cands", ctypes.c_int64), ("bal_exact_entries", ctypes.c_int64)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            if name in ("level_n", "level_m", "level_k"):
                v = list(v)[: self.levels]
            elif name in ("level_kp", "level_U"):
                v = list(v)[: self.clustered]
            d[name] = v
        return d


class Tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in (
        "rate_blocks_per_sm", "hub_degree", "hub_chunk", "ip_blocks_per_sm", "dense_hub_degree", "lp_graphs",
        "hub_bucket", "dense_labels")]


def load():
    """Load libkmp.so (built by __graft_entry__.build()); raise if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError(f"libkmp.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "kmp_config_default": (None, [P]),
        "kmp_set_config": (ctypes.c_int, [P]),
        "kmp_get_config": (ctypes.c_int, [P]),
        "kmp_set_stream": (ctypes.c_int, [P]),
        "kmp_last_error": (ctypes.c_char_p, []),
        "kmp_graph_create": (ctypes.c_int, [i32, P, P, P, P, ctypes.c_int, PP]),
        "kmp_graph_free": (ctypes.c_int, [P]),
        "kmp_graph_get": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "kmp_graph_copy_to_host": (ctypes.c_int, [P, P, P, P, P]),
        "kmp_coarsen_level": (ctypes.c_int, [P, i64, i32, u64, i32, P, P]),
        "kmp_contract": (ctypes.c_int, [P, P, PP, P]),
        "kmp_refine": (ctypes.c_int, [P, i32, P, i32, u64, P, P]),
        "kmp_balance": (ctypes.c_int, [P, i32, P, P, P]),
        "kmp_project": (ctypes.c_int, [i32, P, P, P]),
        "kmp_cut": (ctypes.c_int, [P, P, i32, P, P]),
        "kmp_cut_noalloc": (ctypes.c_int, [P, P, i32, P, P]),
        "kmp_bipartition_blocks": (ctypes.c_int, [P, i32, P, dbl, i64, i32, u64, P, P, P]),
        "kmp_bipartition_each": (ctypes.c_int, [P, i32, P, u64, P]),
        "kmp_partition": (ctypes.c_int, [i32, P, P, P, P, i32, dbl, u64, P]),
        "kmp_partition_graph": (ctypes.c_int, [P, i32, dbl, u64, P, P]),
        "kmp_last_stats": (ctypes.c_int, [P]),
        "kmp_set_profiling": (ctypes.c_int, [ctypes.c_int]),
        "kmp_mpnn_num_params": (ctypes.c_int, []),
        "kmp_mpnn_create": (ctypes.c_int, [u64, PP]),
        "kmp_mpnn_free": (ctypes.c_int, [P]),
        "kmp_mpnn_get_params": (ctypes.c_int, [P, P]),
        "kmp_mpnn_set_params": (ctypes.c_int, [P, P]),
        "kmp_mpnn_forward": (ctypes.c_int, [P, i32, P, P, P, P, P, P, P, P]),
        "kmp_mpnn_gradients": (ctypes.c_int, [P, i32, P, P, P, P, P, P, P, P, P]),
        "kmp_mpnn_train": (ctypes.c_int, [P, i32, P, P, P, P, P, P, P, i32, ctypes.c_float, P]),
        "kmp_set_proposer": (ctypes.c_int, [P]),
        "kmp_sample_sink_open": (ctypes.c_int, [i32, i64, i64]),
        "kmp_sample_sink_count": (ctypes.c_int, [P, P, P, P]),
        "kmp_sample_sink_read": (ctypes.c_int, [P, P, P, P, P, P, P]),
        "kmp_sample_sink_close": (ctypes.c_int, []),
        "kmp_sample_sink_level": (ctypes.c_int, [i32]),
        "kmp_set_tuning": (ctypes.c_int, [P]),
        "kmp_get_tuning": (ctypes.c_int, [P]),
        "kmp_autotune": (ctypes.c_int, [P, i32, dbl, u64, P]),
        "kmp_profile_read": (ctypes.c_int, [P, P, P, ctypes.c_int]),
        "kmp_profile_read_stage": (ctypes.c_int, [P, P, P, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = L
    return L


def _check(rc: int, allow=()):
    if rc != KMP_OK and rc not in allow:
        raise KmpError(rc, load().kmp_last_error().decode())
    return rc


def _stream():
    load().kmp_set_stream(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def config(**kw) -> Config:
    c = Config()
    load().kmp_config_default(ctypes.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def set_config(cfg: Config):
    _check(load().kmp_set_config(ctypes.byref(cfg)))


def get_config() -> Config:
    c = Config()
    _check(load().kmp_get_config(ctypes.byref(c)))
    return c


class DeviceGraph:
    """Owning handle of a kmp_graph (CSR in device memory)."""

    def __init__(self, handle):
        self.h = handle

    @classmethod
    def from_host(cls, g) -> "DeviceGraph":
        L = load()
        _stream()
        xadj = np.ascontiguousarray(g.xadj, np.int64)
        adj = np.ascontiguousarray(g.adjncy, np.int32)
        vw = None if g.vwgt is None else np.ascontiguousarray(g.vwgt, np.int32)
        ew = None if g.adjwgt is None else np.ascontiguousarray(g.adjwgt, np.int32)
        h = ctypes.c_void_p()
        _check(L.kmp_graph_create(g.n, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew), 0, ctypes.byref(h)))
        return cls(h)

    @classmethod
    def from_device(cls, n, xadj: torch.Tensor, adj: torch.Tensor, vw=None, ew=None) -> "DeviceGraph":
        L = load()
        _stream()
        h = ctypes.c_void_p()
        _check(L.kmp_graph_create(n, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew), 1, ctypes.byref(h)))
        return cls(h)

    def info(self):
        n, m = ctypes.c_int32(), ctypes.c_int64()
        _check(load().kmp_graph_get(self.h, ctypes.byref(n), ctypes.byref(m), None, None, None, None))
        return n.value, m.value

    @property
    def n(self):
        return self.info()[0]

    @property
    def m(self):
        return self.info()[1]

    def to_host(self):
        from .graphgen import Graph

        n, m = self.info()
        xadj = np.zeros(n + 1, np.int64)
        adj = np.zeros(max(m, 1), np.int32)
        vw = np.zeros(max(n, 1), np.int32)
        ew = np.zeros(max(m, 1), np.int32)
        _stream()
        _check(load().kmp_graph_copy_to_host(self.h, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew)))
        return Graph(n, xadj, adj[:m], vw[:n], ew[:m], "device")

    def free(self):
        if self.h:
            load().kmp_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _i32(n, device="cuda"):
    return torch.empty(max(int(n), 1), dtype=torch.int32, device=device)[: int(n)]


def coarsen_level(dg: DeviceGraph, U: int, rounds: int, seed: int, level: int, fav=False):
    _stream()
    n = dg.n
    label = _i32(n)
    favt = _i32(n) if fav else None
    _check(load().kmp_coarsen_level(dg.h, int(U), int(rounds), int(seed), int(level), _ptr(label), _ptr(favt)))
    return (label, favt) if fav else label


def contract(dg: DeviceGraph, label: torch.Tensor):
    _stream()
    mp = _i32(label.numel())
    h = ctypes.c_void_p()
    _check(load().kmp_contract(dg.h, _ptr(label), ctypes.byref(h), _ptr(mp)))
    return DeviceGraph(h), mp


def refine(dg: DeviceGraph, k: int, caps, rounds: int, seed: int, part: torch.Tensor) -> int:
    _stream()
    caps = np.ascontiguousarray(caps, np.int64)
    cut = ctypes.c_int64()
    _check(load().kmp_refine(dg.h, int(k), _ptr(caps), int(rounds), int(seed), _ptr(part), ctypes.byref(cut)))
    return cut.value


def balance(dg: DeviceGraph, k: int, caps, part: torch.Tensor) -> int:
    _stream()
    caps = np.ascontiguousarray(caps, np.int64)
    mv = ctypes.c_int64()
    _check(load().kmp_balance(dg.h, int(k), _ptr(caps), _ptr(part), ctypes.byref(mv)))
    return mv.value


def project(mp: torch.Tensor, part_c: torch.Tensor) -> torch.Tensor:
    _stream()
    pf = _i32(mp.numel())
    _check(load().kmp_project(mp.numel(), _ptr(mp), _ptr(part_c), _ptr(pf)))
    return pf


def cut(dg: DeviceGraph, part: torch.Tensor, k: int):
    _stream()
    bw = np.zeros(k, np.int64)
    c = ctypes.c_int64()
    _check(load().kmp_cut(dg.h, _ptr(part), int(k), ctypes.byref(c), _ptr(bw)))
    return c.value, bw


KMP_NOALLOC_MAX_K = 65536


def cut_noalloc(dg: DeviceGraph, part: torch.Tensor, k: int):
    """Same result as cut(), computed without any device allocation (fixed
    library-side scratch; calls must not overlap)."""
    _stream()
    bw = np.zeros(max(int(k), 0), np.int64)
    c = ctypes.c_int64()
    _check(load().kmp_cut_noalloc(dg.h, _ptr(part), int(k), ctypes.byref(c), _ptr(bw) if k > 0 else None))
    return c.value, bw


def bipartition_each(dg: DeviceGraph, nblocks: int, caps, roundkey: int, part: torch.Tensor):
    """Bipartition every block with explicit (t0, t1, L0, L1) caps; part becomes 2b + side."""
    _stream()
    caps = np.ascontiguousarray(caps, np.int32).reshape(-1)
    assert caps.size == 4 * nblocks
    _check(load().kmp_bipartition_each(dg.h, int(nblocks), _ptr(caps), ctypes.c_uint64(roundkey), _ptr(part)))
    return part


def bipartition_blocks(dg: DeviceGraph, nblocks: int, f, eps: float, cV: int, k: int, roundkey: int,
                       part: torch.Tensor):
    _stream()
    f = np.ascontiguousarray(f, np.int32)
    fo = np.zeros(2 * nblocks, np.int32)
    nb = ctypes.c_int32()
    _check(load().kmp_bipartition_blocks(dg.h, int(nblocks), _ptr(f), float(eps), int(cV), int(k),
                                         ctypes.c_uint64(roundkey), _ptr(part), ctypes.byref(nb), _ptr(fo)))
    return nb.value, fo[: nb.value].copy()


def partition(g, k: int, eps: float, seed: int):
    """kmp_partition on a host CSR; returns (part numpy int32, return code)."""
    _stream()
    xadj = np.ascontiguousarray(g.xadj, np.int64)
    adj = np.ascontiguousarray(g.adjncy, np.int32)
    vw = None if g.vwgt is None else np.ascontiguousarray(g.vwgt, np.int32)
    ew = None if g.adjwgt is None else np.ascontiguousarray(g.adjwgt, np.int32)
    part = np.zeros(g.n, np.int32)
    rc = _check(load().kmp_partition(g.n, _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew), int(k), float(eps),
                                     ctypes.c_uint64(seed), _ptr(part)), allow=(KMP_ERR_INFEASIBLE,))
    return part, rc


def partition_graph(dg: DeviceGraph, k: int, eps: float, seed: int, part: torch.Tensor | None = None):
    """kmp_partition_graph on a device graph; returns (part tensor, rc, Stats)."""
    _stream()
    if part is None:
        part = _i32(dg.n)
    st = Stats()
    rc = _check(load().kmp_partition_graph(dg.h, int(k), float(eps), ctypes.c_uint64(seed), _ptr(part),
                                           ctypes.byref(st)), allow=(KMP_ERR_INFEASIBLE,))
    return part, rc, st


def last_stats() -> Stats:
    st = Stats()
    load().kmp_last_stats(ctypes.byref(st))
    return st


def set_tuning(t: Tuning):
    _check(load().kmp_set_tuning(ctypes.byref(t)))


def get_tuning() -> Tuning:
    t = Tuning()
    _check(load().kmp_get_tuning(ctypes.byref(t)))
    return t


def autotune(dg: DeviceGraph, k: int, eps: float, seed: int) -> Tuning:
    _stream()
    t = Tuning()
    _check(load().kmp_autotune(dg.h, int(k), float(eps), ctypes.c_uint64(seed), ctypes.byref(t)))
    return t


def set_profiling(on: bool):
    _check(load().kmp_set_profiling(1 if on else 0))


class Profile:
    """Sums of the live rating profile since the last reset."""

    def __init__(self, rate_ms, rate_bytes, rate_launches, stage_ms, stage_bytes, stage_spans):
        self.rate_ms, self.rate_bytes, self.rate_launches = rate_ms, rate_bytes, rate_launches
        self.stage_ms, self.stage_bytes, self.stage_spans = stage_ms, stage_bytes, stage_spans

    def __iter__(self):  # (ms, bytes, launches) of k_rate alone
        return iter((self.rate_ms, self.rate_bytes, self.rate_launches))

    def as_dict(self, peak_gbs=None):
        gbs = lambda by, ms: by / (ms / 1e3) / 1e9 if ms > 0 else None
        d = {"rate_ms": self.rate_ms, "rate_bytes": self.rate_bytes, "rate_launches": self.rate_launches,
             "rate_bytes_per_launch": self.rate_bytes / self.rate_launches if self.rate_launches else None,
             "rate_gbs": gbs(self.rate_bytes, self.rate_ms), "stage_ms": self.stage_ms,
             "stage_bytes": self.stage_bytes, "stage_spans": self.stage_spans,
             "stage_gbs": gbs(self.stage_bytes, self.stage_ms)}
        d["rate_frac"] = d["rate_gbs"] / peak_gbs if peak_gbs and d["rate_gbs"] else None
        d["stage_frac"] = d["stage_gbs"] / peak_gbs if peak_gbs and d["stage_gbs"] else None
        return d


def profile_read(reset: bool = False) -> Profile:
    """Rating profile sums since the last reset; unpacks as (ms, bytes, launches) of k_rate."""
    ms, by, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    sms, sby, sn = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    L = load()
    _check(L.kmp_profile_read(ctypes.byref(ms), ctypes.byref(by), ctypes.byref(n), 1 if reset else 0))
    _check(L.kmp_profile_read_stage(ctypes.byref(sms), ctypes.byref(sby), ctypes.byref(sn), 1 if reset else 0))
    return Profile(ms.value, by.value, n.value, sms.value, sby.value, sn.value)


# ------------------------------------------------------------ learned proposer
MPNN_PARAMS = 9409


class Batch:
    """Disjoint union of graphs in host arrays (the proposer's batch format)."""

    def __init__(self, noff, xadj, adj, vw, ew, keys, side=None):
        self.noff = np.ascontiguousarray(noff, np.int32)
        self.xadj = np.ascontiguousarray(xadj, np.int64)
        self.adj = np.ascontiguousarray(adj, np.int32)
        self.vw = None if vw is None else np.ascontiguousarray(vw, np.int32)
        self.ew = None if ew is None else np.ascontiguousarray(ew, np.int32)
        self.keys = np.ascontiguousarray(keys, np.uint64)
        self.side = None if side is None else np.ascontiguousarray(side, np.int32)

    @property
    def ng(self):
        return len(self.noff) - 1

    @property
    def n(self):
        return int(self.noff[-1])

    def _args(self):
        return (int(self.ng), _ptr(self.noff), _ptr(self.xadj), _ptr(self.adj), _ptr(self.vw), _ptr(self.ew),
                _ptr(self.keys))

    @staticmethod
    def from_graphs(graphs, keys, sides=None):
        noff, xs, adjs, vws, ews = [0], [np.zeros(1, np.int64)], [], [], []
        nb = eb = 0
        for g in graphs:
            xs.append(np.asarray(g.xadj[1:], np.int64) + eb)
            adjs.append(np.asarray(g.adjncy, np.int32) + nb)
            vws.append(np.ones(g.n, np.int32) if g.vwgt is None else np.asarray(g.vwgt, np.int32))
            ews.append(np.ones(len(g.adjncy), np.int32) if g.adjwgt is None else np.asarray(g.adjwgt, np.int32))
            nb += g.n
            eb += len(g.adjncy)
            noff.append(nb)
        side = None if sides is None else np.concatenate([np.asarray(x, np.int32) for x in sides])
        return Batch(noff, np.concatenate(xs), np.concatenate(adjs) if adjs else np.zeros(0, np.int32),
                     np.concatenate(vws), np.concatenate(ews) if ews else np.zeros(0, np.int32), keys, side)


class Mpnn:
    """A proposer model (device-resident weights, Adam state)."""

    def __init__(self, seed: int = 1):
        _stream()
        h = ctypes.c_void_p()
        _check(load().kmp_mpnn_create(ctypes.c_uint64(seed), ctypes.byref(h)))
        self.h = h

    def free(self):
        if self.h:
            _check(load().kmp_mpnn_free(self.h))
            self.h = None

    def get_params(self):
        p = np.zeros(MPNN_PARAMS, np.float32)
        _check(load().kmp_mpnn_get_params(self.h, _ptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == MPNN_PARAMS
        _check(load().kmp_mpnn_set_params(self.h, _ptr(p)))

    def forward(self, b: Batch, features=False):
        _stream()
        S = np.zeros(max(b.n, 1), np.float32)
        X = np.zeros((max(b.n, 1), 8), np.float32) if features else None
        _check(load().kmp_mpnn_forward(self.h, *b._args(), _ptr(S), _ptr(X)))
        return (S[: b.n], X[: b.n]) if features else S[: b.n]

    def gradients(self, b: Batch):
        _stream()
        loss = ctypes.c_float()
        g = np.zeros(MPNN_PARAMS, np.float32)
        _check(load().kmp_mpnn_gradients(self.h, *b._args(), _ptr(b.side), ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, b: Batch, epochs: int, lr: float):
        _stream()
        losses = np.zeros(max(epochs, 1), np.float32)
        _check(load().kmp_mpnn_train(self.h, *b._args(), _ptr(b.side), int(epochs), ctypes.c_float(lr),
                                     _ptr(losses)))
        return losses[:epochs]


def set_proposer(m: "Mpnn | None"):
    _check(load().kmp_set_proposer(m.h if m is not None else None))


def sample_sink_open(max_graphs: int, max_nodes: int, max_entries: int, item_level: int = 0):
    """Open the sink; item_level 1 records item graphs with their final bipartitions."""
    _stream()
    _check(load().kmp_sample_sink_open(int(max_graphs), int(max_nodes), int(max_entries)))
    _check(load().kmp_sample_sink_level(int(item_level)))


def sample_sink_read():
    """(Batch of the kept samples with their sides, dropped count)."""
    ng, nn, ne, dr = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().kmp_sample_sink_count(ctypes.byref(ng), ctypes.byref(nn), ctypes.byref(ne), ctypes.byref(dr)))
    noff = np.zeros(ng.value + 1, np.int32)
    xadj = np.zeros(nn.value + 1, np.int64)
    adj = np.zeros(max(ne.value, 1), np.int32)
    vw = np.zeros(max(nn.value, 1), np.int32)
    ew = np.zeros(max(ne.value, 1), np.int32)
    keys = np.zeros(max(ng.value, 1), np.uint64)
    side = np.zeros(max(nn.value, 1), np.int32)
    _check(load().kmp_sample_sink_read(_ptr(noff), _ptr(xadj), _ptr(adj), _ptr(vw), _ptr(ew), _ptr(keys), _ptr(side)))
    b = Batch(noff, xadj, adj[: ne.value], vw[: nn.value], ew[: ne.value], keys[: ng.value], side[: nn.value])
    return b, dr.value


def sample_sink_close():
    _check(load().kmp_sample_sink_close())

