"""Seeded synthetic graph generators (inputs for both the CUDA path and the oracle).

Holds no partitioning arithmetic: it builds symmetric CSR graphs with positive
integer weights, the input model of the paper's problem statement (Section 2).
Workload shapes follow the paper's benchmark families (Section 5): 2D random
geometric graphs (mesh-like, local) and R-MAT graphs (skewed degrees).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        from .. import _build

        path = _build.build_graphgen()
        lib = ctypes.CDLL(path)
        i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        p64 = ctypes.POINTER(ctypes.c_int64)
        pp32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
        lib.gg_rgg.argtypes = [i32, dbl, u64, p64, pp32]
        lib.gg_rgg.restype = i64
        lib.gg_rmat.argtypes = [i32, i32, dbl, dbl, dbl, u64, p64, pp32]
        lib.gg_rmat.restype = i64
        lib.gg_grid.argtypes = [i32, i32, p64, pp32]
        lib.gg_grid.restype = i64
        lib.gg_random.argtypes = [i32, i64, u64, p64, pp32]
        lib.gg_random.restype = i64
        lib.gg_hubs.argtypes = [i32, i32, ctypes.c_void_p, i64, u64, p64, pp32]
        lib.gg_hubs.restype = i64
        lib.gg_weights.argtypes = [i32, ctypes.c_void_p, ctypes.c_void_p, i32, i32, u64,
                                   ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_weights.restype = None
        lib.gg_free.argtypes = [ctypes.c_void_p]
        lib.gg_free.restype = None
        _LIB = lib
    return _LIB


@dataclass
class Graph:
    """Undirected graph in CSR form: xadj int64[n+1], adjncy int32[M],
    vwgt int32[n] or None (unit), adjwgt int32[M] or None (unit)."""

    n: int
    xadj: np.ndarray
    adjncy: np.ndarray
    vwgt: np.ndarray | None = None
    adjwgt: np.ndarray | None = None
    name: str = ""

    @property
    def m_directed(self) -> int:
        return int(self.xadj[-1])

    def vw(self) -> np.ndarray:
        return self.vwgt if self.vwgt is not None else np.ones(self.n, np.int32)

    def ew(self) -> np.ndarray:
        return self.adjwgt if self.adjwgt is not None else np.ones(self.m_directed, np.int32)


def _finish(n, xadj, adjp, m, name):
    adj = np.ctypeslib.as_array(adjp, shape=(max(m, 1),))[:m].copy()
    _lib().gg_free(ctypes.cast(adjp, ctypes.c_void_p))
    return Graph(n=n, xadj=xadj, adjncy=adj.astype(np.int32, copy=False), name=name)


def rgg(n: int, avg_deg: float, seed: int) -> Graph:
    """2D random geometric graph: n points uniform in the unit square, radius
    sqrt(avg_deg/(pi n)); ids ordered by grid cell (spatial locality)."""
    xadj = np.zeros(n + 1, np.int64)
    adjp = ctypes.POINTER(ctypes.c_int32)()
    m = _lib().gg_rgg(n, float(avg_deg), seed, xadj.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                      ctypes.byref(adjp))
    return _finish(n, xadj, adjp, m, f"rgg_n{n}_d{avg_deg:g}_s{seed}")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19) -> Graph:
    """R-MAT graph, symmetrised, deduplicated, self-loops removed, ids randomly permuted."""
    n = 1 << scale
    xadj = np.zeros(n + 1, np.int64)
    adjp = ctypes.POINTER(ctypes.c_int32)()
    m = _lib().gg_rmat(scale, edge_factor, a, b, c, seed,
                       xadj.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(adjp))
    return _finish(n, xadj, adjp, m, f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def grid(a: int, b: int) -> Graph:
    """a x b grid graph; vertex (i, j) has id i*b + j."""
    n = a * b
    xadj = np.zeros(n + 1, np.int64)
    adjp = ctypes.POINTER(ctypes.c_int32)()
    m = _lib().gg_grid(a, b, xadj.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(adjp))
    return _finish(n, xadj, adjp, m, f"grid_{a}x{b}")


def path(n: int) -> Graph:
    g = grid(1, n)
    g.name = f"path_{n}"
    return g


def random_graph(n: int, m_samples: int, seed: int) -> Graph:
    xadj = np.zeros(n + 1, np.int64)
    adjp = ctypes.POINTER(ctypes.c_int32)()
    m = _lib().gg_random(n, m_samples, seed, xadj.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                         ctypes.byref(adjp))
    return _finish(n, xadj, adjp, m, f"random_n{n}_m{m_samples}_s{seed}")


def hubs(n: int, hub_degrees, bg_samples: int, seed: int) -> Graph:
    """Sparse random background plus hub vertices 0..h-1 with the given sample
    counts; covers every degree class from isolated to very high degree."""
    hd = np.ascontiguousarray(np.asarray(hub_degrees, np.int32))
    xadj = np.zeros(n + 1, np.int64)
    adjp = ctypes.POINTER(ctypes.c_int32)()
    m = _lib().gg_hubs(n, len(hd), hd.ctypes.data, bg_samples, seed,
                       xadj.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(adjp))
    return _finish(n, xadj, adjp, m, f"hubs_n{n}_s{seed}")


def with_weights(g: Graph, vmax: int, emax: int, seed: int) -> Graph:
    """Attach symmetric random integer weights (vertex 1..vmax, edge 1..emax)."""
    vw = np.zeros(g.n, np.int32) if vmax > 0 else None
    ew = np.zeros(g.m_directed, np.int32) if emax > 0 else None
    _lib().gg_weights(g.n, g.xadj.ctypes.data, g.adjncy.ctypes.data, max(vmax, 1), max(emax, 1), seed,
                      vw.ctypes.data if vw is not None else None,
                      ew.ctypes.data if ew is not None else None)
    return Graph(g.n, g.xadj, g.adjncy, vw, ew, g.name + f"_w{vmax}_{emax}")


def subgraph(g: Graph, vertices) -> Graph:
    """Induced subgraph on the given vertex ids (kept in ascending order)."""
    vs = np.unique(np.asarray(vertices, np.int64))
    loc = -np.ones(g.n, np.int64)
    loc[vs] = np.arange(len(vs))
    rows, adj, ew = [0], [], []
    gew = g.ew()
    for v in vs:
        s, e = g.xadj[v], g.xadj[v + 1]
        nb = g.adjncy[s:e]
        keep = loc[nb] >= 0
        adj.append(loc[nb][keep])
        ew.append(gew[s:e][keep])
        rows.append(rows[-1] + int(keep.sum()))
    adjn = np.concatenate(adj).astype(np.int32) if adj else np.zeros(0, np.int32)
    ewn = np.concatenate(ew).astype(np.int32) if ew else np.zeros(0, np.int32)
    vw = g.vw()[vs].astype(np.int32)
    return Graph(len(vs), np.asarray(rows, np.int64), adjn, vw, ewn, g.name + "_sub")


def from_edges(n: int, edges, vwgt=None, ew=None) -> Graph:
    """Build a symmetric CSR from an undirected edge list [(u, v, w), ...] or [(u, v), ...]."""
    ent = {}
    for e in edges:
        u, v = int(e[0]), int(e[1])
        w = int(e[2]) if len(e) > 2 else 1
        if u == v:
            continue
        ent[(u, v)] = w
        ent[(v, u)] = w
    keys = sorted(ent)
    xadj = np.zeros(n + 1, np.int64)
    for u, _ in keys:
        xadj[u + 1] += 1
    xadj = np.cumsum(xadj).astype(np.int64)
    adj = np.asarray([v for _, v in keys], np.int32)
    wts = np.asarray([ent[k] for k in keys], np.int32)
    has_w = any(len(e) > 2 for e in edges)
    vw = None if vwgt is None else np.asarray(vwgt, np.int32)
    return Graph(n, xadj, adj, vw, wts if has_w else None, "edges")


# Workload shapes used by tests and the bench (synthetic stand-ins for the
# paper's benchmark sets, which are not available here).
def workload_rgg_small(seed: int = 1) -> Graph:
    """2D RGG, n = 2^15, average degree ~8, unit weights (k = 8 case)."""
    return rgg(1 << 15, 8.0, seed)


def workload_rmat20(seed: int = 1) -> Graph:
    """R-MAT scale 20, edge factor 16, (0.57, 0.19, 0.19, 0.05), unit weights (k = 256 case)."""
    return rmat(20, 16, seed)
