"""GPU parity of the batched initial bipartitioner (Algorithm 2 split round),
k-way balancing and the full deep multilevel partition (Algorithm 1) against
the CPU oracle, through the C ABI.  Integer outputs: bit-exact."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2105_02022_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kmp():
    from paper_2105_02022_gb300 import _build
    from paper_2105_02022_gb300 import kmp as K

    _build.build_all()
    O.build()
    assert torch.cuda.is_available()
    K.set_config(K.config())
    return K


def _split_case(name):
    if name == "rgg_root":
        g = gg.rgg(4096, 8, 3)
        return g, np.zeros(g.n, np.int32), [8], 8
    if name == "rgg_16blocks":
        g = gg.rgg(20000, 8, 4)
        return g, (np.arange(g.n) * 16 // g.n).astype(np.int32), [2] * 16, 32
    if name == "weighted_generalk":
        g = gg.with_weights(gg.rgg(6000, 10, 5), 7, 30, 5)
        return g, (np.arange(g.n) * 4 // g.n).astype(np.int32), [3, 2, 1, 5], 11
    if name == "hubs_items":
        g = gg.hubs(8000, [500, 900], 16000, 7)
        return g, (np.arange(g.n) % 3).astype(np.int32), [2, 4, 2], 8
    if name == "tiny_blocks":
        g = gg.rgg(300, 6, 9)
        part = np.zeros(g.n, np.int32)
        part[0] = 1          # a one-node block
        part[1:3] = 2        # a two-node block; block 3 stays empty
        return g, part, [2, 2, 2, 2], 8
    if name == "rmat_blocks":
        g = gg.rmat(13, 8, 3)
        rng = np.random.default_rng(3)
        return g, rng.integers(0, 6, g.n).astype(np.int32), [2, 2, 3, 1, 2, 6], 16
    raise KeyError(name)


SPLITS = ["rgg_root", "rgg_16blocks", "weighted_generalk", "hubs_items", "tiny_blocks", "rmat_blocks"]


@pytest.mark.parametrize("name", SPLITS)
def test_bipartition_blocks_parity(kmp, name):
    g, part, f, k = _split_case(name)
    cV = int(g.vw().sum())
    rk = O.key(5, [3, 1, 0])
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    nb, fo = kmp.bipartition_blocks(dg, len(f), f, 0.03, cV, k, rk, pt)
    rp, rf = O.bipartition_blocks(g, len(f), f, 0.03, cV, k, rk, part)
    assert nb == len(rf) and np.array_equal(fo, rf)
    assert np.array_equal(pt.cpu().numpy(), rp)


@pytest.mark.parametrize("cfgkw", [dict(rep_random=1, rep_bfs=0, rep_ggg=0), dict(fm_passes=0),
                                   dict(ip_lp_rounds=1, subrounds=2), dict(rep_ggg=17, fm_stop=3),
                                   dict(adaptive=1), dict(adaptive=1, rep_random=3, rep_bfs=5, rep_ggg=9),
                                   dict(adaptive=1, rep_random=0, rep_bfs=2, rep_ggg=1)])
def test_bipartition_config_variants(kmp, cfgkw):
    g, part, f, k = _split_case("rgg_16blocks")
    kmp.set_config(kmp.config(**cfgkw))
    try:
        cV = int(g.vw().sum())
        dg = kmp.DeviceGraph.from_host(g)
        pt = torch.from_numpy(part).cuda()
        kmp.bipartition_blocks(dg, len(f), f, 0.03, cV, k, 77, pt)
        rp, _ = O.bipartition_blocks(g, len(f), f, 0.03, cV, k, 77, part, cfg=O.config(**cfgkw))
        assert np.array_equal(pt.cpu().numpy(), rp)
    finally:
        kmp.set_config(kmp.config())


@pytest.mark.parametrize("case", ["rgg", "weighted", "rmat", "hubs_k1024"])
def test_balance_parity(kmp, case):
    k = 6
    if case == "rgg":
        g = gg.rgg(5000, 8, 3)
    elif case == "weighted":
        g = gg.with_weights(gg.rgg(5000, 8, 4), 9, 5, 4)
    elif case == "rmat":
        g = gg.rmat(13, 8, 5)
    else:
        # hubs with more than 256 distinct neighbour blocks: their connectivity
        # tables exceed a warp's shared table (global-table candidate pass,
        # speculation hands them to the exact commit, per-member commit tables)
        g = gg.hubs(30000, [3000, 12000, 700, 2500], 60000, 8)
        k = 1024
    part = (np.arange(g.n) * k // g.n).astype(np.int32)
    part[g.n // 6: g.n // 3] = 0
    part[g.n // 2: g.n // 2 + 300] = 5
    cap = np.full(k, int(1.03 * g.vw().sum() / k), np.int64)
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    mv = kmp.balance(dg, k, cap, pt)
    rp, rmv = O.balance(g, k, cap.astype(np.int32), part)
    assert mv == rmv and mv > 0
    assert np.array_equal(pt.cpu().numpy(), rp)


@pytest.mark.parametrize("name,k", [("rmat15", 512), ("rgg", 2000), ("rmat15_w", 300)])
def test_balance_random_partitions_many_overloaded_blocks(kmp, name, k):
    """A random k-way partition overloads about half of the blocks, nearly all
    of them neighbours (R-MAT) or spatially close (RGG), so most speculated
    moves are fragile and go through the exact commit; bit-exact with the
    oracle."""
    if name == "rmat15":
        g = gg.rmat(15, 16, 3)
    elif name == "rgg":
        g = gg.rgg(40000, 8, 5)
    else:
        g = gg.with_weights(gg.rmat(15, 16, 4), 4, 9, 4)
    rng = np.random.default_rng(k)
    part = rng.integers(0, k, g.n).astype(np.int32)
    cap = np.full(k, int(1.03 * g.vw().sum() / k) + int(g.vw().max()), np.int64)
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    mv = kmp.balance(dg, k, cap, pt)
    rp, rmv = O.balance(g, k, cap.astype(np.int32), part)
    assert mv == rmv and mv > 0
    assert np.array_equal(pt.cpu().numpy(), rp)


def test_balance_many_adjacent_overloaded_blocks(kmp):
    """480 blocks of 15 and 10 nodes alternating over an RGG whose ids are
    spatially local, cap 12: half the blocks are overloaded and most border
    another one, so candidates' connectivities change as earlier blocks are
    emptied (the cases the speculative schedule must hand to the exact commit)"""
    g = gg.rgg(6000, 8, 3)
    k = 480
    sizes = np.where(np.arange(k) % 2 == 0, 15, 10)
    sizes[-1] += g.n - sizes.sum()
    part = np.repeat(np.arange(k), sizes).astype(np.int32)
    cap = np.full(k, int(1.03 * g.n / k), np.int64)
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    mv = kmp.balance(dg, k, cap, pt)
    rp, rmv = O.balance(g, k, cap.astype(np.int32), part)
    assert mv == rmv and mv > 0
    assert np.array_equal(pt.cpu().numpy(), rp)


def _same_schedule(st, rst):
    """Level sizes, k', U and block counts per level equal the oracle's."""
    assert st.levels == rst.levels
    assert list(st.level_n[: st.levels]) == list(rst.level_n[: rst.levels])
    assert list(st.level_k[: st.levels]) == list(rst.level_k[: rst.levels])
    assert st.clustered == rst.clustered
    assert list(st.level_kp[: st.clustered]) == list(rst.level_kp[: rst.clustered])
    assert list(st.level_U[: st.clustered]) == list(rst.level_U[: rst.clustered])


PARTS = [
    ("path", lambda: gg.path(700), [2, 5]),
    ("grid", lambda: gg.grid(40, 60), [2, 4, 7]),
    ("rgg15", lambda: gg.workload_rgg_small(1), [8, 3, 64]),
    ("rgg_w", lambda: gg.with_weights(gg.rgg(12000, 8, 6), 5, 9, 6), [7, 16]),
    ("rmat14", lambda: gg.rmat(14, 16, 2), [32, 5]),
    ("hubs", lambda: gg.hubs(30000, [3000, 12000], 60000, 8), [16, 600]),
    # 16 nodes per block: L_k leaves no slack, so the result may be infeasible
    # (both sides must agree on that too)
    ("rgg15_k2048", lambda: gg.workload_rgg_small(1), [2048]),
]


REPL = [
    ("rgg15", lambda: gg.workload_rgg_small(1), 8, [2, 4, 8]),
    ("rgg_w", lambda: gg.with_weights(gg.rgg(12000, 8, 6), 5, 9, 6), 7, [2, 4]),
    ("rmat14", lambda: gg.rmat(14, 16, 2), 32, [2, 8]),
    ("rgg300", lambda: gg.rgg(300, 8, 6), 2, [2]),
]


@pytest.mark.parametrize("name,make,k,Rs", REPL, ids=[p[0] for p in REPL])
def test_replication_parity(kmp, name, make, k, Rs):
    """Replication of the coarsest levels (Section 3, "Parallelization") on
    the GPU against the oracle, bit for bit"""
    g = make()
    dg = kmp.DeviceGraph.from_host(g)
    try:
        for R in Rs:
            kmp.set_config(kmp.config(replicas=R))
            part, rc, st = kmp.partition_graph(dg, k, 0.03, 1)
            rp, rrc, rst = O.partition(g, k, 0.03, 1, O.config(replicas=R))
            assert np.array_equal(part.cpu().numpy(), rp), (name, R)
            assert rc == rrc and st.cut == rst.cut and st.feasible == rst.feasible
            _same_schedule(st, rst)
    finally:
        kmp.set_config(kmp.config())


@pytest.mark.parametrize("name,make,ks", PARTS, ids=[p[0] for p in PARTS])
def test_partition_parity(kmp, name, make, ks):
    g = make()
    dg = kmp.DeviceGraph.from_host(g)
    for k in ks:
        for seed in (1, 2):
            part, rc, st = kmp.partition_graph(dg, k, 0.03, seed)
            rp, rrc, rst = O.partition(g, k, 0.03, seed)
            got = part.cpu().numpy()
            assert np.array_equal(got, rp), (name, k, seed)
            assert rc == rrc and st.cut == rst.cut and st.feasible == rst.feasible
            _same_schedule(st, rst)


def test_schedule_halving_chain_on_isolated_nodes(kmp):
    """2^15 isolated unit nodes, k = 128, eps = 0.0157: every level is known
    in closed form (Section 4.1 and Algorithm 1, readings D1 and D2; the
    derivation is in the oracle's pin of the same name).  The GPU partition
    is bit-exact with the oracle and its schedule equals the hand values."""
    n = 1 << 15
    g = gg.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), None, None)
    dg = kmp.DeviceGraph.from_host(g)
    part, rc, st = kmp.partition_graph(dg, 128, 0.0157, 1)
    rp, rrc, rst = O.partition(g, 128, 0.0157, 1)
    assert np.array_equal(part.cpu().numpy(), rp) and rc == rrc
    assert list(st.level_n[:7]) == [32768, 8192, 4096, 2048, 1024, 512, 256] and st.levels == 7
    assert list(st.level_kp[:6]) == [128, 64, 32, 16, 8, 4]
    assert list(st.level_U[:6]) == [4, 8, 16, 32, 64, 128]
    assert list(st.level_k[:7]) == [128, 64, 32, 16, 8, 4, 2]
    _same_schedule(st, rst)


@pytest.mark.parametrize("tune", [(4, 1024, 1024, 2, 600, 0, 64, 57344), (8, 2048, 4096, 8, 1 << 30, 1, 1 << 20, 0),
                                  (2, 256, 256, 1, 4096, 0, 0)])
def test_tuning_invariance(kmp, tune):
    """Schedule parameters (grids, hub threshold, chunking) never change results."""
    g = gg.hubs(30000, [700, 3000, 12000], 60000, 8)
    dg = kmp.DeviceGraph.from_host(g)
    old = kmp.get_tuning()
    try:
        kmp.set_tuning(kmp.Tuning(*tune))
        for k in (16, 5):
            part, rc, st = kmp.partition_graph(dg, k, 0.03, 3)
            rp, rrc, _ = O.partition(g, k, 0.03, 3)
            assert np.array_equal(part.cpu().numpy(), rp)
    finally:
        kmp.set_tuning(old)


def test_autotune_then_parity(kmp):
    g = gg.rmat(14, 16, 5)
    dg = kmp.DeviceGraph.from_host(g)
    old = kmp.get_tuning()
    try:
        best = kmp.autotune(dg, 32, 0.03, 1)
        assert best.rate_blocks_per_sm in (4, 6, 8) and best.hub_degree in (1024, 2048)
        part, rc, st = kmp.partition_graph(dg, 32, 0.03, 1)
        rp, rrc, _ = O.partition(g, 32, 0.03, 1)
        assert np.array_equal(part.cpu().numpy(), rp)
    finally:
        kmp.set_tuning(old)


def test_host_partition_entry(kmp):
    g = gg.rgg(6000, 8, 11)
    part, rc = kmp.partition(g, 12, 0.05, 4)
    rp, rrc, _ = O.partition(g, 12, 0.05, 4)
    assert np.array_equal(part, rp) and rc == rrc == 0


def test_partition_edge_cases(kmp):
    g = gg.rgg(2000, 8, 1)
    dg = kmp.DeviceGraph.from_host(g)
    part, rc, st = kmp.partition_graph(dg, 1, 0.03, 1)
    assert rc == 0 and not part.any().item()
    # more blocks than nodes
    small = gg.rgg(40, 6, 2)
    ds = kmp.DeviceGraph.from_host(small)
    part, rc, st = kmp.partition_graph(ds, 64, 0.03, 1)
    rp, rrc, _ = O.partition(small, 64, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), rp) and rc == rrc
    # isolated nodes only
    iso = gg.Graph(500, np.zeros(501, np.int64), np.zeros(0, np.int32), None, None)
    di = kmp.DeviceGraph.from_host(iso)
    part, rc, st = kmp.partition_graph(di, 4, 0.03, 1)
    rp, rrc, _ = O.partition(iso, 4, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), rp) and rc == rrc
    with pytest.raises(kmp.KmpError):
        kmp.partition_graph(dg, 0, 0.03, 1)
    with pytest.raises(kmp.KmpError):
        kmp.partition_graph(dg, 4, 0.0, 1)


def test_full_size_rmat20_k256(kmp):
    """The R-MAT scale-20, k = 256 workload exactly as the benchmark runs it:
    partition, cut and balance bit-exact with the oracle."""
    g = gg.workload_rmat20(1)
    dg = kmp.DeviceGraph.from_host(g)
    part, rc, st = kmp.partition_graph(dg, 256, 0.03, 1)
    rp, rrc, rst = O.partition(g, 256, 0.03, 1)
    assert np.array_equal(part.cpu().numpy(), rp)
    assert rc == rrc == 0 and st.cut == rst.cut and st.feasible == 1


def _golden(name):
    import os

    out = {}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            out[key] = vals if len(vals) > 1 else vals[0]
    return out


def test_full_size_rgg24_k16384(kmp):
    """The large-k case: 2D RGG with 2^24 nodes (average degree ~16), k = 2^14.
    The whole partition is bit-exact with the oracle's: its SHA-256, cut,
    status and level sizes equal the stored record that
    tests/golden/make_partition_golden.py wrote by running the oracle alone.
    Also checked: the input level's coarsening bit-exactly against the oracle
    (the driver's cluster cap), every block within L_k = floor(1.03 ceil(n/k)),
    the reported cut equal to a recount, and the same result on a second run."""
    import hashlib

    rec = _golden("rgg24_k16384_partition.txt")
    g = gg.rgg(1 << 24, 16, 1)
    k = 1 << 14
    dg = kmp.DeviceGraph.from_host(g)
    kp = min(k, g.n // kmp.get_config().C)
    U = int(np.floor(0.03 * g.n / kp))
    label = kmp.coarsen_level(dg, U, 5, 1, 0)
    assert np.array_equal(label.cpu().numpy(), O.cluster(g, U, 5, 1, 0))
    part, rc, st = kmp.partition_graph(dg, k, 0.03, 1)
    part2, rc2, st2 = kmp.partition_graph(dg, k, 0.03, 1)
    assert rc == rc2 == 0 and st.feasible == 1
    assert torch.equal(part, part2) and st.cut == st2.cut
    p = part.cpu().numpy()
    assert p.min() >= 0 and p.max() < k
    Lk = int(np.floor(1.03 * ((g.n + k - 1) // k)))
    assert np.bincount(p, minlength=k).max() <= Lk
    cut, bw = kmp.cut(dg, part, k)
    assert cut == st.cut and int(bw.sum()) == g.n
    assert int(rec["n"]) == g.n and int(rec["m_directed"]) == g.m_directed
    assert hashlib.sha256(np.ascontiguousarray(p, dtype="<i4").tobytes()).hexdigest() == rec["sha256"]
    assert st.cut == int(rec["cut"]) and rc == int(rec["status"])
    assert [int(x) for x in rec["level_n"]] == list(st.level_n[: st.levels])


@pytest.mark.parametrize("name,make,k", [("rgg15", lambda: gg.workload_rgg_small(1), 64),
                                         ("rmat14", lambda: gg.rmat(14, 16, 2), 32),
                                         ("rgg_w", lambda: gg.with_weights(gg.rgg(12000, 8, 6), 5, 9, 6), 16)])
def test_adaptive_partition_parity(kmp, name, make, k):
    """Adaptive portfolio selection (Section 4.2, reading B7) in every split
    round of a full partition: bit-exact with the oracle."""
    g = make()
    dg = kmp.DeviceGraph.from_host(g)
    kmp.set_config(kmp.config(adaptive=1))
    try:
        part, rc, st = kmp.partition_graph(dg, k, 0.03, 1)
    finally:
        kmp.set_config(kmp.config())
    rp, rrc, rst = O.partition(g, k, 0.03, 1, O.config(adaptive=1))
    assert np.array_equal(part.cpu().numpy(), rp)
    assert rc == rrc and st.cut == rst.cut
