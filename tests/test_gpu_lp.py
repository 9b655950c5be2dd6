"""GPU parity of the coarsening / contraction / refinement kernels against the
CPU oracle, called through the C ABI.  Integer work: bit-exact."""
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


def _cases():
    hubs = gg.hubs(20000, [40, 300, 1500, 3000, 9000, 20000], 30000, 3)
    return {
        "path": gg.path(30),
        "grid": gg.grid(12, 17),
        "triangles": gg.from_edges(6, [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (2, 3)]),
        "star_heavy": gg.from_edges(10, [(0, i) for i in range(1, 10)], vwgt=[2] + [1] * 9),
        "isolated": gg.Graph(50, np.zeros(51, np.int64), np.zeros(0, np.int32), None, None),
        "rand_w": gg.with_weights(gg.random_graph(700, 2100, 5), 9, 20, 5),
        "rand_iso": gg.with_weights(gg.random_graph(3000, 1500, 6), 3, 4, 6),
        "hubs": hubs,
        "hubs_w": gg.with_weights(hubs, 4, 7, 2),
        "rgg15": gg.workload_rgg_small(1),
        "rmat14": gg.rmat(14, 16, 2),
    }


CASES = _cases()


def _U(g, frac):
    return max(int(g.vw().max()), int(frac * g.vw().sum()))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("frac", [0.0, 0.004, 0.05])
def test_coarsen_level_parity(kmp, name, frac):
    g = CASES[name]
    U = _U(g, frac)
    dg = kmp.DeviceGraph.from_host(g)
    for seed, level in [(1, 0), (9, 3)]:
        label, fav = kmp.coarsen_level(dg, U, 5, seed, level, fav=True)
        rl, rf, st = O.cluster(g, U, 5, seed, level, stats=True)
        assert np.array_equal(label.cpu().numpy(), rl), (name, U, seed)
        assert np.array_equal(fav.cpu().numpy(), rf), (name, U, seed)
        w = np.bincount(rl, weights=g.vw(), minlength=g.n)
        assert w.max() <= U


@pytest.mark.parametrize("name", ["grid", "rand_w", "hubs", "hubs_w", "rgg15", "rmat14", "isolated"])
def test_contract_parity(kmp, name):
    g = CASES[name]
    U = _U(g, 0.004)
    ref = O.cluster(g, U, 5, 3, 0)
    dg = kmp.DeviceGraph.from_host(g)
    lab = torch.from_numpy(ref).cuda()
    cg, mp = kmp.contract(dg, lab)
    rg, rmp = O.contract(g, ref)
    h = cg.to_host()
    assert np.array_equal(mp.cpu().numpy(), rmp)
    assert h.n == rg.n
    assert np.array_equal(h.xadj, rg.xadj)
    assert np.array_equal(h.adjncy, rg.adjncy)
    assert np.array_equal(h.adjwgt, rg.adjwgt)
    assert np.array_equal(h.vwgt, rg.vwgt)


def _contract_check(kmp, g, lab):
    dg = kmp.DeviceGraph.from_host(g)
    cg, mp = kmp.contract(dg, torch.from_numpy(lab).cuda())
    rg, rmp = O.contract(g, lab)
    h = cg.to_host()
    assert np.array_equal(mp.cpu().numpy(), rmp)
    assert np.array_equal(h.xadj, rg.xadj)
    assert np.array_equal(h.adjncy, rg.adjncy)
    assert np.array_equal(h.adjwgt, rg.adjwgt)
    assert np.array_equal(h.vwgt, rg.vwgt)


@pytest.mark.parametrize("n,m", [(24000, 240000), (240000, 1200000)])
def test_contract_row_classes(kmp, n, m):
    """Weighted clusters whose members' total degree falls in every
    aggregation class (<= 64, 128, 256, 512, 2048, 4096, 8192 and above), filled
    greedily up to each class bound; the other nodes stay singletons, so on
    the larger graph a row's neighbour ids span more than 2^17 coarse ids"""
    g = gg.with_weights(gg.random_graph(n, m, 11), 5, 9, 4)
    deg = np.diff(g.xadj)
    order = np.random.default_rng(3).permutation(g.n)
    lab = np.empty(g.n, np.int32)
    targets = [40, 64, 100, 128, 200, 256, 300, 512, 2048, 4096, 8192, 30000]
    pos, c = 0, 0
    ubs = []
    for t in targets * 3:
        s, start = 0, pos
        while pos < g.n and s + deg[order[pos]] <= t:
            s += deg[order[pos]]
            pos += 1
        if pos == start and pos < g.n:
            s += deg[order[pos]]
            pos += 1
        lab[order[start:pos]] = order[start]
        ubs.append(s)
    lab[order[pos:]] = order[pos:]           # the rest are singletons
    ubs = np.array(ubs)
    bounds = [0, 64, 128, 256, 512, 2048, 4096, 8192, 1 << 40]
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        lo += 1
        assert ((ubs >= lo) & (ubs <= hi)).any(), (lo, hi)
    _contract_check(kmp, g, lab)


def _large_rows_by_distinct(g, lab, rg, rmp):
    """Distinct-entry counts of the coarse rows whose members' total degree is
    above the block path's bound (8192): the rows of the global path"""
    ub = np.bincount(rmp, weights=np.diff(g.xadj), minlength=rg.n)
    return np.diff(rg.xadj)[ub > 8192]


@pytest.mark.parametrize("family", ["rgg_blocks", "random_clusters"])
def test_contract_large_rows_every_sort_class(kmp, family):
    """Rows of the global path whose distinct entries fall in each of its
    three sort classes: at most 2048 (sorted by one CTA of 256 threads in
    shared memory), at most 16384 (1024 threads) and more (key-value radix
    sort over all such rows).  Spatially consecutive RGG nodes give rows with
    a large total degree but few distinct neighbours (only the cluster's
    boundary); clusters of random nodes give about as many as their degree."""
    if family == "rgg_blocks":
        g = gg.with_weights(gg.rgg(300000, 16, 6), 3, 7, 2)
        lab = ((np.arange(g.n) // 1500) * 1500).astype(np.int32)
    else:
        g = gg.with_weights(gg.random_graph(240000, 1500000, 12), 5, 9, 4)
        deg = np.diff(g.xadj)
        order = np.random.default_rng(5).permutation(g.n)
        lab = np.arange(g.n, dtype=np.int32)  # singletons by default
        pos = 0
        for t in [9000, 12000, 20000, 40000, 90000] * 2:
            s, start = 0, pos
            while pos < g.n and s + deg[order[pos]] <= t:
                s += deg[order[pos]]
                pos += 1
            lab[order[start:pos]] = order[start]
    rg, rmp = O.contract(g, lab)
    d = _large_rows_by_distinct(g, lab, rg, rmp)
    if family == "rgg_blocks":
        assert (d <= 2048).any()
    else:
        assert ((d > 2048) & (d <= 16384)).any() and (d > 16384).any()
    _contract_check(kmp, g, lab)


@pytest.mark.parametrize("group", [40, 100, 700])
def test_contract_many_members(kmp, group):
    """Clusters of `group` consecutive nodes of a sparse graph with many
    isolated nodes: rows with more members than a warp or a CTA chunk holds,
    most of them of degree 0"""
    g = CASES["rand_iso"]
    lab = ((np.arange(g.n) // group) * group).astype(np.int32)
    assert (np.diff(g.xadj) == 0).sum() > g.n // 4
    _contract_check(kmp, g, lab)


def test_two_levels_chain(kmp):
    """coarsen -> contract -> coarsen on the GPU's own coarse graph equals the oracle chain"""
    g = CASES["rmat14"]
    dg = kmp.DeviceGraph.from_host(g)
    rg = g
    for level in range(3):
        U = _U(rg, 0.01)
        label = kmp.coarsen_level(dg, U, 5, 4, level)
        ref = O.cluster(rg, U, 5, 4, level)
        assert np.array_equal(label.cpu().numpy(), ref)
        dg, _ = kmp.contract(dg, label)
        rg, _ = O.contract(rg, ref)
        h = dg.to_host()
        assert np.array_equal(h.adjncy, rg.adjncy) and np.array_equal(h.adjwgt, rg.adjwgt)


@pytest.mark.parametrize("name", ["grid", "rand_w", "hubs_w", "rgg15", "rmat14"])
@pytest.mark.parametrize("k", [2, 7, 64])
def test_refine_parity(kmp, name, k):
    g = CASES[name]
    rng = np.random.default_rng(k)
    part = rng.integers(0, k, g.n).astype(np.int32)
    bw = np.bincount(part, weights=g.vw(), minlength=k)
    caps = (np.maximum(bw, 1.03 * g.vw().sum() / k) + int(g.vw().max())).astype(np.int64)
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    cut = kmp.refine(dg, k, caps, 5, 11, pt)
    rp, rc = O.refine(g, k, caps.astype(np.int32), 5, 11, part)
    assert np.array_equal(pt.cpu().numpy(), rp)
    assert cut == rc
    c2, bw2 = kmp.cut(dg, pt, k)
    assert c2 == rc and np.all(bw2 <= caps)


def test_project_and_cut(kmp):
    g = CASES["rgg15"]
    ref = O.cluster(g, 60, 5, 2, 0)
    rg, rmp = O.contract(g, ref)
    pc = np.random.default_rng(1).integers(0, 9, rg.n).astype(np.int32)
    pf = kmp.project(torch.from_numpy(rmp).cuda(), torch.from_numpy(pc).cuda())
    assert np.array_equal(pf.cpu().numpy(), pc[rmp])
    dg = kmp.DeviceGraph.from_host(g)
    c, bw = kmp.cut(dg, pf, 9)
    assert c == O.cut(g, pc[rmp]) == O.cut(rg, pc)
    assert np.array_equal(bw, np.bincount(pc[rmp], minlength=9))


def test_invalid_inputs_are_rejected(kmp):
    g = gg.path(10)
    bad = gg.Graph(10, g.xadj, g.adjncy.copy(), None, None)
    bad.adjncy[0] = 99
    with pytest.raises(kmp.KmpError) as e:
        kmp.DeviceGraph.from_host(bad)
    assert e.value.code == kmp.KMP_ERR_ARG
    dg = kmp.DeviceGraph.from_host(g)
    with pytest.raises(kmp.KmpError):
        kmp.coarsen_level(dg, 0, 5, 1, 0)          # U below max node weight
    lab = torch.full((10,), 50, dtype=torch.int32, device="cuda")
    with pytest.raises(kmp.KmpError):
        kmp.contract(dg, lab)                      # labels out of range


def test_full_size_rmat20_level0(kmp):
    """Level 0 of the R-MAT scale-20 workload in the launch configuration the
    benchmark uses: labels bit-exact with the oracle."""
    g = gg.workload_rmat20(1)
    U = int(np.floor(0.03 * g.n / 256))
    dg = kmp.DeviceGraph.from_host(g)
    label = kmp.coarsen_level(dg, U, 5, 1, 0)
    ref = O.cluster(g, U, 5, 1, 0)
    assert np.array_equal(label.cpu().numpy(), ref)
    _contract_check(kmp, g, ref)


@pytest.mark.parametrize("graphs", [0, 1])
def test_rating_profile_is_consistent(kmp, graphs):
    """The k_rate spans recorded on the device timer (profiling) are positive,
    one per rating launch, and fit inside the wall time of the whole LP call
    measured with CUDA events on the same stream; profiling changes no result."""
    g = gg.rmat(16, 16, 3)
    dg = kmp.DeviceGraph.from_host(g)
    U = int(np.floor(0.03 * g.n / 64))
    old = kmp.get_tuning()
    t = kmp.Tuning(old.rate_blocks_per_sm, old.hub_degree, old.hub_chunk, old.ip_blocks_per_sm,
                   old.dense_hub_degree, graphs, old.hub_bucket, old.dense_labels)
    kmp.set_tuning(t)
    try:
        plain = kmp.coarsen_level(dg, U, 5, 7, 0)
        kmp.set_profiling(True)
        kmp.profile_read(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        prof = kmp.coarsen_level(dg, U, 5, 7, 0)
        e1.record()
        e1.synchronize()
        p = kmp.profile_read(reset=True)
        ms, by, nl = p
    finally:
        kmp.set_profiling(False)
        kmp.set_tuning(old)
    assert torch.equal(plain, prof)
    S = kmp.get_config().subrounds
    assert nl > 0 and nl % S == 0 and nl <= 5 * S
    assert by > 0
    assert 0 < ms <= e0.elapsed_time(e1)
    # the whole rating stage (k_rate and the hub kernels after it) spans at
    # least k_rate's time, one span per sub-round, hub entries included
    assert p.stage_spans == nl and ms <= p.stage_ms <= e0.elapsed_time(e1)
    assert p.stage_bytes > by


@pytest.mark.parametrize("bucket", [32, 256, 1 << 20])
def test_hub_buckets_any_size(kmp, bucket):
    """Hub ratings with many labels aggregate each hub's entries in label
    buckets of about `bucket` entries, one warp each, in rounds of at most a
    table's worth of new labels.  One bucket per hub (2^20) forces several
    rounds for every hub with more distinct neighbour labels than a round
    admits; 32 makes many small buckets.  The bucket size is a schedule
    parameter: labels and favoured clusters stay bit-exact with the oracle."""
    old = kmp.get_tuning()
    t = kmp.Tuning(old.rate_blocks_per_sm, 256, old.hub_chunk, old.ip_blocks_per_sm, old.dense_hub_degree,
                   old.lp_graphs, bucket, 0)
    kmp.set_tuning(t)
    try:
        for name in ("hubs", "hubs_w", "rmat14"):
            g = CASES[name]
            U = _U(g, 0.004)
            dg = kmp.DeviceGraph.from_host(g)
            label, fav = kmp.coarsen_level(dg, U, 5, 4, 0, fav=True)
            rl, rf, _ = O.cluster(g, U, 5, 4, 0, stats=True)
            assert np.array_equal(label.cpu().numpy(), rl), (name, bucket)
            assert np.array_equal(fav.cpu().numpy(), rf), (name, bucket)
    finally:
        kmp.set_tuning(old)


@pytest.mark.parametrize("name", ["hubs_w", "rmat14"])
def test_refine_parity_many_blocks(kmp, name):
    """Refinement with more blocks than a shared table holds labels (k = 3000):
    hub ratings take the bucketed path with blocks as labels."""
    g = CASES[name]
    k = 3000
    rng = np.random.default_rng(5)
    part = rng.integers(0, k, g.n).astype(np.int32)
    bw = np.bincount(part, weights=g.vw(), minlength=k)
    caps = (np.maximum(bw, 1.03 * g.vw().sum() / k) + int(g.vw().max())).astype(np.int64)
    dg = kmp.DeviceGraph.from_host(g)
    pt = torch.from_numpy(part).cuda()
    old = kmp.get_tuning()
    kmp.set_tuning(kmp.Tuning(old.rate_blocks_per_sm, 256, old.hub_chunk, old.ip_blocks_per_sm,
                              old.dense_hub_degree, old.lp_graphs, 64, 0))
    try:
        cut = kmp.refine(dg, k, caps, 5, 11, pt)
    finally:
        kmp.set_tuning(old)
    rp, rc = O.refine(g, k, caps.astype(np.int32), 5, 11, part)
    assert np.array_equal(pt.cpu().numpy(), rp)
    assert cut == rc


@pytest.mark.parametrize("dense_labels", [0, 57344])
def test_dense_hub_rows_for_mid_size_label_sets(kmp, dense_labels):
    """With at most `dense_labels` labels (here every graph of the test), hubs
    rate into dense per-hub rows of label counters instead of label buckets:
    coarsening labels, favoured clusters and a many-block refinement stay
    bit-exact with the oracle either way."""
    old = kmp.get_tuning()
    t = kmp.Tuning(old.rate_blocks_per_sm, 256, old.hub_chunk, old.ip_blocks_per_sm, old.dense_hub_degree,
                   old.lp_graphs, old.hub_bucket, dense_labels)
    kmp.set_tuning(t)
    try:
        for name in ("hubs_w", "rmat14"):
            g = CASES[name]
            U = _U(g, 0.004)
            dg = kmp.DeviceGraph.from_host(g)
            label, fav = kmp.coarsen_level(dg, U, 5, 4, 0, fav=True)
            rl, rf, _ = O.cluster(g, U, 5, 4, 0, stats=True)
            assert np.array_equal(label.cpu().numpy(), rl), name
            assert np.array_equal(fav.cpu().numpy(), rf), name
            k = 3000
            rng = np.random.default_rng(7)
            part = rng.integers(0, k, g.n).astype(np.int32)
            bw = np.bincount(part, weights=g.vw(), minlength=k)
            caps = (np.maximum(bw, 1.03 * g.vw().sum() / k) + int(g.vw().max())).astype(np.int64)
            pt = torch.from_numpy(part).cuda()
            cut = kmp.refine(dg, k, caps, 5, 11, pt)
            rp, rc = O.refine(g, k, caps.astype(np.int32), 5, 11, part)
            assert np.array_equal(pt.cpu().numpy(), rp) and cut == rc, name
    finally:
        kmp.set_tuning(old)
