"""GPU tests of the learned seed proposer through the C ABI: features and
scores bit-exact against the oracle's kernel-precision inference, gradients
against the oracle's fp64 backward within a tolerance derived from fp32
accumulation, learned-mode bipartitions and partitions bit-exact against the
oracle in the same mode, the sample sink, and training on the GPU."""
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
    yield K
    K.set_proposer(None)
    K.set_config(K.config())
    O.set_proposer(None)


def _bf16(x):
    """Round float32 values to the nearest BF16 value (ties to even)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _params(seed, scale=0.25):
    return _bf16(np.random.default_rng(seed).normal(0, scale, O.mpnn_num_params()).astype(np.float32))


def _graphs(seed):
    iso = gg.from_edges(7, [(0, 1, 3), (1, 2, 1), (4, 5, 2)], vwgt=np.array([1, 2, 3, 4, 5, 6, 7], np.int32))
    return [
        gg.with_weights(gg.random_graph(60, 150, seed), 9, 13, seed),
        gg.with_weights(gg.rgg(400, 8, seed), 40, 200, seed + 1),
        gg.path(17),
        iso,
        gg.from_edges(1, []),
        gg.grid(9, 13),
    ]


def _batch(kmp, graphs, seed, sides=None):
    keys = [O.key(seed, [i]) for i in range(len(graphs))]
    return kmp.Batch.from_graphs(graphs, keys, sides), keys


def test_features_and_scores_are_bit_exact(kmp):
    graphs = _graphs(3)
    b, keys = _batch(kmp, graphs, 3)
    P = _params(3)
    m = kmp.Mpnn(1)
    try:
        m.set_params(P)
        assert np.array_equal(m.get_params(), P)
        S, X = m.forward(b, features=True)
    finally:
        m.free()
    off = b.noff
    for i, g in enumerate(graphs):
        Xo = O.mpnn_features(g, keys[i]).astype(np.float32)
        So = O.mpnn_scores_f32(g, keys[i], P)
        assert np.array_equal(X[off[i]:off[i + 1]], Xo), i
        assert np.array_equal(S[off[i]:off[i + 1]], So), i


def test_gradients_match_the_oracle(kmp):
    # tolerance: fp32 sums of at most a few thousand terms per parameter with
    # relative rounding 2^-24 each stay far below 1e-4 of the largest gradient
    graphs = _graphs(5)
    rng = np.random.default_rng(5)
    sides = [rng.integers(0, 2, g.n).astype(np.int32) for g in graphs]
    b, keys = _batch(kmp, graphs, 5, sides)
    P = _params(5)
    m = kmp.Mpnn(2)
    try:
        m.set_params(P)
        loss, grad = m.gradients(b)
    finally:
        m.free()
    ng = len(graphs)
    gref = np.zeros(O.mpnn_num_params())
    lref = 0.0
    for g, key, side in zip(graphs, keys, sides):
        X = O.mpnn_features(g, key)
        S = O.mpnn_forward(g, X, P.astype(np.float64))
        L, gS = O.mpnn_loss(S, side)
        lref += L / ng
        gref += O.mpnn_backward(g, X, P.astype(np.float64), gS) / ng
    assert loss == pytest.approx(lref, rel=1e-5)
    scale = np.max(np.abs(gref))
    assert scale > 0
    assert np.max(np.abs(grad - gref)) <= 1e-4 * scale
    cos = grad @ gref / (np.linalg.norm(grad) * np.linalg.norm(gref))
    assert cos > 0.999999


def _blocks_case(name):
    if name == "rgg_blocks":
        g = gg.with_weights(gg.rgg(30000, 8, 7), 5, 9, 7)
        nb = 24
    elif name == "rmat_blocks":
        g = gg.rmat(13, 16, 8)
        nb = 16
    else:
        g = gg.grid(120, 90)
        nb = 9
    part = (np.arange(g.n) * nb // g.n).astype(np.int32)
    vw = g.vw()
    caps = []
    for bl in range(nb):
        cB = int(vw[part == bl].sum())
        t0 = cB // 2
        L = int(np.floor(1.03 * ((cB + 1) // 2)))
        caps += [t0, cB - t0, L, L]
    return g, part, nb, np.array(caps, np.int32)


def _oracle_each(g, part, nb, caps, roundkey, cfg):
    out = np.zeros(g.n, np.int32)
    for bl in range(nb):
        vs = np.flatnonzero(part == bl)
        sub = gg.subgraph(g, vs)
        c = caps[4 * bl: 4 * bl + 4]
        side, _ = O.bipartition(sub, int(c[2]), int(c[3]), int(c[0]), int(c[1]), O.step(roundkey, bl), cfg)
        out[vs] = 2 * bl + side
    return out


@pytest.mark.parametrize("name", ["rgg_blocks", "rmat_blocks", "grid_blocks"])
@pytest.mark.parametrize("learned", [0, 1, 2])
def test_bipartition_each_parity(kmp, name, learned):
    g, part, nb, caps = _blocks_case(name)
    P = _params(11)
    m = kmp.Mpnn(3)
    try:
        m.set_params(P)
        kmp.set_proposer(m)
        O.set_proposer(P)
        kw = dict(learned=learned)
        kmp.set_config(kmp.config(**kw))
        dg = kmp.DeviceGraph.from_host(g)
        pt = torch.from_numpy(part.copy()).cuda()
        kmp.bipartition_each(dg, nb, caps, 4242, pt)
        want = _oracle_each(g, part, nb, caps, 4242, O.config(**kw))
        assert np.array_equal(pt.cpu().numpy(), want)
    finally:
        kmp.set_proposer(None)
        O.set_proposer(None)
        kmp.set_config(kmp.config())
        m.free()


LEARNED_PARTS = [
    ("rgg15", lambda: gg.workload_rgg_small(1), [8, 64]),
    ("rgg_w", lambda: gg.with_weights(gg.rgg(12000, 8, 6), 5, 9, 6), [7]),
    ("rmat14", lambda: gg.rmat(14, 16, 2), [32]),
]


@pytest.mark.parametrize("learned", [1, 2])
@pytest.mark.parametrize("name,make,ks", LEARNED_PARTS, ids=[p[0] for p in LEARNED_PARTS])
def test_learned_partition_parity(kmp, name, make, ks, learned):
    """Learned mode on the coarsest graph of every item (1) and on the item
    graph itself (2): full partitions bit-exact with the oracle."""
    g = make()
    P = _params(17)
    m = kmp.Mpnn(4)
    try:
        m.set_params(P)
        kmp.set_proposer(m)
        O.set_proposer(P)
        kmp.set_config(kmp.config(learned=learned))
        dg = kmp.DeviceGraph.from_host(g)
        for k in ks:
            part, rc, st = kmp.partition_graph(dg, k, 0.03, 5)
            rp, rrc, rst = O.partition(g, k, 0.03, 5, O.config(learned=learned))
            assert np.array_equal(part.cpu().numpy(), rp), (name, k)
            assert rc == rrc and st.cut == rst.cut
    finally:
        kmp.set_proposer(None)
        O.set_proposer(None)
        kmp.set_config(kmp.config())
        m.free()


def test_learned_mode_without_a_proposer_is_the_plain_method(kmp):
    g = gg.rmat(13, 16, 4)
    dg = kmp.DeviceGraph.from_host(g)
    kmp.set_proposer(None)
    p0, _, _ = kmp.partition_graph(dg, 16, 0.03, 2)
    kmp.set_config(kmp.config(learned=1))
    try:
        p1, _, _ = kmp.partition_graph(dg, 16, 0.03, 2)
    finally:
        kmp.set_config(kmp.config())
    assert torch.equal(p0, p1)


def test_sample_sink_records_every_item(kmp):
    g, part, nb, caps = _blocks_case("rgg_blocks")
    dg = kmp.DeviceGraph.from_host(g)
    kmp.sample_sink_open(nb, 10**6, 10**7)
    try:
        kmp.bipartition_each(dg, nb, caps, 99, torch.from_numpy(part.copy()).cuda())
        b, dropped = kmp.sample_sink_read()
    finally:
        kmp.sample_sink_close()
    assert dropped == 0 and b.ng == nb
    assert np.array_equal(np.sort(b.keys), np.sort([O.step(99, bl) for bl in range(nb)]))
    assert list(b.keys) == sorted(b.keys)
    vw = g.vw()
    want_w = {O.step(99, bl): int(vw[part == bl].sum()) for bl in range(nb)}
    for i in range(b.ng):
        lo, hi = b.noff[i], b.noff[i + 1]
        # coarsening conserves node weight; sides are a bipartition
        assert int(b.vw[lo:hi].sum()) == want_w[int(b.keys[i])]
        assert set(np.unique(b.side[lo:hi])) <= {0, 1}
        # a symmetric CSR inside the graph's own id range
        rows = np.repeat(np.arange(lo, hi), np.diff(b.xadj[lo:hi + 1]))
        cols = b.adj[b.xadj[lo]:b.xadj[hi]]
        assert cols.min(initial=lo) >= lo and cols.max(initial=lo) < hi
        assert not np.any(rows == cols)
        fw = set(zip(rows.tolist(), cols.tolist(), b.ew[b.xadj[lo]:b.xadj[hi]].tolist()))
        bw = set(zip(cols.tolist(), rows.tolist(), b.ew[b.xadj[lo]:b.xadj[hi]].tolist()))
        assert fw == bw


def test_sample_sink_item_level_records_items_and_their_bipartitions(kmp):
    """With the sink at item level, every item is recorded once: its own
    graph (the block's induced subgraph, nodes in ascending id) and the final
    bipartition that the call returned for it."""
    g, part, nb, caps = _blocks_case("rgg_blocks")
    dg = kmp.DeviceGraph.from_host(g)
    kmp.sample_sink_open(nb, 10**6, 10**7, item_level=1)
    try:
        pt = torch.from_numpy(part.copy()).cuda()
        kmp.bipartition_each(dg, nb, caps, 99, pt)
        b, dropped = kmp.sample_sink_read()
    finally:
        kmp.sample_sink_close()
    out = pt.cpu().numpy()
    assert dropped == 0 and b.ng == nb
    for i in range(b.ng):
        bl = [x for x in range(nb) if O.step(99, x) == int(b.keys[i])][0]
        vs = np.flatnonzero(part == bl)
        lo, hi = b.noff[i], b.noff[i + 1]
        assert hi - lo == len(vs)
        sub = gg.subgraph(g, vs)
        assert np.array_equal(b.xadj[lo:hi + 1] - b.xadj[lo], sub.xadj)
        assert np.array_equal(b.adj[b.xadj[lo]:b.xadj[hi]] - lo, sub.adjncy)
        assert np.array_equal(b.vw[lo:hi], sub.vw())
        assert np.array_equal(b.side[lo:hi], out[vs] - 2 * bl)


def test_sink_capacity_drops_and_counts(kmp):
    g, part, nb, caps = _blocks_case("grid_blocks")
    dg = kmp.DeviceGraph.from_host(g)
    kmp.sample_sink_open(3, 10**6, 10**7)
    try:
        kmp.bipartition_each(dg, nb, caps, 5, torch.from_numpy(part.copy()).cuda())
        b, dropped = kmp.sample_sink_read()
    finally:
        kmp.sample_sink_close()
    assert b.ng == 3 and dropped == nb - 3


def test_training_on_method_samples_lowers_the_loss(kmp):
    g, part, nb, caps = _blocks_case("rgg_blocks")
    dg = kmp.DeviceGraph.from_host(g)
    kmp.sample_sink_open(1000, 10**6, 10**7)
    try:
        for key in (1, 2, 3):
            kmp.bipartition_each(dg, nb, caps, key, torch.from_numpy(part.copy()).cuda())
        b, _ = kmp.sample_sink_read()
    finally:
        kmp.sample_sink_close()
    m = kmp.Mpnn(9)
    try:
        losses = m.train(b, 150, 3e-3)
        after, _ = m.gradients(b)
    finally:
        m.free()
    assert np.all(np.isfinite(losses))
    assert after < 0.85 * losses[0]


def _coarse_blocks(kmp, g, seed, levels, k):
    """Blocks of a k-way partition of a coarse level of g (coarsened on the
    GPU), with per-block caps for a bisection at eps = 0.03."""
    dg = kmp.DeviceGraph.from_host(g)
    for lev in range(levels):
        h = dg.to_host()
        U = max(int(h.vw().max()), int(h.vw().sum()) // max(dg.n // 6, 1))
        dg, _ = kmp.contract(dg, kmp.coarsen_level(dg, U, 5, seed, lev))
    part, _, _ = kmp.partition_graph(dg, k, 0.03, seed)
    _, bw = kmp.cut(dg, part, k)
    caps = []
    for b in range(k):
        cB = int(bw[b])
        L = int(np.floor(1.03 * ((cB + 1) // 2)))
        caps += [cB // 2, cB - cB // 2, L, L]
    return dg, part, np.array(caps, np.int32)


def _samples(kmp, sources):
    kmp.sample_sink_open(100000, 10**7, 10**8)
    try:
        for g, seed, levels, k in sources:
            dg, part, caps = _coarse_blocks(kmp, g, seed, levels, k)
            kmp.bipartition_each(dg, k, caps, 777 + seed, part.clone())
        b, dropped = kmp.sample_sink_read()
    finally:
        kmp.sample_sink_close()
    assert dropped == 0
    return b


TRAIN = [(lambda: gg.rgg(1 << 17, 8, 11), 11, 2, 64), (lambda: gg.rmat(15, 16, 12), 12, 1, 48)]
HELD_OUT = [(lambda: gg.rgg(1 << 17, 8, 21), 21, 2, 64), (lambda: gg.rmat(15, 16, 22), 22, 1, 48)]


def _make(srcs):
    return [(f(), s, lv, k) for f, s, lv, k in srcs]


def test_training_is_deterministic(kmp):
    b1 = _samples(kmp, _make(TRAIN[:1]))
    b2 = _samples(kmp, _make(TRAIN[:1]))
    for f in ("noff", "xadj", "adj", "vw", "ew", "keys", "side"):
        assert np.array_equal(getattr(b1, f), getattr(b2, f)), f
    ps = []
    for _ in range(2):
        m = kmp.Mpnn(3)
        try:
            m.train(b1, 60, 3e-3)
            ps.append(m.get_params())
        finally:
            m.free()
    assert np.array_equal(ps[0], ps[1])


def _first_fit(b, S):
    """score-ordered first-fit start of every sample (block 0 filled to
    floor(c/2)); returns (summed cut, weight fraction on the label's side under
    the better orientation, averaged over samples)"""
    total, agree = 0, []
    for i in range(b.ng):
        lo, hi = b.noff[i], b.noff[i + 1]
        vw = b.vw[lo:hi].astype(np.int64)
        t0 = int(vw.sum()) // 2
        keys = np.array([O.mpnn_score_key(s) for s in S[lo:hi]], np.uint64)
        order = np.lexsort((np.arange(hi - lo), keys))
        side = np.ones(hi - lo, np.int32)
        w0 = 0
        for v in order:
            if w0 + vw[v] <= t0:
                side[v] = 0
                w0 += vw[v]
        rows = np.repeat(np.arange(hi - lo), np.diff(b.xadj[lo:hi + 1]))
        cols = b.adj[b.xadj[lo]:b.xadj[hi]] - lo
        w = b.ew[b.xadj[lo]:b.xadj[hi]].astype(np.int64)
        total += int(w[side[rows] != side[cols]].sum()) // 2
        a = float(vw[side == b.side[lo:hi]].sum()) / float(vw.sum())
        agree.append(max(a, 1.0 - a))
    return total, float(np.mean(agree))


def test_trained_proposer_gains_over_the_untrained_one(kmp):
    """What training buys, measured on held-out coarsest graphs of the
    bipartitioner: the loss against the method's own best-of-portfolio
    bipartitions drops, and the trained network's score order puts more node
    weight on the side the portfolio chose than the untrained network does.
    In learned mode the end result of bipartitioning held-out blocks stays
    within 1% of the plain portfolio's cut."""
    train = _samples(kmp, _make(TRAIN))
    held = _samples(kmp, _make(HELD_OUT))
    trained, untrained = kmp.Mpnn(5), kmp.Mpnn(5)
    try:
        losses = trained.train(train, 400, 3e-3)
        held_loss_t, _ = trained.gradients(held)
        held_loss_u, _ = untrained.gradients(held)
        ct, at = _first_fit(held, trained.forward(held))
        cu, au = _first_fit(held, untrained.forward(held))
        cl, al = _first_fit(held, (held.side == 0).astype(np.float32))  # the labels themselves
        cuts = {}
        for name, src in zip(("rgg", "rmat"), _make(HELD_OUT)):
            dg, part, caps = _coarse_blocks(kmp, *src)
            nb = src[3]
            c0, _ = kmp.cut(dg, part, nb)
            for mode, cfg, model in (("plain", kmp.config(), None), ("learned", kmp.config(learned=1), trained)):
                kmp.set_proposer(model)
                kmp.set_config(cfg)
                p = part.clone()
                kmp.bipartition_each(dg, nb, caps, 99, p)
                cuts[(name, mode)] = kmp.cut(dg, p, 2 * nb)[0] - c0
    finally:
        kmp.set_proposer(None)
        kmp.set_config(kmp.config())
        trained.free()
        untrained.free()
    print(f"\nloss train {losses[0]:.4f}->{losses[-1]:.4f}; held-out {held_loss_u:.4f} (untrained) "
          f"{held_loss_t:.4f} (trained); first-fit agreement untrained {au:.3f} trained {at:.3f} "
          f"labels {al:.3f}; first-fit cut untrained {cu} trained {ct} labels {cl}; {cuts}")
    assert held_loss_t < 0.7 * held_loss_u
    assert at > au + 0.05
    for name in ("rgg", "rmat"):
        assert cuts[(name, "learned")] <= 1.01 * cuts[(name, "plain")]
