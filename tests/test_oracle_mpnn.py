"""Pins for the oracle of the learned seed proposer: backward pass against
central finite differences of the loss, features against hand-derived values,
the score-ordered first-fit proposal against a hand case.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2105_02022_gb300 import graphgen as gg


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0, scale, O.mpnn_num_params())


def test_param_count():
    # W1s, W1n (64x8), b1, W2s, W2n (64x64), b2, w_o, b_o
    assert O.mpnn_num_params() == 2 * 64 * 8 + 64 + 2 * 64 * 64 + 64 + 64 + 1


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_backward_matches_finite_differences(seed):
    g = gg.with_weights(gg.random_graph(30, 70, seed), 5, 7, seed)
    X = O.mpnn_features(g, O.key(seed, [9]))
    P = _params(seed)
    side = np.random.default_rng(seed).integers(0, 2, g.n).astype(np.int32)
    S = O.mpnn_forward(g, X, P)
    L, gS = O.mpnn_loss(S, side)
    gP = O.mpnn_backward(g, X, P, gS)
    rng = np.random.default_rng(100 + seed)
    idx = np.concatenate([rng.choice(len(P), 60, replace=False), [len(P) - 1, 0, 600, 1100]])
    h = 1e-6
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        Lp, _ = O.mpnn_loss(O.mpnn_forward(g, X, Pp), side)
        Lm, _ = O.mpnn_loss(O.mpnn_forward(g, X, Pm), side)
        num = (Lp - Lm) / (2 * h)
        assert abs(num - gP[i]) <= 1e-6 + 1e-5 * abs(num), (i, num, gP[i])


def test_loss_is_orientation_symmetric():
    S = np.array([2.0, -1.0, 0.5, -3.0])
    side = np.array([0, 1, 0, 1], np.int32)
    a, _ = O.mpnn_loss(S, side)
    b, _ = O.mpnn_loss(S, 1 - side)
    assert a == pytest.approx(b)
    # closed form: mean softplus(s) - y*s with y = 1 for block 0
    y = (side == 0).astype(float)
    ref = np.mean(np.logaddexp(0, S) - y * S)
    assert a == pytest.approx(ref)


def test_features_on_a_path():
    g = gg.path(5)
    key = O.key(4, [1])
    X = O.mpnn_features(g, key)
    # anchor a = node with the smallest key; BFS hops along a path are |v - a|
    hs = [O.step(key, v) for v in range(5)]
    a = int(np.argmin(hs))
    d1 = np.abs(np.arange(5) - a)
    assert np.allclose(X[:, 4], d1 / (d1.max() + 1))
    b = int(np.argmax(d1))  # farthest from a (ties: smallest id)
    d2 = np.abs(np.arange(5) - b)
    assert np.allclose(X[:, 5], d2 / (d2.max() + 1))
    assert np.allclose(X[:, 0], 1.0)
    assert np.allclose(X[:, 1], 1.0)                      # unit weights: c(v)/mean = 1
    deg = np.diff(g.xadj)
    assert np.allclose(X[:, 2], deg / 2)
    assert np.allclose(X[:, 3], deg / deg.mean())
    assert set(np.unique(X[:, 6:])) <= {-1.0, 1.0}


def test_propose_first_fit_by_score():
    g = gg.Graph(5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.array([3, 1, 2, 2, 1], np.int32), None)
    S = np.array([0.1, 0.9, 0.9, -1.0, 0.5])
    # order: 1 (0.9), 2 (0.9, id 2), 4 (0.5), 0, 3; target 4: 1 (w1) + 2 (w2) -> 3, 4 (w1) -> 4
    side = O.mpnn_propose(g, S, 4)
    assert side.tolist() == [1, 0, 0, 1, 0]


def _bf16(x):
    """Round float32 values to the nearest BF16 value (ties to even)."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def test_bf16_rounding_helper():
    # 1 + 2^-8 is halfway between BF16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    x = np.array([1.0, 1 + 2.0**-8, 1 + 3 * 2.0**-8, -2.5], np.float32)
    assert _bf16(x).tolist() == [1.0, 1.0, 1 + 2.0**-6, -2.5]


@pytest.mark.parametrize("seed", [4, 5])
def test_fp32_scores_follow_the_fp64_network(seed):
    # the kernel-precision path is the same network: it agrees with the fp64
    # forward to fp32 rounding (a wrong index or a dropped term would not)
    g = gg.with_weights(gg.random_graph(60, 150, seed), 9, 13, seed)
    P = _bf16(_params(seed, 0.25).astype(np.float32))
    key = O.key(seed, [3])
    S32 = O.mpnn_scores_f32(g, key, P)
    S64 = O.mpnn_forward(g, O.mpnn_features(g, key), P.astype(np.float64))
    assert np.max(np.abs(S32 - S64)) <= 1e-4 * (1 + np.max(np.abs(S64)))


def test_score_key_orders_descending_and_merges_zeros():
    vals = [3.5, 1.0, 1e-30, 0.0, -1e-30, -2.0, -np.inf]
    keys = [O.mpnn_score_key(v) for v in vals]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    assert O.mpnn_score_key(-0.0) == O.mpnn_score_key(0.0)
    assert O.mpnn_score_key(np.inf) < keys[0]


def _distance_net():
    """score = -d1 / (D1 + 1): only the hop distance from anchor a counts"""
    P = np.zeros(O.mpnn_num_params(), np.float32)
    P[0 * 8 + 4] = 1.0            # W1_self[0][4]: h1_0 = relu(x4)
    P[1088 + 0 * 64 + 0] = 1.0    # W2_self[0][0]: h2_0 = h1_0
    P[9344 + 0] = -1.0            # w_o[0]
    return P


def test_learned_start_grows_from_the_anchor():
    # with the distance network, the learned start is the first fit in
    # (hop distance from anchor a, id) order: on a path, a contiguous segment
    n, t0 = 9, 4
    g = gg.path(n)
    key = O.key(7, [2])
    hs = [O.step(key, v) for v in range(n)]
    a = int(np.argmin(hs))
    order = sorted(range(n), key=lambda v: (abs(v - a), v))
    want = np.ones(n, np.int32)
    want[order[:t0]] = 0
    side = O.learned_initial(g, t0, key, _distance_net())
    assert side.tolist() == want.tolist()


def test_learned_mode_bipartition_is_optimal_on_a_path():
    # learned start alone (no portfolio repetitions), then FM: one cut edge,
    # the brute-force optimum of a balanced path bisection
    g = gg.path(18)
    cfg = O.config()
    cfg.learned, cfg.lrep_random, cfg.lrep_bfs, cfg.lrep_ggg = 1, 0, 0, 0
    O.set_proposer(_distance_net())
    try:
        side, cut = O.bipartition(g, 9, 9, 9, 9, O.key(1, [5]), cfg)
    finally:
        O.set_proposer(None)
    assert cut == O.brute_bisection(g, 9, 9)[0] == 1
    # the bipartitioner's caps allow target + max c(v) (reading B5)
    assert abs(int(np.sum(side == 0)) - 9) <= 1


def test_learned_mode_without_a_proposer_is_the_plain_method():
    g = gg.with_weights(gg.rgg(3000, 8, 3), 4, 6, 3)
    cfg = O.config()
    p0, _, _ = O.partition(g, 8, 0.03, 2, cfg)
    cfg.learned = 1
    p1, _, _ = O.partition(g, 8, 0.03, 2, cfg)
    assert np.array_equal(p0, p1)


def test_item_mode_bipartition_is_optimal_on_a_path():
    """Learned item mode (reading B8): the distance network's start on the
    item graph itself, FM there, no coarsening: one cut edge on a path, the
    brute-force optimum of a balanced path bisection."""
    g = gg.path(20)
    cfg = O.config(learned=2)
    O.set_proposer(_distance_net())
    try:
        side, cut = O.bipartition(g, 10, 10, 10, 10, O.key(3, [5]), cfg)
    finally:
        O.set_proposer(None)
    assert cut == O.brute_bisection(g, 10, 10)[0] == 1
    assert cut == O.cut(g, side)


def test_item_mode_is_fm_of_the_learned_start_when_feasible():
    """Where the refined learned start keeps the caps, it is the result: the
    same as the learned start refined by FM on the item graph directly."""
    g = gg.with_weights(gg.rgg(400, 8, 4), 3, 5, 4)
    cB = int(g.vw().sum())
    t0, t1, L0, L1 = O.split_caps(0.03, cB, 2, cB, 2)
    key = O.key(9, [1])
    P = _params(4).astype(np.float32)
    cfg = O.config(learned=2)
    O.set_proposer(P)
    try:
        side, cut = O.bipartition(g, L0, L1, t0, t1, key, cfg)
        start = O.learned_initial(g, t0, O.step(key, 9), P)
    finally:
        O.set_proposer(None)
    mx = int(g.vw().max())
    c0, c1 = max(L0, t0 + mx), max(L1, t1 + mx)
    ref, rcut = O.fm(g, c0, c1, start, cfg)
    w = g.vw().astype(np.int64)
    assert w[ref == 0].sum() <= c0 and w[ref == 1].sum() <= c1
    assert np.array_equal(side, ref) and cut == rcut


def test_item_mode_falls_back_to_the_plain_method_when_infeasible():
    """Three nodes of weight 10 with targets 1: no bipartition keeps the caps
    (11 each), so learned item mode returns the plain method's result."""
    g = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)], vwgt=[10, 10, 10])
    O.set_proposer(_distance_net())
    try:
        a, ca = O.bipartition(g, 1, 1, 1, 1, O.key(2, [1]), O.config(learned=2))
    finally:
        O.set_proposer(None)
    b, cb = O.bipartition(g, 1, 1, 1, 1, O.key(2, [1]), O.config())
    assert np.array_equal(a, b) and ca == cb


def test_item_mode_without_a_proposer_is_the_plain_method():
    g = gg.with_weights(gg.rgg(3000, 8, 3), 4, 6, 3)
    p0, _, _ = O.partition(g, 8, 0.03, 2, O.config())
    p1, _, _ = O.partition(g, 8, 0.03, 2, O.config(learned=2))
    assert np.array_equal(p0, p1)
