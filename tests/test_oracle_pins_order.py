"""Hand-derived pins for the order-dependent parts of the CPU oracle: the
deterministic commit of LP moves (reading R4), the balancer's candidate
order and target choice (reading D5, Section 4.3) and the coarsening /
uncoarsening schedule (readings D1, D2; Section 4.1 and Algorithm 1).

Every expected value below is derived by hand in the test's docstring from
the reading it pins, on graphs small or regular enough that the derivation
does not depend on hash values.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2105_02022_gb300 import graphgen as gg


def _iso(vw):
    """Graph without edges and with the given node weights."""
    n = len(vw)
    return gg.Graph(n, np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.asarray(vw, np.int32), None)


# ------------------------------------------------------------- commit (R4) --
def test_commit_one_jacobi_round_coarsening():
    """Coarsening, one round, one sub-round (S = 1), U = 10.
    Node t = 0 (c = 7) is joined to a = 1, b = 2, c = 3 (c = 3 each) with
    edge weights 2, 5, 3.  Every node reads the same start state:
      a, b, c each propose t's cluster 0 (7 + 3 = 10 <= U) with gains 2, 5, 3;
      t proposes b's cluster 2 (its heaviest admissible neighbour, 3 + 7 <= U).
    Commit against the start weights: target 0 takes its proposals in
    (gain desc, id asc) order b, c, a with prefix weights 10, 13, 16, so only
    b is accepted; target 2 accepts t (3 + 7 = 10).  Result: label(t) = 2,
    label(b) = 0, a and c stay, and both rejected nodes favour cluster 0.
    (Accepting in id order would move a; rejecting contested targets would
    move nobody into 0; checking the cap after t's departure would take all
    three; a strict cap would accept nothing.)"""
    g = gg.from_edges(4, [(0, 1, 2), (0, 2, 5), (0, 3, 3)], vwgt=[7, 3, 3, 3])
    label, fav, st = O.cluster(g, 10, 1, 5, 0, cfg=O.config(subrounds=1), isolated=False,
                               two_hop=False, stats=True)
    assert label.tolist() == [2, 1, 0, 3]
    assert st.moved[0] == 2
    assert fav[1] == 0 and fav[3] == 0


def _star_refine(ew, vw_leaves, cap0, seed=3):
    """Refinement with S = 1: block 0 = {t} (c = 5), block 1 = leaves 1..3 and
    an isolated anchor 4 (c = 10) whose weight fills block 1 to its cap."""
    g = gg.from_edges(5, [(0, 1, ew[0]), (0, 2, ew[1]), (0, 3, ew[2])], vwgt=[5, *vw_leaves, 10])
    part = np.array([0, 1, 1, 1, 1], np.int32)
    caps = np.array([cap0, sum(vw_leaves) + 10], np.int32)
    return O.refine(g, 2, caps, 5, seed, part, cfg=O.config(subrounds=1))


def test_commit_highest_gain_wins_the_last_unit_of_room():
    """Block 0 has room for one unit (cap 6, weight 5).  Leaves 1, 2, 3 have
    gains 2, 3, 5 towards block 0 (no neighbour in their own block); t cannot
    move (block 1 is at its cap).  The commit accepts leaf 3 (highest gain)
    and rejects 2 and 1 (prefix weights 7, 8 > 6).  Round 1 rates only t
    (neighbour of the mover): r(own) = 5 = r(block 1), no move.  Cut = 2 + 3."""
    part, cut = _star_refine((2, 3, 5), (1, 1, 1), 6)
    assert part.tolist() == [0, 1, 1, 0, 1]
    assert cut == 5


def test_commit_equal_gains_lowest_id_wins():
    """As above with gains 4, 4, 4: the tie goes to the lowest id, leaf 1."""
    part, cut = _star_refine((4, 4, 4), (1, 1, 1), 6)
    assert part.tolist() == [0, 0, 1, 1, 1]
    assert cut == 8


def test_commit_accepts_a_prefix_not_a_first_fit():
    """Room for 3 units (cap 8, weight 5); leaves weigh 1, 2, 2 with gains
    2, 3, 5.  Order: leaf 3 (w 2, prefix 7 <= 8, accepted), leaf 2 (prefix 9,
    rejected), leaf 1 (prefix 10, rejected) -- although leaf 1 alone would
    still fit (5 + 2 + 1 = 8), the accepted set is a prefix of the order."""
    part, cut = _star_refine((2, 3, 5), (1, 2, 2), 8)
    assert part.tolist() == [0, 1, 1, 0, 1]
    assert cut == 5


# ----------------------------------------------------------- balancer (D5) --
def test_balance_nonnegative_gain_ranks_by_d_times_c():
    """Blocks 0 = {anchor 0 (c 10, isolated), x = 1 (c 1), y = 2 (c 2)},
    1 = {p = 3}, 2 = {q = 4}; edges x-p (3), y-q (2); cap0 = 12 < 13.
    Relative gains: x: d = 3, 3*1 = 3; y: d = 2, 2*2 = 4; anchor: d = 0.
    Order y, x, anchor: y leaves first, to q's block 2 (its only connected
    block), and block 0 then fits.  (Ranking by d/c or by d alone would move x.)"""
    g = gg.from_edges(5, [(1, 3, 3), (2, 4, 2)], vwgt=[10, 1, 2, 1, 1])
    part = np.array([0, 0, 0, 1, 2], np.int32)
    out, mv = O.balance(g, 3, np.array([12, 100, 100], np.int32), part)
    assert out.tolist() == [0, 0, 2, 1, 2] and mv == 1


def test_balance_negative_gain_ranks_by_d_over_c():
    """Block 0 = {x = 0 (c 1), y = 1 (c 4), a = 2 (c 1)}, blocks 1 = {3},
    2 = {4} with no edges to block 0; edges x-a (2), y-a (4); cap0 = 5 < 6.
    Every other block has connectivity 0, so d = -conn(own):
    x: -2/1 = -2; y: -4/4 = -1; a: -6/1 = -6.  y leaves first, to block 1
    (connectivity ties go to the lowest id).  (Ranking by d*c: y = -16 would
    come last and x would leave.)"""
    g = gg.from_edges(5, [(0, 2, 2), (1, 2, 4)], vwgt=[1, 4, 1, 1, 1])
    part = np.array([0, 0, 0, 1, 2], np.int32)
    out, mv = O.balance(g, 3, np.array([5, 100, 100], np.int32), part)
    assert out.tolist() == [0, 1, 0, 1, 2] and mv == 1


def test_balance_target_is_the_most_connected_admissible_block():
    """z = 0 (c 1) in overloaded block 0 (with an isolated anchor of c 5;
    cap0 = 5 < 6) has connectivity 1 to block 1 and 5 to block 2.  It moves
    to block 2, not to the lowest-id block 1.  When block 2 is full (cap 1,
    weight 1), block 2 is not admissible and z goes to block 1."""
    g = gg.from_edges(4, [(0, 2, 1), (0, 3, 5)], vwgt=[1, 5, 1, 1])
    part = np.array([0, 0, 1, 2], np.int32)
    out, _ = O.balance(g, 3, np.array([5, 100, 100], np.int32), part)
    assert out.tolist() == [2, 0, 1, 2]
    out, _ = O.balance(g, 3, np.array([5, 100, 1], np.int32), part)
    assert out.tolist() == [1, 0, 1, 2]


# ----------------------------------------------------------- schedule (D1, D2) --
def test_schedule_cfg1_level0():
    """RGG 2^15, k = 8, eps = 0.03, C = 160: k' = min(8, floor(32768/160))
    = 8, not halved (2 * 32768 > 8 * 160), U = floor(0.03 * 32768 / 8) = 122;
    the input level ends with k_i = k = 8 blocks."""
    g = gg.workload_rgg_small(1)
    _, rc, st = O.partition(g, 8, 0.03, 1)
    assert rc == 0
    assert st.level_kp[0] == 8 and st.level_U[0] == 122
    assert st.level_k[0] == 8


def test_schedule_halving_chain_on_isolated_nodes():
    """2^15 isolated unit nodes, k = 128, eps = 0.0157 (eps c(V) = 514.4576).
    Without edges a level is packed in id order into chunks of weight <= U,
    so every level is known in closed form:
      level 0: n = 32768, k' = min(128, 204) = 128, U = floor(4.019) = 4 -> 8192 nodes of weight 4
      level 1: 2*8192 <= 128*160, k' = 64,  U = floor(8.038)  = 8   -> 4096 (weight 8)
      level 2: 2*4096 <= 64*160,  k' = 32,  U = floor(16.077) = 16  -> 2048
      level 3: 2*2048 <= 32*160,  k' = 16,  U = floor(32.15)  = 32  -> 1024
      level 4: 2*1024 <= 16*160,  k' = 8,   U = floor(64.31)  = 64  -> 512
      level 5: 2*512  <= 8*160,   k' = 4,   U = floor(128.6)  = 128 -> 256
      level 6: 256 <= 2C = 320: coarsening stops.
    On the way up k_i = ceil2(n_i / 160) clamped to [2, k], and k on the input:
      256 -> 2, 512 -> 4, 1024 -> 8, 2048 -> 16, 4096 -> 32, 8192 -> 64, input -> 128."""
    n = 1 << 15
    _, _, st = O.partition(_iso([1] * n), 128, 0.0157, 1)
    assert st.levels == 7
    assert list(st.level_n)[:7] == [32768, 8192, 4096, 2048, 1024, 512, 256]
    assert st.clustered == 6
    assert list(st.level_kp)[:6] == [128, 64, 32, 16, 8, 4]
    assert list(st.level_U)[:6] == [4, 8, 16, 32, 64, 128]
    assert list(st.level_k)[:7] == [128, 64, 32, 16, 8, 4, 2]


def test_schedule_k_prime_uses_the_floor_of_n_over_C():
    """2^15 isolated unit nodes, k = 1024, eps = 0.03: k' = min(1024,
    floor(32768/160) = 204) = 204 (a power-of-two rounding would give 256),
    U = floor(983.04 / 204) = 4, so level 1 has 32768 / 4 = 8192 nodes."""
    n = 1 << 15
    _, _, st = O.partition(_iso([1] * n), 1024, 0.03, 1)
    assert st.level_kp[0] == 204 and st.level_U[0] == 4
    assert st.level_n[1] == 8192
    assert st.level_k[0] == 1024


def test_schedule_cap_is_at_least_the_heaviest_node():
    """1000 isolated nodes, node 0 of weight 500 and 999 of weight 1, k = 8:
    k' = min(8, floor(1000/160)) = 6, eps c(V)/k' = 0.03 * 1499 / 6 = 7.495,
    so U = max(7, 500) = 500.  Packing: node 0 fills chunk 0 = [0, 500),
    nodes 1..500 (prefixes 500..999) fill chunk 1 and nodes 501..999
    (prefixes 1000..1498) chunk 2: three coarse nodes, coarsening stops.
    The coarsest level gets k_i = 2, the input level k = 8.  (Without the
    heaviest-node term U = 7 would leave hundreds of coarse nodes.)"""
    _, _, st = O.partition(_iso([500] + [1] * 999), 8, 0.03, 1)
    assert st.level_kp[0] == 6 and st.level_U[0] == 500
    assert st.levels == 2 and list(st.level_n)[:2] == [1000, 3]
    assert list(st.level_k)[:2] == [8, 2]


def test_balance_order_is_fixed_by_the_starting_state():
    """Block 0 = {x = 0, y = 1, z = 2, anchor a = 3 (c 10, isolated)}, unit
    x, y, z; block 1 = {p = 4}, block 2 = {q = 5}; edges x-p (5), x-y (1),
    y-p (1), z-q (1); cap0 = 11 < 13, so two unit nodes must leave.
    Starting-state relative gains: x: 5 - 1 = 4; y: 1 - 1 = 0; z: 1; a: 0.
    Order x, z, y, a: x goes to block 1, then z to block 2, and block 0 fits.
    (Re-rating after x's move would give y: 2 - 0 = 2 > z and move y.)"""
    g = gg.from_edges(6, [(0, 4, 5), (0, 1, 1), (1, 4, 1), (2, 5, 1)], vwgt=[1, 1, 1, 10, 1, 1])
    part = np.array([0, 0, 0, 0, 1, 2], np.int32)
    out, mv = O.balance(g, 3, np.array([11, 100, 100], np.int32), part)
    assert out.tolist() == [1, 0, 2, 0, 1, 2] and mv == 2


# ------------------------------------------------- adaptive portfolio (B7) --
def _keep_by_definition(cuts, best):
    """mean - 2 * population standard deviation <= best, exactly (Fractions)."""
    import statistics
    from fractions import Fraction

    if not cuts:
        return False
    xs = [Fraction(c) for c in cuts]
    mean, var = statistics.mean(xs), statistics.pvariance(xs)
    d = mean - best
    return d <= 0 or d * d <= 4 * var


def test_adaptive_keep_rule():
    """The rule that keeps an algorithm in the adaptive portfolio against its
    statistical definition: cuts 10, 12 have mean 11 and sd 1, so the
    algorithm stays for best >= 9 and stops for best 8; equal cuts (sd 0)
    stay only when they equal the best; no feasible run never stays."""
    assert O.adaptive_keep([10, 12], 9) and not O.adaptive_keep([10, 12], 8)
    assert O.adaptive_keep([9, 13], 7) and not O.adaptive_keep([9, 13], 6)
    assert O.adaptive_keep([5, 5, 5], 5) and not O.adaptive_keep([5, 5, 5], 4)
    assert not O.adaptive_keep([], 100)
    rng = np.random.default_rng(4)
    for _ in range(3000):
        f = int(rng.integers(1, 6))
        cuts = rng.integers(0, 60, f).tolist()
        best = int(rng.integers(0, 60))
        assert O.adaptive_keep(cuts, best) == _keep_by_definition(cuts, best), (cuts, best)
    big = [3_000_000_000, 3_000_000_007]  # sums of squares beyond 64 bits
    assert O.adaptive_keep(big, 2_999_999_996) == _keep_by_definition(big, 2_999_999_996)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_adaptive_with_single_repetitions_is_the_plain_portfolio(seed):
    """With one repetition per algorithm, stage 1 is the whole portfolio."""
    g = gg.with_weights(gg.random_graph(60, 150, seed), 3, 5, seed)
    cB = int(g.vw().sum())
    t0, t1, L0, L1 = O.split_caps(0.03, cB, 2, cB, 2)
    kw = dict(rep_random=1, rep_bfs=1, rep_ggg=1)
    a, ca = O.bipartition(g, L0, L1, t0, t1, 77, cfg=O.config(adaptive=1, **kw))
    b, cb = O.bipartition(g, L0, L1, t0, t1, 77, cfg=O.config(**kw))
    assert ca == cb and np.array_equal(a, b)


@pytest.mark.parametrize("seed", range(1, 9))
def test_adaptive_bipartition_vs_brute_force(seed):
    """The adaptive portfolio's bipartitions keep the caps and never beat the
    exhaustive optimum (n <= 18)."""
    g = gg.with_weights(gg.random_graph(16 + seed % 3, 40, seed), 4, 6, seed)
    cB = int(g.vw().sum())
    t0, t1, L0, L1 = O.split_caps(0.03, cB, 2, cB, 2)
    side, c = O.bipartition(g, L0, L1, t0, t1, 5, cfg=O.config(adaptive=1))
    w = g.vw().astype(np.int64)
    assert w[side == 0].sum() <= L0 + w.max() and w[side == 1].sum() <= L1 + w.max()
    opt, _ = O.brute_bisection(g, L0 + int(w.max()), L1 + int(w.max()))
    assert c >= opt and c == O.cut(g, side)
