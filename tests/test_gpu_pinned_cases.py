"""The hand-derived cases that pin the oracle's commit order (Section 4.1,
reading R4) and balancer (Section 4.3, reading D5), run on the CUDA path
through the C ABI: the GPU must give the hand-derived results too (and so the
oracle's).  The derivations are in the docstrings of
tests/test_oracle_pins_order.py."""
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
    K.set_config(K.config())


def test_commit_one_jacobi_round_coarsening(kmp):
    g = gg.from_edges(4, [(0, 1, 2), (0, 2, 5), (0, 3, 3)], vwgt=[7, 3, 3, 3])
    dg = kmp.DeviceGraph.from_host(g)
    kmp.set_config(kmp.config(subrounds=1, two_hop=0))
    try:
        label, fav = kmp.coarsen_level(dg, 10, 1, 5, 0, fav=True)
    finally:
        kmp.set_config(kmp.config())
    assert label.cpu().tolist() == [2, 1, 0, 3]
    f = fav.cpu().tolist()
    assert f[1] == 0 and f[3] == 0


@pytest.mark.parametrize("ew,vw,cap0,expect", [
    ((2, 3, 5), (1, 1, 1), 6, [0, 1, 1, 0, 1]),   # highest gain wins the last unit of room
    ((4, 4, 4), (1, 1, 1), 6, [0, 0, 1, 1, 1]),   # equal gains: lowest id
    ((2, 3, 5), (1, 2, 2), 8, [0, 1, 1, 0, 1]),   # a prefix, not a first fit
])
def test_commit_refinement_cases(kmp, ew, vw, cap0, expect):
    g = gg.from_edges(5, [(0, 1, ew[0]), (0, 2, ew[1]), (0, 3, ew[2])], vwgt=[5, *vw, 10])
    dg = kmp.DeviceGraph.from_host(g)
    caps = np.array([cap0, sum(vw) + 10], np.int64)
    part = torch.tensor([0, 1, 1, 1, 1], dtype=torch.int32, device="cuda")
    kmp.set_config(kmp.config(subrounds=1))
    try:
        cut = kmp.refine(dg, 2, caps, 5, 3, part)
    finally:
        kmp.set_config(kmp.config())
    assert part.cpu().tolist() == expect
    rp, rcut = O.refine(g, 2, caps.astype(np.int32), 5, 3, np.array([0, 1, 1, 1, 1], np.int32),
                        cfg=O.config(subrounds=1))
    assert rp.tolist() == expect and cut == rcut


BALANCE_CASES = [
    # d >= 0 ranks by d * c(v)
    (5, [(1, 3, 3), (2, 4, 2)], [10, 1, 2, 1, 1], [0, 0, 0, 1, 2], [12, 100, 100], [0, 0, 2, 1, 2]),
    # d < 0 ranks by d / c(v)
    (5, [(0, 2, 2), (1, 2, 4)], [1, 4, 1, 1, 1], [0, 0, 0, 1, 2], [5, 100, 100], [0, 1, 0, 1, 2]),
    # most connected admissible block, and a full block is not admissible
    (4, [(0, 2, 1), (0, 3, 5)], [1, 5, 1, 1], [0, 0, 1, 2], [5, 100, 100], [2, 0, 1, 2]),
    (4, [(0, 2, 1), (0, 3, 5)], [1, 5, 1, 1], [0, 0, 1, 2], [5, 100, 1], [1, 0, 1, 2]),
    # the order is fixed by the starting state
    (6, [(0, 4, 5), (0, 1, 1), (1, 4, 1), (2, 5, 1)], [1, 1, 1, 10, 1, 1], [0, 0, 0, 0, 1, 2],
     [11, 100, 100], [1, 0, 2, 0, 1, 2]),
]


@pytest.mark.parametrize("n,edges,vw,part0,caps,expect", BALANCE_CASES)
def test_balance_hand_cases(kmp, n, edges, vw, part0, caps, expect):
    g = gg.from_edges(n, edges, vwgt=vw)
    dg = kmp.DeviceGraph.from_host(g)
    part = torch.tensor(part0, dtype=torch.int32, device="cuda")
    kmp.balance(dg, 3, np.array(caps, np.int64), part)
    assert part.cpu().tolist() == expect
    rp, _ = O.balance(g, 3, np.array(caps, np.int32), np.array(part0, np.int32))
    assert rp.tolist() == expect
