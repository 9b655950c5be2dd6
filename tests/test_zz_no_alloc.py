"""kmp_cut_noalloc: the cut and block weights of kmp_cut computed without any
device allocation.  It serves callers that cannot let a library allocate
device memory when it is called: their memory belongs to another allocator or
a fixed arena, they reserved all of it up front, or they cannot take an
allocation's synchronisation or failure inside a loop.  Its scratch is a fixed
device array inside the library.

Each case is checked against the CPU oracle's cut and against block weights
summed on the host, and against the allocating entry point, on calls in a row
(the array keeps the previous call's contents).

Collected last on purpose (file name); it builds and loads the library itself,
so it also passes when run alone in a fresh process."""
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
    return K


def _host_block_weights(g, part, k):
    w = np.ones(g.n, np.int64) if g.vwgt is None else g.vwgt.astype(np.int64)
    return np.bincount(part, weights=w, minlength=k).astype(np.int64)


def test_noalloc_matches_oracle_and_cut_on_calls_in_a_row(kmp):
    g = gg.with_weights(gg.rgg(20000, 8, 5), 7, 9, 5)
    dg = kmp.DeviceGraph.from_host(g)
    rng = np.random.default_rng(3)
    # calls in a row with shrinking and growing k: no call may see an earlier
    # call's sums; k = KMP_NOALLOC_MAX_K fills the array to its end, and
    # 300 / 8 take the shared-memory staging path
    for k in (300, 8, kmp.KMP_NOALLOC_MAX_K, 5):
        hp = rng.integers(0, k, g.n).astype(np.int32)
        part = torch.from_numpy(hp).cuda()
        cut, bw = kmp.cut_noalloc(dg, part, k)
        assert cut == O.cut(g, hp), k
        assert np.array_equal(bw, _host_block_weights(g, hp, k)), k
        ref_cut, ref_bw = kmp.cut(dg, part, k)
        assert cut == ref_cut and np.array_equal(bw, ref_bw), k


def test_noalloc_unit_weights_and_large_k(kmp):
    g = gg.rmat(14, 16, 4)
    dg = kmp.DeviceGraph.from_host(g)
    rng = np.random.default_rng(9)
    for k in (4096, 2):  # above the staged range (global atomics), then below it
        hp = rng.integers(0, k, g.n).astype(np.int32)
        cut, bw = kmp.cut_noalloc(dg, torch.from_numpy(hp).cuda(), k)
        assert cut == O.cut(g, hp), k
        assert np.array_equal(bw, _host_block_weights(g, hp, k)), k


def test_noalloc_second_call_commits_no_device_memory(kmp):
    g = gg.rgg(50000, 8, 11)
    dg = kmp.DeviceGraph.from_host(g)
    part = torch.from_numpy((np.arange(g.n) % 64).astype(np.int32)).cuda()
    kmp.cut_noalloc(dg, part, 64)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        kmp.cut_noalloc(dg, part, 64)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_limits(kmp):
    g = gg.rgg(1000, 8, 2)
    dg = kmp.DeviceGraph.from_host(g)
    part = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(kmp.KmpError) as e:
        kmp.cut_noalloc(dg, part, kmp.KMP_NOALLOC_MAX_K + 1)
    assert e.value.code == kmp.KMP_ERR_ARG
    with pytest.raises(kmp.KmpError) as e:
        kmp.cut_noalloc(dg, part, 0)
    assert e.value.code == kmp.KMP_ERR_ARG
    part[5] = 7
    with pytest.raises(kmp.KmpError):
        kmp.cut_noalloc(dg, part, 4)
    # the entry point stays usable after a rejected call
    part[5] = 0
    cut, bw = kmp.cut_noalloc(dg, part, 4)
    assert cut == 0 and bw[0] == g.n
