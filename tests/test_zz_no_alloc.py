"""kmp_cut_noalloc: the cut and block weights of kmp_cut computed without any
device allocation (scratch in a fixed device array), for callers whose device
memory is owned elsewhere or who cannot afford an allocation at call time.

Collected last on purpose (file name); it builds and loads the library itself,
so it also passes when run alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2105_02022_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kmp():
    from paper_2105_02022_gb300 import _build
    from paper_2105_02022_gb300 import kmp as K

    _build.build_all()
    assert torch.cuda.is_available()
    return K


def test_noalloc_matches_cut_on_two_calls(kmp):
    g = gg.with_weights(gg.rgg(20000, 8, 5), 7, 9, 5)
    dg = kmp.DeviceGraph.from_host(g)
    rng = np.random.default_rng(3)
    # two calls in a row; the second one (smaller k) must not see the first one's sums
    for k in (300, 8):
        part = torch.from_numpy(rng.integers(0, k, g.n).astype(np.int32)).cuda()
        ref_cut, ref_bw = kmp.cut(dg, part, k)
        cut, bw = kmp.cut_noalloc(dg, part, k)
        assert cut == ref_cut
        assert np.array_equal(bw, ref_bw)


def test_noalloc_limits(kmp):
    g = gg.rgg(1000, 8, 2)
    dg = kmp.DeviceGraph.from_host(g)
    part = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(kmp.KmpError) as e:
        kmp.cut_noalloc(dg, part, kmp.KMP_NOALLOC_MAX_K + 1)
    assert e.value.code == kmp.KMP_ERR_ARG
    part[5] = 7
    with pytest.raises(kmp.KmpError):
        kmp.cut_noalloc(dg, part, 4)
