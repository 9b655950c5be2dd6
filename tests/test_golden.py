"""The oracle against the stored fixtures under tests/golden/ (each file states
where its values come from).  CPU only."""
import itertools
import os

import pytest

import oracle as O
from paper_2105_02022_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def _graph(family, a, b):
    if family == "path":
        return gg.path(a)
    if family == "cycle":
        return gg.from_edges(a, [(i, (i + 1) % a) for i in range(a)])
    if family == "complete":
        return gg.from_edges(a, list(itertools.combinations(range(a), 2)))
    if family == "grid":
        return gg.grid(a, b)
    raise ValueError(family)


@pytest.mark.parametrize("row", list(_rows("min_bisection.txt")), ids=lambda r: "-".join(r[:3]))
def test_min_bisection_fixture(row):
    family, a, b, want = row[0], int(row[1]), (int(row[2]) if row[2] != "-" else 0), int(row[3])
    g = _graph(family, a, b)
    half = g.n // 2
    cut, side = O.brute_bisection(g, half, half)
    assert cut == want
    assert O.cut(g, side) == want


@pytest.mark.parametrize("row", list(_rows("hash_vectors.txt")), ids=lambda r: "-".join(r[:2]))
def test_hash_fixture(row):
    fn, x, want = row[0], int(row[1], 0), int(row[2], 16)
    if fn == "splitmix64":
        assert O.key(x, []) == want
    else:
        assert O.lib().kmpo_perm32(0, x) == want


def test_full_size_partition_record_is_complete():
    """The stored oracle record of the large-k partition (written by
    tests/golden/make_partition_golden.py from oracle/ alone) has every field
    the GPU test compares, and its level sizes start at the input graph."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rgg24_k16384_partition.txt")
    rec = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        key, *vals = line.split()
        rec[key] = vals
    for key in ("n", "m_directed", "sha256", "cut", "status", "feasible", "max_block", "level_n"):
        assert key in rec, key
    assert len(rec["sha256"][0]) == 64
    assert int(rec["level_n"][0]) == int(rec["n"][0]) == 1 << 24
    assert int(rec["max_block"][0]) <= int(1.03 * ((1 << 24) // (1 << 14)))
