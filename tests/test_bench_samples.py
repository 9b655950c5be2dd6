"""CPU checks of the measurement plumbing: the oracle's timing-only sample
options, which bound the benchmark's CPU baseline and reference arm, and the
committed DRAM-traffic record the bench line scales by its own algorithmic
bytes."""
import hashlib
import json
import os

import numpy as np
import pytest

import bench
import oracle as O
from paper_2105_02022_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rmat():
    O.build()
    return gg.rmat(14, 16, 1)


def _scanned(g, U, **kw):
    _, _, st = O.cluster(g, U, 1, 1, 0, cfg=O.config(sample_subrounds=1, **kw), isolated=False,
                         two_hop=False, stats=True)
    return int(st.scanned[0])


def test_sample_nodes_bounds_the_sampled_subround(rmat):
    """sample_nodes rates only nodes below it in the sampled sub-round: fewer
    entries than the whole sub-round, more with more nodes, the whole
    sub-round at n (or 0)."""
    g = rmat
    U = bench.level0_cap(g, 256)
    full = _scanned(g, U)
    assert full > 0
    assert _scanned(g, U, sample_nodes=0) == full
    assert _scanned(g, U, sample_nodes=g.n) == full
    third, half = _scanned(g, U, sample_nodes=g.n // 3), _scanned(g, U, sample_nodes=g.n // 2)
    assert 0 < third < half < full
    # one sub-round of S = 8 rates about an eighth of the entries
    assert full < 0.25 * g.m_directed


def test_sample_nodes_without_sampling_changes_nothing(rmat):
    """Outside a timing sample (sample_subrounds = 0) the option is inert:
    the labels equal those of the default configuration."""
    g = rmat
    U = bench.level0_cap(g, 256)
    ref = O.cluster(g, U, 3, 1, 0)
    got = O.cluster(g, U, 3, 1, 0, cfg=O.config(sample_nodes=g.n // 5))
    assert np.array_equal(ref, got)


def test_traffic_record_is_tied_to_its_workload_and_source():
    """The bench reports DRAM traffic from the committed record only for the
    workload it was captured on and only while the LP source is the one it was
    captured from; the per-span figure is the record's bytes per algorithmic
    byte times the run's own algorithmic bytes."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "lp_rate_traffic.json")))
    for w in rec["applies_to"]:
        assert w in bench.WORKLOADS
    src = open(os.path.join(ROOT, "paper_2105_02022_gb300", "csrc", "kmp_lp.cu"), "rb").read()
    same_source = hashlib.sha256(src).hexdigest() == rec["kmp_lp_cu_sha256"]
    w = rec["applies_to"][0]
    for key in ("stage", "k_rate"):
        got = bench.recorded_rate_traffic(w, 1.0e9, key)
        if same_source:
            assert got == pytest.approx(rec[key]["dram_bytes_per_algorithmic_byte"] * 1.0e9)
        else:
            assert got is None
    other = next(n for n in bench.WORKLOADS if n not in rec["applies_to"])
    assert bench.recorded_rate_traffic(other, 1.0e9, "stage") is None
    # the record's own figures are consistent
    st = rec["stage"]
    assert st["dram_bytes_per_algorithmic_byte"] == pytest.approx(
        st["dram_bytes_per_step"] / st["algorithmic_bytes_per_step"])
    assert st["dram_bytes_per_span"] == pytest.approx(st["dram_bytes_per_step"] / rec["spans_per_step"])
    per = rec["per_kernel"]
    assert sum(v["dram_read_bytes"] + v["dram_write_bytes"] for v in per.values()) == st["dram_bytes_per_step"]
