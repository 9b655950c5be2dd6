"""The seeded input generators: their output does not depend on the number of
host threads that build it.  CPU only."""
import hashlib
import os
import subprocess
import sys

from paper_2105_02022_gb300 import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SNIPPET = (
    "import hashlib, sys; sys.path.insert(0, %r)\n"
    "from paper_2105_02022_gb300 import graphgen as gg\n"
    "g = gg.rmat(17, 16, 5)\n"
    "print(hashlib.sha256(g.xadj.tobytes() + g.adjncy.tobytes()).hexdigest())\n" % ROOT
)


def _digest(g):
    return hashlib.sha256(g.xadj.tobytes() + g.adjncy.tobytes()).hexdigest()


def test_rmat_same_with_one_and_many_threads():
    here = _digest(gg.rmat(17, 16, 5))
    for threads in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=threads)
        out = subprocess.run([sys.executable, "-c", _SNIPPET], env=env, capture_output=True, text=True,
                             check=True).stdout.strip()
        assert out == here, threads


def test_rmat_same_when_the_runtime_gives_fewer_threads():
    """The work is split into as many chunks as threads were asked for; a
    runtime that grants fewer (a thread limit, dynamic teams) must still
    process every chunk."""
    here = _digest(gg.rmat(17, 16, 5))
    for env_extra in ({"OMP_NUM_THREADS": "4", "OMP_THREAD_LIMIT": "2"},
                      {"OMP_NUM_THREADS": "6", "OMP_DYNAMIC": "true", "OMP_THREAD_LIMIT": "3"}):
        env = dict(os.environ, **env_extra)
        out = subprocess.run([sys.executable, "-c", _SNIPPET], env=env, capture_output=True, text=True,
                             check=True).stdout.strip()
        assert out == here, env_extra


def test_rmat_csr_is_symmetric_sorted_and_loop_free():
    g = gg.rmat(14, 16, 3)
    import numpy as np

    src = np.repeat(np.arange(g.n), np.diff(g.xadj))
    assert not np.any(src == g.adjncy)
    pairs = set(zip(src.tolist(), g.adjncy.tolist()))
    assert all((v, u) in pairs for u, v in pairs)
    for v in range(0, g.n, 97):
        row = g.adjncy[g.xadj[v]:g.xadj[v + 1]]
        assert np.all(np.diff(row) > 0)
