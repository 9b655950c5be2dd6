"""Writes the stored expected values of the full-size large-k partition test:
the CPU oracle's partition of the 2D random geometric graph with 2^24 nodes
(average degree 16, seed 1) into k = 2^14 blocks at eps = 0.03, seed 1
(Algorithm 1 under the deterministic readings of oracle/).  Only the input
generator and the oracle run here; nothing comes from the CUDA path.

    python tests/golden/make_partition_golden.py

takes tens of minutes on one core and writes rgg24_k16384_partition.txt:
the SHA-256 of the partition (int32 little-endian, node order), the cut, the
status, the level sizes and the largest block weight."""
import hashlib
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2105_02022_gb300 import graphgen as gg  # noqa: E402

N_LOG, DEG, K, EPS, SEED = 24, 16, 1 << 14, 0.03, 1


def main():
    t0 = time.time()
    g = gg.rgg(1 << N_LOG, DEG, SEED)
    part, rc, st = O.partition(g, K, EPS, SEED)
    part = np.ascontiguousarray(part, dtype="<i4")
    bw = np.bincount(part, minlength=K)
    out = os.path.join(HERE, "rgg24_k16384_partition.txt")
    with open(out, "w") as f:
        f.write("# CPU oracle partition of rgg(2^24, deg 16, seed 1), k = 2^14, eps = 0.03, seed 1\n")
        f.write("# written by tests/golden/make_partition_golden.py (oracle/ and the input generator only)\n")
        f.write(f"n {g.n}\nm_directed {g.m_directed}\n")
        f.write(f"sha256 {hashlib.sha256(part.tobytes()).hexdigest()}\n")
        f.write(f"cut {int(st.cut)}\nstatus {rc}\nfeasible {int(st.feasible)}\n")
        f.write(f"max_block {int(bw.max())}\n")
        f.write("level_n " + " ".join(str(x) for x in list(st.level_n)[: st.levels]) + "\n")
        f.write(f"oracle_seconds {time.time() - t0:.0f}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
