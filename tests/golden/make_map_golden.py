#!/usr/bin/env python3
"""Writes the expected result of a complete multilevel map, computed by the
CPU oracle alone, for workloads too large for the oracle to run inside a test
(a serial map of R-MAT scale 22 takes tens of minutes).

The file records, per hierarchy level, the vertex count, the CSR entries, the
Alg. 6 iterations and J after refining that level, then the final J, the
SHA-256 of the final mapping (int32, little-endian) and the mapping at 4096
seeded sample positions, so that a mismatch can be located.

Usage:  python tests/golden/make_map_golden.py rmat22
Only ``oracle/`` and the seeded input generators are used; nothing here
touches the CUDA library.
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_2510_12196_gb300 import inputs as I  # noqa: E402

WORKLOADS = {"rmat22": lambda: I.workload_rmat(22)}
SAMPLE = 4096


def golden_path(key: str) -> str:
    return os.path.join(HERE, f"map_{key}.json")


def sample_positions(n: int, seed: int) -> np.ndarray:
    return np.unique((I.splitmix64(seed, np.arange(SAMPLE, dtype=np.uint64)) % np.uint64(n)).astype(np.int64))


def main(key: str) -> None:
    w = WORKLOADS[key]()
    g, t = w.graph, w.topo
    prm = O.default_params(w.seed)
    t0 = time.time()
    pi, J, st = O.map_run(g, t.hier, t.dist, t.eps, prm)
    secs = time.time() - t0
    pos = sample_positions(g.n, w.seed)
    out = {
        "workload": w.name, "seed": w.seed, "n": g.n, "m_dir": g.m_dir,
        "hier": list(t.hier), "dist": list(t.dist), "eps": t.eps,
        "params": "oracle default_params(seed): label-propagation clustering, breadth-first initial mapping, "
                  "G >= 0 filter, edge-cut rebalancing",
        "levels": [{"n": st.n[i], "m_dir": st.m_dir[i], "iters": st.iters[i], "J": st.J[i]}
                   for i in range(st.levels)],
        "J": J,
        "pi_sha256": hashlib.sha256(np.ascontiguousarray(pi, dtype="<i4").tobytes()).hexdigest(),
        "sample_positions_seed": w.seed, "sample_pi": pi[pos].tolist(),
        "oracle_seconds": round(secs, 1),
    }
    with open(golden_path(key), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(f"{key}: J={J} levels={[l['n'] for l in out['levels']]} in {secs:.0f} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "rmat22")
