"""Writes net22_oracle_sets0_9999.txt.gz: the oracle's steady-state statuses
and distinct-state counts on sets 0..9999 of the 22-node / 82-edge workload
(100,000 solves), the reference the GPU path's distinct-state counts are
checked against at a size the oracle cannot re-run inside the test suite.

Calls only the oracle (oracle/, FP64 Dormand-Prince 5(4) at rtol 1e-10, atol
1e-13, t_end 200, ss_tol 1e-6, Newton polish, dedupe tol 1e-2: GRiNS Sec.
2.1.3 and Sec. 3.1) on the seeded inputs of paper_2503_18356_gb300.workloads
(topology seed 1002, parameter and IC seed 2002, Table 1 ranges).  Re-run it
whenever the oracle's arithmetic changes:

    python tests/golden/make_net22_reference.py

One line per set: the set index, the oracle's n_unique and its ten status
digits (0 converged, 1 t_end, 2 max_steps, 3 non-finite, 4 polish failed).
"""
import gzip
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2503_18356_gb300 import workloads as W  # noqa: E402

PATH = os.path.join(HERE, "net22_oracle_sets0_9999.txt.gz")
N_SETS = 10_000


def load(path=PATH):
    """-> (status uint8 [S, 10], n_unique int32 [S]) of the stored reference."""
    st, nu = [], []
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("#"):
                continue
            s, n, digits = line.split()
            nu.append(int(n))
            st.append([int(c) for c in digits])
    return np.array(st, dtype=np.uint8), np.array(nu, dtype=np.int32)


def main():
    w = W.net22_workload()
    net = O.Network(*w["topology"].edges())
    u = O.sample_ics(w["topology"].n_nodes, w["ic_seed"], w["n_ics"])
    t0 = time.time()
    chunks = []
    for a in range(0, N_SETS, 1000):
        p = O.sample_params(net, w["param_seed"], 1000, set0=a)
        chunks.append(O.run_sets_parallel(net, p, u))
        print("sets %d..%d done, %.0f s" % (a, a + 999, time.time() - t0), flush=True)
    status = np.concatenate([c["status"] for c in chunks])
    n_unique = np.concatenate([c["n_unique"] for c in chunks])
    with gzip.open(PATH, "wt") as f:
        f.write("# oracle (FP64 DP5 rtol 1e-10, polish, dedupe tol 1e-2) on sets 0..%d of the 22-node "
                "workload; written by make_net22_reference.py\n" % (N_SETS - 1))
        for s in range(N_SETS):
            f.write("%d %d %s\n" % (s, n_unique[s], "".join(str(int(x)) for x in status[s])))


if __name__ == "__main__":
    main()
