"""Seeded synthetic networks shaped like the paper's workloads.

This module draws signed directed topologies only; it holds none of the
RACIPE arithmetic (parameters and initial conditions are drawn by the
sampler from a seed).  Both the CUDA path and the CPU oracle consume its
edge lists.  numpy's PCG64 generator is used, seeded per workload.

Workloads (GRiNS, arXiv 2503.18356):
  * toggle switch (TS, mutual inhibition) and TS with self-activation
    (TSSA), Sec. 3.1;
  * a random 22-node / 82-edge signed network standing in for the EMT
    network of Sec. 3.2 (whose edge list is not reproduced here): about 40 %
    inhibitory edges, three self-activations, every node on some edge;
  * random signed networks of a given density, for batched and streamed
    ensembles of uneven networks.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Topology:
    n_nodes: int
    src: np.ndarray   # int32 [E]
    dst: np.ndarray   # int32 [E]
    sign: np.ndarray  # int8 [E], +1 activation / -1 inhibition
    name: str = ""

    @property
    def n_edges(self) -> int:
        return int(self.src.size)

    def edges(self):
        return self.n_nodes, self.src, self.dst, self.sign


def _topo(n, edges, name):
    e = np.array(edges, dtype=np.int64).reshape(-1, 3)
    return Topology(n, e[:, 0].astype(np.int32), e[:, 1].astype(np.int32),
                    e[:, 2].astype(np.int8), name)


def toggle_switch() -> Topology:
    """A -| B and B -| A (Sec. 3.1, Fig. 2A i)."""
    return _topo(2, [(0, 1, -1), (1, 0, -1)], "TS")


def toggle_switch_self_activation() -> Topology:
    """TS plus A -> A and B -> B (Sec. 3.1, Fig. 2A ii)."""
    return _topo(2, [(0, 1, -1), (1, 0, -1), (0, 0, 1), (1, 1, 1)], "TSSA")


def cascade(sign: int) -> Topology:
    """A -> B (sign +1) or A -| B (sign -1)."""
    return _topo(2, [(0, 1, sign)], "cascade%+d" % sign)


def random_network(seed: int, n_nodes: int, n_edges: int, n_inhibitory: int,
                   n_self_activations: int = 0, name: str = "") -> Topology:
    """Random signed network with exact counts.

    ``n_self_activations`` distinct nodes get a self-activating loop; the
    remaining ``n_edges - n_self_activations`` edges are distinct ordered
    pairs (i != j), ``n_inhibitory`` of them inhibitory.  Redrawn until every
    node lies on at least one edge.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_pairs = n_edges - n_self_activations
    assert 0 <= n_pairs <= n_nodes * (n_nodes - 1)
    assert 0 <= n_inhibitory <= n_pairs
    for _ in range(10_000):
        selfs = rng.choice(n_nodes, size=n_self_activations, replace=False)
        flat = rng.choice(n_nodes * (n_nodes - 1), size=n_pairs, replace=False)
        i = flat // (n_nodes - 1)
        j = flat % (n_nodes - 1)
        j = j + (j >= i)                      # skip the diagonal
        sign = np.ones(n_pairs, dtype=np.int64)
        sign[rng.choice(n_pairs, size=n_inhibitory, replace=False)] = -1
        src = np.concatenate([selfs, i]).astype(np.int32)
        dst = np.concatenate([selfs, j]).astype(np.int32)
        sg = np.concatenate([np.ones(n_self_activations, dtype=np.int64), sign]).astype(np.int8)
        touched = np.zeros(n_nodes, dtype=bool)
        touched[src] = True
        touched[dst] = True
        if touched.all():
            return Topology(n_nodes, src, dst, sg, name)
    raise RuntimeError("could not draw a connected network")


def density_network(seed: int, n_nodes: int, density: float, name: str = "") -> Topology:
    """E = round(d * N * (N - 1)) distinct non-self pairs, signs 50/50."""
    E = int(round(density * n_nodes * (n_nodes - 1)))
    E = max(E, (n_nodes + 1) // 2)            # enough edges to touch every node
    E = min(E, n_nodes * (n_nodes - 1))
    return random_network(seed, n_nodes, E, E // 2, 0, name)


# ----------------------------------------------------------------- workloads
def ts_workload():
    """Toggle switch, 500 sets x 20 ICs, plain FP64."""
    return dict(topology=toggle_switch(), n_sets=500, n_ics=20, param_seed=2000, ic_seed=2000)


def net5_workload():
    """Random N=5, E=10 (5 activating / 5 inhibiting, no self-loops), 10k x 100."""
    topo = random_network(1001, 5, 10, 5, 0, "rand5x10")
    return dict(topology=topo, n_sets=10_000, n_ics=100, param_seed=2001, ic_seed=2001)


def net22_workload():
    """Random N=22, E=82 (33 inhibitory, 3 self-activations), 100k x 10."""
    topo = random_network(1002, 22, 82, 33, 3, "rand22x82")
    return dict(topology=topo, n_sets=100_000, n_ics=10, param_seed=2002, ic_seed=2002)


def batched_workload(n_networks: int = 64, seed: int = 1003):
    """Uneven networks: N ~ U{2..40}, density ~ U[0.1, 0.3], sets log-uniform
    over [100, 10k], 10 ICs each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(n_networks):
        N = int(rng.integers(2, 41))
        d = float(rng.uniform(0.1, 0.3))
        S = int(round(np.exp(rng.uniform(np.log(100), np.log(10_000)))))
        topo = density_network(seed * 1000 + b, N, d, "batch%d" % b)
        out.append(dict(topology=topo, n_sets=S, n_ics=10, param_seed=2003 + b, ic_seed=2003 + b))
    return out


def serving_stream(rate_hz: float = 20.0, duration_s: float = 60.0, seed: int = 3004):
    """Poisson arrivals; each request a network of N ~ U{2..60}, density
    ~ U[0.05, 0.3], sets log-uniform over [1k, 50k], ICs ~ U{1..20}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    reqs = []
    while True:
        t += float(rng.exponential(1.0 / rate_hz))
        if t >= duration_s:
            break
        r = len(reqs)
        N = int(rng.integers(2, 61))
        d = float(rng.uniform(0.05, 0.3))
        S = int(round(np.exp(rng.uniform(np.log(1_000), np.log(50_000)))))
        I = int(rng.integers(1, 21))
        topo = density_network(seed * 10_000 + r, N, d, "req%d" % r)
        reqs.append(dict(arrival_s=t, topology=topo, n_sets=S, n_ics=I,
                         param_seed=4000 + r, ic_seed=4000 + r))
    return reqs


def sobol_direction_table():
    """The published Sobol initialisation table of Joe and Kuo (2008), as
    scipy ships it (21,201 dimensions): (poly int64 [D], m int64 [D, 18]),
    poly[d] the primitive polynomial of dimension d with bit j the
    coefficient of x^j, m[d, k-1] the initial direction integer m_k.  Data
    only: the direction numbers are derived from it by the sampler and,
    independently, by the oracle."""
    import os

    import scipy.stats
    path = os.path.join(os.path.dirname(scipy.stats.__file__), "_sobol_direction_numbers.npz")
    with np.load(path) as z:
        return (np.ascontiguousarray(z["poly"], dtype=np.int64),
                np.ascontiguousarray(z["vinit"], dtype=np.int64))
