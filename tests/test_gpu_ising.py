"""GPU Boolean Ising (Eq. 3) against the oracle, bit for bit: synchronous and
asynchronous modes, both encodings, random and given initial states, from
one node up to the 64-node limit."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def gpu(h, n, **kw):
    fin, stp, st = h.ising_run(n, **kw)
    torch.cuda.synchronize()
    return fin.cpu().numpy().view(np.uint64), stp.cpu().numpy(), st.cpu().numpy()


def check(topo, n, seed, max_steps, init=None):
    from paper_2503_18356_gb300 import api
    h = PT.gpu_handle(topo)
    net = O.Network(*topo.edges())
    dinit = None if init is None else torch.tensor(init.view(np.int64), device="cuda")
    for mode in (api.GRINS_ISING_SYNC, api.GRINS_ISING_ASYNC):
        for enc01 in (False, True):
            g = gpu(h, n, mode=mode, seed=seed, init=dinit, max_steps=max_steps, enc01=enc01)
            o = O.ising_run(net, mode=mode, seed=seed, n_traj=n, init=init, max_steps=max_steps, enc01=enc01)
            for a, b in zip(g, o):
                assert np.array_equal(a, b), (mode, enc01)
            print(topo.n_nodes, mode, enc01, "converged", np.mean(g[2] == 0), "mean steps", g[1].mean())


def test_ising_net22_random_initial_states():
    check(W.net22_workload()["topology"], 2000, 31, 300)


def test_ising_given_states_small_and_wide():
    ts = W.toggle_switch()
    check(ts, 4, 1, 9, init=np.arange(4, dtype=np.uint64))
    one = W.random_network(2, 1, 1, 0, 1)
    check(one, 2, 3, 5, init=np.array([0, 1], dtype=np.uint64))
    wide = W.random_network(8, 64, 200, 100, 2)
    rng = np.random.default_rng(0)
    init = rng.integers(0, 2 ** 63, 500, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 500, dtype=np.uint64)
    check(wide, 500, 7, 200, init=init)


def test_ising_argument_errors():
    from paper_2503_18356_gb300 import api
    h = PT.gpu_handle(W.toggle_switch())
    with pytest.raises(api.GrinsError):
        h.ising_run(4, mode=2)
    with pytest.raises(api.GrinsError):
        h.ising_run(4, max_steps=-1)
