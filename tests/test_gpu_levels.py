"""GPU parity of the levels path (G/k histogram, level labels, distinct
states per set, multistability histogram) with the oracle, bit-exact,
through the C ABI."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu

U64MAX = np.iinfo(np.uint64).max


def gpu_levels(h, params, states, status, n_bins, bounds):
    counts = h.gk_histogram(params, states, status, n_bins=n_bins)
    lab, ns, mh = h.level_states(params, states, status, bounds, n_bins=n_bins)
    torch.cuda.synchronize()
    return (counts.cpu().numpy().view(np.uint64), lab.cpu().numpy().view(np.uint64), ns.cpu().numpy(),
            mh.cpu().numpy().view(np.uint64))


def check(h, params, states, status, G, k, n_bins, bounds):
    counts, lab, ns, mh = gpu_levels(h, params, states, status, n_bins, bounds)
    st, stat = states.cpu().numpy(), status.cpu().numpy()
    assert np.array_equal(counts, O.gk_histogram(st, stat, G, k, n_bins))
    olab, ons, omh = O.level_states(st, stat, G, k, np.asarray(bounds, np.int32), n_bins)
    assert np.array_equal(lab, olab)
    assert np.array_equal(ns, ons)
    assert np.array_equal(mh, omh)
    return counts, lab, ns, mh


def test_levels_on_integrated_net22_states():
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    S, I = 300, 10
    params, ic, p, _ = PT.gpu_sample(h, w["param_seed"], S, I)
    out = h.integrate(params, ic)
    torch.cuda.synchronize()
    counts = h.gk_histogram(params, out["states"], out["status"], n_bins=100)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint64)
    bounds = api.level_boundaries(c, half_width=4, max_boundaries=3)
    assert list(bounds) == list(O.level_boundaries(c, m=4, max_b=3))
    print("boundaries", bounds, "histogram", c[:5], c[-5:])
    _, lab, ns, mh = check(h, params, out["states"], out["status"], p.G, p.k, 100, bounds)
    assert mh.sum() == S
    # the counts add up: every converged solve's nodes, one histogram
    conv = int((out["status"] == 0).sum().item())
    assert c.sum() == conv * 22


def test_levels_on_bin_edges_and_accumulation():
    topo = W.random_network(3, 6, 14, 6, 0)
    h = PT.gpu_handle(topo)
    S, I, N, B = 64, 40, 6, 64
    params, _, p, _ = PT.gpu_sample(h, 5, S, I)
    rng = np.random.default_rng(0)
    v = rng.integers(0, B + 1, (S, I, N)) / B              # values on bin edges, 0 and 1 included
    v[::5, 3, 2] = -0.25
    v[::7, 1, 0] = 1.5
    x = v * p.G[:, None, :] / p.k[:, None, :]
    status = (rng.uniform(size=(S, I)) < 0.2).astype(np.uint8)
    xs = torch.tensor(x, device="cuda"); ss = torch.tensor(status, device="cuda")
    check(h, params, xs, ss, p.G, p.k, B, [10, 31, 50])
    # two half batches add up to the whole histogram
    half = S // 2
    counts = h.gk_histogram(params[:half], xs[:half], ss[:half], n_bins=B)
    h.gk_histogram(params[half:], xs[half:], ss[half:], n_bins=B, counts=counts)
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy().view(np.uint64), O.gk_histogram(x, status, p.G, p.k, B))


def test_levels_edge_cases():
    from paper_2503_18356_gb300 import api
    # nothing converged: sentinel labels, no states
    topo = W.random_network(4, 3, 5, 2, 0)
    h = PT.gpu_handle(topo)
    params, _, p, _ = PT.gpu_sample(h, 1, 8, 4)
    x = torch.ones((8, 4, 3), dtype=torch.float64, device="cuda")
    st = torch.full((8, 4), 1, dtype=torch.uint8, device="cuda")
    counts, lab, ns, mh = gpu_levels(h, params, x, st, 50, [20])
    assert counts.sum() == 0 and np.all(lab == U64MAX) and np.all(ns == 0) and mh[0] == 8
    # 64 nodes: one boundary fills the 64-bit label, two do not fit
    big = W.random_network(9, 64, 128, 64, 0)
    hb = PT.gpu_handle(big)
    params, _, p, _ = PT.gpu_sample(hb, 2, 4, 3)
    v = np.random.default_rng(1).uniform(0, 1, (4, 3, 64))
    xb = torch.tensor(v * p.G[:, None, :] / p.k[:, None, :], device="cuda")
    sb = torch.zeros((4, 3), dtype=torch.uint8, device="cuda")
    check(hb, params, xb, sb, p.G, p.k, 100, [50])
    with pytest.raises(api.GrinsError):
        hb.level_states(params, xb, sb, [30, 60], n_bins=100)
    with pytest.raises(api.GrinsError):
        h.level_states(params[:1], x[:1], st[:1], [30, 20], n_bins=50)   # not increasing
