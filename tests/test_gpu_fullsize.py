"""Parity at the full workload sizes, in the launch configuration the
benchmark times: every set of the workload is sampled, integrated (FP32 +
FP64 polish, or plain FP64 for the toggle switch) and deduplicated on the
GPU in one call each; the oracle then recomputes a spread of sampled sets one
by one, and properties that hold at any size are checked on all of them.

Bars (the same as the small parity tests):
  * sampler: bit-exact on every sampled set;
  * polished states: relative 1e-6 (floor 1e-6 G/k); plain FP64: 1e-3 on the
    G/k scale;
  * distinct steady states per set: every mismatch explained by a solve
    whose status differs, and mismatches within 0.1 % of the sampled sets
    (none at these sample sizes);
  * at full size: statuses valid, converged states finite and within
    [0, G/k] (up to 1e-4 of G/k: unpolished states stop within the
    steady-state tolerance), state ids and counts consistent; on the sampled
    sets the polished states meet the residual certificate under the
    oracle's own Eq. 1.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def sampled_sets(S, n):
    """n set indices spread over [0, S), the last set included."""
    return np.unique(np.concatenate([np.linspace(0, S - 1, n).round().astype(np.int64), [S - 1]]))


def check_full_size(w, precision, polish, n_sample, rel_tol, normalised, method=0):
    topo = w["topology"]
    S, I, N = w["n_sets"], w["n_ics"], topo.n_nodes
    net = O.Network(*topo.edges())
    h = PT.gpu_handle(topo)
    params, ic = h.sample_params(w["param_seed"], S, I)
    out = h.integrate(params, ic, precision=precision, polish=polish, method=method)
    sid, nu = h.unique_states(params, out["states"], out["status"])
    torch.cuda.synchronize()
    G, k = (x.cpu().numpy() for x in h.unpack_params(params)[:2])
    states = out["states"].cpu().numpy()
    status = out["status"].cpu().numpy()
    sid, nu = sid.cpu().numpy(), nu.cpu().numpy()

    # properties of every solve and set
    assert states.shape == (S, I, N) and status.shape == (S, I)
    assert np.all(status <= 4)
    conv = status == 0
    x = states[conv]
    gk = (G / k)[:, None, :].repeat(I, axis=1)[conv]
    assert np.all(np.isfinite(x))
    assert np.all(x >= -1e-4 * gk) and np.all(x <= gk * (1 + 1e-4))
    n_conv = conv.sum(axis=1)
    assert np.all(nu <= n_conv) and np.all((nu >= 1) == (n_conv >= 1))
    assert np.all(sid[~conv] == -1) and np.all(sid[conv] >= 0)
    assert np.all(sid.max(axis=1) == nu - 1)

    # the oracle on a spread of sampled sets, one by one
    pick = sampled_sets(S, n_sample)
    ref_p = [O.sample_params(net, w["param_seed"], 1, set0=int(s)) for s in pick]
    Tg, lg, ng = (x.cpu().numpy() for x in h.unpack_params(params[torch.as_tensor(pick, device=params.device)])[2:])
    for q, s in enumerate(pick):
        r = ref_p[q]
        assert np.array_equal(G[s], r.G[0]) and np.array_equal(k[s], r.k[0])
        assert np.array_equal(Tg[q], r.T[0]) and np.array_equal(lg[q], r.lam[0])
        assert np.array_equal(ng[q].astype(np.int32), r.n[0])
    icn = ic.cpu().numpy()
    assert np.array_equal(icn, O.sample_ics(N, w["param_seed"], I))
    p = O.ParamSet(*(np.concatenate([getattr(r, f) for r in ref_p]) for f in ("G", "k", "T", "lam", "n")))
    o = O.run_sets_parallel(net, p, icn, threads=PT.THREADS, polish=bool(polish), method=method)
    g = dict(states=states[pick], status=status[pick])
    c = PT.compare_states(g, o, p, rel_tol, net, normalised=normalised)
    print(w["topology"].name, "sampled", len(pick), c)
    assert c["max_err"] <= rel_tol and c["n_uncertified"] == 0
    assert c["n_basin"] <= 0.01 * g["status"].size
    assert c["status_agree"] >= 0.98
    if polish:
        # the polish certificate, recomputed in FP64 by the oracle's Eq. 1
        both = (g["status"] == 0)
        worst = 0.0
        for q, c_ in zip(*np.nonzero(both)):
            f = O.rhs(net, p, g["states"][q, c_], s=q)
            worst = max(worst, float(np.max(np.abs(f) * p.k[q] / p.G[q])))
        assert worst < 1e-11, worst
    bad = np.flatnonzero(nu[pick] != o["n_unique"])
    st_diff = np.any(g["status"] != o["status"], axis=1)
    print("n_unique mismatches on the sampled sets", [int(pick[b]) for b in bad])
    assert len(bad) <= 0.001 * len(pick)
    assert all(st_diff[b] for b in bad), [int(pick[b]) for b in bad]


def test_net22_full_size_fp32_polish():
    """100,000 sets x 10 ICs of the 22-node network, FP32 + FP64 polish."""
    check_full_size(W.net22_workload(), precision=1, polish=1, n_sample=120, rel_tol=1e-6, normalised=False)


def test_net22_full_size_tsit5_polish():
    """The same full workload with the paper's Tsitouras 5(4) pair on both
    sides (FP32 + FP64 polish on the GPU)."""
    check_full_size(W.net22_workload(), precision=1, polish=1, n_sample=60, rel_tol=1e-6, normalised=False,
                    method=1)


def test_net5_full_size_fp32_polish():
    """10,000 sets x 100 ICs of the 5-node network, FP32 + FP64 polish."""
    check_full_size(W.net5_workload(), precision=1, polish=1, n_sample=80, rel_tol=1e-6, normalised=False)


def test_toggle_switch_full_size_fp64():
    """500 sets x 20 ICs of the toggle switch, plain FP64, every set."""
    check_full_size(W.ts_workload(), precision=0, polish=0, n_sample=500, rel_tol=1e-3, normalised=True)


def test_levels_full_size_net22():
    """The levels row on every solve of the full 22-node workload: histogram,
    boundaries, labels, distinct level states and the multistability
    histogram bit-exact with the oracle's over all 1,000,000 solves."""
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    topo = w["topology"]
    S, I = w["n_sets"], w["n_ics"]
    h = PT.gpu_handle(topo)
    params, ic = h.sample_params(w["param_seed"], S, I)
    out = h.integrate(params, ic)
    counts = h.gk_histogram(params, out["states"], out["status"], n_bins=100)
    torch.cuda.synchronize()
    c = counts.cpu().numpy().view(np.uint64)
    bounds = api.level_boundaries(c, half_width=4, max_boundaries=3)
    lab, ns, mh = h.level_states(params, out["states"], out["status"], bounds, n_bins=100)
    torch.cuda.synchronize()
    G, k = (x.cpu().numpy() for x in h.unpack_params(params)[:2])
    st, stat = out["states"].cpu().numpy(), out["status"].cpu().numpy()
    assert np.array_equal(c, O.gk_histogram(st, stat, G, k, 100))
    assert list(bounds) == list(O.level_boundaries(c, m=4, max_b=3))
    olab, ons, omh = O.level_states(st, stat, G, k, np.asarray(bounds, np.int32), 100)
    assert np.array_equal(lab.cpu().numpy().view(np.uint64), olab)
    assert np.array_equal(ns.cpu().numpy(), ons)
    assert np.array_equal(mh.cpu().numpy().view(np.uint64), omh)
    assert int(omh.sum()) == S and int(c.sum()) == int((stat == 0).sum()) * topo.n_nodes


def is_fixed_point(topo, final, enc01=False):
    """No node of any state would change under Eq. 3 (ties keep the state):
    the field J s of every node agrees in sign with the node's state."""
    N = topo.n_nodes
    bits = ((final[:, None] >> np.arange(N, dtype=np.uint64)[None, :]) & np.uint64(1)).astype(bool)
    s = np.where(bits, 1.0, 0.0 if enc01 else -1.0).astype(np.float32)
    J = np.zeros((N, N), dtype=np.float32)                 # J[src, dst]
    np.add.at(J, (topo.src, topo.dst), topo.sign.astype(np.float32))
    field = s @ J
    return ~np.any((field > 0) & ~bits, axis=1) & ~np.any((field < 0) & bits, axis=1)


def test_ising_full_size_net22():
    """1,000,000 trajectories of the 22-node network, synchronous and
    asynchronous: every converged final state is a fixed point of Eq. 3;
    synchronous trajectories spread over the index range, restarted by the
    oracle from their initial states, and the first asynchronous ones (the
    node choices are drawn per trajectory index) are bit-exact."""
    from paper_2503_18356_gb300 import api
    topo = W.net22_workload()["topology"]
    net = O.Network(*topo.edges())
    h = PT.gpu_handle(topo)
    n, seed = 1_000_000, 31
    init, _, _ = O.ising_run(net, mode=0, seed=seed, n_traj=n, max_steps=0)   # the initial states
    for mode, max_steps in ((api.GRINS_ISING_SYNC, 200), (api.GRINS_ISING_ASYNC, 2000)):
        fin, stp, st = h.ising_run(n, mode=mode, seed=seed, max_steps=max_steps)
        torch.cuda.synchronize()
        fin, stp, st = fin.cpu().numpy().view(np.uint64), stp.cpu().numpy(), st.cpu().numpy()
        conv = st == 0
        assert conv.mean() > 0.9
        assert np.all(is_fixed_point(topo, fin[conv])) and not np.any(is_fixed_point(topo, fin[~conv]))
        assert np.all(stp[~conv] == max_steps)
        if mode == api.GRINS_ISING_SYNC:
            pick = sampled_sets(n, 20_000)
            o = O.ising_run(net, mode=mode, seed=seed, n_traj=len(pick), init=init[pick], max_steps=max_steps)
            got = (fin[pick], stp[pick], st[pick])
        else:
            o = O.ising_run(net, mode=mode, seed=seed, n_traj=3000, max_steps=max_steps)
            got = (fin[:3000], stp[:3000], st[:3000])
        for a, b in zip(got, o):
            assert np.array_equal(a, b), mode
