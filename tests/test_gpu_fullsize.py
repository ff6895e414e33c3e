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
    whose status differs, and mismatches below 2 % of the sampled sets;
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


def check_full_size(w, precision, polish, n_sample, rel_tol, normalised):
    topo = w["topology"]
    S, I, N = w["n_sets"], w["n_ics"], topo.n_nodes
    net = O.Network(*topo.edges())
    h = PT.gpu_handle(topo)
    params, ic = h.sample_params(w["param_seed"], S, I)
    out = h.integrate(params, ic, precision=precision, polish=polish)
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
    o = O.run_sets_parallel(net, p, icn, threads=PT.THREADS, polish=bool(polish))
    g = dict(states=states[pick], status=status[pick])
    c = PT.compare_states(g, o, p, rel_tol, normalised=normalised)
    print(w["topology"].name, "sampled", len(pick), c)
    assert c["max_rel"] <= rel_tol
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
    assert len(bad) <= 0.02 * len(pick)
    assert all(st_diff[b] for b in bad), [int(pick[b]) for b in bad]


def test_net22_full_size_fp32_polish():
    """100,000 sets x 10 ICs of the 22-node network, FP32 + FP64 polish."""
    check_full_size(W.net22_workload(), precision=1, polish=1, n_sample=120, rel_tol=1e-6, normalised=False)


def test_net5_full_size_fp32_polish():
    """10,000 sets x 100 ICs of the 5-node network, FP32 + FP64 polish."""
    check_full_size(W.net5_workload(), precision=1, polish=1, n_sample=80, rel_tol=1e-6, normalised=False)


def test_toggle_switch_full_size_fp64():
    """500 sets x 20 ICs of the toggle switch, plain FP64, every set."""
    check_full_size(W.ts_workload(), precision=0, polish=0, n_sample=500, rel_tol=1e-3, normalised=True)
