"""Batched launch (grins_racipe_plan_*): many uneven networks in one
persistent launch (of the kernel compiled for every job's layout, or of the
run-time-layout kernel), or each on its own compiled kernel on a graph
branch, under a captured CUDA graph, checked job by job against the CPU
oracle and against the single-network path.

Bars as in test_gpu_parity.py: FP32 + FP64 polish relative 1e-6 (floor
1e-6 G/k) against the oracle; distinct-state counts equal the oracle's
except where a solve's status differs; a replay of the graph reproduces the
first run bit for bit (every solve's arithmetic is independent of which
warp runs it).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _jobs(n_networks, max_sets, seed=1003):
    from paper_2503_18356_gb300 import api
    jobs = []
    for wl in W.batched_workload(n_networks, seed=seed):
        topo = wl["topology"]
        h = api.Racipe.from_topology(topo)
        S = min(wl["n_sets"], max_sets)
        params, ic = h.sample_params(wl["param_seed"], S, wl["n_ics"])
        jobs.append(dict(net=h, params=params, ic_unit=ic, topo=topo))
    return jobs


def _np(out):
    return {k: v.cpu().numpy() for k, v in out.items() if v is not None}


@pytest.mark.parametrize("autotune", [1, 2, 3, 0])
def test_plan_matches_oracle_and_replays_exactly(autotune):
    """Every form of the plan against the oracle: the autotuner's pick (1),
    per-network compiled kernels on graph branches (2), one persistent
    launch of a kernel compiled for every job's layout (3) and one
    persistent launch of the run-time-layout kernel (0)."""
    from paper_2503_18356_gb300 import api
    jobs = _jobs(8, 48)
    plan = api.Plan(jobs, autotune=autotune)
    info = plan.info()
    print(info)
    if autotune == 1:
        assert "autotuned" in info and "per-network compiled kernels:" in info and "one compiled launch" in info
    elif autotune == 2:
        assert "per-network compiled" in info
    elif autotune == 3:
        assert "one persistent launch of a kernel compiled" in info
    else:
        assert "batched lane-group" in info
    res1 = [_np(j["out"]) for j in plan.run()]
    torch.cuda.synchronize()
    res2 = [_np(j["out"]) for j in plan.run()]
    torch.cuda.synchronize()
    for a, b in zip(res1, res2):
        for k in ("states", "status", "n_steps", "state_id", "n_unique"):
            assert np.array_equal(a[k], b[k]), k
    for jb, g in zip(jobs, res1):
        h, topo = jb["net"], jb["topo"]
        S = min(16, jb["params"].shape[0])
        G, k, T, lam, n = (x[:S].cpu().numpy() for x in h.unpack_params(jb["params"]))
        p = O.ParamSet(G, k, T, lam, n.astype(np.int32))
        o = O.run_sets_parallel(O.Network(*topo.edges()), p, jb["ic_unit"].cpu().numpy(), threads=PT.THREADS)
        gs = {kk: v[:S] for kk, v in g.items()}
        c = PT.compare_states(gs, o, p, 1e-6, O.Network(*topo.edges()))
        print(topo.name, topo.n_nodes, topo.n_edges, c)
        assert c["max_err"] <= 1e-6 and c["n_uncertified"] == 0
        assert c["n_basin"] <= max(1, 0.01 * gs["status"].size)
        assert c["status_agree"] >= 0.95
        bad = np.where(gs["n_unique"] != o["n_unique"])[0]
        st_diff = np.any(gs["status"] != o["status"], axis=1)
        assert all(st_diff[s] for s in bad), bad
    plan.close()


@pytest.mark.parametrize("autotune", [0, 3])
def test_plan_agrees_with_single_network_path(autotune):
    from paper_2503_18356_gb300 import api
    jobs = _jobs(5, 64, seed=77)
    plan = api.Plan(jobs, autotune=autotune)
    res = [_np(j["out"]) for j in plan.run()]
    torch.cuda.synchronize()
    for jb, g in zip(jobs, res):
        h = jb["net"]
        single = _np(h.integrate(jb["params"], jb["ic_unit"], tail_rtol=0.0))   # plans run no re-pass
        torch.cuda.synchronize()
        both = (g["status"] == 0) & (single["status"] == 0)
        assert both.mean() >= 0.9 * (single["status"] == 0).mean()
        G, k = (x.cpu().numpy() for x in h.unpack_params(jb["params"])[:2])
        v1 = g["states"] * k[:, None, :] / G[:, None, :]
        v2 = single["states"] * k[:, None, :] / G[:, None, :]
        same = both & (np.abs(v1 - v2).max(axis=2) <= 1e-2)      # same basin
        err = PT.rel_err(g["states"], single["states"], G[:, None, :], k[:, None, :])
        assert same.sum() >= 0.98 * both.sum()
        assert err[same].max() <= 2e-6
    plan.close()


def test_plan_rejects_unsupported_options():
    from paper_2503_18356_gb300 import api
    jobs = _jobs(2, 4)
    with pytest.raises(api.GrinsError):
        api.Plan(jobs, opts=api.default_opts(precision=api.GRINS_FP64))
    grid = np.linspace(0, 1, 3)
    o = api.default_opts()
    o.t_grid = grid.ctypes.data_as(api.C.POINTER(api.C.c_double))
    o.n_t = 3
    with pytest.raises(api.GrinsError):
        api.Plan(jobs, opts=o)
