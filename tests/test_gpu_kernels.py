"""The FP32 integrator's kernel variants, each through the C ABI against the
CPU oracle on the same seeded inputs:

  * lane-group layouts with 2, 4 and 8 lanes per solve (GRINS_GRP_L), which
    change the node rows, the edge positions and the lane mapping;
  * the kernels compiled for the network at run time -- records in
    registers (the default) and records in shared memory (GRINS_JIT_KIND)
    -- and the run-time-layout kernel (GRINS_JIT=0).

Bars as in test_gpu_parity.py: FP32 + FP64 polish relative 1e-6 (floor
1e-6 G/k); raw FP32 1e-3 on the G/k scale.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _check(h, params, ic, p, o, net):
    for polish, tol in [(1, 1e-6), (0, 1e-3)]:
        g = PT.to_numpy(h.integrate(params, ic, precision=1, polish=polish))
        torch.cuda.synchronize()
        c = PT.compare_states(g, o, p, tol, net, normalised=not polish)
        print(h.integrator(), polish, c)
        assert c["max_err"] <= tol and c["n_uncertified"] == 0
        assert c["n_basin"] <= max(1, 0.01 * g["status"].size)
        assert c["status_agree"] >= 0.97


@pytest.mark.parametrize("L", [2, 4, 8])
def test_lane_group_layouts_match_oracle(L, monkeypatch):
    monkeypatch.setenv("GRINS_GRP_L", str(L))
    w = W.net22_workload()
    topo = w["topology"]
    h = PT.gpu_handle(topo)
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 40, 10)
    o = O.run_sets_parallel(O.Network(*topo.edges()), p, icn, threads=PT.THREADS)
    _check(h, params, ic, p, o, O.Network(*topo.edges()))
    assert "L=%d lanes" % L in h.integrator()
    h.close()


@pytest.mark.parametrize("jit", ["rr", "grp", "0"])
@pytest.mark.parametrize("wl", ["ts", "net5", "net22"])
def test_compiled_and_runtime_layout_kernels(jit, wl, monkeypatch):
    if jit == "0":
        monkeypatch.setenv("GRINS_JIT", "0")
    else:
        monkeypatch.setenv("GRINS_JIT_KIND", jit)
    w = {"ts": W.ts_workload, "net5": W.net5_workload, "net22": W.net22_workload}[wl]()
    topo = w["topology"]
    h = PT.gpu_handle(topo)
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 40, min(w["n_ics"], 10))
    o = O.run_sets_parallel(O.Network(*topo.edges()), p, icn, threads=PT.THREADS)
    _check(h, params, ic, p, o, O.Network(*topo.edges()))
    info = h.integrator()
    if jit == "0":
        assert "run-time layout" in info, info
    else:
        assert "compiled for this network at run time" in info, info
        kind = "registers" if jit == "rr" else "shared memory"
        assert "records in " + kind in info, info
    h.close()


@pytest.mark.parametrize("jit", ["1", "0"])
@pytest.mark.parametrize("wl", ["ts", "net5", "net22"])
def test_fp64_compiled_and_generic_kernels(jit, wl, monkeypatch):
    """The plain FP64 solver: the register-record kernel compiled in FP64
    (exact power-table edge terms) and the generic FP64 kernel, raw states
    against the oracle on the G/k scale (1e-3, as for FP32)."""
    monkeypatch.setenv("GRINS_JIT", jit)
    w = {"ts": W.ts_workload, "net5": W.net5_workload, "net22": W.net22_workload}[wl]()
    topo = w["topology"]
    h = PT.gpu_handle(topo)
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 40, min(w["n_ics"], 10))
    o = O.run_sets_parallel(O.Network(*topo.edges()), p, icn, threads=PT.THREADS)
    g = PT.to_numpy(h.integrate(params, ic, precision=0, polish=0))
    torch.cuda.synchronize()
    c = PT.compare_states(g, o, p, 1e-3, O.Network(*topo.edges()), normalised=True)
    info = h.integrator()
    print(info, c)
    assert c["max_err"] <= 1e-3 and c["n_uncertified"] == 0
    assert c["n_basin"] <= max(1, 0.01 * g["status"].size)
    assert c["status_agree"] >= 0.97
    if jit == "1":
        assert "FP64, records in registers" in info, info
    h.close()


def _hub_topology(n_reg=12):
    """Node 0 regulated by nodes 1..n_reg (alternating activation and
    inhibition), those nodes a chain 1 -> 2 -> ... -> n_reg + 1 -> 1 with 0 -| n_reg + 1."""
    N = n_reg + 2
    e = [(k, 0, 1 if k % 2 else -1) for k in range(1, n_reg + 1)]
    e += [(k, k + 1, 1) for k in range(1, N - 1)] + [(N - 1, 1, 1), (0, N - 1, -1)]
    a = np.array(e, dtype=np.int64)
    return W.Topology(N, a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int8), "hub12")


@pytest.mark.parametrize("L", [0, 2])
def test_hub_node_beyond_eight_factors(L, monkeypatch):
    """A node with 12 regulators (Eq. 1's product of 12 shifted Hill
    factors): with the library's layout the hub's edges continue in a second
    row; with L = 2 (no free slot to continue in) its row of 12 positions
    takes a chunk of eight factors, too many for one division (its two
    halves are divided apart), and one of four.  The
    polish folds the hub's running products after eight factors and the
    borderline re-pass rescales them every third.

    Bars: polished states (FP32 and FP64 integration) relative 1e-6 against
    the oracle's; raw states 1e-3 on the G/k scale where both sides stopped
    at the same fixed point.  The hub's slow modes let the stop rule
    (residual below ss_tol) end some solves more than 1e-2 G/k from the
    fixed point -- the oracle's own unpolished states stop as far (printed;
    on these sets 8 at 0.015 G/k and one at 0.98 G/k).  Each such raw state
    must be a certified near-equilibrium (residual below 10 ss_tol under the
    oracle's Eq. 1); within polish_max_move (0.1 G/k) of the fixed point its
    polish must land there, beyond it the polish either lands there or
    refuses the step (POLISH_FAIL, raw state kept)."""
    if L:
        monkeypatch.setenv("GRINS_GRP_L", str(L))
    topo = _hub_topology()
    net = O.Network(*topo.edges())
    h = PT.gpu_handle(topo)
    params, ic, p, icn = PT.gpu_sample(h, 23, 40, 8)
    o = O.run_sets_parallel(net, p, icn, threads=PT.THREADS)
    o_raw = O.run_sets_parallel(net, p, icn, threads=PT.THREADS, polish=False)
    Gk = (p.G / p.k)[:, None, :]
    conv_o = o["status"] == O.CONVERGED
    far_o = conv_o & (o_raw["status"] == O.CONVERGED) & (np.max(np.abs(o_raw["states"] - o["states"]) / Gk, axis=2) > 1e-2)
    print(h.integrator(), "oracle raw stops > 1e-2 G/k from its fixed point:", int(far_o.sum()), "of", far_o.size)
    if L:
        assert "L=%d lanes" % L in h.integrator()
    for prec in (1, 0):
        gp = PT.to_numpy(h.integrate(params, ic, precision=prec, polish=1))
        g = PT.to_numpy(h.integrate(params, ic, precision=prec, polish=0))
        torch.cuda.synchronize()
        c = PT.compare_states(gp, o, p, 1e-6, net)
        print(prec, "polished", c)
        assert c["max_err"] <= 1e-6 and c["n_uncertified"] == 0
        assert c["n_basin"] <= max(1, 0.01 * gp["status"].size) and c["status_agree"] >= 0.97
        c = PT.compare_states(g, o, p, 1e-3, net, normalised=True)
        far = (g["status"] == O.CONVERGED) & conv_o & (np.max(np.abs(g["states"] - o["states"]) / Gk, axis=2) > 1e-2)
        print(prec, "raw", c, "stops > 1e-2 G/k from the fixed point:", int(far.sum()))
        assert c["max_err"] <= 1e-3 and c["n_uncertified"] == 0 and c["status_agree"] >= 0.97
        dist = np.max(np.abs(g["states"] - o["states"]) / Gk, axis=2)
        rel = PT.rel_err(gp["states"], o["states"], p.G[:, None, :], p.k[:, None, :]).max(axis=2)
        landed = (gp["status"] == O.CONVERGED) & (rel <= 1e-6)
        refused = (gp["status"] == O.POLISH_FAIL) & np.all(gp["states"] == g["states"], axis=2)
        assert np.all(landed[far & (dist <= 0.1)]), (dist[far], rel[far], gp["status"][far])
        assert np.all((landed | refused)[far & (dist > 0.1)]), (dist[far], rel[far], gp["status"][far])
    h.close()
