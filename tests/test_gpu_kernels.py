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
