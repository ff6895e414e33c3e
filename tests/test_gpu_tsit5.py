"""The Tsitouras 5(4) pair (the paper's Tsit5) on the GPU against the
oracle's Tsit5, through the C ABI: FP32 raw and polished, the plain FP64
solver, a time series, and the calls that take Dormand-Prince only."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def run(h, params, ic, **opt):
    out = h.integrate(params, ic, **opt)
    torch.cuda.synchronize()
    return PT.to_numpy(out)


@pytest.mark.parametrize("wl,S", [("net5", 60), ("net22", 60)])
def test_tsit5_fp32_polished_and_raw(wl, S):
    from paper_2503_18356_gb300 import api
    w = {"net5": W.net5_workload, "net22": W.net22_workload}[wl]()
    h = PT.gpu_handle(w["topology"])
    I = min(w["n_ics"], 10)
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], S, I)
    o = O.run_sets_parallel(O.Network(*w["topology"].edges()), p, icn, threads=PT.THREADS, method=1)
    for polish, tol in [(1, 1e-6), (0, 1e-3)]:
        g = run(h, params, ic, precision=1, polish=polish, method=api.GRINS_METHOD_TSIT5)
        c = PT.compare_states(g, o, p, tol, O.Network(*w["topology"].edges()), normalised=not polish)
        print(wl, polish, h.integrator(), c)
        assert c["max_err"] <= tol and c["n_uncertified"] == 0
        assert c["n_basin"] <= max(1, 0.01 * g["status"].size)
        assert c["status_agree"] >= 0.97


def test_tsit5_fp64_and_series():
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 24, 8)
    net = O.Network(*w["topology"].edges())
    o = O.run_sets_parallel(net, p, icn, threads=PT.THREADS, method=1)
    g = run(h, params, ic, precision=0, polish=0, method=api.GRINS_METHOD_TSIT5)
    c = PT.compare_states(g, o, p, 1e-3, net, normalised=True)
    print("fp64", h.integrator(), c)
    assert "FP64 solver compiled" in h.integrator()
    assert c["max_err"] <= 1e-3 and c["status_agree"] >= 0.97 and c["n_uncertified"] == 0
    grid = np.linspace(0.0, 30.0, 16)
    small = W.net5_workload()
    hs = PT.gpu_handle(small["topology"])
    params, ic, p, icn = PT.gpu_sample(hs, small["param_seed"], 20, 6)
    gs = run(hs, params, ic, precision=1, polish=0, t_grid=grid, method=api.GRINS_METHOD_TSIT5)
    os_ = O.run_sets_parallel(O.Network(*small["topology"].edges()), p, icn, threads=PT.THREADS,
                              series=True, t_grid=grid, method=1)
    G = p.G[:, None, None, :]; k = p.k[:, None, None, :]
    err = PT.rel_err(gs["series"], os_["series"], G, k, floor=1e-6)
    assert np.max(err) < 1e-3


def test_tsit5_refused_where_only_dormand_prince_runs(monkeypatch):
    from paper_2503_18356_gb300 import api
    w = W.net5_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, _, _ = PT.gpu_sample(h, w["param_seed"], 4, 3)
    with pytest.raises(api.GrinsError):
        h.integrate(params, ic, method=7)
    monkeypatch.setenv("GRINS_JIT", "0")
    h0 = PT.gpu_handle(w["topology"])
    params0, ic0, _, _ = PT.gpu_sample(h0, w["param_seed"], 4, 3)
    with pytest.raises(api.GrinsError):
        h0.integrate(params0, ic0, method=api.GRINS_METHOD_TSIT5)
    monkeypatch.delenv("GRINS_JIT")
    opts = api.default_opts(method=api.GRINS_METHOD_TSIT5)
    with pytest.raises(api.GrinsError):
        api.Plan([dict(net=h, params=params, ic_unit=ic)], opts=opts)
