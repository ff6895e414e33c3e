"""Request server (grins_racipe_server_*): continuous batching of ensemble
requests on one GPU.

  * each request's results are the same alone and in a mix of concurrent
    requests (bit for bit: a solve's arithmetic does not depend on what else
    runs), and requests in the mix overlap on the device;
  * admission respects the HBM budget, and a request larger than the whole
    budget is refused;
  * a served request agrees with the CPU oracle (FP32 + FP64 polish,
    relative 1e-6 with a floor of 1e-6 G/k), on the run-time-layout kernel
    and on kernels compiled in the background at submission.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _requests(n, max_sets=200, seed=3004):
    from paper_2503_18356_gb300 import api
    reqs = []
    for r in W.serving_stream(rate_hz=20.0, duration_s=60.0, seed=seed)[:n]:
        net = api.Racipe.from_topology(r["topology"])
        reqs.append(dict(net=net, topo=r["topology"], seed=r["param_seed"], S=min(r["n_sets"], max_sets),
                         I=min(r["n_ics"], 8)))
    return reqs


def _np(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def test_results_same_alone_and_in_mix():
    from paper_2503_18356_gb300 import api
    reqs = _requests(6)
    sv = api.Server(max_inflight=8)
    alone = []
    for r in reqs:
        rid = sv.submit(r["net"], r["seed"], r["S"], r["I"])
        sv.wait(rid)
        alone.append(_np(sv.results(rid)))
        sv.release(rid)
    ids = [sv.submit(r["net"], r["seed"], r["S"], r["I"]) for r in reqs]
    infos = [sv.wait(i) for i in ids]
    mix = [_np(sv.results(i)) for i in ids]
    torch.cuda.synchronize()
    for a, m in zip(alone, mix):
        for k in ("states", "status", "n_unique", "state_id"):
            assert np.array_equal(a[k], m[k]), k
    # requests submitted together ran concurrently: some request was admitted
    # before another one finished
    lat = [x["latency_s"] for x in infos]
    que = [x["queued_s"] for x in infos]
    print("latency", np.round(lat, 4), "queued", np.round(que, 4))
    assert any(que[j] < lat[i] for i in range(len(ids)) for j in range(len(ids)) if i != j)
    for i in ids:
        sv.release(i)
    sv.close()


def test_admission_by_budget():
    from paper_2503_18356_gb300 import api
    reqs = _requests(3)
    sizes = []
    sv = api.Server(max_inflight=8, hbm_budget_bytes=1 << 40)
    for r in reqs:
        rid = sv.submit(r["net"], r["seed"], r["S"], r["I"])
        sizes.append(sv.wait(rid)["bytes"])
        sv.release(rid)
    sv.close()
    # a budget that holds one request at a time: the others queue until the
    # running one is released
    budget = max(sizes) + 1024
    sv = api.Server(max_inflight=8, hbm_budget_bytes=budget)
    ids = [sv.submit(r["net"], r["seed"], r["S"], r["I"]) for r in reqs]
    first = sv.wait(ids[0])
    assert first["state"] == api.REQ_DONE
    second = sv.wait(ids[1], timeout_s=0.2)
    assert second["state"] == api.REQ_QUEUED      # waits for memory
    sv.release(ids[0])
    for i in ids[1:]:
        assert sv.wait(i)["state"] == api.REQ_DONE
        sv.release(i)
    big = reqs[0]
    with pytest.raises(api.GrinsError) as e:
        sv.submit(big["net"], big["seed"], 10 * big["S"], big["I"])
    assert e.value.status == api.GRINS_E_BUDGET
    sv.close()


def test_served_request_matches_oracle():
    from paper_2503_18356_gb300 import api
    r = _requests(2, max_sets=24)[1]
    sv = api.Server()
    rid = sv.submit(r["net"], r["seed"], r["S"], r["I"])
    sv.wait(rid)
    g = _np(sv.results(rid))
    sv.release(rid)
    sv.close()
    topo = r["topo"]
    net = O.Network(*topo.edges())
    p = O.sample_params(net, r["seed"], r["S"])
    ic = O.sample_ics(topo.n_nodes, r["seed"], r["I"])
    o = O.run_sets_parallel(net, p, ic, threads=PT.THREADS)
    c = PT.compare_states(g, o, p, 1e-6, net)
    print(topo.n_nodes, topo.n_edges, c)
    assert c["max_err"] <= 1e-6 and c["n_uncertified"] == 0
    assert c["n_compared"] > 0
    assert c["n_basin"] <= max(1, 0.01 * g["status"].size)
    # a status mismatch is a slow solve meeting the steady-state condition
    # before t_end on one side only (converged, possibly with a polish that
    # could not certify it, vs t_end), never a non-finite or step-limit stop
    diff = g["status"] != o["status"]
    seen = set(g["status"][diff].tolist()) | set(o["status"][diff].tolist())
    assert seen <= {O.CONVERGED, O.TEND, O.POLISH_FAIL}, seen
    assert c["status_agree"] >= 0.9


def test_requests_on_compiled_kernels():
    """With jit_min_work = 0 every FP32 request starts a background compile of
    its network's integrator at submission and is admitted once it is done:
    results agree with the oracle as on the run-time-layout kernel, and a
    second request on the same network finds the kernel compiled."""
    from paper_2503_18356_gb300 import api
    reqs = _requests(3, max_sets=24)[1:]
    sv = api.Server(jit_min_work=0.0, jit_max_wait_s=60.0)
    ids = [sv.submit(r["net"], r["seed"], r["S"], r["I"]) for r in reqs]
    infos = [sv.wait(i) for i in ids]
    assert all(x["state"] == api.REQ_DONE for x in infos), infos
    res = [_np(sv.results(i)) for i in ids]
    for i in ids:
        sv.release(i)
    r = reqs[0]
    again = sv.submit(r["net"], r["seed"], r["S"], r["I"])
    info2 = sv.wait(again)
    g2 = _np(sv.results(again))
    sv.release(again)
    sv.close()
    print("queued", [round(x["queued_s"], 3) for x in infos], "second", round(info2["queued_s"], 4))
    assert info2["queued_s"] < infos[0]["queued_s"] + 0.5
    for k in ("states", "status", "n_unique", "state_id"):
        assert np.array_equal(res[0][k], g2[k]), k
    for r, g in zip(reqs, res):
        topo = r["topo"]
        net = O.Network(*topo.edges())
        p = O.sample_params(net, r["seed"], r["S"])
        ic = O.sample_ics(topo.n_nodes, r["seed"], r["I"])
        o = O.run_sets_parallel(net, p, ic, threads=PT.THREADS)
        c = PT.compare_states(g, o, p, 1e-6, net)
        print(topo.n_nodes, topo.n_edges, c)
        assert c["max_err"] <= 1e-6 and c["n_uncertified"] == 0
        assert c["n_compared"] > 0
        assert c["n_basin"] <= max(1, 0.01 * g["status"].size)
        diff = g["status"] != o["status"]
        seen = set(g["status"][diff].tolist()) | set(o["status"][diff].tolist())
        assert seen <= {O.CONVERGED, O.TEND, O.POLISH_FAIL}, seen


def test_request_keeps_its_own_copy_of_the_ranges_tables():
    """A request with Sobol sets, a per-parameter table and initial-condition
    rows: the caller overwrites its arrays right after submitting, and the
    served results still match the same work run directly on the handle
    (the server may run another kernel for a request this small, so the
    polished states agree to the polish tolerance, not bit for bit)."""
    from paper_2503_18356_gb300 import api
    r = _requests(1)[0]
    net, S, I = r["net"], r["S"], r["I"]
    poly, m = W.sobol_direction_table()
    rows = net.param_range_table()
    rows[0] = (api.GRINS_DIST_LOGUNIFORM, 0, 5.0, 50.0)
    icr = np.zeros(net.n_nodes, dtype=api.PARAM_RANGE_DTYPE)
    icr[:] = (0, 0, 0.1, 0.9)

    def ranges(poly, m, rows, icr):
        return api.default_ranges(sobol=api.GRINS_SOBOL_SCRAMBLED, sobol_table=(poly, m), param_ranges=rows,
                                  ic_ranges=icr)

    params, ic = net.sample_params(r["seed"], S, I, ranges=ranges(poly, m, rows, icr))
    out = net.integrate(params, ic)
    _, nu = net.unique_states(params, out["states"], out["status"])
    direct = dict(states=out["states"].cpu().numpy(), status=out["status"].cpu().numpy(), n_unique=nu.cpu().numpy())

    p2, m2, rows2, icr2 = poly.copy(), m.copy(), rows.copy(), icr.copy()
    rr = ranges(p2, m2, rows2, icr2)
    sv = api.Server(max_inflight=4)
    rid = sv.submit(net, r["seed"], S, I, ranges=rr)
    p2[:] = 0; m2[:] = 0; rows2["lo"] = -1.0; icr2["hi"] = 7.0       # the caller's arrays change at once
    info = sv.wait(rid)
    served = _np(sv.results(rid))
    print("request", info)
    both = (served["status"] == 0) & (direct["status"] == 0)
    assert np.mean(served["status"] == direct["status"]) >= 0.97
    G, k = (x.cpu().numpy() for x in net.unpack_params(params)[:2])
    gk = np.broadcast_to((G / k)[:, None, :], direct["states"].shape)
    d = np.abs(served["states"] - direct["states"])[both]
    scale = np.maximum(np.abs(direct["states"][both]), 1e-6 * gk[both])
    assert both.sum() > 0 and np.all(d <= 1e-6 * scale)
    assert np.mean(served["n_unique"] == direct["n_unique"]) >= 0.95
    sv.release(rid)
    sv.close()
