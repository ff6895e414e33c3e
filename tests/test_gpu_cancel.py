"""Cancellation, driven from the host only: a call's cancel flag
(grins_solver_opts.cancel) set before or while it runs, and
grins_racipe_server_cancel on a queued and on a running request.  The
kernels stop taking work; solves in flight finish; the rest are marked
GRINS_SS_CANCELLED; no call hangs (each wait here has a limit)."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _flag(value=0):
    return torch.full((1,), value, dtype=torch.int32, device="cuda")


def test_cancel_flag_set_before_the_call():
    from paper_2503_18356_gb300 import api
    w = W.net5_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, _, _ = PT.gpu_sample(h, w["param_seed"], 200, 8)
    flag = _flag(1)
    for prec in (api.GRINS_FP32, api.GRINS_FP64):
        o = api.default_opts(precision=prec)
        o.cancel = flag.data_ptr()
        out = h.integrate(params, ic, opts=o)
        torch.cuda.synchronize()
        st = out["status"].cpu().numpy()
        assert np.all(st == api.CANCELLED), np.bincount(st.ravel())
    h.close()


def _set_later(flag, delay_s, done):
    """Writes 1 into the device flag after delay_s, by a copy on a side
    stream (the copy engine, not a kernel: it runs beside the integrator)."""
    side = torch.cuda.Stream()
    one = torch.ones((1,), dtype=torch.int32).pin_memory()
    time.sleep(delay_s)
    with torch.cuda.stream(side):
        flag.copy_(one, non_blocking=True)
    side.synchronize()
    done.set()


@pytest.mark.parametrize("jit", ["1", "0"])
def test_cancel_flag_set_while_running(jit, monkeypatch):
    """1,000,000 solves of the 22-node workload (the compiled kernel, and the
    run-time-layout kernel with GRINS_JIT=0): the flag set after a fifth of
    the uncancelled run's time ends the call early, with cancelled solves;
    every solve that did run equals the uncancelled run's result."""
    from paper_2503_18356_gb300 import api
    monkeypatch.setenv("GRINS_JIT", jit)
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    S = 100_000 if jit == "1" else 50_000
    params, ic = h.sample_params(w["param_seed"], S, w["n_ics"])
    o = api.default_opts(polish=0, tail_rtol=0.0)
    flag = _flag(0)
    o.cancel = flag.data_ptr()          # the same kernel (one that polls a flag) for every run
    ref = h.integrate(params, ic, opts=o)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = PT.to_numpy(h.integrate(params, ic, opts=o, out=ref))
    t_full = time.perf_counter() - t0
    assert not np.any(ref["status"] == api.CANCELLED)
    done = threading.Event()
    th = threading.Thread(target=_set_later, args=(flag, 0.2 * t_full, done))
    t0 = time.perf_counter()
    th.start()
    out = h.integrate(params, ic, opts=o)
    torch.cuda.synchronize()
    t_cut = time.perf_counter() - t0
    th.join(timeout=30)
    assert done.is_set()
    got = PT.to_numpy(out)
    cancelled = got["status"] == api.CANCELLED
    print("full %.3f s, cancelled run %.3f s, cancelled solves %d of %d" % (t_full, t_cut, cancelled.sum(),
                                                                          cancelled.size))
    assert cancelled.sum() > 0.2 * cancelled.size
    assert t_cut < 0.8 * t_full
    ran = ~cancelled
    assert ran.sum() > 0
    for k in ("states", "status", "n_steps"):
        assert np.array_equal(got[k][ran], ref[k][ran]), k
    h.close()


def _wait_state(sv, rid, states, limit_s=60.0):
    t0 = time.time()
    while time.time() - t0 < limit_s:
        info = sv.wait(rid, timeout_s=0.005)
        if info["state"] in states:
            return info
    raise AssertionError("request %d did not reach %s" % (rid, states))


def test_server_cancel_queued_and_running():
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    sv = api.Server(max_inflight=1)
    nets = [api.Racipe.from_topology(w["topology"]), api.Racipe.from_topology(w["topology"])]
    # the first request takes the only slot; the second, submitted once the
    # first runs, waits in the queue
    r1 = sv.submit(nets[0], w["param_seed"], 1_500_000, 10)      # about 1.4 s of work
    _wait_state(sv, r1, (api.REQ_RUNNING, api.REQ_DONE))
    r2 = sv.submit(nets[1], w["param_seed"], 1_000, 10)
    assert sv.wait(r2, timeout_s=0.0)["state"] in (api.REQ_QUEUED, api.REQ_RUNNING, api.REQ_DONE)
    queued = sv.wait(r2, timeout_s=0.0)["state"] == api.REQ_QUEUED
    sv.cancel(r2)
    if queued:
        info2 = _wait_state(sv, r2, (api.REQ_CANCELLED,), limit_s=5.0)
        assert info2["error"] == api.GRINS_E_CANCELLED
        with pytest.raises(api.GrinsError):
            sv.results(r2)                   # never ran: no results
    else:                                    # r1 finished first: r2 ran (or runs); let it end
        _wait_state(sv, r2, (api.REQ_CANCELLED, api.REQ_DONE), limit_s=60.0)
    sv.cancel(r1)
    t0 = time.time()
    info1 = _wait_state(sv, r1, (api.REQ_CANCELLED, api.REQ_DONE), limit_s=60.0)
    print("running request ended %.3f s after the cancel, state %d" % (time.time() - t0, info1["state"]))
    if info1["state"] == api.REQ_CANCELLED:
        assert info1["error"] == api.GRINS_E_CANCELLED
        res = sv.results(r1, keys=("status", "n_unique"))
        torch.cuda.synchronize()
        st = res["status"].cpu().numpy()
        assert np.any(st == api.CANCELLED)
        assert set(np.unique(st).tolist()) <= {api.CONVERGED, api.TEND, api.MAXSTEPS, api.NONFINITE,
                                              api.POLISH_FAIL, api.CANCELLED}
    sv.release(r1)
    sv.release(r2)
    # the slot is reusable: a new request on it runs to completion
    r3 = sv.submit(nets[0], w["param_seed"], 500, 10)
    info3 = _wait_state(sv, r3, (api.REQ_DONE,), limit_s=60.0)
    st3 = sv.results(r3, keys=("status",))["status"].cpu().numpy()
    assert not np.any(st3 == api.CANCELLED)
    sv.release(r3)
    sv.close()
    for h in nets:
        h.close()
