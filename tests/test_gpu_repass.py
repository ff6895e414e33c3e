"""The borderline re-pass of grins_racipe_integrate (grins_solver_opts.tail_*):
the FP32 pass keeps a checkpoint per solve and lists the solves whose
steady-state decision falls near t_end; an FP64 pass re-integrates only
those from their checkpoints.  These tests check that it touches only the
listed solves, reports what it did, and validates its options; its effect
on parity is held by test_n_unique_bar_net22_10k_sets and the parity tests,
which run with it (the default)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_18356_gb300 import workloads as W
from tests import parity as PT

pytestmark = pytest.mark.gpu


def _run(h, params, ic, **opt):
    out = h.integrate(params, ic, polish=0, **opt)
    torch.cuda.synchronize()
    return PT.to_numpy(out)


def test_repass_changes_only_listed_solves():
    """Solves the FP32 pass does not list come out bit-identical with and
    without the re-pass; listed ones carry the FP64 pass's attempts on top of
    the FP32 pass's (d_n_steps counts both) and end converged or at t_end."""
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 300, 10)
    off = _run(h, params, ic, tail_rtol=0.0)
    assert h.tail_stats() == (0, 0)
    assert "borderline re-pass: off" in h.integrator()
    on = _run(h, params, ic)
    n_tail, a_tail = h.tail_stats()
    print(h.integrator(), n_tail, a_tail)
    assert "borderline re-pass: FP64" in h.integrator()
    assert n_tail > 0 and a_tail > 0
    extra = on["n_steps"].astype(np.int64) - off["n_steps"]
    assert np.all(extra >= 0)
    assert extra.sum() == a_tail
    listed = extra > 0
    assert 0 < listed.sum() <= n_tail
    # a listed solve the FP64 pass decides without a step (its checkpoint at
    # t_end, or already below ss_tol in FP64) has no extra attempts: at most
    # n_tail - listed.sum() of the others may differ
    same = ~listed
    differ = (~np.all(on["states"] == off["states"], axis=2) | (on["status"] != off["status"])
              | (on["t_final"] != off["t_final"]))
    assert differ[same].sum() <= n_tail - listed.sum()
    assert np.all(np.isin(on["status"][listed], [O.CONVERGED, O.TEND]))
    assert np.all(on["t_final"][listed] <= 200.0)
    # the FP32 pass's decision was borderline: t_end reached, or converged late
    assert np.all((off["status"][listed] == O.TEND) | (off["t_final"][listed] > 100.0))
    h.close()


def test_repass_skipped_with_time_series_and_for_fp64():
    w = W.net5_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, _, _ = PT.gpu_sample(h, w["param_seed"], 20, 4)
    g = _run(h, params, ic, t_grid=np.linspace(0.0, 50.0, 6))
    assert h.tail_stats() == (0, 0)
    assert "not run (time series requested)" in h.integrator()
    _run(h, params, ic, precision=0)            # FP64 integrations take no re-pass
    assert h.tail_stats() == (0, 0)
    assert g["series"].shape == (20, 4, 6, w["topology"].n_nodes)
    h.close()


@pytest.mark.parametrize("bad", [dict(tail_rtol=-1e-9), dict(tail_start=0.5), dict(tail_rho=-1.0),
                                 dict(tail_late=-0.1), dict(tail_work=-1), dict(tail_rtol=float("nan"))])
def test_repass_rejects_bad_options(bad):
    from paper_2503_18356_gb300 import api
    h = PT.gpu_handle(W.toggle_switch())
    params, ic = h.sample_params(1, 4, 3)
    with pytest.raises(api.GrinsError) as e:
        h.integrate(params, ic, **bad)
    assert e.value.status == api.GRINS_E_INVALID_ARG
    assert "re-pass" in str(e.value)
    h.close()
