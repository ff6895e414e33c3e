"""The borderline re-pass of grins_racipe_integrate (grins_solver_opts.tail_*):
the FP32 pass keeps a checkpoint per solve and lists the solves whose
steady-state decision falls near t_end; a wide pass (double-float by default, or FP64) re-integrates only
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
    without the re-pass; listed ones carry the re-pass's attempts on top of
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
    assert "borderline re-pass: double-float" in h.integrator()
    assert n_tail > 0 and a_tail > 0
    extra = on["n_steps"].astype(np.int64) - off["n_steps"]
    assert np.all(extra >= 0)
    assert extra.sum() == a_tail
    listed = extra > 0
    assert 0 < listed.sum() <= n_tail
    # a listed solve the re-pass decides without a step (its checkpoint at
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


def test_double_float_repass_matches_fp64_repass():
    """The double-float re-pass (default) and the FP64 one take the same list
    (the FP32 pass is the same) and integrate it at the same tolerances: their
    statuses agree and their states agree to far below the parity floor
    (1e-6 of G/k), the difference being rounding of the right-hand side
    (about 2^-44 against 2^-53 relative) and the double-float kernel's clamp
    of saturated edge powers at 2^40."""
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, p, icn = PT.gpu_sample(h, w["param_seed"], 2000, 10)
    dd_ = _run(h, params, ic)
    n_dd = h.tail_stats()
    assert "double-float" in h.integrator()
    f64 = _run(h, params, ic, tail_precision=api.GRINS_TAIL_FP64)
    n_64 = h.tail_stats()
    assert "FP64" in h.integrator().split("borderline re-pass:")[1]
    print("dd", n_dd, "fp64", n_64)
    assert n_dd[0] == n_64[0] > 0                     # the same list
    listed = (dd_["n_steps"] != f64["n_steps"]) | (dd_["status"] != f64["status"])
    same_status = dd_["status"] == f64["status"]
    assert same_status.mean() >= 0.999, (~same_status).sum()
    G = p.G[:, None, :]
    k = p.k[:, None, :]
    both = same_status & np.isin(dd_["status"], [O.CONVERGED, O.TEND])
    diff = np.abs(dd_["states"] - f64["states"]) * k / G
    print("listed or differing solves", listed.sum(), "max normalised state difference", diff[both].max())
    assert diff[both].max() <= 1e-6
    # attempts of the two re-passes agree to within a few percent overall
    assert abs(n_dd[1] - n_64[1]) <= 0.05 * n_64[1]
    h.close()


def test_polish_beside_repass_equals_polish_after():
    """integrate with the polish runs it beside the re-pass (the solves the
    FP32 pass did not list) and on the listed solves after it; the results
    are bit-identical to integrate without the polish followed by the polish
    call, and no status carries the internal mark of a listed solve."""
    from paper_2503_18356_gb300 import api
    w = W.net22_workload()
    h = PT.gpu_handle(w["topology"])
    params, ic, _, _ = PT.gpu_sample(h, w["param_seed"], 3000, 10)
    a = h.integrate(params, ic, polish=1)
    torch.cuda.synchronize()
    a = PT.to_numpy(a)
    n_a = h.tail_stats()
    b = h.integrate(params, ic, polish=0)
    h.polish(params, b["states"], b["status"], b["err_est"], opts=api.default_opts())
    torch.cuda.synchronize()
    b = PT.to_numpy(b)
    assert n_a == h.tail_stats() and n_a[0] > 0
    for k in ("states", "status", "err_est", "n_steps", "t_final"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    assert a["status"].max() <= api.CANCELLED
    assert np.any(a["status"] == O.CONVERGED)
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
                                 dict(tail_late=-0.1), dict(tail_work=-1), dict(tail_rtol=float("nan")),
                                 dict(tail_precision=2)])
def test_repass_rejects_bad_options(bad):
    from paper_2503_18356_gb300 import api
    h = PT.gpu_handle(W.toggle_switch())
    params, ic = h.sample_params(1, 4, 3)
    with pytest.raises(api.GrinsError) as e:
        h.integrate(params, ic, **bad)
    assert e.value.status == api.GRINS_E_INVALID_ARG
    assert "re-pass" in str(e.value)
    h.close()
