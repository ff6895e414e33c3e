"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare them."""
from __future__ import annotations

import os

import numpy as np

import oracle as O

THREADS = max(1, min(16, os.cpu_count() or 1))


def gpu_handle(topo):
    from paper_2503_18356_gb300 import api
    return api.Racipe.from_topology(topo)


def gpu_sample(h, seed, n_sets, n_ics, set0=0, ranges=None):
    params, ic = h.sample_params(seed, n_sets, n_ics, set0=set0, ranges=ranges)
    G, k, T, lam, n = (x.cpu().numpy() for x in h.unpack_params(params))
    return params, ic, O.ParamSet(G, k, T, lam, n.astype(np.int32)), ic.cpu().numpy()


def rel_err(x, ref, G, k, floor=1e-6):
    """|x - x*| / max(|x*|, floor * G/k), elementwise (floor for states near 0)."""
    scale = np.maximum(np.abs(ref), floor * (G / k))
    return np.abs(x - ref) / scale


def compare_states(gpu, orc, p: O.ParamSet, tol, net: O.Network, basin_tol=None, normalised=False):
    """Compares converged states set by set.  Returns a dict with the max
    error over solves converged on both sides and at the same fixed point,
    the number of such solves, the count of solves that reached different
    fixed points, how many of those are not certified equilibria, and the
    status agreement rate.

    `max_rel` is always the relative error with a floor for states near
    zero, |x - x*| / max(|x*|, 1e-6 G/k), and `max_gk` the error on the G/k scale,
    |x - x*| k / G.  `max_err` is the one the caller's bar is stated in:
    relative for polished states; with `normalised` the G/k scale, which is
    how unpolished states are judged -- they stop at max_i |f_i| k_i / G_i <
    ss_tol, which bounds their distance to the fixed point in units of G/k,
    not relative to a small steady level (a node near zero can be 1e-4 G/k
    from its fixed point and many times its own level off; the oracle's own
    unpolished states show the same, see test_oracle_pins).

    Same fixed point: G/k-normalised distance <= basin_tol, by default 1e-2
    for unpolished states and 1e-5 for polished ones (fixed points to ~1e-12;
    near a saddle-node bifurcation a stable node and its saddle can lie
    1e-4 .. 1e-2 apart, and a solve that the two sides send to different
    ones is a basin mismatch, not an accuracy error -- but only if both
    states are equilibria: each side's state must pass the oracle's residual
    certificate, max_i |f_i| k_i / G_i in FP64 below 1e-10 for polished
    states and below 10 ss_tol = 1e-5 for unpolished ones, else it counts in
    `n_uncertified`)."""
    if basin_tol is None:
        basin_tol = 1e-2 if normalised else 1e-5
    G = p.G[:, None, :]
    k = p.k[:, None, :]
    both = (gpu["status"] == O.CONVERGED) & (orc["status"] == O.CONVERGED)
    vg = gpu["states"] * k / G
    vo = orc["states"] * k / G
    dist = np.max(np.abs(vg - vo), axis=2)
    same = both & (dist <= basin_tol)
    rel = rel_err(gpu["states"], orc["states"], G, k)
    gk = np.abs(vg - vo)
    err = gk if normalised else rel
    cert = 1e-5 if normalised else 1e-10
    n_unc = 0
    for s_, c_ in zip(*np.nonzero(both & ~same)):
        for x in (gpu["states"][s_, c_], orc["states"][s_, c_]):
            if not (O.rho(net, p, x, s_) < cert):
                n_unc += 1
                break

    def mx(e):
        return float(np.max(e[same])) if same.any() else 0.0

    return dict(max_err=mx(err), max_rel=mx(rel), max_gk=mx(gk), n_compared=int(same.sum()),
                n_basin=int((both & ~same).sum()), n_uncertified=n_unc,
                status_agree=float(np.mean(gpu["status"] == orc["status"])),
                share_rel_above_1e3=float(np.mean(rel.max(axis=-1)[same] > 1e-3)) if same.any() else 0.0,
                p999=float(np.quantile(err[same].max(axis=-1), 0.999)) if same.any() else 0.0)


def to_numpy(out):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items() if v is not None}
