"""RACIPE oracle: plain FP64 CPU implementation of the ensemble path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library (``paper_2503_18356_gb300``) and never imports
it.  The arithmetic lives in ``racipe_oracle.c`` (compiled with gcc,
``-ffp-contract=off``); this module only marshals numpy arrays.

Functions mirror the paper (GRiNS, arXiv 2503.18356):
  * ``shifted_hill`` / ``rhs``         -- Eq. 2 / Eq. 1 (Sec. 2.1.1)
  * ``median`` / ``sample_params`` / ``sample_ics`` -- Sec. 2.1.2, Table 1
  * ``solve``                           -- Dormand-Prince 5(4) to steady state
                                           and time series (Sec. 2.1.3)
  * ``polish``                          -- Newton on Eq. 1 = 0
  * ``dedupe``                          -- unique steady states (Sec. 3.1)
  * ``ising_run``                       -- Boolean Ising formalism (Sec. 2.2, Eq. 3)
  * ``gk_histogram`` / ``level_boundaries`` / ``level_states``
                                        -- levels of G/k-normalised expression,
                                           state labels and multistability
                                           (Sec. 2.1.3 analysis, Sec. 3.1)
  * ``run_sets`` / ``run_sets_parallel``-- the whole path over sets
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "racipe_oracle.c")
_LIB = os.path.join(_HERE, "libracipe_oracle.so")

CONVERGED, TEND, MAXSTEPS, NONFINITE, POLISH_FAIL = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into this folder."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_lock = threading.Lock()


class Ranges(C.Structure):
    _fields_ = [("G_min", C.c_double), ("G_max", C.c_double),
                ("k_min", C.c_double), ("k_max", C.c_double),
                ("lam_act_min", C.c_double), ("lam_act_max", C.c_double),
                ("lam_inh_min", C.c_double), ("lam_inh_max", C.c_double),
                ("n_min", C.c_int32), ("n_max", C.c_int32),
                ("thr_lo", C.c_double), ("thr_hi", C.c_double),
                ("median_samples", C.c_int32), ("median_mode", C.c_int32),
                ("dist_G", C.c_int32), ("dist_k", C.c_int32),
                ("dist_lam_act", C.c_int32), ("dist_lam_inh", C.c_int32),
                ("lhs_sets", C.c_int64),
                ("sobol", C.c_int32), ("sobol_dims", C.c_int32),
                ("sobol_poly", C.POINTER(C.c_int64)), ("sobol_m", C.POINTER(C.c_int64)),
                ("sobol_m_cols", C.c_int32),
                ("param_ranges", C.c_void_p)]


# one row of a per-parameter range table (dist, reserved, lo, hi)
PARAM_ROW = np.dtype([("dist", np.int32), ("reserved", np.int32), ("lo", np.float64), ("hi", np.float64)])


class Net(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_edges", C.c_int32),
                ("src", C.POINTER(C.c_int32)), ("dst", C.POINTER(C.c_int32)),
                ("sign", C.POINTER(C.c_int8))]


class Params(C.Structure):
    _fields_ = [("G", C.POINTER(C.c_double)), ("k", C.POINTER(C.c_double)),
                ("T", C.POINTER(C.c_double)), ("lam", C.POINTER(C.c_double)),
                ("n", C.POINTER(C.c_int32))]


class Opts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("t0", C.c_double),
                ("t_end", C.c_double), ("ss_tol", C.c_double), ("max_steps", C.c_int64),
                ("t_grid", C.POINTER(C.c_double)), ("n_t", C.c_int32),
                ("h_fixed", C.c_double), ("method", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("t_final", C.c_double),
                ("n_attempts", C.c_int64), ("n_accepted", C.c_int64)]


class PathOpts(C.Structure):
    _fields_ = [("polish", C.c_int32), ("polish_tol", C.c_double),
                ("polish_iters", C.c_int32), ("dedupe_tol", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            l = C.CDLL(build())
            P = C.POINTER
            l.orc_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
            l.orc_u01.argtypes = [C.c_uint64]; l.orc_u01.restype = C.c_double
            l.orc_uint_range.argtypes = [C.c_uint64, C.c_int32, C.c_int32]
            l.orc_uint_range.restype = C.c_int32
            l.orc_default_ranges.argtypes = [P(Ranges)]
            l.orc_shifted_hill.argtypes = [C.c_double] * 4; l.orc_shifted_hill.restype = C.c_double
            l.orc_rhs.argtypes = [P(Net), P(Params), P(C.c_double), P(C.c_double)]
            l.orc_rho.argtypes = [P(Net), P(Params), P(C.c_double)]; l.orc_rho.restype = C.c_double
            l.orc_median_samples.argtypes = [C.c_int32, C.c_int32, P(Ranges), C.c_double, P(C.c_double)]
            l.orc_median.argtypes = [C.c_int32, C.c_int32, P(Ranges)]; l.orc_median.restype = C.c_double
            l.orc_sample_params.argtypes = [P(Net), P(Ranges), C.c_uint64, C.c_int64, C.c_int64,
                                            P(C.c_double), P(C.c_double), P(C.c_double),
                                            P(C.c_double), P(C.c_int32)]
            l.orc_lhs_stratum.argtypes = [C.c_uint64] * 4; l.orc_lhs_stratum.restype = C.c_uint64
            l.orc_sobol_x.argtypes = [P(Ranges), C.c_uint64, C.c_uint64, C.c_uint64]
            l.orc_sobol_x.restype = C.c_uint32
            l.orc_node_medians.argtypes = [P(Net), P(Ranges), P(C.c_double)]
            l.orc_sample_ics.argtypes = [C.c_int32, C.c_uint64, C.c_int32, P(C.c_double)]
            l.orc_sample_ics_ranges.argtypes = [C.c_int32, C.c_uint64, C.c_int32, C.c_void_p, P(C.c_double)]
            l.orc_solve.argtypes = [P(Net), P(Params), P(C.c_double), P(Opts), P(C.c_double),
                                    P(C.c_double)]
            l.orc_solve.restype = Result
            l.orc_polish.argtypes = [P(Net), P(Params), P(C.c_double), C.c_double, C.c_int32,
                                     P(C.c_double), P(C.c_double)]
            l.orc_polish.restype = C.c_int32
            l.orc_dedupe.argtypes = [C.c_int32, C.c_int32, P(C.c_double), P(C.c_uint8),
                                     P(C.c_double), P(C.c_double), C.c_double, P(C.c_int32)]
            l.orc_dedupe.restype = C.c_int32
            l.orc_ising_run.argtypes = [P(Net), C.c_int32, C.c_int32, C.c_uint64, C.c_int64, P(C.c_uint64),
                                        C.c_int32, P(C.c_uint64), P(C.c_int32), P(C.c_uint8)]
            l.orc_ising_run.restype = C.c_int32
            l.orc_tableau.argtypes = [C.c_int32, P(C.c_double), P(C.c_double), P(C.c_double), P(C.c_double)]
            l.orc_gk_bin.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int32]
            l.orc_gk_bin.restype = C.c_int32
            l.orc_gk_histogram.argtypes = [C.c_int32, C.c_int32, C.c_int64, P(C.c_double), P(C.c_uint8),
                                           P(C.c_double), P(C.c_double), C.c_int32, P(C.c_uint64)]
            l.orc_level_boundaries.argtypes = [P(C.c_uint64), C.c_int32, C.c_int32, C.c_int32, P(C.c_int32)]
            l.orc_level_boundaries.restype = C.c_int32
            l.orc_level_states.argtypes = [C.c_int32, C.c_int32, C.c_int64, P(C.c_double), P(C.c_uint8),
                                           P(C.c_double), P(C.c_double), C.c_int32, P(C.c_int32), C.c_int32,
                                           P(C.c_uint64), P(C.c_int32), P(C.c_uint64)]
            l.orc_level_states.restype = C.c_int32
            l.orc_run_sets.argtypes = [P(Net), P(C.c_double), P(C.c_double), P(C.c_double),
                                       P(C.c_double), P(C.c_int32), C.c_int64, P(C.c_double),
                                       C.c_int32, P(Opts), P(PathOpts), P(C.c_double),
                                       P(C.c_uint8), P(C.c_double), P(C.c_int64), P(C.c_double),
                                       P(C.c_int32), P(C.c_int32)]
            _lib = l
    return _lib


def _p(a, ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- helpers
def default_ranges(sobol_table=None, param_ranges=None, **over) -> Ranges:
    """Table 1's ranges with fields overridden; `sobol_table` = (poly, m)
    int64 arrays for the Sobol modes; `param_ranges` = a PARAM_ROW array of
    2N + 3E rows (kept alive with the struct)."""
    r = Ranges()
    lib().orc_default_ranges(C.byref(r))
    for k, v in over.items():
        setattr(r, k, v)
    r._rows = None
    if param_ranges is not None:
        r._rows = np.ascontiguousarray(param_ranges, dtype=PARAM_ROW)
        r.param_ranges = r._rows.ctypes.data
    if sobol_table is not None:
        poly = np.ascontiguousarray(sobol_table[0], dtype=np.int64)
        m = np.ascontiguousarray(sobol_table[1], dtype=np.int64)
        r._keep = (poly, m)
        r.sobol_dims, r.sobol_m_cols = int(poly.shape[0]), int(m.shape[1])
        r.sobol_poly = _p(poly, C.c_int64)
        r.sobol_m = _p(m, C.c_int64)
    return r


class Network:
    """Signed directed edge list (Sec. 2.1.1) held for the oracle."""

    def __init__(self, n_nodes, src, dst, sign):
        self.n_nodes = int(n_nodes)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.sign = np.ascontiguousarray(sign, dtype=np.int8)
        self.n_edges = int(self.src.size)
        self.c = Net(self.n_nodes, self.n_edges, _p(self.src, C.c_int32),
                     _p(self.dst, C.c_int32), _p(self.sign, C.c_int8))


class ParamSet:
    """Parameters of sets: G, k [S, N]; T, lam [S, E] (float64); n [S, E] (int32)."""

    def __init__(self, G, k, T, lam, n):
        self.G = _f64(G); self.k = _f64(k); self.T = _f64(T); self.lam = _f64(lam)
        self.n = np.ascontiguousarray(n, dtype=np.int32)

    @property
    def n_sets(self):
        return self.G.shape[0]

    def one(self, s):
        return ParamSet(self.G[s:s + 1], self.k[s:s + 1], self.T[s:s + 1],
                        self.lam[s:s + 1], self.n[s:s + 1])

    def c_one(self, s=0):
        G, k, T, lam, n = self.G[s], self.k[s], self.T[s], self.lam[s], self.n[s]
        keep = (G, k, T, lam, n)
        return Params(_p(G, C.c_double), _p(k, C.c_double), _p(T, C.c_double),
                      _p(lam, C.c_double), _p(n, C.c_int32)), keep


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c, C.c_uint64), _p(k, C.c_uint64), _p(out, C.c_uint64))
    return out


def u01(r):
    return lib().orc_u01(C.c_uint64(int(r)))


def uint_range(r, lo, hi):
    return lib().orc_uint_range(C.c_uint64(int(r)), lo, hi)


def shifted_hill(B, B0, n, lam):
    return lib().orc_shifted_hill(float(B), float(B0), float(n), float(lam))


def rhs(net: Network, p: ParamSet, x, s=0):
    x = _f64(x)
    f = np.zeros(net.n_nodes)
    cp, keep = p.c_one(s)
    lib().orc_rhs(C.byref(net.c), C.byref(cp), _p(x, C.c_double), _p(f, C.c_double))
    return f


def rho(net: Network, p: ParamSet, x, s=0):
    x = _f64(x)
    cp, keep = p.c_one(s)
    return lib().orc_rho(C.byref(net.c), C.byref(cp), _p(x, C.c_double))


def median_samples(a, b, ranges=None, M0=0.0):
    r = ranges or default_ranges()
    out = np.zeros(r.median_samples)
    lib().orc_median_samples(a, b, C.byref(r), float(M0), _p(out, C.c_double))
    return out


def median(a, b, ranges=None):
    r = ranges or default_ranges()
    return lib().orc_median(a, b, C.byref(r))


def sample_params(net: Network, seed, n_sets, set0=0, ranges=None) -> ParamSet:
    r = ranges or default_ranges()
    N, E = net.n_nodes, net.n_edges
    G = np.zeros((n_sets, N)); k = np.zeros((n_sets, N))
    T = np.zeros((n_sets, E)); lam = np.zeros((n_sets, E))
    n = np.zeros((n_sets, E), dtype=np.int32)
    lib().orc_sample_params(C.byref(net.c), C.byref(r), C.c_uint64(seed), set0, n_sets,
                            _p(G, C.c_double), _p(k, C.c_double), _p(T, C.c_double),
                            _p(lam, C.c_double), _p(n, C.c_int32))
    return ParamSet(G, k, T, lam, n)


def lhs_stratum(seed, d, s, S):
    """The Latin-hypercube stratum of draw d of set s among S sets: a keyed
    permutation of [0, S) in s (Feistel network with cycle walking)."""
    return int(lib().orc_lhs_stratum(C.c_uint64(seed), C.c_uint64(d), C.c_uint64(s), C.c_uint64(S)))


def node_medians(net: Network, ranges=None):
    """The half-functional median M_j of every node."""
    r = ranges or default_ranges()
    M = np.zeros(net.n_nodes)
    lib().orc_node_medians(C.byref(net.c), C.byref(r), _p(M, C.c_double))
    return M


def sobol_x(ranges, seed, d, s):
    """Coordinate d of Sobol point s (32-bit), plain or scrambled per
    `ranges.sobol`."""
    return int(lib().orc_sobol_x(C.byref(ranges), C.c_uint64(seed), C.c_uint64(d), C.c_uint64(s)))


def sample_ics(n_nodes, seed, n_ics, ic_ranges=None):
    """Unit initial conditions [n_ics, N] (fractions of G/k), uniform on
    [0, 1) or from per-node PARAM_ROW rows."""
    u = np.zeros((n_ics, n_nodes))
    if ic_ranges is None:
        lib().orc_sample_ics(n_nodes, C.c_uint64(seed), n_ics, _p(u, C.c_double))
    else:
        rows = np.ascontiguousarray(ic_ranges, dtype=PARAM_ROW)
        lib().orc_sample_ics_ranges(n_nodes, C.c_uint64(seed), n_ics, rows.ctypes.data, _p(u, C.c_double))
    return u


def make_opts(rtol=1e-10, atol=1e-13, t0=0.0, t_end=200.0, ss_tol=1e-6, max_steps=10_000_000,
              t_grid=None, h_fixed=0.0, method=0):
    """method: 0 Dormand-Prince 5(4), 1 Tsitouras 5(4) (the paper's Tsit5)."""
    g = None if t_grid is None else _f64(t_grid)
    o = Opts(rtol, atol, t0, t_end, ss_tol, max_steps, _p(g, C.c_double),
             0 if g is None else g.size, h_fixed, method)
    return o, g


def tableau(method=0):
    """(c [7], a [7, 7], b5 [7], b4 [7]) of a 5(4) pair (0 Dormand-Prince,
    1 Tsitouras)."""
    c, b5, b4 = np.zeros(7), np.zeros(7), np.zeros(7)
    a = np.zeros((7, 7))
    lib().orc_tableau(method, _p(c, C.c_double), _p(a, C.c_double), _p(b5, C.c_double), _p(b4, C.c_double))
    return c, a, b5, b4


def solve(net: Network, p: ParamSet, x0, s=0, **opt):
    """One trajectory; returns dict(x, status, t_final, n_attempts, n_accepted, series)."""
    o, g = make_opts(**opt)
    x0 = _f64(x0)
    x = np.zeros(net.n_nodes)
    series = None if g is None else np.zeros((g.size, net.n_nodes))
    cp, keep = p.c_one(s)
    r = lib().orc_solve(C.byref(net.c), C.byref(cp), _p(x0, C.c_double), C.byref(o),
                        _p(x, C.c_double), _p(series, C.c_double))
    return dict(x=x, status=r.status, t_final=r.t_final, n_attempts=r.n_attempts,
                n_accepted=r.n_accepted, series=series)


def polish(net: Network, p: ParamSet, x, s=0, tol=1e-13, max_iter=8):
    x = _f64(x).copy()
    rho_ = C.c_double(0.0); step = C.c_double(0.0)
    cp, keep = p.c_one(s)
    rc = lib().orc_polish(C.byref(net.c), C.byref(cp), _p(x, C.c_double), tol, max_iter,
                          C.byref(rho_), C.byref(step))
    return dict(x=x, rc=rc, rho=rho_.value, step=step.value)


def dedupe(states, status, G, k, tol=1e-2):
    """states [I, N], status [I], G, k [N] of one set -> (state_id [I], n_unique)."""
    st = _f64(states)
    I, N = st.shape
    stat = np.ascontiguousarray(status, dtype=np.uint8)
    G = _f64(G); k = _f64(k)
    sid = np.zeros(I, dtype=np.int32)
    nu = lib().orc_dedupe(N, I, _p(st, C.c_double), _p(stat, C.c_uint8), _p(G, C.c_double),
                          _p(k, C.c_double), tol, _p(sid, C.c_int32))
    return sid, nu


def gk_bin(x, k, G, n_bins):
    """Bin of one normalised value (x k) / G among n_bins equal bins on [0, 1]."""
    return lib().orc_gk_bin(float(x), float(k), float(G), int(n_bins))


def gk_histogram(states, status, G, k, n_bins=100, counts=None):
    """states [S, I, N], status [S, I], per-set G, k [S, N] -> counts [n_bins]
    (added to ``counts`` when given)."""
    st = _f64(states)
    S, I, N = st.shape
    stat = np.ascontiguousarray(status, dtype=np.uint8)
    G = _f64(G); k = _f64(k)
    out = np.zeros(n_bins, dtype=np.uint64) if counts is None else counts
    lib().orc_gk_histogram(N, I, S, _p(st, C.c_double), _p(stat, C.c_uint8), _p(G, C.c_double),
                           _p(k, C.c_double), n_bins, _p(out, C.c_uint64))
    return out


def level_boundaries(counts, m=4, max_b=3):
    """Boundary bins of a histogram of normalised values (binomial smoothing
    of half-width m, at most max_b valleys)."""
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    out = np.zeros(max(1, max_b), dtype=np.int32)
    n = lib().orc_level_boundaries(_p(c, C.c_uint64), c.size, m, max_b, _p(out, C.c_int32))
    return out[:n].copy()


def level_states(states, status, G, k, bounds, n_bins=100):
    """-> (labels [S, I] uint64, n_states [S], multi_hist [I + 1]); None when
    the levels of N nodes do not fit in 64 bits."""
    st = _f64(states)
    S, I, N = st.shape
    stat = np.ascontiguousarray(status, dtype=np.uint8)
    G = _f64(G); k = _f64(k)
    b = np.ascontiguousarray(bounds, dtype=np.int32)
    labels = np.zeros((S, I), dtype=np.uint64)
    ns = np.zeros(S, dtype=np.int32)
    mh = np.zeros(I + 1, dtype=np.uint64)
    rc = lib().orc_level_states(N, I, S, _p(st, C.c_double), _p(stat, C.c_uint8), _p(G, C.c_double),
                                _p(k, C.c_double), n_bins, _p(b, C.c_int32) if b.size else None, b.size,
                                _p(labels, C.c_uint64), _p(ns, C.c_int32), _p(mh, C.c_uint64))
    return None if rc != 0 else (labels, ns, mh)


def ising_run(net: Network, mode=0, seed=0, n_traj=1, init=None, max_steps=1000, enc01=False):
    """Boolean Ising trajectories (Eq. 3) -> (final uint64 [n_traj], steps
    int32, status uint8); mode 0 synchronous, 1 asynchronous; init: uint64
    states (bit i = node i active) or None for random ones from seed."""
    fin = np.zeros(n_traj, dtype=np.uint64)
    stp = np.zeros(n_traj, dtype=np.int32)
    st = np.zeros(n_traj, dtype=np.uint8)
    ini = None if init is None else np.ascontiguousarray(init, dtype=np.uint64)
    rc = lib().orc_ising_run(C.byref(net.c), mode, int(bool(enc01)), seed, n_traj,
                             _p(ini, C.c_uint64), max_steps, _p(fin, C.c_uint64), _p(stp, C.c_int32),
                             _p(st, C.c_uint8))
    assert rc == 0
    return fin, stp, st


def run_sets(net: Network, p: ParamSet, ic_unit, polish=True, polish_tol=1e-13,
             polish_iters=8, dedupe_tol=1e-2, series=False, **opt):
    """Whole path over every set of ``p``; returns a dict of arrays."""
    o, g = make_opts(**opt)
    S, N, I = p.n_sets, net.n_nodes, ic_unit.shape[0]
    ic = _f64(ic_unit)
    out = dict(states=np.zeros((S, I, N)), status=np.zeros((S, I), dtype=np.uint8),
               t_final=np.zeros((S, I)), n_attempts=np.zeros((S, I), dtype=np.int64),
               state_id=np.zeros((S, I), dtype=np.int32), n_unique=np.zeros(S, dtype=np.int32))
    out["series"] = np.zeros((S, I, g.size, N)) if (series and g is not None) else None
    po = PathOpts(1 if polish else 0, polish_tol, polish_iters, dedupe_tol)
    lib().orc_run_sets(C.byref(net.c), _p(p.G, C.c_double), _p(p.k, C.c_double),
                       _p(p.T, C.c_double), _p(p.lam, C.c_double), _p(p.n, C.c_int32), S,
                       _p(ic, C.c_double), I, C.byref(o), C.byref(po),
                       _p(out["states"], C.c_double), _p(out["status"], C.c_uint8),
                       _p(out["t_final"], C.c_double), _p(out["n_attempts"], C.c_int64),
                       _p(out["series"], C.c_double), _p(out["state_id"], C.c_int32),
                       _p(out["n_unique"], C.c_int32))
    return out


def run_sets_parallel(net: Network, p: ParamSet, ic_unit, threads=None, **kw):
    """``run_sets`` with the sets split over host threads (ctypes drops the GIL)."""
    S = p.n_sets
    threads = max(1, min(threads or os.cpu_count() or 1, S))
    bounds = np.linspace(0, S, threads + 1).astype(int)

    def part(i):
        a, b = bounds[i], bounds[i + 1]
        sub = ParamSet(p.G[a:b], p.k[a:b], p.T[a:b], p.lam[a:b], p.n[a:b])
        return run_sets(net, sub, ic_unit, **kw)

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(part, range(threads)))
    out = {}
    for key in parts[0]:
        if parts[0][key] is None:
            out[key] = None
        else:
            out[key] = np.concatenate([q[key] for q in parts], axis=0)
    return out
