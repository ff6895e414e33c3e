"""Thin Python binding of libgrins_racipe.so (the C ABI in include/grins_racipe.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors allocated here; the CUDA
stream is torch's current stream unless one is given.  The library must be
built (``paper_2503_18356_gb300.build.build()``); importing this module
raises if it is missing -- there is no fallback.

Low-level functions carry the C names (``grins_racipe_create``, ...); the
``Racipe`` class wraps a handle for everyday use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# GRINS_RACIPE_LIB selects another build of the same library (the tests use it
# to load the index-checked variant); the default is the in-tree release build.
LIB_PATH = os.environ.get("GRINS_RACIPE_LIB") or os.path.join(_HERE, "libgrins_racipe.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libgrins_racipe.so is not built; run paper_2503_18356_gb300.build.build()")

_lib = C.CDLL(LIB_PATH)

GRINS_OK, GRINS_E_INVALID_ARG, GRINS_E_TOPOLOGY, GRINS_E_NOMEM, GRINS_E_CUDA, GRINS_E_BUDGET, \
    GRINS_E_CANCELLED = range(7)
CONVERGED, TEND, MAXSTEPS, NONFINITE, POLISH_FAIL, CANCELLED = range(6)
GRINS_FP64, GRINS_FP32 = 0, 1
GRINS_TAIL_DD, GRINS_TAIL_FP64 = 0, 1
GRINS_METHOD_DOPRI5, GRINS_METHOD_TSIT5 = 0, 1
GRINS_ISING_SYNC, GRINS_ISING_ASYNC = 0, 1
GRINS_DIST_TABLE1, GRINS_DIST_LOGUNIFORM, GRINS_DIST_NORMAL, GRINS_DIST_LOGNORMAL = 0, 1, 2, 3
GRINS_SOBOL_OFF, GRINS_SOBOL_PLAIN, GRINS_SOBOL_SCRAMBLED = 0, 1, 2
MEDIAN_PER_INDEGREE, MEDIAN_UNREGULATED = 0, 1
GRINS_STATIC_MAX_GRID = 4096        # largest time grid of grins_racipe_integrate_static


class grins_param_range(C.Structure):
    _fields_ = [("dist", C.c_int32), ("reserved", C.c_int32), ("lo", C.c_double), ("hi", C.c_double)]


# numpy mirror of grins_param_range (one row per parameter, layout order)
PARAM_RANGE_DTYPE = np.dtype([("dist", np.int32), ("reserved", np.int32), ("lo", np.float64), ("hi", np.float64)])


class grins_racipe_ranges(C.Structure):
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
                ("sobol_m_cols", C.c_int32), ("reserved", C.c_int32),
                ("param_ranges", C.POINTER(grins_param_range)),
                ("ic_ranges", C.POINTER(grins_param_range))]


class grins_solver_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("polish", C.c_int32),
                ("rtol", C.c_double), ("atol", C.c_double),
                ("t0", C.c_double), ("t_end", C.c_double), ("ss_tol", C.c_double),
                ("max_steps", C.c_int64),
                ("t_grid", C.POINTER(C.c_double)), ("n_t", C.c_int32),
                ("polish_tol", C.c_double), ("polish_iters", C.c_int32),
                ("polish_max_move", C.c_double), ("ss_tighten", C.c_double), ("method", C.c_int32),
                ("tail_rtol", C.c_double), ("tail_start", C.c_double), ("tail_rho", C.c_double),
                ("tail_late", C.c_double), ("tail_work", C.c_int32), ("tail_precision", C.c_int32),
                ("pass_event", C.c_void_p),
                ("cancel", C.c_void_p)]


class grins_racipe_job(C.Structure):
    _fields_ = [("net", C.c_void_p), ("d_params", C.c_void_p), ("n_sets", C.c_int64),
                ("d_ic_unit", C.c_void_p), ("n_ics", C.c_int32),
                ("d_states", C.c_void_p), ("d_status", C.c_void_p), ("d_t_final", C.c_void_p),
                ("d_n_steps", C.c_void_p), ("d_err_est", C.c_void_p), ("d_state_id", C.c_void_p),
                ("d_n_unique", C.c_void_p), ("dedupe_tol", C.c_double)]


class grins_server_config(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("hbm_budget_bytes", C.c_int64), ("jit", C.c_int32),
                ("jit_min_work", C.c_double), ("jit_max_wait_s", C.c_double)]


class grins_request_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("error", C.c_int32), ("n_sets", C.c_int64), ("n_ics", C.c_int32),
                ("bytes", C.c_int64), ("queued_s", C.c_double), ("latency_s", C.c_double)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)

_H = C.c_void_p
_P = C.c_void_p
_S = C.c_int32

_sig = {
    "grins_racipe_default_ranges": (None, [C.POINTER(grins_racipe_ranges)]),
    "grins_solver_default_opts": (None, [C.POINTER(grins_solver_opts)]),
    "grins_last_error": (C.c_char_p, []),
    "grins_version": (C.c_char_p, []),
    "grins_device_allocations": (C.c_int64, []),
    "grins_unit_rates": (_S, [C.POINTER(C.c_double), _P]),
    "grins_racipe_create": (_S, [C.c_int32, C.c_int32, _P, _P, _P, C.POINTER(_H)]),
    "grins_racipe_destroy": (_S, [_H]),
    "grins_racipe_param_stride": (C.c_int64, [_H]),
    "grins_racipe_integrator": (C.c_char_p, [_H]),
    "grins_racipe_node_medians": (_S, [_H, C.POINTER(grins_racipe_ranges), _P]),
    "grins_racipe_sample_params": (_S, [_H, C.POINTER(grins_racipe_ranges), C.c_uint64, C.c_int64,
                                        C.c_int64, C.c_int32, _P, _P, _P]),
    "grins_racipe_integrate": (_S, [_H, C.POINTER(grins_solver_opts), _P, C.c_int64, _P, C.c_int32,
                                    _P, _P, _P, _P, _P, _P, _P]),
    "grins_racipe_integrate_static": (_S, [_H, C.POINTER(grins_solver_opts), _P, C.c_int64, _P,
                                           C.c_int32, _P, _P, _P, _P, _P, _P, _P]),
    "grins_racipe_plan_create": (_S, [C.POINTER(grins_solver_opts), C.POINTER(grins_racipe_job), C.c_int32,
                                      C.c_int32, _P, C.POINTER(_H)]),
    "grins_racipe_plan_run": (_S, [_H, _P]),
    "grins_racipe_plan_info": (C.c_char_p, [_H]),
    "grins_racipe_plan_destroy": (_S, [_H]),
    "grins_server_default_config": (None, [C.POINTER(grins_server_config)]),
    "grins_racipe_server_create": (_S, [C.POINTER(grins_server_config), C.POINTER(_H)]),
    "grins_racipe_server_submit": (_S, [_H, _H, C.POINTER(grins_racipe_ranges), C.c_uint64, C.c_int64, C.c_int32,
                                        C.POINTER(grins_solver_opts), C.c_double, C.POINTER(C.c_int64)]),
    "grins_racipe_server_wait": (_S, [_H, C.c_int64, C.c_double, C.POINTER(grins_request_info)]),
    "grins_racipe_server_copy_results": (_S, [_H, C.c_int64, _P, _P, _P, _P, _P, _P]),
    "grins_racipe_server_release": (_S, [_H, C.c_int64]),
    "grins_racipe_server_cancel": (_S, [_H, C.c_int64]),
    "grins_racipe_server_destroy": (_S, [_H]),
    "grins_racipe_tail_stats": (_S, [_H, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "grins_racipe_polish": (_S, [_H, C.POINTER(grins_solver_opts), _P, C.c_int64, C.c_int32, _P, _P, _P, _P]),
    "grins_racipe_unique_states": (_S, [_H, _P, _P, _P, C.c_int64, C.c_int32, C.c_double, _P, _P, _P]),
    "grins_racipe_gk_histogram": (_S, [_H, _P, _P, _P, C.c_int64, C.c_int32, C.c_int32, _P, _P]),
    "grins_level_boundaries": (_S, [C.POINTER(C.c_ulonglong), C.c_int32, C.c_int32, C.c_int32,
                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "grins_racipe_level_states": (_S, [_H, _P, _P, _P, C.c_int64, C.c_int32, C.c_int32, C.POINTER(C.c_int32),
                                       C.c_int32, _P, _P, _P, _P]),
    "grins_ising_run": (_S, [_H, C.c_int32, C.c_int32, C.c_uint64, C.c_int64, _P, C.c_int32, _P, _P, _P, _P]),
}
EXPORTED = tuple(_sig)
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class GrinsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("grins status %d: %s" % (status, msg))
        self.status = status


def device_allocations() -> int:
    """grins_device_allocations: device allocations the library has made so far."""
    return int(_lib.grins_device_allocations())


def _check(st):
    if st != GRINS_OK:
        raise GrinsError(st, _lib.grins_last_error().decode())


UNIT_RATE_NAMES = ("ex2", "lg2", "rcp", "ffma", "dfma", "dmul", "dadd")


def unit_rates(stream=None) -> dict:
    """grins_unit_rates: measured issue rates (operations per clock per SM) of
    ex2.approx, lg2.approx, rcp.approx, FP32 FMA, FP64 FMA, FP64 multiply and
    FP64 add on the current device, keyed by those names."""
    r = (C.c_double * len(UNIT_RATE_NAMES))()
    _check(_lib.grins_unit_rates(r, _stream(stream)))
    return dict(zip(UNIT_RATE_NAMES, (float(x) for x in r)))


def default_ranges(sobol_table=None, param_ranges=None, ic_ranges=None, **over) -> grins_racipe_ranges:
    """Table 1's ranges with fields overridden by keyword.  `sobol_table` =
    (poly [D], m [D, cols]) int64 arrays, e.g. workloads.sobol_direction_table(),
    for the Sobol modes (`sobol=GRINS_SOBOL_PLAIN` or `GRINS_SOBOL_SCRAMBLED`);
    `param_ranges` = a PARAM_RANGE_DTYPE array of 2N + 3E rows (see
    Racipe.param_range_table); `ic_ranges` = N rows for the initial
    conditions (fractions of G/k).  The arrays are kept alive with the struct."""
    r = grins_racipe_ranges()
    _lib.grins_racipe_default_ranges(C.byref(r))
    for k, v in over.items():
        setattr(r, k, v)
    keep = []
    if param_ranges is not None:
        rows = np.ascontiguousarray(param_ranges, dtype=PARAM_RANGE_DTYPE)
        keep.append(rows)
        r.param_ranges = rows.ctypes.data_as(C.POINTER(grins_param_range))
    if ic_ranges is not None:
        icr = np.ascontiguousarray(ic_ranges, dtype=PARAM_RANGE_DTYPE)
        keep.append(icr)
        r.ic_ranges = icr.ctypes.data_as(C.POINTER(grins_param_range))
    if sobol_table is not None:
        poly = np.ascontiguousarray(sobol_table[0], dtype=np.int64)
        m = np.ascontiguousarray(sobol_table[1], dtype=np.int64)
        keep += [poly, m]
        r.sobol_dims = int(poly.shape[0])
        r.sobol_m_cols = int(m.shape[1])
        r.sobol_poly = poly.ctypes.data_as(C.POINTER(C.c_int64))
        r.sobol_m = m.ctypes.data_as(C.POINTER(C.c_int64))
    r._keep = keep
    return r


def default_opts(**over) -> grins_solver_opts:
    o = grins_solver_opts()
    _lib.grins_solver_default_opts(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Racipe:
    """A RACIPE network handle (signed directed edge list, Sec. 2.1.1)."""

    def __init__(self, n_nodes, src, dst, sign, device=None):
        self.device = torch.device(device or "cuda")
        self.n_nodes = int(n_nodes)
        self.src = np.ascontiguousarray(src, dtype=np.int32)
        self.dst = np.ascontiguousarray(dst, dtype=np.int32)
        self.sign = np.ascontiguousarray(sign, dtype=np.int8)
        self.n_edges = int(self.src.size)
        h = _H()
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_create(self.n_nodes, self.n_edges,
                                            self.src.ctypes.data, self.dst.ctypes.data,
                                            self.sign.ctypes.data, C.byref(h)))
        self._h = h
        self.param_stride = int(_lib.grins_racipe_param_stride(h))

    @classmethod
    def from_topology(cls, topo, device=None):
        return cls(*topo.edges(), device=device)

    def param_range_table(self, ranges=None):
        """The per-parameter range table (the generated range file) that the
        class fields of `ranges` describe: rows G[N], k[N], T[E], lam[E], n[E]
        as a PARAM_RANGE_DTYPE array, to be edited and passed back as
        default_ranges(param_ranges=...)."""
        r = ranges if ranges is not None else default_ranges()
        N, E = self.n_nodes, self.n_edges
        t = np.zeros(2 * N + 3 * E, dtype=PARAM_RANGE_DTYPE)
        t[:N] = (r.dist_G, 0, r.G_min, r.G_max)
        t[N:2 * N] = (r.dist_k, 0, r.k_min, r.k_max)
        t[2 * N:2 * N + E] = (0, 0, r.thr_lo, r.thr_hi)
        for e in range(E):
            t[2 * N + E + e] = ((r.dist_lam_act, 0, r.lam_act_min, r.lam_act_max) if self.sign[e] > 0
                                else (r.dist_lam_inh, 0, r.lam_inh_min, r.lam_inh_max))
        t[2 * N + 2 * E:] = (0, 0, float(r.n_min), float(r.n_max))
        return t

    def integrator(self) -> str:
        """Which FP32 integrator kernel this handle uses (grins_racipe_integrator)."""
        return _lib.grins_racipe_integrator(self._h).decode()

    def close(self):
        if getattr(self, "_h", None):
            _lib.grins_racipe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ sampling
    def node_medians(self, ranges=None):
        out = np.zeros(self.n_nodes)
        r = C.byref(ranges) if ranges is not None else None
        _check(_lib.grins_racipe_node_medians(self._h, r, out.ctypes.data))
        return out

    def sample_params(self, seed, n_sets, n_ics, set0=0, ranges=None, stream=None, params=None,
                      ic_unit=None):
        """Returns (params uint8 [n_sets, stride], ic_unit float64 [n_ics, N])."""
        if params is None:
            params = torch.empty((n_sets, self.param_stride), dtype=torch.uint8, device=self.device)
        if ic_unit is None and n_ics > 0:
            ic_unit = torch.empty((n_ics, self.n_nodes), dtype=torch.float64, device=self.device)
        r = C.byref(ranges) if ranges is not None else None
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_sample_params(self._h, r, seed, set0, n_sets, n_ics, _ptr(params),
                                                   _ptr(ic_unit), _stream(stream)))
        return params, ic_unit

    def unpack_params(self, params):
        """Views of a parameter block: G, k [S, N]; T, lam [S, E] float64; n [S, E] uint8."""
        N, E = self.n_nodes, self.n_edges
        S = params.shape[0]
        flat = params.view(S, -1)
        f64 = flat[:, : 16 * N + 16 * E].contiguous().view(torch.float64)
        G, k = f64[:, :N], f64[:, N:2 * N]
        T, lam = f64[:, 2 * N:2 * N + E], f64[:, 2 * N + E:2 * N + 2 * E]
        n = flat[:, 16 * N + 16 * E:16 * N + 17 * E]
        return G, k, T, lam, n

    def pack_params(self, G, k, T, lam, n):
        """Inverse of unpack_params (device tensors or arrays) -> uint8 [S, stride]."""
        G = torch.as_tensor(G, dtype=torch.float64, device=self.device)
        S = G.shape[0]
        f64 = torch.cat([G, torch.as_tensor(k, dtype=torch.float64, device=self.device),
                         torch.as_tensor(T, dtype=torch.float64, device=self.device).reshape(S, -1),
                         torch.as_tensor(lam, dtype=torch.float64, device=self.device).reshape(S, -1)],
                        dim=1)
        out = torch.zeros((S, self.param_stride), dtype=torch.uint8, device=self.device)
        nb = f64.shape[1] * 8
        out[:, :nb] = f64.contiguous().view(torch.uint8).view(S, nb)
        out[:, nb:nb + self.n_edges] = torch.as_tensor(n, device=self.device).to(torch.uint8).reshape(S, -1)
        return out

    # ---------------------------------------------------------- integrate
    def integrate(self, params, ic_unit, opts=None, stream=None, out=None, **over):
        """Integrates every (set, IC); returns a dict of device tensors."""
        o = opts if opts is not None else default_opts()
        t_grid = over.pop("t_grid", None)
        for k, v in over.items():
            setattr(o, k, v)
        grid = None
        if t_grid is not None:
            grid = np.ascontiguousarray(t_grid, dtype=np.float64)
            o.t_grid = grid.ctypes.data_as(C.POINTER(C.c_double))
            o.n_t = grid.size
        S, I, N = params.shape[0], ic_unit.shape[0], self.n_nodes
        dev = self.device
        if out is None:
            out = dict(states=torch.empty((S, I, N), dtype=torch.float64, device=dev),
                       status=torch.empty((S, I), dtype=torch.uint8, device=dev),
                       t_final=torch.empty((S, I), dtype=torch.float64, device=dev),
                       err_est=torch.empty((S, I), dtype=torch.float32, device=dev),
                       n_steps=torch.empty((S, I), dtype=torch.int32, device=dev),
                       series=(torch.empty((S, I, o.n_t, N), dtype=torch.float64, device=dev)
                               if o.n_t > 0 else None))
        with torch.cuda.device(dev):
            _check(_lib.grins_racipe_integrate(
                self._h, C.byref(o), _ptr(params), S, _ptr(ic_unit), I, _ptr(out["states"]),
                _ptr(out["status"]), _ptr(out.get("t_final")), _ptr(out.get("err_est")),
                _ptr(out.get("n_steps")), _ptr(out.get("series")), _stream(stream)))
        return out

    def integrate_static(self, params, ic_unit, out, opts=None, stream=None):
        """grins_racipe_integrate_static: the same integration with the library's
        fixed scratch array instead of any device allocation.  ``out`` holds
        caller-allocated buffers (keys as returned by ``integrate``)."""
        o = opts if opts is not None else default_opts()
        S, I = params.shape[0], ic_unit.shape[0]
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_integrate_static(
                self._h, C.byref(o), _ptr(params), S, _ptr(ic_unit), I, _ptr(out["states"]),
                _ptr(out["status"]), _ptr(out.get("t_final")), _ptr(out.get("err_est")),
                _ptr(out.get("n_steps")), _ptr(out.get("series")), _stream(stream)))
        return out

    def tail_stats(self, stream=None):
        """(solves, attempts) of the last FP32 integrate's borderline re-pass."""
        n, a = C.c_int64(0), C.c_int64(0)
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_tail_stats(self._h, _stream(stream), C.byref(n), C.byref(a)))
        return n.value, a.value

    def polish(self, params, states, status, err_est=None, opts=None, stream=None, **over):
        """FP64 Newton polish in place of converged states (see grins_racipe_polish)."""
        o = opts if opts is not None else default_opts()
        for k, v in over.items():
            setattr(o, k, v)
        S, I = status.shape
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_polish(self._h, C.byref(o), _ptr(params), S, I, _ptr(states),
                                            _ptr(status), _ptr(err_est), _stream(stream)))
        return states, status, err_est

    def unique_states(self, params, states, status, tol=1e-2, stream=None, out=None):
        S, I = status.shape
        if out is None:
            out = (torch.empty((S, I), dtype=torch.int32, device=self.device),
                   torch.empty((S,), dtype=torch.int32, device=self.device))
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_unique_states(self._h, _ptr(params), _ptr(states), _ptr(status),
                                                   S, I, tol, _ptr(out[0]), _ptr(out[1]),
                                                   _stream(stream)))
        return out


    def gk_histogram(self, params, states, status, n_bins=100, counts=None, stream=None):
        """Adds the bins of the converged solves' G/k-normalised values to
        ``counts`` (uint64 [n_bins] on the device; zeros when None)."""
        S, I = status.shape
        if counts is None:
            counts = torch.zeros((n_bins,), dtype=torch.int64, device=self.device)
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_gk_histogram(self._h, _ptr(params), _ptr(states), _ptr(status), S, I,
                                                  n_bins, _ptr(counts), _stream(stream)))
        return counts

    def ising_run(self, n_traj, mode=GRINS_ISING_SYNC, seed=0, init=None, max_steps=1000, enc01=False,
                  stream=None, out=None):
        """Boolean Ising trajectories (grins_ising_run) -> (final states uint64
        as int64 [n_traj], steps int32, status uint8); init: a device int64
        tensor of states (bit i = node i on) or None for random ones."""
        if out is None:
            out = (torch.empty((n_traj,), dtype=torch.int64, device=self.device),
                   torch.empty((n_traj,), dtype=torch.int32, device=self.device),
                   torch.empty((n_traj,), dtype=torch.uint8, device=self.device))
        with torch.cuda.device(self.device):
            _check(_lib.grins_ising_run(self._h, mode, int(bool(enc01)), seed, n_traj, _ptr(init), max_steps,
                                        _ptr(out[0]), _ptr(out[1]), _ptr(out[2]), _stream(stream)))
        return out

    def level_states(self, params, states, status, bounds, n_bins=100, stream=None, out=None):
        """-> (labels uint64 [S, I] as int64, n_states int32 [S], multi_hist
        uint64 [I + 1] as int64, accumulated into ``out[2]`` when given)."""
        S, I = status.shape
        if out is None:
            out = (torch.empty((S, I), dtype=torch.int64, device=self.device),
                   torch.empty((S,), dtype=torch.int32, device=self.device),
                   torch.zeros((I + 1,), dtype=torch.int64, device=self.device))
        b = (C.c_int32 * max(1, len(bounds)))(*[int(x) for x in bounds])
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_level_states(self._h, _ptr(params), _ptr(states), _ptr(status), S, I, n_bins,
                                                  b, len(bounds), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                                                  _stream(stream)))
        return out


def level_boundaries(counts, half_width=4, max_boundaries=3):
    """Boundary bins of a histogram of normalised values (host; see
    grins_level_boundaries)."""
    import numpy as np
    c = np.ascontiguousarray(np.asarray(counts).astype(np.uint64))
    bins = (C.c_int32 * max_boundaries)()
    n = C.c_int32(0)
    _check(_lib.grins_level_boundaries(c.ctypes.data_as(C.POINTER(C.c_ulonglong)), c.size, half_width,
                                       max_boundaries, bins, C.byref(n)))
    return [bins[t] for t in range(n.value)]


class Plan:
    """A batched launch over many networks (grins_racipe_plan_*).

    ``autotune``: 0/False one persistent launch of the run-time-layout
    kernel, 1/True time every form and its knobs and keep the fastest, 2 the
    per-network compiled kernels on graph branches without timing, 3 one
    persistent launch of a kernel compiled for every job's layout.

    ``jobs``: list of dicts with keys net (a Racipe), params, ic_unit and,
    optionally, out (buffers as returned by ``Racipe.integrate``; allocated
    here when absent), dedupe (bool, default True) and dedupe_tol.  The
    buffers live as long as the plan."""

    def __init__(self, jobs, opts=None, autotune=True, stream=None):
        self.opts = opts if opts is not None else default_opts()
        self.jobs = []
        arr = (grins_racipe_job * len(jobs))()
        for b, jb in enumerate(jobs):
            net, params, ic = jb["net"], jb["params"], jb["ic_unit"]
            S, I, N = params.shape[0], ic.shape[0], net.n_nodes
            dev = net.device
            out = jb.get("out") or dict(
                states=torch.empty((S, I, N), dtype=torch.float64, device=dev),
                status=torch.empty((S, I), dtype=torch.uint8, device=dev),
                t_final=torch.empty((S, I), dtype=torch.float64, device=dev),
                err_est=torch.empty((S, I), dtype=torch.float32, device=dev),
                n_steps=torch.empty((S, I), dtype=torch.int32, device=dev))
            if jb.get("dedupe", True):
                out.setdefault("state_id", torch.empty((S, I), dtype=torch.int32, device=dev))
                out.setdefault("n_unique", torch.empty((S,), dtype=torch.int32, device=dev))
            self.jobs.append(dict(net=net, params=params, ic_unit=ic, out=out))
            arr[b] = grins_racipe_job(net._h.value, params.data_ptr(), S, ic.data_ptr(), I,
                                      out["states"].data_ptr(), out["status"].data_ptr(),
                                      out["t_final"].data_ptr() if out.get("t_final") is not None else None,
                                      out["n_steps"].data_ptr() if out.get("n_steps") is not None else None,
                                      out["err_est"].data_ptr() if out.get("err_est") is not None else None,
                                      out["state_id"].data_ptr() if out.get("state_id") is not None else None,
                                      out["n_unique"].data_ptr() if out.get("n_unique") is not None else None,
                                      float(jb.get("dedupe_tol", 1e-2)))
        self._arr = arr
        h = _H()
        _check(_lib.grins_racipe_plan_create(C.byref(self.opts), arr, len(jobs), int(autotune),
                                             _stream(stream), C.byref(h)))
        self._p = h

    def run(self, stream=None):
        _check(_lib.grins_racipe_plan_run(self._p, _stream(stream)))
        return self.jobs

    def info(self) -> str:
        return _lib.grins_racipe_plan_info(self._p).decode()

    def close(self):
        if getattr(self, "_p", None):
            _lib.grins_racipe_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (grins_racipe_server_*)."""

    def __init__(self, max_inflight=8, hbm_budget_bytes=32 << 30, device=None, jit=True, jit_min_work=None,
                 jit_max_wait_s=None):
        self.device = torch.device(device or "cuda")
        cfg = grins_server_config()
        _lib.grins_server_default_config(C.byref(cfg))
        cfg.max_inflight, cfg.hbm_budget_bytes, cfg.jit = max_inflight, hbm_budget_bytes, 1 if jit else 0
        if jit_min_work is not None:
            cfg.jit_min_work = jit_min_work
        if jit_max_wait_s is not None:
            cfg.jit_max_wait_s = jit_max_wait_s
        h = _H()
        with torch.cuda.device(self.device):
            _check(_lib.grins_racipe_server_create(C.byref(cfg), C.byref(h)))
        self._s = h
        self._nets = {}

    def submit(self, net, seed, n_sets, n_ics, opts=None, ranges=None, dedupe_tol=1e-2):
        o = opts if opts is not None else default_opts()
        rid = C.c_int64()
        r = C.byref(ranges) if ranges is not None else None
        _check(_lib.grins_racipe_server_submit(self._s, net._h, r, seed, n_sets, n_ics, C.byref(o),
                                               dedupe_tol, C.byref(rid)))
        self._nets[rid.value] = (net, n_sets, n_ics)
        return rid.value

    def wait(self, rid, timeout_s=-1.0):
        info = grins_request_info()
        _check(_lib.grins_racipe_server_wait(self._s, rid, timeout_s, C.byref(info)))
        return dict(state=info.state, error=info.error, n_sets=info.n_sets, n_ics=info.n_ics, bytes=info.bytes,
                    queued_s=info.queued_s, latency_s=info.latency_s)

    def results(self, rid, stream=None, keys=("states", "status", "n_unique", "state_id", "n_steps")):
        """Copies a finished request's results (the given keys of states,
        status, n_unique, state_id, n_steps) into new tensors."""
        net, S, I = self._nets[rid]
        dev = net.device
        shapes = dict(states=((S, I, net.n_nodes), torch.float64), status=((S, I), torch.uint8),
                      n_unique=((S,), torch.int32), state_id=((S, I), torch.int32), n_steps=((S, I), torch.int32))
        out = {k: torch.empty(shapes[k][0], dtype=shapes[k][1], device=dev) for k in keys}
        with torch.cuda.device(dev):
            _check(_lib.grins_racipe_server_copy_results(self._s, rid, _ptr(out.get("states")),
                                                         _ptr(out.get("status")), _ptr(out.get("n_unique")),
                                                         _ptr(out.get("state_id")), _ptr(out.get("n_steps")),
                                                         _stream(stream)))
        return out

    def cancel(self, rid):
        """grins_racipe_server_cancel: stop a queued or running request."""
        _check(_lib.grins_racipe_server_cancel(self._s, rid))

    def release(self, rid):
        _check(_lib.grins_racipe_server_release(self._s, rid))
        self._nets.pop(rid, None)

    def close(self):
        if getattr(self, "_s", None):
            _lib.grins_racipe_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
