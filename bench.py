"""RACIPE ensemble benchmark: steady-state solves per second on one GB300.

Workload (one "step" = the whole hot path over one batch): the seeded random
22-node / 82-edge signed network (33 inhibitory edges, 3 self-activations;
stand-in for the paper's EMT network, Sec. 3.2), 100,000 parameter sets x 10
initial conditions = 1,000,000 solves per step:
  sample parameters + ICs -> FP32 Dormand-Prince 5(4) to steady state ->
  double-float re-pass of the solves whose steady-state decision fell near
  t_end, with the FP64 Newton polish of the other solves beside it, then of
  the re-passed ones -> distinct steady states per set.
Under torchrun each rank integrates its own 100,000 sets (set offset rank x
100,000; weak scaling, no collective on the data path).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
plain FP64 implementation under oracle/) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the headline metric, the same string on both arms (the reference arm times
# the oracle on a bounded sample of the same workload)
METRIC = "RACIPE steady-state solves/s (22-node network, FP32 + FP64 polish)"
N_SETS = 100_000
N_ICS = 10
TOL = dict(rtol=1e-6, atol=1e-9, t_end=200.0, ss_tol=1e-6)
# DRAM bytes (read + write) of one FP32 integrator launch per solve, from an
# ncu capture of the same kernel on a 20,000-set launch of this workload
# (35.75 MB read + 0.64 MB written for 200,000 solves,
# profiles/grins_grp_ct_rr_rand22x82_20k.md); traffic grows with the solves
# per launch.  None while no capture of the current kernel exists.
INTEGRATOR_DRAM_BYTES_PER_SOLVE = (35.753e6 + 0.639e6) / 200_000
# Executed FP64 instructions (DADD + DMUL + DFMA, thread level) of the FP64
# kernels per unit of work, from an ncu capture of the same 20,000-set
# launch (profiles/fp64_kernels_rand22x82_20k.md): the polish per solve it
# polishes (its two launches of the step, beside the re-pass and after it;
# converged before the polish: 127,247), the re-pass per FP64 step
# attempt (254,532), the dedupe per converged solve (127,243).
# (DADD, DMUL, DFMA) counts of each kernel; the per-unit figure is their sum
# over the units, the peak the issue rate of that mix (each kind at its own
# measured rate)
POLISH_FP64_MIX = (5_834_202, 142_128_522, 72_993_468)
REPASS_FP64_MIX = (253_617_128, 766_275_305, 786_803_446)
UNIQUE_FP64_MIX = (2_580_512, 5_598_692, 19_595_422)
POLISH_FP64_INSTR_PER_SOLVE = sum(POLISH_FP64_MIX) / 127_247
REPASS_FP64_INSTR_PER_ATTEMPT = sum(REPASS_FP64_MIX) / 254_532
UNIQUE_FP64_INSTR_PER_SOLVE = sum(UNIQUE_FP64_MIX) / 127_243
# Executed warp instructions of the double-float re-pass kernel per solve
# step attempt, from an ncu capture of the same 20,000-set launch
# (801,912,638 warp instructions for 254,533 attempts,
# profiles/fp64_kernels_rand22x82_20k.md); None while no capture of the
# current kernel exists.
REPASS_DD_WARP_INSTR_PER_ATTEMPT = 801_912_638 / 254_533


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--sets", type=int, default=N_SETS)
    ap.add_argument("--tail-precision", default="dd", choices=["dd", "fp64"],
                    help="arithmetic of the borderline re-pass: double-float (default) or FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sets", type=int, default=1000, help="sets of the oracle sample (sets 0..n-1)")
    ap.add_argument("--ref-sets", type=int, default=200,
                    help="sets per step of the reference arm (the oracle timed on the host cores)")
    ap.add_argument("--fp64-sets", type=int, default=N_SETS,
                    help="sets of the plain FP64 GPU solver's timed run (default: the whole workload)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the Poisson request stream of the serving measurement (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=20.0, help="requests per second of that stream")
    ap.add_argument("--batch-reps", type=int, default=3,
                    help="timed replays of the batched 64-network plan (0: skip)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0])); smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None,
                    sm_max_mhz=max(smax) if smax else None, reasons=sorted(reasons),
                    samples=len(sm))


# ------------------------------------------------------------ CPU baseline
def oracle_sample(n_sets, threads):
    """The oracle as it stands on the first n_sets sets of the workload."""
    import numpy as np
    import oracle as O
    from paper_2503_18356_gb300 import workloads as W
    w = W.net22_workload()
    net = O.Network(*w["topology"].edges())
    p = O.sample_params(net, w["param_seed"], n_sets)
    ic = O.sample_ics(w["topology"].n_nodes, w["ic_seed"], N_ICS)
    t0 = time.perf_counter()
    out = O.run_sets_parallel(net, p, ic, threads=threads)
    dt = time.perf_counter() - t0
    return n_sets * N_ICS / dt, dt, out


def oracle_tolerance_floor(n_sets, orc):
    """The oracle itself at the GPU solver's tolerances (TOL, FP64, same
    polish and dedupe) on the same sets, against the oracle at rtol 1e-10:
    the status and distinct-state agreement that these tolerances allow any
    solver, whatever its precision."""
    import numpy as np
    import oracle as O
    from paper_2503_18356_gb300 import workloads as W
    w = W.net22_workload()
    net = O.Network(*w["topology"].edges())
    p = O.sample_params(net, w["param_seed"], n_sets)
    ic = O.sample_ics(w["topology"].n_nodes, w["ic_seed"], N_ICS)
    lo = O.run_sets_parallel(net, p, ic, threads=os.cpu_count() or 1, **TOL)
    return dict(status_agree=float((lo["status"] == orc["status"][:n_sets]).mean()),
                n_unique_agree=float((lo["n_unique"] == orc["n_unique"][:n_sets]).mean()),
                note="the FP64 oracle run at the GPU solver's tolerances (rtol %g, atol %g), against the "
                     "oracle at rtol 1e-10" % (TOL["rtol"], TOL["atol"]))


def cpu_baseline(n_sets):
    """The timed oracle sample; also returns the oracle's results."""
    threads = os.cpu_count() or 1
    v, dt, out = oracle_sample(n_sets, threads)
    return dict(value=v, unit="solves/s", cores=threads, kind="oracle",
                sample="sets 0..%d of the workload x %d ICs (%d solves), FP64 DP5 rtol 1e-10 + "
                       "Newton polish + dedupe, %.1f s" % (n_sets - 1, N_ICS, n_sets * N_ICS, dt)), out


def parity_figures(gpu, orc, G, k, params_slice):
    """Per-result error of the GPU path against the oracle on the same sets,
    over solves converged on both sides at the same fixed point (G/k-
    normalised distance <= 1e-2 raw, 1e-5 polished):
      * raw states (the integrator's stopping point, before the polish):
        relative error with a floor, |x - x*| / max(|x*|, 1e-6 G/k) -- the
        relative 1e-3 scale -- with the share of solves above 1e-3, and the
        error on the G/k scale beside it (the steady-state test bounds the
        distance to the fixed point in units of G/k);
      * polished states: relative, floor 1e-6 G/k;
    the basin-mismatch rate (both converged, different fixed points) and how
    many of those fail the oracle's residual certificate, the status
    agreement and the share of sets with the same number of distinct steady
    states."""
    import numpy as np
    import oracle as O
    from paper_2503_18356_gb300 import workloads as W
    net = O.Network(*W.net22_workload()["topology"].edges())
    G = G[:, None, :]
    k = k[:, None, :]
    vo = orc["states"] * k / G
    res = {}
    for name, states, status, tol, cert in (("fp32_raw", gpu["raw_states"], gpu["raw_status"], 1e-2, 1e-5),
                                            ("fp32_polish", gpu["states"], gpu["status"], 1e-5, 1e-10)):
        both = (status == 0) & (orc["status"] == 0)
        vg = states * k / G
        dist = np.abs(vg - vo).max(axis=2)
        same = both & (dist <= tol)
        rel = (np.abs(states - orc["states"]) / np.maximum(np.abs(orc["states"]), 1e-6 * G)).max(axis=2)
        gk = np.abs(vg - vo).max(axis=2)
        e = rel[same]
        unc = 0
        for s_, c_ in zip(*np.nonzero(both & ~same)):
            if not all(O.rho(net, params_slice, x, s_) < cert for x in (states[s_, c_], orc["states"][s_, c_])):
                unc += 1
        res[name] = dict(max=float(e.max()) if e.size else None,
                         p999=float(np.quantile(e, 0.999)) if e.size else None,
                         share_above_1e3=float((e > 1e-3).mean()) if e.size else None,
                         compared=int(same.sum()), basin_mismatch_rate=float((both & ~same).mean()),
                         basin_mismatch_uncertified=unc,
                         status_agree=float((status == orc["status"]).mean()),
                         error="relative, floor 1e-6 G/k")
        if name == "fp32_raw":
            res[name]["gk_scale"] = dict(max=float(gk[same].max()) if e.size else None,
                                         p999=float(np.quantile(gk[same], 0.999)) if e.size else None)
    res["n_unique_agree"] = float((gpu["n_unique"] == orc["n_unique"]).mean())
    if "fp64_n_unique" in gpu:
        # the same figures for the plain FP64 GPU solver at the same tolerances
        res["fp64_solver"] = dict(status_agree=float((gpu["fp64_status"] == orc["status"]).mean()),
                                  n_unique_agree=float((gpu["fp64_n_unique"] == orc["n_unique"]).mean()))
    return res


def oracle_unpolished_share(n_sets):
    """The oracle's own integration stopping point (rtol 1e-10, no polish)
    against its polished fixed point on the first n_sets sets, on the same
    relative scale: what the steady-state test alone leaves on nodes near
    zero, whatever the arithmetic."""
    import numpy as np
    import oracle as O
    from paper_2503_18356_gb300 import workloads as W
    w = W.net22_workload()
    net = O.Network(*w["topology"].edges())
    p = O.sample_params(net, w["param_seed"], n_sets)
    ic = O.sample_ics(w["topology"].n_nodes, w["ic_seed"], N_ICS)
    raw = O.run_sets_parallel(net, p, ic, polish=False)
    pol = O.run_sets_parallel(net, p, ic, polish=True)
    G, k = p.G[:, None, :], p.k[:, None, :]
    both = (raw["status"] == 0) & (pol["status"] == 0)
    rel = (np.abs(raw["states"] - pol["states"]) / np.maximum(np.abs(pol["states"]), 1e-6 * G / k)).max(axis=2)[both]
    gk = (np.abs(raw["states"] - pol["states"]) * k / G).max(axis=2)[both]
    return dict(sets=n_sets, compared=int(both.sum()), share_above_1e3=float((rel > 1e-3).mean()),
                max=float(rel.max()), gk_max=float(gk.max()),
                note="the oracle's own unpolished states (rtol 1e-10, stopped at max|f| k/G < 1e-6) against its "
                     "polished ones, relative with floor 1e-6 G/k")


def levels_measurement(h, params, out, stream, dev, S, I, n_bins=100, reps=3):
    """The levels row on the step's polished states: G/k histogram (device),
    level boundaries (host), labels, distinct states per set and the
    multistability histogram (device); CUDA-event times of the two device
    passes, the boundaries found and the share of sets by number of states."""
    import numpy as np
    import torch
    from paper_2503_18356_gb300 import api
    cnt = torch.zeros((n_bins,), dtype=torch.int64, device=dev)
    lab = torch.empty((S, I), dtype=torch.int64, device=dev)
    nst = torch.empty((S,), dtype=torch.int32, device=dev)
    mh = torch.zeros((I + 1,), dtype=torch.int64, device=dev)
    t_hist, t_states = [], []
    for r in range(reps + 1):                 # the first pass is a warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        cnt.zero_(); mh.zero_()
        ev[0].record(stream)
        h.gk_histogram(params, out["states"], out["status"], n_bins=n_bins, counts=cnt, stream=stream)
        ev[1].record(stream)
        torch.cuda.synchronize()
        bounds = api.level_boundaries(cnt.cpu().numpy().view(np.uint64), half_width=4, max_boundaries=3)
        ev[2].record(stream)
        h.level_states(params, out["states"], out["status"], bounds, n_bins=n_bins, stream=stream,
                       out=(lab, nst, mh))
        ev[3].record(stream)
        torch.cuda.synchronize()
        if r:
            t_hist.append(ev[0].elapsed_time(ev[1])); t_states.append(ev[2].elapsed_time(ev[3]))
    hist = mh.cpu().numpy()
    ms = float(np.mean(t_hist) + np.mean(t_states))
    return dict(ms_histogram=float(np.mean(t_hist)), ms_states=float(np.mean(t_states)),
                solves_per_s=S * I / (ms / 1e3), n_bins=n_bins,
                boundaries=[(b + 0.5) / n_bins for b in bounds],
                share_of_sets_by_states={str(k): float(v) / S for k, v in enumerate(hist) if v},
                reading="one G/k histogram over all nodes of all converged solves, binomial smoothing of "
                        "half-width 4, modes merged by persistence (a boundary where the absorbed peak is at "
                        "least twice the valley and 1/64 of the highest count), at most 3 boundaries")


def tsit5_measurement(h, params, ic, out, stream, S, I, reps=2):
    """The paper's own 5(4) pair (Tsitouras, diffrax's Tsit5) on the same
    workload and tolerances: FP32 integrate + FP64 polish, CUDA events."""
    import numpy as np
    import torch
    from paper_2503_18356_gb300 import api
    opts = api.default_opts(method=api.GRINS_METHOD_TSIT5, **TOL)
    h.integrate(params, ic, opts=opts, stream=stream, out=out)       # compile and warm up
    ts = []
    for _ in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        h.integrate(params, ic, opts=opts, stream=stream, out=out)
        ev[1].record(stream)
        torch.cuda.synchronize()
        ts.append(ev[0].elapsed_time(ev[1]))
    ms = float(np.mean(ts))
    st = out["status"].cpu().numpy()
    return dict(ms_integrate_polish=ms, solves_per_s=S * I / (ms / 1e3),
                step_attempts_per_solve=float(out["n_steps"].float().mean().item()),
                converged_share=float((st == 0).mean()), kernel=h.integrator())


def ising_measurement(h, stream, N, n_traj=1_000_000, reps=3):
    """The Boolean Ising formalism (Eq. 3) on the same network: random
    initial states, synchronous and asynchronous modes, CUDA events."""
    import numpy as np
    import torch
    from paper_2503_18356_gb300 import api
    res = {}
    for name, mode, max_steps in (("sync", api.GRINS_ISING_SYNC, 200), ("async", api.GRINS_ISING_ASYNC, 2000)):
        out = h.ising_run(n_traj, mode=mode, seed=77, max_steps=max_steps, stream=stream)   # warm-up
        ts = []
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            h.ising_run(n_traj, mode=mode, seed=77, max_steps=max_steps, stream=stream, out=out)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        ms = float(np.mean(ts))
        fin = out[0].cpu().numpy()
        steps = out[1].cpu().numpy().astype(np.int64)
        conv = out[2].cpu().numpy() == 0
        vals, cnt = np.unique(fin[conv], return_counts=True)
        # node updates: every node of every synchronous step, one node an asynchronous step
        updates = float(steps.sum() * (N if mode == api.GRINS_ISING_SYNC else 1))
        res[name] = dict(ms=ms, trajectories_per_s=n_traj / (ms / 1e3), node_updates_per_s=updates / (ms / 1e3),
                         max_steps=max_steps, converged_share=float(conv.mean()),
                         distinct_fixed_points=int(vals.size),
                         top_state_share=float(cnt.max() / conv.sum()) if cnt.size else 0.0)
    res["trajectories"] = n_traj
    return res


def sampler_measurement(h, stream, S, reps=3):
    """The parameter sampler of the workload under each distribution of
    every continuous class (Table 1, log-uniform, normal, log-normal), under
    a Latin hypercube over the S sets and as scrambled Sobol points (Table 1
    classes): CUDA-event time of one call for all S sets (the medians are
    cached; the Sobol call includes building and uploading its table)."""
    import numpy as np
    import torch
    from paper_2503_18356_gb300 import api
    res = {}
    from paper_2503_18356_gb300 import workloads as W
    tab = W.sobol_direction_table()
    for name, d, lhs, sob in (("table1", 0, 0, 0), ("loguniform", 1, 0, 0), ("normal", 2, 0, 0),
                              ("lognormal", 3, 0, 0), ("lhs_table1", 0, S, 0), ("sobol_scrambled", 0, 0, 2)):
        r = api.default_ranges(dist_G=d, dist_k=d, dist_lam_act=d, dist_lam_inh=d, lhs_sets=lhs, sobol=sob,
                               sobol_table=tab if sob else None)
        params, _ = h.sample_params(2000, S, 1, ranges=r, stream=stream)       # medians, warm-up
        ts = []
        for _ in range(reps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            h.sample_params(2000, S, 1, ranges=r, stream=stream, params=params)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        res[name] = dict(ms=float(np.mean(ts)), sets_per_s=S / (float(np.mean(ts)) / 1e3))
    return res


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_sample(max(2, args.ref_sets // 4), os.cpu_count() or 1)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, _ = oracle_sample(args.ref_sets, os.cpu_count() or 1)
        vals.append(v); times.append(dt)
    total = args.ref_sets * N_ICS * args.steps
    value = total / sum(times)
    cores = os.cpu_count() or 1
    line = dict(impl="reference", metric=METRIC,
                value=value, unit="solves/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1000 * sum(times) / args.steps, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload="rand22x82: 22 nodes, 82 edges; %d sets x %d ICs per step "
                                     "(bounded CPU sample of the 100000 x 10 workload)" % (args.ref_sets, N_ICS)),
                cpu_baseline=dict(value=value, unit="solves/s", cores=cores, kind="oracle",
                                  sample="sets 0..%d x %d ICs per step" % (args.ref_sets - 1, N_ICS)),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


# ------------------------------------------------------------------ batched
def batched_measurement(dev, reps, rcp_rate, f_mhz):
    """One plan over the 64 uneven networks of the batched workload (2-40
    nodes, density 0.1-0.3, 100-10k sets log-uniform, 10 ICs each), captured
    in a CUDA graph and autotuned at creation (untimed; the autotuner's pick
    -- normally one persistent launch of the kernel compiled for every job's
    layout -- then each job's polish and dedupe).  Timed: `reps` replays of
    the graph after one warm-up replay, CUDA events on the stream."""
    import torch
    from paper_2503_18356_gb300 import api, workloads as W

    jobs = []
    solves = 0
    for wl in W.batched_workload(64):
        h = api.Racipe.from_topology(wl["topology"], device=dev)
        params, ic = h.sample_params(wl["param_seed"], wl["n_sets"], wl["n_ics"])
        jobs.append(dict(net=h, params=params, ic_unit=ic))
        solves += wl["n_sets"] * wl["n_ics"]
    stream = torch.cuda.current_stream()
    plan = api.Plan(jobs, stream=stream)
    plan.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    info = plan.info()
    # the SFU work of record over the jobs (W_SFU = 6E + N per step attempt
    # of one solve), per replay, against the SFU peak (the measured reciprocal
    # rate at the timed steps' median SM clock):
    # a lower bound on the integrator's fraction, the replay also holding the
    # jobs' polish and dedupe
    work = 0.0
    for jb in plan.jobs:
        h = jb["net"]
        work += float(jb["out"]["n_steps"].double().sum().item()) * (6 * h.n_edges + h.n_nodes)
    props = torch.cuda.get_device_properties(dev)
    peak = rcp_rate * props.multi_processor_count * f_mhz * 1e6
    achieved = work / (ms / 1e3)
    plan.close()
    return dict(networks=len(jobs), solves=solves, ms_per_replay=ms, solves_per_s=solves / (ms / 1e3),
                plan=info, reps=reps,
                roofline=dict(bound="alu", achieved=achieved / 1e9, peak=peak / 1e9, unit="Gop/s (MUFU, SFU pipe)",
                              frac=achieved / peak,
                              basis="sum over jobs of step attempts x (6E + N) per replay / replay time (polish "
                                    "and dedupe included) / (%.2f rcp.approx/clk/SM measured x %d SMs x %.0f MHz, "
                                    "the median SM clock of the timed steps)"
                                    % (rcp_rate, props.multi_processor_count, f_mhz)),
                workload="64 seeded random signed networks of 2-40 nodes, density 0.1-0.3, 100-10k sets "
                         "(log-uniform) x 10 ICs, FP32 + FP64 polish + dedupe, one CUDA-graph replay")


# ------------------------------------------------------------------ serving
def serving_measurement(dev, seconds, rate, rcp_rate, f_mhz):
    """Request server under the Poisson stream of ensemble requests (networks
    of 2-60 nodes, density 0.05-0.3, 1k-50k sets x 1-20 ICs, FP32 + FP64
    polish + dedupe).  At each request's arrival time the submitting thread
    creates the network handle from its edge list and submits the request; a
    second thread waits for each request and releases it (handles are freed
    at the end: freeing one synchronises the device).
    Latency = scheduled arrival -> results ready on the device (so a busy
    submitting thread counts against it); `server_p50_ms`/`server_p99_ms`
    are the server's own submission -> ready times.  solves/s = all solves
    of the stream / wall time from the first arrival to the last completion.
    The first request of the process compiles nothing in advance: kernels
    and median tables are built as requests need them."""
    import threading as th
    import numpy as np
    from paper_2503_18356_gb300 import api, workloads as W

    stream = W.serving_stream(rate_hz=rate, duration_s=seconds)
    sv = api.Server(max_inflight=16, hbm_budget_bytes=64 << 30, device=dev)
    w = W.net5_workload()                          # warm-up request (not timed)
    wnet = api.Racipe.from_topology(w["topology"], device=dev)
    rid = sv.submit(wnet, 1, 100, 2)
    sv.wait(rid)
    sv.release(rid)
    n = len(stream)
    ids, nets, infos, t_ret = [None] * n, [None] * n, [None] * n, [0.0] * n
    work = [0.0] * n              # SFU work of record: step attempts x (6E + N)
    ready = th.Semaphore(0)

    def releaser():
        for k in range(n):
            ready.acquire()
            infos[k] = sv.wait(ids[k])
            if infos[k]["state"] == api.REQ_DONE:
                steps = sv.results(ids[k], keys=("n_steps",))["n_steps"]
                work[k] = float(steps.double().sum().item()) * (6 * nets[k].n_edges + nets[k].n_nodes)
            sv.release(ids[k])

    t = th.Thread(target=releaser)
    t.start()
    solves = 0
    start = time.perf_counter()
    for k, r in enumerate(stream):
        dt = r["arrival_s"] - (time.perf_counter() - start)
        if dt > 0:
            time.sleep(dt)
        nets[k] = api.Racipe.from_topology(r["topology"], device=dev)
        ids[k] = sv.submit(nets[k], r["param_seed"], r["n_sets"], r["n_ics"])
        t_ret[k] = time.perf_counter() - start
        solves += r["n_sets"] * r["n_ics"]
        ready.release()
    t.join()
    wall = time.perf_counter() - start
    sv.close()
    for h in nets:
        h.close()
    props = __import__("torch").cuda.get_device_properties(dev)
    peak = rcp_rate * props.multi_processor_count * f_mhz * 1e6
    offered = sum(r["n_sets"] * r["n_ics"] for r in stream) / seconds
    srv = np.array([x["latency_s"] for x in infos]) * 1e3
    lat = srv + (np.array(t_ret) - np.array([r["arrival_s"] for r in stream])) * 1e3
    que = np.array([x["queued_s"] for x in infos]) * 1e3
    return dict(requests=n, rate_hz=rate, stream_s=seconds, wall_s=wall, solves=solves,
                solves_per_s=solves / wall, offered_solves_per_s=offered,
                roofline=dict(bound="alu", frac=sum(work) / wall / peak, achieved=sum(work) / wall / 1e9,
                              peak=peak / 1e9, unit="Gop/s (MUFU, SFU pipe)",
                              basis="sum over requests of step attempts x (6E + N) / wall time from the first "
                                    "arrival to the last completion (sampling, polish, dedupe, compiles and idle "
                                    "gaps included) / (%.2f rcp.approx/clk/SM measured x %d SMs x %.0f MHz, the "
                                    "median SM clock of the timed steps)"
                                    % (rcp_rate, props.multi_processor_count, f_mhz)),
                p50_ms=float(np.percentile(lat, 50)),
                p99_ms=float(np.percentile(lat, 99)), max_ms=float(lat.max()),
                server_p50_ms=float(np.percentile(srv, 50)), server_p99_ms=float(np.percentile(srv, 99)),
                queued_p50_ms=float(np.percentile(que, 50)), queued_p99_ms=float(np.percentile(que, 99)),
                failed=int(sum(x["state"] != api.REQ_DONE for x in infos)),
                workload="Poisson stream at %g req/s for %g s: seeded random signed networks of 2-60 nodes, "
                         "density 0.05-0.3, 1k-50k sets x 1-20 ICs each, FP32 + FP64 polish + dedupe; "
                         "handle created at arrival; admitted by HBM budget (64 GB), up to 16 in flight"
                         % (rate, seconds))


# ------------------------------------------------------------------ native
def run_native(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2503_18356_gb300 import build as B
    B.build()
    from paper_2503_18356_gb300 import api, shard, workloads as W

    w = W.net22_workload()
    topo = w["topology"]
    S, I, N, E = args.sets, N_ICS, topo.n_nodes, topo.n_edges
    set0, _ = shard.rank_sets(S, rank)
    h = api.Racipe.from_topology(topo, device=dev)
    stream = torch.cuda.current_stream()
    params = torch.empty((S, h.param_stride), dtype=torch.uint8, device=dev)
    ic = torch.empty((I, N), dtype=torch.float64, device=dev)
    out = dict(states=torch.empty((S, I, N), dtype=torch.float64, device=dev),
               status=torch.empty((S, I), dtype=torch.uint8, device=dev),
               t_final=torch.empty((S, I), dtype=torch.float64, device=dev),
               err_est=torch.empty((S, I), dtype=torch.float32, device=dev),
               n_steps=torch.empty((S, I), dtype=torch.int32, device=dev), series=None)
    sid = torch.empty((S, I), dtype=torch.int32, device=dev)
    nu = torch.empty((S,), dtype=torch.int32, device=dev)
    opts = api.default_opts(precision=api.GRINS_FP32, polish=0, **TOL)
    opts.tail_precision = api.GRINS_TAIL_FP64 if args.tail_precision == "fp64" else api.GRINS_TAIL_DD
    popts = api.default_opts()

    # the step as a user runs it: one integrate call with the polish, which
    # runs the polish beside the re-pass
    opts_p = api.default_opts(precision=api.GRINS_FP32, polish=1, **TOL)
    opts_p.tail_precision = opts.tail_precision

    def step(ev=None, separate=False):
        # events: 0 start, 1 sampled, 2 FP32 pass done (recorded by the
        # library between its passes), 3 integrate done, 4 polished, 5
        # deduped.  separate: the polish as its own call after the re-pass
        # (per-kernel times for the secondary rooflines); else 3 = 4
        o = opts if separate else opts_p
        if ev:
            ev[0].record(stream)
            o.pass_event = ev[2].cuda_event
        h.sample_params(w["param_seed"], S, I, set0=set0, params=params, ic_unit=ic, stream=stream)
        if ev: ev[1].record(stream)
        h.integrate(params, ic, opts=o, stream=stream, out=out)
        o.pass_event = None
        if ev: ev[3].record(stream)
        if separate:
            h.polish(params, out["states"], out["status"], out["err_est"], opts=popts, stream=stream)
        if ev: ev[4].record(stream)
        h.unique_states(params, out["states"], out["status"], stream=stream, out=(sid, nu))
        if ev: ev[5].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
            torch.cuda.synchronize()

    # the first step is cold: it computes the half-functional median table
    # and compiles the network's kernels (FP32 pass and re-pass) at run time;
    # its wall time is reported beside the steady-state figures
    t_cold = time.perf_counter()
    step()
    barrier()
    first_step_s = time.perf_counter() - t_cold
    for _ in range(max(3, args.warmup) - 1):
        step()
    barrier()
    # issue rates of the units the kernels are bound by (per clock per SM),
    # measured on this device before the timed region
    rates = api.unit_rates(stream)

    props = torch.cuda.get_device_properties(dev)
    uuid = str(getattr(props, "uuid", "") or "")
    clk = ClockSampler(("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else (uuid or str(dev.index)))
    clk.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    for e in evs:                    # create the events the library records (torch creates them lazily)
        e[2].record(stream)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    barrier()
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    stop.record(stream)
    barrier()
    clocks = clk.stop()
    elapsed_ms = shard.max_over_ranks(start.elapsed_time(stop), dev)
    per_kernel = np.array([[e[i].elapsed_time(e[i + 1]) for i in range(5)] for e in evs])  # ms
    # the last timed step's re-pass (every step integrates the same sets)
    n_tail, a_tail = h.tail_stats(stream)
    # one more (untimed) step with the polish as its own call: the re-pass
    # and the polish timed apart
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    sev[2].record(stream)
    step(sev, separate=True)
    torch.cuda.synchronize()
    sep_ms = [sev[i].elapsed_time(sev[i + 1]) for i in range(5)]

    # the first sets of one more (untimed) step, raw and polished, for the
    # per-result comparison with the oracle
    snap = None
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        P = min(S, args.cpu_sets)
        h.sample_params(w["param_seed"], S, I, set0=set0, params=params, ic_unit=ic, stream=stream)
        h.integrate(params, ic, opts=opts, stream=stream, out=out)
        snap = dict(raw_states=out["states"][:P].cpu().numpy(), raw_status=out["status"][:P].cpu().numpy())
        h.polish(params, out["states"], out["status"], out["err_est"], opts=popts, stream=stream)
        h.unique_states(params, out["states"], out["status"], stream=stream, out=(sid, nu))
        G, k = (x[:P].cpu().numpy() for x in h.unpack_params(params[:P])[:2])
        Tt, lt, nt = (x[:P].cpu().numpy() for x in h.unpack_params(params[:P])[2:])
        snap.update(states=out["states"][:P].cpu().numpy(), status=out["status"][:P].cpu().numpy(),
                    n_unique=nu[:P].cpu().numpy(), G=G, k=k, T=Tt, lam=lt, n=nt,
                    n_unique_all=nu.cpu().numpy(), status_all=out["status"].cpu().numpy())
    kern_ms = per_kernel.mean(axis=0)
    # the timed step's step attempts and statuses, before later legs reuse the
    # buffers; d_n_steps counts both passes, the roofline the FP32 pass's
    attempts_all = int(out["n_steps"].sum().item())
    attempts = attempts_all - a_tail
    kernel_desc = h.integrator()          # the timed step's kernels, before the Tsit5 leg
    status = out["status"].cpu().numpy()
    levels = levels_measurement(h, params, out, stream, dev, S, I) if rank == 0 else None
    tsit5 = tsit5_measurement(h, params, ic, out, stream, S, I) if rank == 0 else None
    ising = ising_measurement(h, stream, N) if rank == 0 else None
    samplers = sampler_measurement(h, stream, S) if rank == 0 else None

    # algorithmic work of the FP32 integrator (per step attempt of one solve)
    w32 = 35 * E + 45 * N
    wsfu = 6 * E + N
    sms = props.multi_processor_count
    f_mhz = clocks.get("sm_mhz") or 1440.0
    t_int = kern_ms[1] / 1e3
    # the SFU term at the reciprocal-class rate (rcp and lg2; ex2 runs at
    # about twice it) against the FP32 term at the FMA rate, both measured
    sfu_rate, fma_rate = rates["rcp"], rates["ffma"]
    sfu_bound = wsfu / sfu_rate >= w32 / fma_rate
    if sfu_bound:
        achieved = attempts * wsfu / t_int / 1e9
        peak = sfu_rate * sms * f_mhz * 1e6 / 1e9
        unit = "Gop/s (MUFU, SFU pipe)"
    else:
        achieved = attempts * w32 / t_int / 1e9
        peak = fma_rate * sms * f_mhz * 1e6 / 1e9
        unit = "Gop/s (FP32 pipe)"
    # the FP64 kernels against the FP64 FMA issue rate: executed FP64
    # instructions per unit (ncu counts, constants above) x units / time
    hist = np.bincount(status.ravel(), minlength=5)
    n_conv = int(hist[0])

    def issue_roof(att, ms):
        # the double-float re-pass runs FP32 instructions: executed warp
        # instructions (ncu count per attempt) against one per clock per
        # scheduler, 4 per SM
        ipk = REPASS_DD_WARP_INSTR_PER_ATTEMPT
        peak_i = 4 * sms * f_mhz * 1e6 / 1e9
        if ipk is None or ms <= 0:
            return dict(bound="issue", achieved=None, peak=peak_i, unit="G warp instr/s", frac=None,
                        basis="no ncu count of the current double-float kernel")
        ach = ipk * att / (ms / 1e3) / 1e9
        return dict(bound="issue", achieved=ach, peak=peak_i, unit="G warp instr/s", frac=ach / peak_i,
                    basis="%.0f warp instructions per step attempt x %d attempts / the re-pass time (ordering + "
                          "double-float kernel); peak 4 warp instructions per clock per SM" % (ipk, att))

    # the FP64 kernels against the FP64 issue rate of their instruction mix:
    # executed FP64 instructions per unit (ncu counts, constants above) x
    # units / time, over the rate at which the SMs issue that mix of DADD,
    # DMUL and DFMA (each kind at its measured rate)
    def mix_peak(mix):
        per_clk = sum(mix) / sum(n / r for n, r in zip(mix, (rates["dadd"], rates["dmul"], rates["dfma"])))
        return per_clk * sms * f_mhz * 1e6 / 1e9

    def fp64_roof(instr, ms, what, mix):
        peak_m = mix_peak(mix)
        ach = instr / (ms / 1e3) / 1e9 if ms > 0 else 0.0
        return dict(bound="fp64", achieved=ach, peak=peak_m, unit="G FP64 instr/s", frac=ach / peak_m,
                    basis=what)

    solves = S * I * ws
    value = solves * args.steps / (elapsed_ms / 1e3)

    # end to end through the C ABI with host buffers: every step creates its
    # handle from the host edge list, runs the path and copies every result
    # back to pinned host memory.  Two sets of output buffers: step k's
    # results go to the host on a second stream while step k+1 computes; the
    # handles are closed once the last results are in (closing frees device
    # memory, which waits for the device).
    def host_set():
        return dict(states=torch.empty((S, I, N), dtype=torch.float64, pin_memory=True),
                    status=torch.empty((S, I), dtype=torch.uint8, pin_memory=True),
                    sid=torch.empty((S, I), dtype=torch.int32, pin_memory=True),
                    nu=torch.empty((S,), dtype=torch.int32, pin_memory=True))
    hosts = [host_set(), host_set()]
    outs = [out, {k: (torch.empty_like(v) if v is not None else None) for k, v in out.items()}]
    dsets = [(sid, nu), (torch.empty_like(sid), torch.empty_like(nu))]
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [None, None]
    h2d = 4 * E * 2 + E
    d2h = sum(t.numel() * t.element_size() for t in hosts[0].values())

    def e2e_step(k, handles):
        b = k % 2
        o, (sd, nd), hb = outs[b], dsets[b], hosts[b]
        if copied[b] is not None:
            stream.wait_event(copied[b])        # step k-2's results have left these buffers
        hh = api.Racipe.from_topology(topo, device=dev)
        hh.sample_params(w["param_seed"], S, I, set0=set0, params=params, ic_unit=ic, stream=stream)
        hh.integrate(params, ic, opts=opts_p, stream=stream, out=o)             # with the polish
        hh.unique_states(params, o["states"], o["status"], stream=stream, out=(sd, nd))
        done = torch.cuda.Event()
        done.record(stream)
        copy_stream.wait_event(done)
        with torch.cuda.stream(copy_stream):
            hb["states"].copy_(o["states"], non_blocking=True)
            hb["status"].copy_(o["status"], non_blocking=True)
            hb["sid"].copy_(sd, non_blocking=True)
            hb["nu"].copy_(nd, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(copy_stream)
        copied[b] = ev
        handles.append(hh)

    warm = []
    e2e_step(0, warm)
    torch.cuda.synchronize()
    for hh in warm:
        hh.close()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 4))
    handles = []
    for k in range(e2e_steps):
        e2e_step(k, handles)
    torch.cuda.synchronize()
    for hh in handles:
        hh.close()
    barrier()
    e2e_s = shard.max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = solves * e2e_steps / e2e_s

    # the plain FP64 GPU solver (FP64 Dormand-Prince end to end, no polish)
    # on the same sets as the step (the whole workload by default), for the
    # FP32 + polish ratio
    f64_sets = max(1, min(S, args.fp64_sets))
    opts64 = api.default_opts(precision=api.GRINS_FP64, polish=0, **TOL)
    out64 = {k: (v[:f64_sets] if v is not None else None) for k, v in out.items()}
    h.integrate(params[:min(f64_sets, 2000)], ic, opts=opts64, stream=stream,
                out={k: (v[:min(f64_sets, 2000)] if v is not None else None) for k, v in out.items()})
    e64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    barrier()
    e64[0].record(stream)
    h.integrate(params[:f64_sets], ic, opts=opts64, stream=stream, out=out64)
    e64[1].record(stream)
    barrier()
    fp64_ms = e64[0].elapsed_time(e64[1])
    fp64_value = f64_sets * I / (fp64_ms / 1e3)
    a64 = int(out64["n_steps"].sum().item())        # the FP64 solver's step attempts
    if snap is not None and f64_sets >= snap["n_unique"].shape[0]:
        # the plain FP64 solver's statuses and distinct-state counts on the
        # oracle's sets (polished and deduplicated as the FP32 path is)
        P = snap["n_unique"].shape[0]
        o64 = {k: (v[:P] if v is not None else None) for k, v in out.items()}
        h.polish(params[:P], o64["states"], o64["status"], o64["err_est"], opts=popts, stream=stream)
        h.unique_states(params[:P], o64["states"], o64["status"], stream=stream, out=(sid[:P], nu[:P]))
        snap.update(fp64_status=o64["status"].cpu().numpy(), fp64_n_unique=nu[:P].cpu().numpy())

    if rank == 0:
        line = dict(
            metric=METRIC,
            value=value, unit="solves/s", n_gpus=ws, steps=args.steps, warmup=max(3, args.warmup),
            ms_per_step=elapsed_ms / args.steps, higher_is_better=True, scaling="weak",
            vs_baseline=None, dtype="f32", data="synthetic",
            config=dict(workload="rand22x82: seeded random signed network, 22 nodes, 82 edges "
                                 "(33 inhibitory, 3 self-activations); %d sets x %d ICs per GPU" % (S, I),
                        solver="Dormand-Prince 5(4) FP32, rtol 1e-6, atol 1e-9, t_end 200, "
                               "ss_tol 1e-6; FP64 Newton polish; dedupe tol 1e-2",
                        l2="inputs larger than L2: parameter block %.0f MB, states %.0f MB" % (
                            S * h.param_stride / 1e6, S * I * N * 8 / 1e6),
                        parallelism="dp%d (sets sharded by rank)" % ws),
            kernel_ms=dict(sample=kern_ms[0], integrate_fp32=kern_ms[1], repass_and_polish=kern_ms[2] + kern_ms[3],
                           unique=kern_ms[4],
                           apart=dict(repass=sep_ms[2], polish_fp64=sep_ms[3],
                                      what="one more step with the polish as its own call after the re-pass "
                                           "(in the timed steps the polish runs beside the re-pass)")),
            step_attempts_per_solve=attempts / (S * I),
            repass=dict(solves=n_tail, share=n_tail / (S * I), attempts=a_tail, ms=sep_ms[2],
                        precision="FP64" if opts.tail_precision == api.GRINS_TAIL_FP64 else "double-float",
                        what="solves whose steady-state decision fell near t_end, re-integrated at rtol %g from "
                             "their first state with residual below %g ss_tol (ordering kernel + re-pass "
                             "kernel)" % (opts.tail_rtol, opts.tail_start)),
            status_hist=hist.tolist(),
            roofline=dict(bound="alu", achieved=achieved, peak=peak, unit=unit, frac=achieved / peak,
                          traffic=(INTEGRATOR_DRAM_BYTES_PER_SOLVE * S * I
                                   if INTEGRATOR_DRAM_BYTES_PER_SOLVE else None), kernel=kernel_desc,
                          peak_basis="%d SMs x %.2f %s/clk/SM x %.0f MHz (median SM clock sampled in the "
                                     "timed region); per-clock rates measured on this GPU by grins_unit_rates"
                                     % (sms, sfu_rate if sfu_bound else fma_rate,
                                        "rcp.approx" if sfu_bound else "FFMA", f_mhz),
                          unit_rates_per_clk_per_sm=rates,
                          work_per_attempt=dict(fp32=w32, sfu=wsfu)),
            secondary_rooflines=dict(
                polish=fp64_roof(POLISH_FP64_INSTR_PER_SOLVE * (n_conv + int(hist[4])), sep_ms[3],
                                 "%.0f FP64 instructions per polished solve x %d solves / the polish kernel's "
                                 "time" % (POLISH_FP64_INSTR_PER_SOLVE, n_conv + int(hist[4])), POLISH_FP64_MIX),
                repass=(fp64_roof(REPASS_FP64_INSTR_PER_ATTEMPT * a_tail, sep_ms[2],
                                  "%.0f FP64 instructions per FP64 step attempt x %d attempts / the re-pass "
                                  "time (ordering + FP64 kernel)" % (REPASS_FP64_INSTR_PER_ATTEMPT, a_tail),
                                  REPASS_FP64_MIX)
                        if opts.tail_precision == api.GRINS_TAIL_FP64 else issue_roof(a_tail, sep_ms[2])),
                unique=fp64_roof(UNIQUE_FP64_INSTR_PER_SOLVE * n_conv, kern_ms[4],
                                 "%.0f FP64 instructions per converged solve x %d solves / the dedupe "
                                 "kernel's time" % (UNIQUE_FP64_INSTR_PER_SOLVE, n_conv), UNIQUE_FP64_MIX),
                peak_basis="%d SMs x the kernel's DADD/DMUL/DFMA mix at %.2f / %.2f / %.2f per clk per SM "
                           "(grins_unit_rates) x %.0f MHz" % (sms, rates["dadd"], rates["dmul"], rates["dfma"],
                                                             f_mhz)),
            e2e=dict(value=e2e_value, unit="solves/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                     first_step_s=first_step_s,
                     steps=e2e_steps,
                     note="steady state: each timed step creates its handle, but the process-wide caches "
                          "(compiled kernels, median table) are warm; step k's results are copied to the "
                          "host on a second stream while step k+1 computes (two buffer sets), every copy "
                          "inside the timed region; first_step_s is the first step of the process, with "
                          "the median table and the run-time compiles"),
            # per step: parameter and IC samplers, FP32 pass, re-pass ordering
            # and kernel, the polish beside it and the list-mode polish after
            # it, dedupe
            gpu_launches=(8 if opts.tail_rtol > 0 else 5) * args.steps,
            fp64_gpu_solver=dict(value=fp64_value, unit="solves/s", ms=fp64_ms,
                                 sample="sets 0..%d x %d ICs (the step's sets), FP64 Dormand-Prince 5(4) on the "
                                        "GPU, same tolerances, no polish" % (f64_sets - 1, I),
                                 ratio=value / fp64_value, step_attempts_per_solve=a64 / (f64_sets * I),
                                 roofline=fp64_roof(REPASS_FP64_INSTR_PER_ATTEMPT * a64, fp64_ms,
                                                    "%.0f FP64 instructions per step attempt (the same FP64 "
                                                    "kernel body as the re-pass) x %d attempts / its time"
                                                    % (REPASS_FP64_INSTR_PER_ATTEMPT, a64), REPASS_FP64_MIX)),
            clocks=clocks)
        if levels is not None:
            line["levels"] = levels
        if tsit5 is not None:
            line["tsit5"] = tsit5
        if ising is not None:
            line["ising"] = ising
        if samplers is not None:
            line["samplers"] = samplers
        if args.batch_reps > 0 and ws == 1:
            line["batched"] = batched_measurement(dev, args.batch_reps, rates["rcp"], f_mhz)
        if args.serve_seconds > 0 and ws == 1:
            line["serving"] = serving_measurement(dev, args.serve_seconds, args.serve_rate, rates["rcp"], f_mhz)
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"], orc = cpu_baseline(args.cpu_sets)
            P = snap["G"].shape[0]
            orc = {kk: (v[:P] if hasattr(v, "shape") else v) for kk, v in orc.items()}
            import oracle as O
            pslice = O.ParamSet(snap["G"], snap["k"], snap["T"], snap["lam"], snap["n"].astype(np.int32))
            line["parity"] = dict(sets=P, solves=P * I, against="the oracle (FP64 CPU, rtol 1e-10, Newton "
                                  "polish) on the same sets", **parity_figures(snap, orc, snap["G"], snap["k"],
                                                                               pslice))
            line["parity"]["oracle_at_solver_tolerances"] = oracle_tolerance_floor(P, orc)
            line["parity"]["oracle_unpolished"] = oracle_unpolished_share(min(P, 200))
            # distinct-state counts on sets 0..9999 against the oracle's,
            # stored by tests/golden/make_net22_reference.py (which calls only
            # the oracle; too long to recompute here)
            from tests.golden import make_net22_reference as R
            ref_status, ref_nu = R.load()
            M = min(ref_nu.size, S)
            g_nu, g_st = snap["n_unique_all"][:M], snap["status_all"][:M]
            line["parity"]["n_unique_10k"] = dict(
                sets=M, agree=float((g_nu == ref_nu[:M]).mean()), mismatched_sets=int((g_nu != ref_nu[:M]).sum()),
                converged_status_agree=float(((g_st == 0) == (ref_status[:M] == 0)).mean()),
                against="the oracle's stored counts (tests/golden/net22_oracle_sets0_9999.txt.gz)")
        print(json.dumps(line))
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
