"""Benchmark: checkerboard Cabibbo-Marinari SU(3) heatbath sweeps on GB300.

Workload (one GPU): a 32^4 periodic lattice, beta = 6.0, Haar-random (hot)
start from the seed, FP32 12-real link storage with FP64 re-unitarisation
and FP64 measurement reductions, FHKP with 2 hits.  One step = 10 sweeps,
then a re-unitarisation and a plaquette + Polyakov-loop measurement (the
re-unitarise-every-10 cadence of the workload), all inside the library's
stage machine; 100 steps = the 1000-sweep run.  The links (201 MB) are
larger than the 129 MB L2, so no flush is needed between steps.

Metric: SU(3) link updates per second (whole job over all ranks).
With --gpus N > 1 every rank runs its own chain (replicas: the method needs
no exchange between independent chains), weak scaling.

--impl reference times the plain double-precision CPU oracle on this
workload (a bounded slice of it per step) on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DIMS = [32, 32, 32, 32]
BETA = 6.0
HITS = 2
SWEEPS_PER_STEP = 10
SEED = 20090406
METRIC = "SU(3) link updates/s"
UNIT = "link updates/s"
WORKLOAD = "32^4 PBC SU(3) Wilson, beta=6.0, hot start, CM heatbath with FHKP 2 hits, FP32 12-real links, " \
           "FP64 reunitarize + plaquette/Polyakov every 10 sweeps; step = 10 sweeps"


def nlinks():
    n = 1
    for d in DIMS:
        n *= d
    return n * len(DIMS)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_hash():
    """Hash of the kernel sources with comments and blank lines removed, so
    that recorded ncu counters stay valid across comment edits."""
    h = hashlib.sha256()
    for f in ("su3_device.cuh", "su3_kernels.cu", "su3_engine.h"):
        with open(os.path.join(ROOT, "paper_0904_0642_gb300", "csrc", f)) as fh:
            src = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for ln in src.splitlines():
            ln = ln.split("//", 1)[0].rstrip()
            if ln:
                h.update(ln.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    h = kernel_hash()
    for ln in lines:
        t = ln.split()
        if len(t) >= 3 and not ln.startswith("#") and t[0] == kernel and t[1] == h:
            return float(t[2])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        return False

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for ln in open(self.path):
            t = [x.strip() for x in ln.split(",")]
            if len(t) < 9:
                continue
            try:
                rows.append((float(t[1]), float(t[2]), float(t[3]), t[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        loaded = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[2] for r in rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle as the reference arm: each step updates one bounded slice
    (2^17 sites of one checkerboard colour, i.e. 65536 links) of the 32^4
    hot-start lattice in double precision on one host core."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    lat = oracle.Lattice(DIMS).hot_start(SEED)
    slice_sites = 1 << 17
    V = lat.V
    ups = []
    t_total = 0.0
    for step in range(args.warmup + args.steps):
        colour = step % 2
        mu = (step // 2) % 4
        s0 = (step * slice_sites) % V
        t0 = time.perf_counter()
        prop, acc = lat.phase(BETA, HITS, SEED, sweep=0, colour=colour, mu=mu, s_begin=s0, s_end=s0 + slice_sites)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            t_total += dt
            ups.append(slice_sites // 2)
    value = sum(ups) / t_total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_step": "one FP64 oracle update of 65536 links "
                                                               "(one colour, one direction, 2^17 sites)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} slices of 65536 link updates of the 32^4 hot-start lattice"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """One full oracle sweep of the 32^4 hot-start lattice on one core, and
    the same sweep with the oracle's OpenMP loop over the sites of a phase
    on every host core (identical links)."""
    import oracle
    lat = oracle.Lattice(DIMS).hot_start(SEED)
    t0 = time.perf_counter()
    lat.sweep(BETA, HITS, SEED, n=1)
    dt = time.perf_counter() - t0
    out = {"value": lat.nlinks / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "one full sweep (4194304 link updates) of the 32^4 hot-start lattice, single thread, FP64",
           "seconds": dt}
    ncores = oracle.available_threads()
    if ncores > 1:
        lat = oracle.Lattice(DIMS).hot_start(SEED)
        oracle.set_threads(ncores)
        try:
            t0 = time.perf_counter()
            lat.sweep(BETA, HITS, SEED, n=1)
            dt = time.perf_counter() - t0
        finally:
            oracle.set_threads(1)
        out["all_cores"] = {"value": lat.nlinks / dt, "unit": UNIT, "cores": ncores, "seconds": dt,
                            "sample": "the same sweep, OpenMP over the sites of each phase"}
    return out


def graph_stage_times(su3, torch, stream, seed, step_ms):
    """Per-stage device times of the 32^4 step, all from CUDA-graph-timed
    runs (CUDA events on the lattice's stream), so that they add up to the
    timed step: a lattice re-unitarised every 10 sweeps runs 80 update ticks
    + 1 re-unitarisation per 10-sweep call (T10), one re-unitarised every 20
    sweeps 160 + 1 per 20-sweep call (T20); neither measures.  Then
    update tick = (T20 - T10) / 80, re-unitarisation = T10 - 80 x tick (it
    carries the call's one-block arm kernel), measurement = step - T10.
    T10 and T20 are each the fastest of three alternating timings: a single
    pair moved the derived tick by ~1 us between runs."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lats = {}
    for every in (10, 20):
        lats[every] = su3.Lattice(DIMS, beta=BETA, seed=seed, hits=HITS, storage=su3.SU3_FP32_12,
                                  start=su3.SU3_START_HOT, reunit_every=every, stream=stream)
        lats[every].autotune()
        lats[every].sweep(every)
    per_call = {10: float("inf"), 20: float("inf")}
    for _ in range(3):
        for every, calls in ((10, 12), (20, 6)):
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(calls):
                lats[every].sweep(every)
            e1.record(stream)
            torch.cuda.synchronize()
            per_call[every] = min(per_call[every], e0.elapsed_time(e1) / calls)
    for lat in lats.values():
        lat.close()
    ticks = 2 * len(DIMS) * SWEEPS_PER_STEP
    tick_ms = (per_call[20] - per_call[10]) / ticks
    reunit_ms = per_call[10] - ticks * tick_ms
    return {"update_tick_us": 1e3 * tick_ms, "reunit_us": 1e3 * reunit_ms,
            "measure_us": 1e3 * (step_ms - per_call[10]), "T10_ms": per_call[10], "T20_ms": per_call[20],
            "sum_ms": ticks * tick_ms + reunit_ms + (step_ms - per_call[10]), "step_ms": step_ms}


# ---------------------------------------------------------------- other workloads
# Each is reported as an extra key of the bench line (same JSON line).


def bench_ensemble(su3, torch, stream, peaks):
    """256 independent 8^4 chains, beta_c ~ U[5.5, 6.5], FP32, one fused
    persistent launch per phase, graph-captured, autotuned; against the same
    chains swept one after another as single-chain lattices."""
    import numpy as np
    rng = np.random.default_rng(2009)
    betas = rng.uniform(5.5, 6.5, 256)
    sweeps = 200
    cfgs = [su3.make_config([8, 8, 8, 8], beta=float(b), seed=5000 + c, storage=su3.SU3_FP32_12,
                            start=su3.SU3_START_HOT, hits=HITS, reunit_every=10) for c, b in enumerate(betas)]
    ens = su3.Ensemble(cfgs, stream=stream)
    var, thr, ctas, _ = ens.autotune()
    ens.sweep(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ens.sweep(sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_ens = e0.elapsed_time(e1) * 1e-3
    links = 256 * 8 ** 4 * 4
    # the update ticks' share of the graph-timed run: the run's re-unitarisation
    # ticks (every 10 sweeps) are timed with per-tick events and taken out
    ens.set_profiling(True)
    ens.profile(reset=True)
    ens.sweep(10)
    prof = ens.profile(reset=True)
    ens.set_profiling(False)
    reunit_ms = prof["reunit_ms"] / max(1, prof["reunit_launches"])
    n_upd = sweeps * 2 * 4
    tick_s = (1e3 * t_ens - (sweeps // 10) * reunit_ms) / n_upd * 1e-3
    alg = 256 * (8 ** 4 // 2) * (2 * 4 + 1) * 48
    # 256 sequential single-chain runs (fewer sweeps each, same per-sweep work)
    seq_sweeps = 20
    lats = [su3.Lattice([8, 8, 8, 8], beta=float(b), seed=5000 + c, storage=su3.SU3_FP32_12,
                        start=su3.SU3_START_HOT, hits=HITS, reunit_every=10, stream=stream)
            for c, b in enumerate(betas)]
    for lat in lats:
        lat.sweep(1)
    torch.cuda.synchronize()
    e0.record(stream)
    for lat in lats:
        lat.sweep(seq_sweeps)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) * 1e-3
    for lat in lats:
        lat.close()
    meas = ens.measure()
    ens.close()
    fused = sweeps * links / t_ens
    seq = seq_sweeps * links / t_seq
    return {"workload": "256 chains of 8^4 PBC, beta ~ U[5.5,6.5], FP32, 200 sweeps, fused + graph",
            "value": fused, "unit": UNIT, "sequential_single_chain": seq, "speedup": fused / seq,
            "launch": {"variant": var, "threads": thr, "ctas_per_sm": ctas},
            "update_tick_us": tick_s * 1e6, "alg_bytes_per_update_tick": alg,
            "achieved_gbs": alg / tick_s / 1e9, "hbm_frac": alg / tick_s / 1e9 / peaks["hbm_gbs"],
            "tick_source": "graph-timed 200 sweeps minus 20 event-timed re-unitarisation ticks, over 1600 "
                           "update ticks (524288 link updates x (2D+1) x 48 B each)",
            "plaquette_mean": float(meas[:, 0].mean())}


def bench_divided(su3, torch, stream):
    """The 32^4 workload on a lattice cut into 2^4 sublattice boxes with
    halo exchange (the paper's MPI decomposition, on one device), against
    the undivided lattice: 10 sweeps + re-unitarisation per step."""
    out = {}
    for name, ndiv in (("undivided", [1, 1, 1, 1]), ("2x2x2x2", [2, 2, 2, 2])):
        lat = su3.Lattice(DIMS, beta=BETA, seed=SEED, hits=HITS, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                          reunit_every=SWEEPS_PER_STEP, ndiv=ndiv, stream=stream)
        lat.autotune()
        lat.sweep(SWEEPS_PER_STEP)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            lat.sweep(SWEEPS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = 3 * SWEEPS_PER_STEP * lat.nlinks / (e0.elapsed_time(e1) * 1e-3)
        lat.close()
    return {"workload": "32^4 PBC beta=6 FP32, cut into 2x2x2x2 sublattice boxes (16^4 interiors + halos)",
            "value": out["2x2x2x2"], "unit": UNIT, "undivided": out["undivided"],
            "ratio": out["2x2x2x2"] / out["undivided"]}


def bench_fp32_18(su3, torch, stream, peaks):
    """The 32^4 workload with all 18 reals of every link stored in float (72
    bytes a link instead of 48: row 3 is loaded, not rebuilt): throughput of
    the step and of the update kernel against the HBM peak, with its own
    algorithmic bytes (2D + 1) x 72 per update."""
    lat = su3.Lattice(DIMS, beta=BETA, seed=SEED, hits=HITS, storage=su3.SU3_FP32_18, start=su3.SU3_START_HOT,
                      reunit_every=SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP, stream=stream)
    var, thr, ctas, _ = lat.autotune()
    lat.sweep(SWEEPS_PER_STEP)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(3):
        lat.sweep(SWEEPS_PER_STEP)
    e1.record(stream)
    torch.cuda.synchronize()
    value = 3 * SWEEPS_PER_STEP * lat.nlinks / (e0.elapsed_time(e1) * 1e-3)
    lat.set_profiling(True)
    lat.profile(reset=True)
    lat.sweep(SWEEPS_PER_STEP)
    prof = lat.profile(reset=True)
    upd_us = 1e3 * prof["update_ms"] / max(1, prof["update_launches"])
    alg = (lat.nlinks // len(DIMS) // 2) * (2 * len(DIMS) + 1) * 72
    plaq = lat.plaquette()[0]
    lat.close()
    return {"workload": "32^4 PBC beta=6 hot start, FP32 18-real storage, 10 sweeps + re-unitarisation per step",
            "value": value, "unit": UNIT, "update_us": upd_us, "alg_bytes_per_update_launch": alg,
            "hbm_frac": alg / (upd_us * 1e-6) / 1e9 / peaks["hbm_gbs"], "plaquette": plaq,
            "launch": {"variant": var, "threads": thr, "ctas_per_sm": ctas}}


def bench_dlt_and_d3(su3, torch, stream):
    out = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, kw, sweeps in (
            ("dlt_2x16^3x4_time_glued_b5.7", dict(dims=[16, 16, 16, 4], boundary=su3.SU3_DLT, glue_mask=0b1000,
                                                   beta=5.7), 500),
            ("pbc_64^3_d3_b10", dict(dims=[64, 64, 64], beta=10.0), 500)):
        lat = su3.Lattice(storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, seed=SEED, hits=HITS, reunit_every=10,
                          stream=stream, **kw)
        var, thr, ctas, _ = lat.autotune()
        lat.sweep(5)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.sweep(sweeps)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        rec = {"value": sweeps * lat.nlinks / t, "unit": UNIT, "sweeps": sweeps, "links": lat.nlinks,
               "launch": {"variant": var, "threads": thr, "ctas_per_sm": ctas}}
        for layer in range(lat.nlayers):
            p = lat.plaquette(layer)
            q = lat.polyakov(layer)
            rec[f"layer{layer}"] = {"plaquette": p[0], "space": p[1], "time": p[2], "polyakov": [q.real, q.imag]}
        out[name] = rec
        lat.close()
    return out


SERVE_SHAPES = [[8, 8, 8, 8], [12, 12, 12, 12], [16, 16, 16, 4], [24, 24, 24, 24], [32, 32, 32, 8], [48, 48, 48]]


def serving_jobs(su3, n, rate, seed):
    """n jobs with Poisson arrivals at `rate` per second: shape uniform over
    the six serving shapes, DLT with probability 0.2, beta ~ U[5.6, 6.4],
    sweeps ~ U{50..500}; (arrival s, dims, boundary, beta, sweeps, seed)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    jobs, t = [], 0.0
    for j in range(n):
        t += rng.exponential(1 / rate)
        dims = SERVE_SHAPES[rng.integers(len(SERVE_SHAPES))]
        boundary = su3.SU3_DLT if rng.random() < 0.2 else su3.SU3_PBC
        jobs.append((t, dims, boundary, float(rng.uniform(5.6, 6.4)), int(rng.integers(50, 501)), 7000 + j))
    return jobs


def _links(su3, dims, boundary):
    n = len(dims) * (2 if boundary == su3.SU3_DLT else 1)
    for d in dims:
        n *= d
    return n


def serve_fp32(su3, jobs, peaks, window=(0.0, 1.0)):
    """The jobs through the continuous-batching server as they arrive.
    Latency = completion - submission (host clock).  p50 / p99 over the jobs
    whose arrival rank lies in `window` (a steady-state window excludes the
    ramp-up and ramp-down); throughput over the whole run; the HBM fraction
    over the device time of the server's rounds."""
    import numpy as np
    srv = su3.Server(max_slots=64)
    t0 = time.perf_counter()
    ids = []
    for (ta, dims, b, beta, sw, seed) in jobs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        cfg = su3.make_config(dims, boundary=b, beta=beta, seed=seed, storage=su3.SU3_FP32_12,
                              start=su3.SU3_START_HOT, hits=HITS, reunit_every=10)
        ids.append(srv.submit(cfg, sw))
    res = [srv.wait(j, timeout_s=900) for j in ids]
    t_all = time.perf_counter() - t0
    rounds, dev_ms = srv.stats()
    srv.close()
    lat_s = np.array([r.finish_s - r.submit_s for r in res])
    lo, hi = int(window[0] * len(jobs)), int(window[1] * len(jobs))
    upd = sum(_links(su3, d, b) * sw for (_, d, b, _, sw, _) in jobs)
    alg = sum(_links(su3, d, b) * sw * (2 * len(d) + 1) * 48 for (_, d, b, _, sw, _) in jobs)
    return {"jobs": len(jobs), "offered_jobs_per_s": len(jobs) / jobs[-1][0], "jobs_per_s": len(jobs) / t_all,
            "link_updates_per_s": upd / t_all, "latency_p50_s": float(np.percentile(lat_s[lo:hi], 50)),
            "latency_p99_s": float(np.percentile(lat_s[lo:hi], 99)), "latency_jobs": hi - lo,
            "rounds": rounds, "device_s": dev_ms * 1e-3, "achieved_gbs": alg / (dev_ms * 1e-3) / 1e9,
            "hbm_frac": alg / (dev_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "statuses_ok": all(r.status == su3.SU3_OK for r in res),
            "plaquettes": [float(r.plaquette[0]) for r in res]}


def serve_fp64_one_at_a_time(su3, torch, jobs):
    """The plain FP64 baseline under the same arrivals: one FP64 18-real
    single-chain lattice at a time, in arrival order; a job waits for the
    previous one.  Latency = completion - arrival, measured."""
    import numpy as np
    t0 = time.perf_counter()
    lat_s, plaq, busy = [], [], 0.0
    for (ta, dims, b, beta, sw, seed) in jobs:
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        s0 = time.perf_counter()
        lat = su3.Lattice(dims, boundary=b, beta=beta, seed=seed, storage=su3.SU3_FP64_18, start=su3.SU3_START_HOT,
                          hits=HITS, reunit_every=10)
        lat.sweep(sw)
        plaq.append(lat.plaquette()[0])  # synchronises
        lat.close()
        done = time.perf_counter()
        busy += done - s0
        lat_s.append(done - t0 - ta)
    upd = sum(_links(su3, d, b) * sw for (_, d, b, _, sw, _) in jobs)
    return {"jobs": len(jobs), "latency_p50_s": float(np.percentile(lat_s, 50)),
            "latency_p99_s": float(np.percentile(lat_s, 99)), "link_updates_per_s_busy": upd / busy,
            "plaquettes": plaq}


def bench_serving(su3, torch, peaks):
    """BASELINE config 5: Poisson arrivals of mixed jobs into the
    continuous-batching server (FP32 12-real links, FP64 re-unitarisation
    and reductions), against a plain FP64 one-job-at-a-time loop under the
    same arrivals."""
    import numpy as np
    out = {"workload": "Poisson jobs, shapes 8^4/12^4/16^3x4/24^4/32^3x8/48^3, 20% DLT, beta U[5.6,6.4], "
                       "50-500 sweeps, FP32 + FP64 reunitarize/reductions"}
    # the same 50 jobs at 50/s: served in FP32, and one at a time in FP64
    jobs50 = serving_jobs(su3, 50, 50.0, 50)
    a = serve_fp32(su3, jobs50, peaks)
    b = serve_fp64_one_at_a_time(su3, torch, jobs50)
    d = np.array(a.pop("plaquettes")) - np.array(b.pop("plaquettes"))
    out["fp32_50_jobs_at_50_per_s"] = a
    out["fp64_one_at_a_time_50_jobs_at_50_per_s"] = b
    # observable accuracy: the FP32 and FP64 chains of a job start alike but
    # decorrelate over tens of sweeps, so their final plaquettes are two
    # samples of the same distribution; their mean difference over the jobs
    # must be consistent with zero
    out["plaquette_fp32_minus_fp64"] = {"mean": float(d.mean()), "stderr": float(d.std(ddof=1) / np.sqrt(len(d))),
                                        "max_abs": float(np.abs(d).max())}
    # 500 jobs at 50/s: above the server's capacity (the queue grows; the
    # latencies include the growing wait)
    c = serve_fp32(su3, serving_jobs(su3, 500, 50.0, 51), peaks)
    c.pop("plaquettes")
    c["note"] = "offered load above capacity: no steady state, latencies include the growing queue"
    out["fp32_500_jobs_at_50_per_s"] = c
    # 500 jobs at 25/s: sustainable; latencies over the steady-state window
    # (arrival ranks 10 %..90 %)
    e = serve_fp32(su3, serving_jobs(su3, 500, 25.0, 52), peaks, window=(0.1, 0.9))
    e.pop("plaquettes")
    out["fp32_500_jobs_at_25_per_s"] = e
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / FP64 / roofline passes")
    ap.add_argument("--no-autotune", action="store_true", help="default launch shape (for profiler runs)")
    ap.add_argument("--variant", type=int, default=None, help="with --no-autotune: kernel variant")
    ap.add_argument("--threads", type=int, default=128, help="with --no-autotune: CTA width")
    ap.add_argument("--ctas", type=int, default=0, help="with --no-autotune: CTAs per SM (0: one per tile)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
        return

    import numpy as np
    import torch

    import paper_0904_0642_gb300 as su3

    from paper_0904_0642_gb300.replicas import Replicas

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    reps = Replicas("nccl", device=torch.device("cuda", local))
    barrier = reps.barrier
    max_over_ranks = reps.max

    stream = torch.cuda.Stream()
    lat = su3.Lattice(DIMS, beta=BETA, seed=reps.seed(SEED), hits=HITS, storage=su3.SU3_FP32_12,
                      start=su3.SU3_START_HOT, reunit_every=SWEEPS_PER_STEP, measure_every=SWEEPS_PER_STEP,
                      measure_capacity=4096, stream=stream)
    if args.no_autotune:
        variant, threads, ctas, us = (args.variant or 0), args.threads, args.ctas, None
        lat.set_launch(threads, ctas, variant=variant)
    else:
        variant, threads, ctas, us = lat.autotune()
    links = lat.nlinks
    for _ in range(args.warmup):
        lat.sweep(SWEEPS_PER_STEP)
    torch.cuda.synchronize()

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            lat.sweep(SWEEPS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms)
    value = world * args.steps * SWEEPS_PER_STEP * links / (ms_max * 1e-3)
    meas = lat.measurements()
    plaq_last = float(meas[-1, 1, 0]) if len(meas) else float("nan")
    launches = args.steps * (2 * len(DIMS) * SWEEPS_PER_STEP + 3)  # k_arm + 80 update + reunit + measure ticks

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": "x".join(map(str, DIMS)), "links": links,
                       "sweeps_per_step": SWEEPS_PER_STEP, "storage": "FP32 12-real", "hits": HITS, "beta": BETA,
                       "l2": "inputs larger than L2 (201 MB of links vs 129 MB L2); no flush",
                       "launch": {"variant": variant, "threads": threads, "ctas_per_sm": ctas,
                                  "autotune_us_per_sweep": us},
                       "graph": True, "parallelism": f"replicas x{world}"},
            "gpu_launches": launches, "plaquette_last": plaq_last}
    clocks = clk.summary()
    line["clocks"] = clocks

    if not args.no_extras:
        # Roofline of the dominant kernel, the update tick.  Its duration comes
        # from graph-timed runs (CUDA events on the launching stream, the
        # launch overlap of the timed step included), so that 80 ticks + the
        # re-unitarisation + the measurement add up to ms_per_step; the
        # per-tick event timing (each tick wrapped in its own events, which
        # loses the overlap of consecutive launches) is reported beside it.
        peaks, peak_src = measured_peaks()
        st = graph_stage_times(su3, torch, stream, reps.seed(SEED), ms_max / args.steps)
        lat.set_profiling(True)
        lat.profile(reset=True)
        lat.sweep(SWEEPS_PER_STEP)
        prof = lat.profile(reset=True)
        lat.set_profiling(False)
        upd_ms = st["update_tick_us"] * 1e-3
        V = links // len(DIMS)
        alg_bytes = (V // 2) * (2 * len(DIMS) + 1) * 48
        achieved = alg_bytes / (upd_ms * 1e-3) / 1e9
        line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": achieved / peaks["hbm_gbs"], "traffic": recorded_traffic("k_tick_fp32_update"),
                            "peak_source": f"hbm_gbs of {peak_src}", "kernel": "k_tick<StoreF32x12> update phase",
                            "alg_bytes_per_launch": alg_bytes, "avg_launch_us": upd_ms * 1e3,
                            "tick_source": "graph-timed: (T(20 sweeps, re-unitarised every 20) - T(10 sweeps, "
                                           "every 10)) / 80 update ticks",
                            "reunit_us": st["reunit_us"], "measure_us": st["measure_us"],
                            "stages_sum_ms": st["sum_ms"], "step_ms": st["step_ms"],
                            "event_timed_us": {
                                "update": 1e3 * prof["update_ms"] / max(1, prof["update_launches"]),
                                "reunit": 1e3 * prof["reunit_ms"] / max(1, prof["reunit_launches"]),
                                "measure": 1e3 * prof["measure_ms"] / max(1, prof["measure_launches"])}}

        # End to end through the C ABI: every step uploads that step's input
        # configuration from pinned host memory (su3_stage_links_ex on the
        # library's copy stream: the upload of step k+1 runs while step k
        # sweeps), applies it (su3_apply_links), runs the 10 sweeps +
        # re-unitarisation + measurement, and copies that step's plaquette
        # and Polyakov loop back to pinned host memory
        # (su3_measurement_latest_async, 80 bytes), which the host reads
        # while the next step runs; the last step's result is read before
        # the clock stops.  The
        # input is the two-row FP32 form of the configuration (12 floats per
        # link, the storage format of this workload); the canonical FP64
        # layout (18 doubles per link) is timed the same way beside it.
        canon = lat.get_links()
        k_e2e = max(3, args.steps // 5)

        def e2e_run(fmt):
            if fmt == su3.SU3_LINKS_FP32_12:
                host = torch.empty((links * 12,), dtype=torch.float32, pin_memory=True).numpy()
                host[:] = canon[..., :2, :, :].reshape(-1)
            else:
                host = torch.empty((links * 18,), dtype=torch.float64, pin_memory=True).numpy()
                host[:] = canon.reshape(-1)
            nres = 5 * (lat.nlayers + 1)
            outs = [torch.empty(nres, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
            evs = [torch.cuda.Event() for _ in range(2)]
            # untimed warm-up steps of the same cycle: the first copies from a
            # freshly pinned buffer ran at 40-55 GB/s against ~210 GB/s after
            for _ in range(2):
                lat.stage_links(host, fmt=fmt)
                lat.apply_links()
                lat.sweep(SWEEPS_PER_STEP)
                lat.latest_measurement_async(outs[0])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.stage_links(host, fmt=fmt)
            for k in range(k_e2e):
                lat.apply_links()
                lat.sweep(SWEEPS_PER_STEP)
                # the next input first: a copy queued behind this step's
                # result copy could wait for this step's sweeps
                if k + 1 < k_e2e:
                    lat.stage_links(host, fmt=fmt)
                lat.latest_measurement_async(outs[k % 2])  # this step's result, copied in stream order
                evs[k % 2].record(stream)
                if k >= 1:  # the previous step's result, read while this step runs
                    evs[(k - 1) % 2].synchronize()
                    result = outs[(k - 1) % 2].copy()
            evs[(k_e2e - 1) % 2].synchronize()
            result = outs[(k_e2e - 1) % 2].copy()
            t = max_over_ranks(time.perf_counter() - t0)
            # one upload alone (copy + apply + a synchronising read), for its bandwidth
            torch.cuda.synchronize()
            u0 = time.perf_counter()
            lat.stage_links(host, fmt=fmt)
            lat.apply_links()
            lat.stats()  # synchronises
            upload_s = time.perf_counter() - u0
            return {"value": world * k_e2e * SWEEPS_PER_STEP * links / t, "unit": UNIT,
                    "h2d_bytes_per_step": int(host.nbytes), "d2h_bytes_per_step": int(result.size) * 8,
                    "steps": k_e2e, "upload_apply_ms": 1e3 * upload_s}

        line["e2e"] = e2e_run(su3.SU3_LINKS_FP32_12)
        line["e2e"]["input"] = "pinned host, rows 1-2 of every link as FP32 (12 floats), copy stream overlapping the previous step"
        line["e2e_fp64_canonical_input"] = e2e_run(su3.SU3_LINKS_FP64_18)

        # Plain FP64 single chain, 18-real storage, same workload and seed.
        lat64 = su3.Lattice(DIMS, beta=BETA, seed=SEED + rank, hits=HITS, storage=su3.SU3_FP64_18,
                            start=su3.SU3_START_HOT, reunit_every=SWEEPS_PER_STEP, stream=stream)
        ref32 = su3.Lattice(DIMS, beta=BETA, seed=SEED + rank, hits=HITS, storage=su3.SU3_FP32_12,
                            start=su3.SU3_START_HOT, reunit_every=SWEEPS_PER_STEP, stream=stream)
        lat64.sweep(SWEEPS_PER_STEP)
        ref32.sweep(SWEEPS_PER_STEP)
        p64, s64, t64 = lat64.plaquette()
        p32, s32, t32 = ref32.plaquette()
        l64, l32 = lat64.polyakov(), ref32.polyakov()
        torch.cuda.synchronize()
        k64 = 3
        e0.record(stream)
        for _ in range(k64):
            lat64.sweep(SWEEPS_PER_STEP)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        line["fp64_single_chain"] = {"value": world * k64 * SWEEPS_PER_STEP * links / (ms64 * 1e-3), "unit": UNIT,
                                     "steps": k64, "storage": "FP64 18-real"}
        line["plaquette_fp32_vs_fp64_after_10_sweeps"] = {"fp32": p32, "fp64": p64, "abs_diff": abs(p32 - p64)}
        line["fp32_vs_fp64_after_10_sweeps"] = {  # same start and random numbers; every observable
            "plaquette": abs(p32 - p64), "space": abs(s32 - s64), "time": abs(t32 - t64),
            "polyakov": abs(l32 - l64), "polyakov_fp64": [l64.real, l64.imag]}
        ref32.close()
        lat64.close()
        if rank == 0 and world == 1:
            line["ensemble_256x8^4"] = bench_ensemble(su3, torch, stream, peaks)
            line["fp32_18_32^4"] = bench_fp32_18(su3, torch, stream, peaks)
            line["divided_32^4_2x2x2x2"] = bench_divided(su3, torch, stream)
            line.update(bench_dlt_and_d3(su3, torch, stream))
            line["serving"] = bench_serving(su3, torch, peaks)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    lat.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()


if __name__ == "__main__":
    main()
