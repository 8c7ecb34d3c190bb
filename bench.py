"""Throughput of the GRMHD predictor-corrector step on GB300.

A "step" is one full predictor-corrector cycle of the whole hot path over
the workload grid.  Default workload: the 128^3 Fishbone-Moncrief torus
around a Kerr black hole (a = 0.9375) in modified Kerr-Schild coordinates
(h = 0.3, R_out = 50), WENO5, FP64, poloidal field at beta = 100, 4% seeded
perturbation of u (synthetic, generated in-process).  The metric is
zone-cycles/s (zones advanced by one full cycle per second).  The timed
region is one grmhd_step call of K cycles, which replays a CUDA graph of one
cycle (what a caller of the library gets); a second pass over K cycles with
a CUDA event around each kernel class gives the roofline's per-kernel times.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torchrun, one process per GPU; every rank advances its own
replica (the single-grid path is not decomposed), scaling "weak".  Rank 0
prints one JSON line.  Besides the headline it carries the same workload in
the mixed-precision and float-float modes ("mixed", "float_float"), 64
uneven flat 2D grids stepped as one
batch against the same grids stepped one by one ("batched"), and the
mixed-precision error of 100 cycles of the 288x128x128 torus against the
FP64 path ("mixed_accuracy"), and a prefix of the serving workload's
request stream through the serving loop ("served": p50/p99 time-to-result,
aggregate zone-cycles/s, offered vs served load); --no-extras skips them.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "zone-cycles/s on 1 GB300 (FP64 vs mixed, single vs batched); served p50/p99"
UNIT = "zone-cycles/s"

WORKLOADS = {
    "torus128": dict(n=(128, 128, 128), recon=1, label="fm_torus_128x128x128_weno5_mks_fp64",
                     r_out=50.0),
    "torus288": dict(n=(288, 128, 128), recon=1, label="fm_torus_288x128x128_weno5_mks_fp64",
                     r_out=1000.0),
    "mode64": dict(n=(64, 64, 1), recon=0, label="linear_fast_mode_64x64_mc_fp64"),
}


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each FP64-bound kernel class on the 128^3 torus: the mean over the class's
# launches (the three directions of kp_recon and kp_face, both stages of
# kp_update) in the one-pass ncu launch list of the 2-cycle bench command.
# The figures hold while the kernel sources hash to src_hash; otherwise the
# bench reports the traffic as unknown (null).
NCU_TRAFFIC = {"src_hash": "5e804b7ef44b62a1",
               "torus128": {"recon": 187957174 + 238592572, "flux": 295317248 + 110696210,
                            "update": 727520073 + 204079488}}
# sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active of full ncu
# captures of single launches (kp_recon<0> and <1>, the X3 walk taken as X2's;
# kp_face<0,0>; kp_update): the hardware's view of the same kernels, as a
# fraction of the nominal 2 FP64 instructions per SM per clock
NCU_FP64_PIPE = {"torus128": {"recon": 0.858, "flux": 0.905, "update": 0.888}}


def kernel_source_hash():
    """Hash of the translation unit that compiles the step kernels (plan.cu,
    every header under csrc/, the public header): the measured kernels'
    source, not the host-side files that only launch or hold them."""
    import glob
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_10191_gb300", "csrc")
    files = [os.path.join(csrc, "plan.cu")] + sorted(glob.glob(os.path.join(csrc, "*.h")) +
                                                   glob.glob(os.path.join(csrc, "*.cuh")))
    files.append(os.path.join(ROOT, "include", "grmhd.h"))
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def make_problem(name, n3_override=None):
    from paper_2110_10191_gb300 import problems as pb
    w = WORKLOADS[name]
    if name == "mode64":
        return pb.linear_mode(64)
    n1, n2, n3 = w["n"]
    pr = pb.fm_torus(n1, n2, n3 if n3_override is None else n3_override, recon=w["recon"],
                     r_out=w["r_out"])
    if n3_override is not None:
        # same zone shape: a slab of n3_override of the n3 zones in phi
        pr.xmax = (pr.xmax[0], pr.xmax[1], 2 * math.pi * n3_override / n3)
    return pr


def faces_per_launch(n):
    """Faces computed by the flux kernel of each direction (flux-CT needs one
    extra transverse layer on each side)."""
    out = []
    for d in range(3):
        f = 1
        for e in range(3):
            f *= (n[e] + 1) if e == d else (n[e] + 2)
        out.append(f)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.lines = []

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[2][q].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(name, steps, count=True):
    """The oracle as it stands on a bounded sample of the workload: a slab of
    8 of the 128 zones in phi (same zones, same per-zone work), one warm-up
    step, then `steps` timed steps, single-threaded.  With count=True the
    counting build also gives the algorithmic FP64 operations per face of the
    flux phase and per zone-cycle."""
    import oracle
    oracle.build()
    n3s = 8 if WORKLOADS[name]["n"][2] > 8 else WORKLOADS[name]["n"][2]
    pr = make_problem(name, n3_override=n3s) if name != "mode64" else make_problem(name)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(1)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    zones = pr.n[0] * pr.n[1] * pr.n[2]
    out = {"value": zones * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "%d step(s) of a %dx%dx%d slab of the workload grid (same zones and "
                     "per-zone work), after 1 warm-up step, 1 thread" % ((steps,) + tuple(pr.n)),
           "seconds": dt}
    if count:
        c = oracle.Oracle(pr, counting=True)
        c.set_prims(pr.P)
        c.step(1)
        oracle.op_counts(reset=True)
        c.step(1)
        ops = oracle.op_counts(reset=True)
        faces = 2 * sum(faces_per_launch(pr.n))  # two stages
        tot = {k: sum(v.values()) for k, v in ops.items()}
        out["_face_flops_per_face"] = tot["flux"] / faces
        out["_recon_flops_per_face"] = tot["recon"] / faces
        out["_update_flops_per_zone_stage"] = tot["update"] / (2 * zones)
        out["_flops_per_zone_cycle"] = sum(tot.values()) / zones
    return out


def _oracle_slab_worker(name, steps, barrier, out_q):
    """One host core's share of the all-cores oracle baseline: the same slab
    sample as cpu_oracle_sample, timed after a barrier with the others."""
    import oracle
    n3s = 8 if WORKLOADS[name]["n"][2] > 8 else WORKLOADS[name]["n"][2]
    pr = make_problem(name, n3_override=n3s) if name != "mode64" else make_problem(name)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(1)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(steps)
    out_q.put((time.perf_counter() - t0, pr.n[0] * pr.n[1] * pr.n[2]))


def cpu_oracle_all_cores(name, steps):
    """The oracle as it stands on every host core this process may use: one
    slab sample per core in separate processes (started with spawn, so no
    CUDA state is inherited), all timed together; aggregate = the zone-cycles
    of all slabs / the slowest slab's time."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    q = ctx.Queue()
    procs = [ctx.Process(target=_oracle_slab_worker, args=(name, steps, barrier, q))
             for _ in range(cores)]
    for p in procs:
        p.start()
    res = [q.get(timeout=900) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    wall = max(r[0] for r in res)
    zones = res[0][1]
    return {"value": cores * zones * steps / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d independent %d-step samples of the same slab, one process per core, "
                      "timed together (aggregate over the slowest)" % (cores, steps),
            "seconds": wall}


def reference_arm(args, rank, world):
    """--impl reference: the oracle, timed on the host cores, one bounded
    sample (a slab of the workload) per step."""
    if rank != 0:
        return
    name = args.config
    import oracle
    oracle.build()
    n3s = 8 if WORKLOADS[name]["n"][2] > 8 else WORKLOADS[name]["n"][2]
    pr = make_problem(name, n3_override=n3s) if name != "mode64" else make_problem(name)
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    zones = pr.n[0] * pr.n[1] * pr.n[2]
    v = zones * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(name),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: one cycle of a %dx%dx%d slab of the workload "
                                       "grid, 1 thread" % tuple(pr.n)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def reduce_max(x, world, device):
    """The maximum of x over the ranks of the default process group (the
    slowest rank's time); x itself when world == 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(zones_per_rank, steps, world, seconds):
    """Whole-job zone-cycles/s: every rank advances its own replica of
    zones_per_rank zones by `steps` cycles; seconds is the slowest rank's."""
    return world * zones_per_rank * steps / seconds


def _timed(stream, fn):
    """Device time (ms) of the work fn enqueues on stream."""
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


PREC_DTYPE = {
    1: "mixed: FP32 reconstruction, fluid states, signal speeds, LLF fluxes; "
       "FP64 geometry, flux-CT, update, 1D_W inversion, bounds",
    3: "mixed + float-float update: FP32 reconstruction, fluid states, signal speeds, LLF "
       "fluxes; float-float U(P), geometric source and 1D_W inversion; FP64 state, geometry, "
       "flux divergence, flux-CT, bounds",
    2: "float-float: reconstruction, fluid states, signal speeds, LLF fluxes, U(P), geometric "
       "source and 1D_W inversion in pairs of FP32 words (~48 significant bits); FP64 state, "
       "geometry, flux divergence, flux-CT, bounds",
}


def mixed_throughput(grmhd, pr, steps, warmup, stream, precision=1):
    """The same workload in the mixed-precision (1) or float-float (2) mode,
    with the device time of each kernel class."""
    import dataclasses
    pm = dataclasses.replace(pr, precision=precision)
    s = grmhd.Sim(pm, stream=stream)
    s.set_prims(pm.P)
    s.step(warmup)
    ms = _timed(stream, lambda: s.step(steps, sync=False))
    s.profile(True)
    s.get_profile(reset=True)
    s.step(2, sync=False)
    prof = s.get_profile(reset=True)
    s.close()
    z = pr.n[0] * pr.n[1] * pr.n[2]
    return {"value": z * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "dtype": PREC_DTYPE[precision], "steps": steps,
            "kernel_ms_per_step": {k: v[0] / 2 for k, v in prof.items()}}


def variant_throughput(grmhd, pr, steps, warmup, stream, what):
    """The FP64 workload with a variant switched on: the bounds in the drift
    frame ("drift") or electron entropies with the Kawazura heating model
    ("electrons"), with the device time of each kernel class."""
    pv = apply_variant(pr, what)
    if what == "drift":
        desc = "bounds in the drift frame (floor parcel added in U and inverted)"
    else:
        desc = ("electron entropies carried with the mass, Kawazura et al. heating, "
                "T_p/T_e in [1e-3, 1e3], P_gas/rho^gamma <= 3")
    s = grmhd.Sim(pv, stream=stream)
    s.set_prims(pv.P)
    if pv.electrons:
        s.set_electrons(pv.K)
    s.step(warmup)
    ms = _timed(stream, lambda: s.step(steps, sync=False))
    s.profile(True)
    s.get_profile(reset=True)
    s.step(2, sync=False)
    prof = s.get_profile(reset=True)
    st = s.stats()
    s.close()
    z = pr.n[0] * pr.n[1] * pr.n[2]
    return {"variant": desc, "value": z * steps / (ms * 1e-3), "unit": UNIT,
            "ms_per_step": ms / steps, "dtype": "f64", "steps": steps,
            "floor_hits": st["floor_hits"], "inv_failures": st["inv_failures"],
            "kernel_ms_per_step": {k: v[0] / 2 for k, v in prof.items()}}


def decomposed(grmhd, pr, steps, warmup, stream, nblocks=(2, 2, 2)):
    """The FP64 workload split into blocks on one GPU (the paper's domain
    decomposition; bitwise the whole grid): cycle time against the whole
    grid's, i.e. the cost of the edge exchanges and the shared time step."""
    d = grmhd.Decomp(pr, nblocks, stream=stream)
    d.set_prims(pr.P)
    d.step(warmup)
    ms = _timed(stream, lambda: d.step(steps)) / steps
    d.close()
    z = pr.n[0] * pr.n[1] * pr.n[2]
    return {"blocks": list(nblocks), "ms_per_step": ms, "value": z / (ms * 1e-3), "unit": UNIT,
            "steps": steps}


def small_single(grmhd, steps, stream):
    """The 64x64 fast mode (the accuracy workload, far too small to fill the
    GPU) stepped alone: one grmhd_step call of `steps` cycles (a graph
    replay per cycle) against `steps` calls of one cycle (one host launch per
    kernel)."""
    import dataclasses
    pr = dataclasses.replace(make_problem("mode64"), t_final=0.0)  # no end time: every cycle works
    out = {}
    for graph in (True, False):
        s = grmhd.Sim(pr, stream=stream)
        s.set_prims(pr.P)
        s.step(3)
        if graph:
            out[graph] = _timed(stream, lambda: s.step(steps, sync=False)) / steps
        else:
            out[graph] = _timed(stream, lambda: [s.step(1, sync=False) for _ in range(steps)]) / steps
        s.close()
    z = pr.n[0] * pr.n[1] * pr.n[2]
    return {"workload": WORKLOADS["mode64"]["label"], "steps": steps,
            "graph_ms_per_step": out[True], "direct_ms_per_step": out[False],
            "graph_value": z / (out[True] * 1e-3), "unit": UNIT,
            "speedup": out[False] / out[True]}


def batched_throughput(grmhd, steps, warmup, stream, nmin=32, nmax=256):
    """64 uneven flat 2D grids (slow/Alfven/fast modes, Orszag-Tang) stepped
    as one batch (one CUDA graph per step), before and after the autotuner,
    and, for comparison, one after the other as single simulations."""
    from paper_2110_10191_gb300 import problems as pb
    probs = pb.batch_2d(ngrid=64, nmin=nmin, nmax=nmax, seed=0)
    zones = sum(p.zones for p in probs)
    sims = [grmhd.Sim(p, stream=stream) for p in probs]
    for s, p in zip(sims, probs):
        s.set_prims(p.P)
        s.step(warmup, sync=False)
    ms_single = _timed(stream, lambda: [s.step(steps, sync=False) for s in sims])
    b = grmhd.Batch(sims)
    b.step(warmup, graph=True, sync=True)
    ms_untuned = _timed(stream, lambda: b.step(steps, graph=True))
    b.autotune(trials=3)
    b.step(1, graph=True, sync=True)
    l0 = b.info()["launches"]
    ms_batch = _timed(stream, lambda: b.step(steps, graph=True))
    info = b.info()
    b.close()
    for s in sims:
        s.close()
    return {"workload": "64 flat periodic 2D grids, N uniform in [%d, %d] (seed 0), equal shares of "
                        "slow/Alfven/fast linear modes and Orszag-Tang vortices, MC or WENO5 per grid"
                        % (nmin, nmax),
            "zones": zones, "value": zones * steps / (ms_batch * 1e-3), "unit": UNIT,
            "ms_per_step": ms_batch / steps, "launches_per_step": info["launches_per_step"],
            "gpu_launches": info["launches"] - l0, "cuda_graph": bool(info["graph"]),
            "autotuned": bool(info["tuned"]), "untuned_ms_per_step": ms_untuned / steps,
            "singles_value": zones * steps / (ms_single * 1e-3),
            "singles_ms_per_step": ms_single / steps,
            "speedup_vs_singles": ms_single / ms_batch, "steps": steps}


def serving_run(grmhd, nreq, zone_cap, quantum, policy=0):
    """The serving workload: the first `nreq` requests of the 200-request
    Poisson stream (4/s; 60% tori a ~ U[0, 0.98], N^3, N ~ U{64..192}; 40%
    Bondi, N^3, N ~ U{96..160}; 20..200 cycles; FP64 / mixed 50/50) submitted to
    the serving loop at their arrival times.  Time-to-result runs from the
    scheduled arrival to the result in host memory."""
    import numpy as np
    from paper_2110_10191_gb300 import problems as pb
    stream = pb.serving_stream(nreq=200, rate=4.0, seed=0)[:nreq]
    srv = grmhd.Server(max_active_zones=zone_cap, quantum=quantum, policy=policy)
    t0 = srv.now()
    results = []

    def collect(wait_ms):
        for r in srv.poll(64, wait_ms=wait_ms):
            r.pop("P", None)
            results.append(r)

    work = 0.0
    late = 0.0
    for r in stream:
        while srv.now() - t0 < r["t_arrival"]:
            collect(int(max(1, min(50, 1e3 * (r["t_arrival"] - (srv.now() - t0))))))
        pr = pb.serving_problem(r)
        late = max(late, srv.now() - t0 - r["t_arrival"])
        srv.submit(r["id"], pr, r["steps"], t_arrival=t0 + r["t_arrival"])
        work += float(pr.zones) * r["steps"]
        del pr
    while len(results) < len(stream):
        collect(200)
    st = srv.stats()
    srv.close()
    lat = np.array([r["t_done"] - r["t_arrival"] for r in results])
    end = max(r["t_done"] for r in results) - t0
    span = stream[-1]["t_arrival"]
    ok = sum(1 for r in results if r["status"] in (0, -4))
    return {"workload": "first %d of 200 Poisson requests at 4/s (seed 0): 60%% FM tori (a ~ U[0, 0.98], "
                        "N^3, N ~ U{64..192}), 40%% Bondi (N^3, N ~ U{96..160}), 20..200 cycles, "
                        "FP64/mixed 50/50" % nreq,
            "requests": len(stream), "completed": ok,
            "failed_zones_reported": sum(1 for r in results if r["status"] == -4),
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "max_s": float(lat.max()),
            "aggregate_value": st["zone_cycles"] / end, "unit": UNIT,
            "offered_load": work / span, "served_load": work / end,
            "zone_cycles": st["zone_cycles"], "seconds": end, "gpu_busy_fraction": st["busy_seconds"] / end,
            "max_submission_lag_s": late, "peak_active": st["peak_active"],
            "peak_hbm_bytes": st["peak_bytes"], "rounds": st["rounds"], "gpu_launches": st["launches"],
            "policy": "%s admission by HBM footprint, at most %d zones in flight (one request always "
                      "admitted), rounds of <= %d cycles as one batch step (CUDA graph)"
                      % ("smallest-work-first" if policy else "FIFO", zone_cap, quantum)}


def corner_divb(P, gdet, dx, n):
    """max |div(sqrt(-g) B)| at interior zone corners, the discrete
    divergence flux-CT keeps at round-off, and the scale max|sqrt(-g) B|/dx."""
    import numpy as np
    GB = P[5:8] * gdet[None, None]
    ng = 3

    def box(comp, off, d):
        tot = 0.0
        for a in (0, -1):
            for b in (0, -1):
                o3 = [a, b]
                o3.insert(d, off)
                tot = tot + GB[comp][ng + o3[2]: ng + n[2] + o3[2], ng + o3[1]: ng + n[1] + o3[1],
                                     ng + o3[0]: ng + n[0] + o3[0]]
        return tot
    div = 0.0
    for d in range(3):
        if n[d] > 1:
            div = div + (box(d, 0, d) - box(d, -1, d)) / (4 * dx[d])
    return (float(np.abs(div[1:-1, 1:-1, 1:-1]).max()),
            float(np.abs(GB).max() / min(dx[d] for d in range(3) if n[d] > 1)))


def mixed_accuracy(grmhd, steps, stream):
    """The 288x128x128 torus (R_out = 1000) advanced `steps` cycles in FP64,
    in the mixed mode and in the mixed mode with the float-float update:
    per-primitive L1 and Linf of the difference from FP64, relative to the
    FP64 state's mean |value| and max |value|, and the corner divergence."""
    import dataclasses
    import numpy as np
    pr = make_problem("torus288")
    states = {}
    for prec in (0, 1, 3):
        p = dataclasses.replace(pr, precision=prec)
        s = grmhd.Sim(p, stream=stream)
        s.set_prims(p.P)
        s.step(steps)
        states[prec] = s.get_prims(with_ghosts=True)
        gdet = s.geom(0)[32]
        s.close()
    names = ["rho", "u", "u1", "u2", "u3", "B1", "B2", "B3"]
    b = states[0][:, 3:-3, 3:-3, 3:-3]
    body = b[0] > 1e-2  # the torus itself (max rho = 1), without the floor-held atmosphere
    # group scales: mean over zones of |rho|, |u|, the velocity norm, the field norm
    grp = {0: np.abs(b[0]).mean(), 1: np.abs(b[1]).mean(),
           2: np.sqrt((b[2:5] ** 2).sum(axis=0)).mean(), 5: np.sqrt((b[5:8] ** 2).sum(axis=0)).mean()}

    def norms(a):
        out = {}
        for v, nm in enumerate(names):
            d = np.abs(a[v] - b[v])
            gs = grp[0 if v == 0 else 1 if v == 1 else 2 if v < 5 else 5]
            out[nm] = {"group_l1_rel": float(d.mean() / max(gs, 1e-300)),
                       "l1_rel": float(d.mean() / max(np.abs(b[v]).mean(), 1e-300)),
                       "linf_rel": float(d.max() / max(np.abs(b[v]).max(), 1e-300)),
                       "torus_l1_rel": float(d[body].mean() / max(np.abs(b[v][body]).mean(), 1e-300)),
                       "torus_linf_rel": float(d[body].max() / max(np.abs(b[v][body]).max(), 1e-300))}
        return out

    out = norms(states[1][:, 3:-3, 3:-3, 3:-3])
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    for prec, key in ((0, "divb_fp64"), (1, "divb_mixed"), (3, "divb_mixed_ff")):
        m, sc = corner_divb(states[prec], gdet, dx, pr.n)
        out[key] = {"max": m, "scale": sc, "rel": m / sc}
    return {"workload": WORKLOADS["torus288"]["label"].replace("_fp64", ""), "steps": steps,
            "reference": "the FP64 path (parity-tested against the FP64 oracle)",
            "norms": "group_l1_rel: mean |mixed - fp64| / mean of the group's magnitude (rho; u; "
                     "|utilde|; |B|); l1_rel: / mean |fp64| of the component; linf_rel: max / max; "
                     "over all interior zones; torus_*: over zones with rho > 1e-2",
            "primitives": out,
            "mixed_ff_primitives": norms(states[3][:, 3:-3, 3:-3, 3:-3])}


def mode_accuracy(grmhd, stream):
    """The 64x64 fast mode (MC, CFL 0.9) run for one period on the GPU and on
    the oracle: per-primitive L1 of the difference from the analytic
    eigenmode at t_final (mean over zones of |P - P_exact|), their sum, and
    the sum relative to the mode's amplitude (1e-4)."""
    import numpy as np
    import oracle
    pr = make_problem("mode64")
    ex = pr.exact(pr.t_final)
    s = grmhd.Sim(pr, stream=stream)
    s.set_prims(pr.P)
    st = s.step(100000)
    Pg = s.get_prims()
    s.close()
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    o.step(100000)
    Po = o.get_prims()
    t_o, _, n_o = o.time()
    o.close()
    names = ["rho", "u", "u1", "u2", "u3", "B1", "B2", "B3"]
    eg = np.abs(Pg - ex).mean(axis=(1, 2, 3))
    eo = np.abs(Po - ex).mean(axis=(1, 2, 3))
    amp = pr.info["amp"]
    return {"workload": WORKLOADS["mode64"]["label"] + "_one_period",
            "t_final": pr.t_final, "cycles_gpu": st["steps"], "cycles_oracle": n_o,
            "l1_gpu": {nm: float(v) for nm, v in zip(names, eg)},
            "l1_oracle": {nm: float(v) for nm, v in zip(names, eo)},
            "l1_sum_gpu": float(eg.sum()), "l1_sum_oracle": float(eo.sum()),
            "l1_sum_over_amplitude_gpu": float(eg.sum() / amp),
            "l1_sum_over_amplitude_oracle": float(eo.sum() / amp),
            "gpu_vs_oracle_rel": float(abs(eg.sum() - eo.sum()) / eo.sum()),
            "norm": "mean over the 64x64 zones of |P_v - P_exact,v| at t = one period; "
                    "amplitude 1e-4 of the eigenvector (unit norm)"}


def mixed_vs_oracle(grmhd, steps, stream):
    """The 288x128x128 torus (R_out = 1000) advanced `steps` cycles by the
    oracle (FP64, one host core) and on the GPU in FP64, in the mixed mode
    and in the mixed mode with the float-float update, every GPU run on the
    oracle's geometry: per-primitive L1 and Linf of each GPU state's
    difference from the oracle's, relative to the oracle state's mean and
    largest magnitude, over all interior zones and over the torus (rho >
    1e-2), and the corner divergence of each."""
    import dataclasses
    import numpy as np
    import oracle
    pr = make_problem("torus288")
    t0 = time.perf_counter()
    o = oracle.Oracle(pr)
    o.set_prims(pr.P)
    geoms = [o.geom(loc) for loc in range(4)]
    o.step(steps)
    ref = o.get_prims()
    o.close()
    oracle_s = time.perf_counter() - t0
    names = ["rho", "u", "u1", "u2", "u3", "B1", "B2", "B3"]
    body = ref[0] > 1e-2
    dx = [(pr.xmax[d] - pr.xmin[d]) / pr.n[d] for d in range(3)]
    out = {"workload": WORKLOADS["torus288"]["label"].replace("_fp64", ""), "steps": steps,
           "reference": "the oracle (FP64, CPU), same geometry", "oracle_seconds": oracle_s}
    for prec, key in ((0, "fp64"), (1, "mixed"), (3, "mixed_ff")):
        p = dataclasses.replace(pr, precision=prec)
        s = grmhd.Sim(p, stream=stream)
        for loc in range(4):
            s.set_geom(loc, geoms[loc])
        s.set_prims(p.P)
        s.step(steps)
        a = s.get_prims()
        Pgh = s.get_prims(with_ghosts=True)
        s.close()
        res = {}
        for v, nm in enumerate(names):
            d = np.abs(a[v] - ref[v])
            res[nm] = {"l1_rel": float(d.mean() / max(np.abs(ref[v]).mean(), 1e-300)),
                       "linf_rel": float(d.max() / max(np.abs(ref[v]).max(), 1e-300)),
                       "torus_l1_rel": float(d[body].mean() / max(np.abs(ref[v][body]).mean(), 1e-300)),
                       "torus_linf_rel": float(d[body].max() / max(np.abs(ref[v][body]).max(), 1e-300))}
        m, sc = corner_divb(Pgh, geoms[0][32], dx, pr.n)
        res["divb_rel"] = m / sc
        out[key] = res
    out["norms"] = ("l1_rel: mean |gpu - oracle| / mean |oracle| of the component; linf_rel: max / "
                    "max; over all interior zones; torus_*: over zones with rho > 1e-2")
    return out


def long_run_health(grmhd, cycles, stream):
    """Health of long runs of the 128^3 torus: `cycles` cycles in each
    precision mode and cycles/2 with each variant (bounds in the drift
    frame; electrons with Kawazura heating), one grmhd_step call each:
    unrecoverable zones, whether every primitive is finite, inversion
    failures and bound hits per cycle, and the corner divergence of sqrt(-g)
    B relative to max|sqrt(-g) B| / min dX."""
    import dataclasses
    import numpy as np
    base = make_problem("torus128")
    dx = min((base.xmax[d] - base.xmin[d]) / base.n[d] for d in range(3))
    runs = [("fp64", dataclasses.replace(base, precision=0), cycles),
            ("mixed", dataclasses.replace(base, precision=1), cycles),
            ("float_float", dataclasses.replace(base, precision=2), cycles),
            ("mixed_ff", dataclasses.replace(base, precision=3), cycles),
            ("drift_frame", apply_variant(base, "drift"), cycles // 2),
            ("electrons", apply_variant(base, "electrons"), cycles // 2)]
    out = {}
    for name, pr, n in runs:
        s = grmhd.Sim(pr, stream=stream)
        s.set_prims(pr.P)
        if pr.electrons:
            s.set_electrons(pr.K)
        t0 = time.perf_counter()
        s.step(n, sync=False)
        st = s.stats()
        sec = time.perf_counter() - t0
        P = s.get_prims()
        dv, gb = s.divb()
        rec = {"cycles": st["steps"], "t": st["t"], "seconds": sec,
               "unrecoverable": st["unrecoverable"], "all_finite": bool(np.isfinite(P).all()),
               "inv_failures": st["inv_failures"], "floor_hits_per_stage": st["floor_hits"] / max(2 * n, 1),
               "divb_rel": dv * dx / gb if gb > 0 else None}
        if pr.electrons:
            rec["electrons_finite"] = bool(np.isfinite(s.get_electrons()).all())
        s.close()
        out[name] = rec
    return {"workload": WORKLOADS["torus128"]["label"].replace("_fp64", ""), "runs": out,
            "note": "floor_hits_per_stage: zones in which a bound acted, per stage (two per cycle)"}


def apply_variant(pr, variant):
    """The workload with a variant of the step switched on: the bounds in the
    drift frame, or electron entropies heated by the Kawazura et al. model
    with T_p/T_e in [1e-3, 1e3] and P_gas/rho^gamma <= 3."""
    import dataclasses
    from paper_2110_10191_gb300 import problems as pb
    if variant == "drift":
        return dataclasses.replace(pr, floor_frame=1)
    if variant == "electrons":
        return pb.with_electrons(pr, model=pb.ELEC_KAWAZURA)
    return pr


def workload_config(name, variant="none"):
    w = WORKLOADS[name]
    cfg = {"workload": w["label"], "grid": list(w["n"]), "dtype": "fp64",
           "recon": "weno5" if w["recon"] == 1 else "mc"}
    if variant != "none":
        cfg["variant"] = variant
    if name.startswith("torus"):
        cfg.update({"metric": "kerr_mks", "a": 0.9375, "hslope": 0.3, "r_out": w["r_out"],
                    "r_in_torus": 6.0, "r_max_torus": 12.0, "beta": 100.0, "perturbation": 0.04,
                    "seed": 0, "l2": "inputs larger than L2 (one primitive set %.0f MB > 129 MB)"
                    % (8 * 8 * (w["n"][0] + 6) * (w["n"][1] + 6) * (w["n"][2] + 6) / 1e6)})
    cfg["step"] = "one full predictor-corrector cycle of the grid"
    return cfg


# FP64 peak from the nominal unit counts and clock: 152 SMs, 2 DFMA per SM
# per clock (ncu sm__sass_thread_inst_executed_op_dfma_pred_on.sum.peak_sustained
# = 304 per GPU), 2 flops per DFMA, 2070 MHz maximum SM clock
FP64_PEAK_NOMINAL = 152 * 2 * 2 * 2070e6
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def fp64_peak_sustained(rate_per_sm_clock, nsm=SM_COUNT, mhz=SM_MAX_MHZ):
    """FP64 peak from the unit count and clock, with the FP64 issue rate per
    SM per clock measured (grmhd_fp64_probe) instead of the nominal 2: nsm x
    rate x 2 flops x the maximum SM clock."""
    return nsm * rate_per_sm_clock * 2.0 * mhz * 1e6


def fp64_issue_sweep(grmhd, iters=1 << 14):
    """The FP64 issue rate per SM per clock (and the SM clock measured in
    the kernel) for FMA with 1, 8 and 16 independent chains per thread on 1,
    8 and 16 blocks per SM, and for add and multiply."""
    out = []
    for op, chains, bps in ((0, 8, 8), (0, 1, 1), (0, 1, 8), (0, 16, 16), (1, 8, 8), (2, 8, 8)):
        r, mhz = grmhd.fp64_probe(op, chains, bps, iters)
        out.append({"op": ("fma", "add", "mul")[op], "chains": chains, "blocks_per_sm": bps,
                    "ops_per_sm_clock": r, "sm_mhz": mhz})
    return out


def build_roofline(prof, cpu, pr, zones, fp64, config, variant="none"):
    """Roofline of the FP64-bound kernel classes from the live per-class
    device times (prof: class -> (total ms, launches)), the counting
    oracle's algorithmic flops (cpu) and the FP64 peak fp64 = {"rate": FP64
    instructions per SM per clock measured by the probe, "mhz": the SM clock
    the probe measured}: the peak is the unit count (152 SMs) x that rate x
    2 flops x the maximum SM clock; the nominal peak (2 per SM per clock) is
    reported beside it.  Returns (roofline of the dominant class, per-class
    figures, algorithmic flops per zone-cycle of this grid)."""
    peak = fp64_peak_sustained(fp64["rate"])
    flops_zc = None
    if cpu is not None and variant == "none" and pr.precision == 0:
        # the oracle counts on a thin slab, whose extended-range faces weigh
        # more per zone than the workload grid's: scale the per-unit counts
        flops_zc = 2 * ((cpu["_face_flops_per_face"] + cpu["_recon_flops_per_face"]) *
                        sum(faces_per_launch(pr.n)) +
                        cpu["_update_flops_per_zone_stage"] * zones) / zones
    roofline = None
    kernels = {}
    if cpu is not None and pr.precision == 0 and variant == "none":
        # the FP64 kernels' algorithmic count
        faces = faces_per_launch(pr.n)
        hbm = 6791e9
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                hbm = float(json.load(f)["hbm_gbs"]) * 1e9
        except (OSError, KeyError, ValueError):
            pass
        # algorithmic work and bytes per launch of each FP64-bound kernel class:
        # face: two states in, one flux out (24 doubles per face); recon: the
        # primitives in, two face values out (24 doubles per zone of the
        # extended range); update: predictor 48, corrector 56 doubles per zone
        work = {
            "flux": ("kp_face (LLF face fluxes from reconstructed states)",
                     cpu["_face_flops_per_face"] * sum(faces) / 3.0, 24 * 8 * sum(faces) / 3.0),
            "recon": ("kp_recon (WENO5 face states, both faces of every zone)",
                      cpu["_recon_flops_per_face"] * sum(faces) / 3.0,
                      24 * 8 * (pr.n[0] + 2) * (pr.n[1] + 2) * (pr.n[2] + 2)),
            "update": ("kp_update (conserved update + 1D_W inversion + bounds)",
                       cpu["_update_flops_per_zone_stage"] * zones, 52 * 8 * zones),
        }
        same_src = kernel_source_hash() == NCU_TRAFFIC["src_hash"]
        traffic = NCU_TRAFFIC.get(config) if same_src else None
        pipe = NCU_FP64_PIPE.get(config) if same_src else None
        for cls, (label, flops, nbytes) in work.items():
            ms_c, n_c = prof[cls]
            if not n_c:
                continue
            avg = ms_c / n_c
            kernels[cls] = {"kernel": label, "avg_launch_ms": avg, "launches": n_c,
                            "achieved_tflops": flops / (avg * 1e-3) / 1e12,
                            "frac": flops / (avg * 1e-3) / peak,
                            "frac_of_nominal": flops / (avg * 1e-3) / FP64_PEAK_NOMINAL,
                            "hbm_frac": nbytes / (avg * 1e-3) / hbm,
                            "algorithmic_bytes": nbytes,
                            "traffic": None if traffic is None else traffic.get(cls),
                            "fp64_pipe_ncu": None if pipe is None else pipe.get(cls)}
        dom = max(kernels, key=lambda k: prof[k][0]) if kernels else None
        if dom:
            kd = kernels[dom]
            roofline = {"bound": "alu", "kernel": kd["kernel"],
                        "achieved": kd["achieved_tflops"], "peak": peak / 1e12,
                        "unit": "TFLOP/s", "frac": kd["frac"],
                        "peak_source": "derived: 152 SMs x %.3f FP64 instructions per SM per clock "
                                       "(measured in this run by grmhd_fp64_probe, the same for any "
                                       "number of chains, blocks and FP64 operation) x 2 flop x "
                                       "2.07 GHz" % fp64["rate"],
                        "peak_nominal": FP64_PEAK_NOMINAL / 1e12,
                        "frac_of_nominal": kd["frac_of_nominal"],
                        "nominal_source": "152 SMs x 2 DFMA/clk (ncu peak_sustained) x 2 flop x "
                                          "2.07 GHz",
                        "work": "algorithmic FP64 flops of the oracle's counting build",
                        "avg_launch_ms": kd["avg_launch_ms"], "hbm_frac": kd["hbm_frac"],
                        "algorithmic_bytes": kd["algorithmic_bytes"], "traffic": kd["traffic"],
                        "fp64_pipe_ncu": kd["fp64_pipe_ncu"],
                        "note": "algorithmic flops are the counting oracle's (adds, multiplies, "
                                "divisions and square roots counted as one each); the kernel spends "
                                "several FP64 instructions on each division and square root and a "
                                "lone add or multiply takes an issue slot worth two flops, while an "
                                "FMA does two counted flops in one slot and the kernels form fewer "
                                "terms than the oracle's plain order (shared differences of the "
                                "reconstruction walk), so a saturated kernel can read above 1",
                        "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per "
                                          "launch of %s, mean over its launches in the ncu launch "
                                          "list of this workload" % kd["kernel"].split()[0]}
    return roofline, kernels, flops_zc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="torus128", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "ff", "mixed_ff"],
                    help="arithmetic of the flux stage of the timed workload (fp64: the headline)")
    ap.add_argument("--variant", default="none", choices=["none", "drift", "electrons"],
                    help="run the timed workload with the bounds in the drift frame or with "
                         "electron entropies (Kawazura heating); none: the headline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mixed-precision, batched and accuracy legs")
    ap.add_argument("--accuracy-steps", type=int, default=100)
    ap.add_argument("--only", default="", choices=["", "batched", "batched_small"],
                    help="run only this leg (no headline) and print its figures as one JSON line")
    ap.add_argument("--long-run", type=int, default=0,
                    help="instead of the benchmark, run this many cycles of the 128^3 torus in "
                         "every precision mode (half as many with each variant) and print their "
                         "health as one JSON line")
    ap.add_argument("--oracle-steps", type=int, default=2,
                    help="cycles of the 288x128x128 torus run by the oracle for the precision "
                         "modes' error against it (0: skip)")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the 200-request serving stream to run (0: skip)")
    ap.add_argument("--serve-zone-cap", type=int, default=1 << 22)
    ap.add_argument("--serve-quantum", type=int, default=8)
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2110_10191_gb300 import grmhd

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    if args.long_run > 0:
        if rank == 0:
            print(json.dumps({"long_run": long_run_health(grmhd, args.long_run,
                                                         torch.cuda.current_stream())}))
        return
    if args.only:
        # one leg alone (for profiling captures of it)
        st0 = torch.cuda.current_stream()
        legs = {"batched": lambda: batched_throughput(grmhd, max(args.steps // 2, 5), args.warmup, st0),
                "batched_small": lambda: batched_throughput(grmhd, args.steps, args.warmup, st0,
                                                            nmin=32, nmax=48)}
        if rank == 0:
            print(json.dumps({args.only: legs[args.only]()}))
        return

    pr = apply_variant(make_problem(args.config), args.variant)
    pr.precision = {"fp64": 0, "mixed": 1, "ff": 2, "mixed_ff": 3}[args.precision]
    zones = pr.n[0] * pr.n[1] * pr.n[2]
    stream = torch.cuda.current_stream()
    sim = grmhd.Sim(pr, stream=stream)
    sim.set_prims(pr.P)
    if pr.electrons:
        sim.set_electrons(pr.K)
    sim.step(args.warmup)

    # ---- per-class pass: K steps with a CUDA event around each kernel class
    # on the launching stream (direct launches); the roofline's per-kernel
    # times and the launch count ----
    sim.profile(True)
    sim.get_profile(reset=True)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    prof_ms = reduce_max(e0.elapsed_time(e1), world, "cuda")
    prof = sim.get_profile(reset=True)
    sim.profile(False)

    # ---- timed region: the same K steps as one grmhd_step call, which
    # replays a CUDA graph of one cycle (the library's own path), device
    # resident ----
    sim.step(2)  # captures the graph (untimed)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(args.steps, sync=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    st = sim.stats()
    ms = reduce_max(ms, world, "cuda")
    value = job_value(zones, args.steps, world, ms * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    io_bytes = 8 * 8 * zones
    e2e_s = None
    if not args.no_e2e:
        host_in = torch.from_numpy(np.ascontiguousarray(pr.P)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        sim2 = grmhd.Sim(pr, stream=stream)
        sim2.set_prims(host_in)
        if pr.electrons:
            sim2.set_electrons(pr.K)
        sim2.step(1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.set_prims(host_in)
        sim2.step(args.steps, sync=False)
        sim2.get_prims(out=host_out)
        t1 = time.perf_counter()
        e2e_s = t1 - t0
        e2e_s = reduce_max(e2e_s, world, "cuda")
        sim2.close()

    fp64_sweep = fp64_issue_sweep(grmhd)
    fp64 = {"rate": fp64_sweep[0]["ops_per_sm_clock"], "mhz": fp64_sweep[0]["sm_mhz"]}

    extras = {}
    if not args.no_extras:
        extras["mixed"] = mixed_throughput(grmhd, pr, args.steps, args.warmup, stream, 1)
        extras["float_float"] = mixed_throughput(grmhd, pr, args.steps, args.warmup, stream, 2)
        extras["mixed_ff"] = mixed_throughput(grmhd, pr, args.steps, args.warmup, stream, 3)
        extras["float_float"]["parity"] = ("one step against the FP64 oracle within 3e-11 of each "
                                           "primitive group's scale (tests/test_gpu_ff.py)")
        extras["drift_frame"] = variant_throughput(grmhd, pr, max(args.steps // 2, 5), args.warmup,
                                                   stream, "drift")
        extras["electrons"] = variant_throughput(grmhd, pr, max(args.steps // 2, 5), args.warmup,
                                                 stream, "electrons")
        extras["single_small"] = small_single(grmhd, 200, stream)
        extras["decomposed"] = decomposed(grmhd, pr, max(args.steps // 5, 5), args.warmup, stream)
        extras["batched"] = batched_throughput(grmhd, max(args.steps // 2, 5), args.warmup, stream)
        extras["batched_small"] = batched_throughput(grmhd, args.steps, args.warmup, stream,
                                                     nmin=32, nmax=48)
        if rank == 0:
            extras["mixed_accuracy"] = mixed_accuracy(grmhd, args.accuracy_steps, stream)
        if args.serve_requests > 0:
            extras["served"] = serving_run(grmhd, args.serve_requests, args.serve_zone_cap,
                                           args.serve_quantum, policy=0)
            extras["served_swf"] = serving_run(grmhd, args.serve_requests, args.serve_zone_cap,
                                               args.serve_quantum, policy=1)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # the oracle leg: the CPU baseline, and the accuracy of the GPU path and
    # of the oracle itself against the analytic mode and against each other
    cpu = None
    cpu_all = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(args.config, steps=2)
        if not args.no_extras:
            cpu_all = cpu_oracle_all_cores(args.config, steps=2)
            extras["mode_accuracy"] = mode_accuracy(grmhd, stream)
            if args.oracle_steps > 0:
                extras["mixed_vs_oracle"] = mixed_vs_oracle(grmhd, args.oracle_steps, stream)

    launches = sum(v[1] for v in prof.values())
    roofline, kernels, flops_zc = build_roofline(prof, cpu, pr, zones, fp64, args.config,
                                                 args.variant)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if pr.precision == 0 else PREC_DTYPE[pr.precision],
            "data": "synthetic", "config": workload_config(args.config, args.variant),
            "e2e": None if e2e_s is None else {
                "value": job_value(zones, args.steps, world, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": io_bytes / args.steps,
                "d2h_bytes_per_step": io_bytes / args.steps,
                "note": "set_prims(pinned host) + %d steps + get_prims(pinned host) per job"
                        % args.steps},
            "gpu_launches": launches,
            "timed_path": "one grmhd_step call of K cycles with profiling off: a CUDA-graph "
                          "replay of one cycle, the library's own path; gpu_launches counts "
                          "the same K cycles' kernels in the per-class pass",
            "per_class_pass": {"value": job_value(zones, args.steps, world, prof_ms * 1e-3),
                               "unit": UNIT, "ms_per_step": prof_ms / args.steps,
                               "note": "the same K steps launched directly, each kernel class "
                                       "between CUDA events on its stream: the per-kernel "
                                       "times of kernel_ms and the roofline"},
            "kernel_ms": {k: v[0] for k, v in prof.items()},
            "roofline": roofline,
            "kernels": kernels,
            "cpu_baseline": None if cpu is None else {k: v for k, v in cpu.items() if not k.startswith("_")},
            "cpu_baseline_all_cores": cpu_all,
            "algorithmic_fp64_flops_per_zone_cycle": flops_zc,
            "fp64_ceiling": None if flops_zc is None else {
                "value": fp64_peak_sustained(fp64["rate"]) / flops_zc, "unit": UNIT,
                "frac": value * flops_zc / fp64_peak_sustained(fp64["rate"]),
                "frac_of_nominal": value * flops_zc / FP64_PEAK_NOMINAL,
                "note": "FP64 peak (measured issue rate) / algorithmic FP64 flops per zone-cycle "
                        "of this grid (the oracle's counts per face and per zone-stage, scaled to "
                        "its faces and zones)"},
            "fp64_issue_rate": fp64_sweep,
            "clocks": clk,
            "sim": {"t": st["t"], "steps": st["steps"], "inv_failures": st["inv_failures"],
                    "floor_hits": st["floor_hits"]}}
    line.update(extras)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
