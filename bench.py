"""Throughput of the GRMHD predictor-corrector step on GB300.

A "step" is one full predictor-corrector cycle of the whole hot path over
the workload grid.  Default workload: the 128^3 Fishbone-Moncrief torus
around a Kerr black hole (a = 0.9375) in modified Kerr-Schild coordinates
(h = 0.3, R_out = 50), WENO5, FP64, poloidal field at beta = 100, 4% seeded
perturbation of u (synthetic, generated in-process).  The metric is
zone-cycles/s (zones advanced by one full cycle per second).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

N > 1 runs under torchrun, one process per GPU; every rank advances its own
replica (the single-grid path is not decomposed), scaling "weak".  Rank 0
prints one JSON line.
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


def workload_config(name):
    w = WORKLOADS[name]
    cfg = {"workload": w["label"], "grid": list(w["n"]), "dtype": "fp64",
           "recon": "weno5" if w["recon"] == 1 else "mc"}
    if name.startswith("torus"):
        cfg.update({"metric": "kerr_mks", "a": 0.9375, "hslope": 0.3, "r_out": w["r_out"],
                    "r_in_torus": 6.0, "r_max_torus": 12.0, "beta": 100.0, "perturbation": 0.04,
                    "seed": 0, "l2": "inputs larger than L2 (one primitive set %.0f MB > 129 MB)"
                    % (8 * 8 * (w["n"][0] + 6) * (w["n"][1] + 6) * (w["n"][2] + 6) / 1e6)})
    cfg["step"] = "one full predictor-corrector cycle of the grid"
    return cfg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default="torus128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
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

    pr = make_problem(args.config)
    zones = pr.n[0] * pr.n[1] * pr.n[2]
    stream = torch.cuda.current_stream()
    sim = grmhd.Sim(pr, stream=stream)
    sim.set_prims(pr.P)
    sim.step(args.warmup)

    # ---- timed region: K steps, device resident ----
    clocks = ClockSampler(local)
    clocks.start()
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
    ms = e0.elapsed_time(e1)
    prof = sim.get_profile(reset=True)
    sim.profile(False)
    clk = clocks.stop()
    st = sim.stats()
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * zones * args.steps / (ms * 1e-3)

    # ---- end to end through the C ABI with host buffers ----
    io_bytes = 8 * 8 * zones
    e2e_s = None
    if not args.no_e2e:
        host_in = torch.from_numpy(np.ascontiguousarray(pr.P)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        sim2 = grmhd.Sim(pr, stream=stream)
        sim2.set_prims(host_in)
        sim2.step(1)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.set_prims(host_in)
        sim2.step(args.steps, sync=False)
        sim2.get_prims(out=host_out)
        t1 = time.perf_counter()
        e2e_s = t1 - t0
        if world > 1:
            t = torch.tensor([e2e_s], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        sim2.close()

    peak_fp64 = grmhd.fp64_peak(1 << 16)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(args.config, steps=2)

    launches = sum(v[1] for v in prof.values())
    roofline = None
    kernels = {}
    if cpu is not None:
        faces = faces_per_launch(pr.n)
        hbm = 6791e9
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                hbm = float(json.load(f)["hbm_gbs"]) * 1e9
        except (OSError, KeyError, ValueError):
            pass
        # algorithmic work and bytes per launch of each FP64-bound kernel class
        work = {
            "flux": ("k_face (LLF face fluxes from reconstructed states)",
                     cpu["_face_flops_per_face"] * sum(faces) / 3.0, 16 * 8 * sum(faces) / 3.0),
            "recon": ("k_recon (WENO5 face states, both faces of every zone)",
                      cpu["_recon_flops_per_face"] * sum(faces) / 3.0,
                      24 * 8 * (pr.n[0] + 2) * (pr.n[1] + 2) * (pr.n[2] + 2)),
            "update": ("k_update (conserved update + 1D_W inversion + bounds)",
                       cpu["_update_flops_per_zone_stage"] * zones, 8 * (8 * 2 + 8 * 6 + 8) * zones),
        }
        for cls, (label, flops, nbytes) in work.items():
            ms_c, n_c = prof[cls]
            if not n_c:
                continue
            avg = ms_c / n_c
            kernels[cls] = {"kernel": label, "avg_launch_ms": avg, "launches": n_c,
                            "achieved_tflops": flops / (avg * 1e-3) / 1e12,
                            "frac": flops / (avg * 1e-3) / peak_fp64,
                            "hbm_frac": nbytes / (avg * 1e-3) / hbm}
        dom = max(kernels, key=lambda k: prof[k][0]) if kernels else None
        if dom:
            kd = kernels[dom]
            roofline = {"bound": "alu", "kernel": kd["kernel"],
                        "achieved": kd["achieved_tflops"], "peak": peak_fp64 / 1e12,
                        "unit": "TFLOP/s", "frac": kd["frac"],
                        "peak_source": "measured FP64 FMA throughput (grmhd_fp64_peak, this run); "
                                       "nominal 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz = 1.259",
                        "work": "algorithmic FP64 flops of the oracle's counting build",
                        "avg_launch_ms": kd["avg_launch_ms"], "hbm_frac": kd["hbm_frac"],
                        "traffic": None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args.config),
            "e2e": None if e2e_s is None else {
                "value": world * zones * args.steps / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": io_bytes / args.steps,
                "d2h_bytes_per_step": io_bytes / args.steps,
                "note": "set_prims(pinned host) + %d steps + get_prims(pinned host) per job"
                        % args.steps},
            "gpu_launches": launches,
            "kernel_ms": {k: v[0] for k, v in prof.items()},
            "roofline": roofline,
            "kernels": kernels,
            "cpu_baseline": None if cpu is None else {k: v for k, v in cpu.items() if not k.startswith("_")},
            "algorithmic_fp64_flops_per_zone_cycle": None if cpu is None else cpu["_flops_per_zone_cycle"],
            "clocks": clk,
            "sim": {"t": st["t"], "steps": st["steps"], "inv_failures": st["inv_failures"],
                    "floor_hits": st["floor_hits"]}}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
