"""Benchmark of the UGKS hot path on GB300: cell-velocity updates per second.

Default workload: the 3D Mach-8 X38-like lifting body at Kn 0.005 and 20
degrees angle of attack (seeded tetrahedral mesh of ~1.05M cells, unstructured
tetrahedral velocity mesh of ~4,550 cells), the largest configuration that fits
one GPU, in the FP32-storage / FP64-moment form; the plain FP64 path is timed
beside it, and the 2D Mach-5 cylinder (~30,000 triangles, 60x50 velocities) is
reported as a secondary line.  One step = one full UGKS time step (all kernels
of Algorithm 1) of the whole case.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ugks|reference]

Prints one JSON line (rank 0).  N > 1 runs one independent replica per GPU
(the method needs no exchange between independent cases): value = all cells x
velocities updated by all ranks / max-over-ranks time.
"""
from __future__ import annotations

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
sys.path.insert(0, ROOT)

METRIC = "cell-velocity updates/s"
UNIT = "cvu/s"
WORKLOAD = "x38_Ma8_Kn0.005_tet1.05M_v4548"
CYLINDER = "cylinder_Ma5_Kn0.1_tri30k_v60x50"
E2E_MAX_BYTES = 32e9      # largest host copy of f the e2e leg stages in pinned memory
LARGE_CVU = 2e9           # cases above this many cell-velocities get a fixed FP64 tiling
X38_SMALL_H0 = 0.2        # first layer of the X38-like mesh for the ~100k-cell profiling instance
# gather tiling (patch cells, velocity tile, threads per CTA, tile group) of the benchmark's workloads:
# the autotuner's choice on GB300 (it varies between near-equal tile groups from run to run), fixed so
# that the committed ncu traffic figure applies and no trial launches run before the timed steps
BENCH_TILING = {WORKLOAD: (48, 64, 512, 64), CYLINDER: (48, 64, 512, 8)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _fp32_peak(torch, sm_max_mhz):
    """FP32 ceiling from the device's unit counts and clock: SMs x 128 FP32
    lanes x 2 flops per FMA x the maximum SM clock (nvidia-smi's clocks.max.sm,
    sampled during the run)."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(sm_max_mhz) if sm_max_mhz else None
    if not mhz:
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.max.sm",
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            mhz = float(out.stdout.strip().splitlines()[0])
        except Exception:
            mhz = None
    if not mhz:
        return None, n_sm, None
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12, n_sm, mhz


def _gather_flops_per_cvu(D, NC, nf):
    """FP32 arithmetic of the gather pass per cell-velocity, counted from its
    formulas (add, sub, mul 1 flop; FMA 2; exp2 and division 1): the limited
    slope of the cell, the flux of each of its nf faces (the gather evaluates
    every face of a cell, so an interior face twice over the mesh), stage 1 and
    the residual moments.  Ring slopes, address arithmetic, compares and
    selects are not counted."""
    slope = NC * (nf * (1 + 2 * D)                 # differences and least-squares sums
                  + nf * (2 * D + 10)              # Venkatakrishnan function at each face
                  + 3 * D + 3)                     # foot point, positivity scaling
    poly = D * D + 6 * D + 2                       # per-face polynomial of degree 3 in c
    face = ((2 * D - 1)                            # u . n
            + NC * (4 * D - 1)                     # upwind value and u . grad f
            + D + (2 * D - 1) + 3                  # c, |c|^2, H0
            + NC * (poly + 6)                      # flux of each component
            + 2 * NC)                              # residual
    stage1 = (D + 2 * (2 * D - 1) + 9 + (5 if NC == 2 else 0)   # Shakhov f+
              + 4 * NC                                          # stage-1 update
              + (2 * D - 1) + 2 + 2 * D + (5 if NC == 2 else 3))  # moments of the residual
    return slope + nf * face + stage1


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower().startswith("active")})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def _dist(backend="nccl"):
    """One process per GPU (torchrun): every rank runs its own replica of the
    workload; the only collectives are the timing barriers and reductions."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group(backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _workload(name):
    from paper_2412_06546_gb300 import cases
    if name == CYLINDER:
        return cases.cylinder_case(n_cells=30000, nvx=60, nvy=50, mach=5.0, Kn=0.1, seed=2)
    if name == "cylinder_Ma5_Kn0.1_tri8k_v60x50":       # the same flow on 8k cells (profiling captures)
        return cases.cylinder_case(n_cells=8000, nvx=60, nvy=50, mach=5.0, Kn=0.1, seed=2)
    if name == "cavity20_v24":
        return cases.cavity_case()
    if name == "sphere_Ma4_Kn0.1_tet150k_v28":
        return cases.sphere_case()
    if name == "sphere_Ma4_Kn0.1_tet20k_v28":           # the same flow on 20k cells (profiling captures)
        return cases.sphere_case(n_cells=20000)
    if name == "cylinder_E1_Ma5_Kn0.1_tri30k_dvs2060":    # the paper's unstructured velocity meshes
        return cases.cylinder_dvs_case("E1", n_cells=30000)
    if name == "cylinder_E2_Ma15_Kn0.01_tri30k_dvs3420":
        return cases.cylinder_dvs_case("E2", n_cells=30000)
    if name == WORKLOAD:
        return cases.x38_case()
    if name == "x38_Ma8_Kn0.005_tet100k_v4548":         # the same flow on ~100k cells (profiling captures)
        return cases.x38_case(h0=X38_SMALL_H0, n_surface=100000)
    raise SystemExit(f"unknown workload {name}")


def _time_steps(torch, g, steps, warmup, dist, sampler_index, profile=True):
    g.step(warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        g.profile_begin(steps)
    st = torch.cuda.ExternalStream(g.stream) if g.stream else torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(sampler_index) as cs:
        e0.record(st)
        g.step(steps)
        e1.record(st)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    groups, n = g.profile_end() if profile else ({}, 0)
    return ms, groups, cs.summary()


def _max_over_ranks(torch, dist, v, device="cuda"):
    if not dist:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _gather_sources():
    """The gather pass's code: its section of ugks_kernels.cu (from the
    "gather pass" to the "W update" marker) and all of ugks_device.cuh."""
    csrc = os.path.join(ROOT, "paper_2412_06546_gb300", "csrc")
    with open(os.path.join(csrc, "ugks_kernels.cu"), "rb") as fh:
        k = fh.read()
    a = k.index(b"// ------------------------------------------------------------ gather pass")
    b = k.index(b"// ------------------------------------------------------------ W update")
    with open(os.path.join(csrc, "ugks_device.cuh"), "rb") as fh:
        return k[a:b] + fh.read()


# committed ncu summaries holding the gather's DRAM traffic per launch, by workload
TRAFFIC_PROFILES = {CYLINDER: "k_gather_cylinder30k_fp32.md", WORKLOAD: "k_gather_x38_fp32.md"}


def _gather_traffic(workload, patch, vtile, threads, group):
    """DRAM bytes of one gather launch from the committed ncu summary of the
    workload, while the gather's sources and tiling are those the counters were
    taken on (else None: the kernel changed since)."""
    import hashlib
    if workload not in TRAFFIC_PROFILES:
        return None
    prof = os.path.join(ROOT, "profiles", TRAFFIC_PROFILES[workload])
    if not os.path.exists(prof):
        return None
    h = hashlib.sha256()
    h.update(_gather_sources())
    fields = {}
    for line in open(prof):
        if ":" in line and line.split(":")[0] in ("gather-sources-sha256-16", "traffic-bytes-per-launch",
                                                  "traffic-tiling"):
            k, v = line.split(":", 1)
            fields[k] = v.strip()
    if fields.get("gather-sources-sha256-16") != h.hexdigest()[:16]:
        return None
    if fields.get("traffic-tiling") != f"patch {patch}, vtile {vtile}, threads {threads}, group {group}":
        return None
    return int(fields["traffic-bytes-per-launch"])


def _cpu_baseline(case, steps=1, max_cvu=3e8):
    """The oracle on the host cores.  Cases up to max_cvu cell-velocities take
    whole steps; larger ones the local problem of a seeded sample of cells
    (the sample, two face rings and every face of the inner ring; one step of
    it gives the full-mesh step at the sample), sized to about 1.5e8
    cell-velocities (several seconds of oracle work) and timed per
    cell-velocity of the local problem."""
    import oracle
    from paper_2412_06546_gb300 import cases
    oracle.build()
    cores = os.cpu_count() or 1
    mesh, C0, Nv0 = case["mesh"], len(case["mesh"]["cell_vol"]), len(case["vgrid"]["w"])
    if C0 * Nv0 <= max_cvu:
        o = oracle.OracleCase(mesh, case["vgrid"], case["params"], case["init"], n_threads=cores)
        what = f"{steps} full step(s) of the same case"
    else:
        n = max(48, min(C0 // 4, int(1.5e8 / Nv0 / 12)))
        sub, s2, _ = cases.local_problem(mesh, cases.pick_sample(mesh, n, 1))
        o = oracle.OracleCase(sub, case["vgrid"], case["params"], case["init"][s2], n_threads=cores)
        what = (f"{steps} step(s) of the local problem of {n} seeded cells of the same case "
                f"({len(s2)} of {C0} cells, all {Nv0} velocities)")
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return {"value": o.C * o.Nv * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} on the host cores (OpenMP), {dt:.1f} s"}


def _e2e(torch, g, args, dist, ws, C, Nv, info):
    """The metric through the public API with host buffers: the state in
    pinned host memory -> ugks_set_state(_f32) -> ugks_step -> ugks_moments.
    f travels in the case's storage precision (FP32 for the FP32 form)."""
    import numpy as np
    from paper_2412_06546_gb300 import _lib
    f_h, W_h = g.state(f_dtype=np.float32 if info["precision"] == _lib.FP32 else np.float64)
    f_pin = torch.from_numpy(f_h).pin_memory().numpy()
    W_pin = torch.from_numpy(W_h).pin_memory().numpy()
    g.set_state(f_pin, W_pin)
    g.step(1)
    g.moments()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        g.set_state(f_pin, W_pin)
        g.step(1)
        g.moments()
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks(torch, dist, time.perf_counter() - t0) / args.e2e_steps
    return {"value": ws * C * Nv / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(f_pin.nbytes + W_pin.nbytes),
            "d2h_bytes_per_step": int(C * (2 * info["dim"] + 2) * 8)}


def _shard(items, rank, ws):
    """The requests a rank serves: independent cases go to independent GPUs."""
    return list(items)[rank::ws]


def _combine_serving(dist, lat, span, cvu, conv):
    """Merge the ranks' serving results: all latencies, the longest makespan,
    the summed cell-velocity updates and converged counts."""
    if not dist:
        return list(lat), span, cvu, conv
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, (list(map(float, lat)), float(span), int(cvu), int(conv)))
    return ([x for p in parts for x in p[0]], max(p[1] for p in parts), sum(p[2] for p in parts),
            sum(p[3] for p in parts))


def _serving(args, torch, lib, dist=None, rank=0, ws=1):
    """Serving leg: closed run (all requests at t = 0) to calibrate capacity,
    then Poisson arrivals at 1.5x that capacity; p50 / p99 of the time from
    arrival to completion and the aggregate cell-velocity rate.  With several
    ranks each serves its share of the stream on its own GPU."""
    import numpy as np
    from paper_2412_06546_gb300 import serving
    spec = ({"c_lo": 1000, "c_hi": 4000, "n_lo": 16, "n_hi": 32} if args.serve_stream == "small"
            else {"c_lo": 1000, "c_hi": 40000, "n_lo": 16, "n_hi": 64})
    reqs = _shard(serving.request_stream(args.serve_n, seed=4, **spec), rank, ws)
    budget = int(args.serve_budget_gb * (1 << 30))

    def run(arrivals):
        srv = lib.Server(budget, args.serve_slots, args.serve_tick)
        t0 = srv.stats()["clock"]
        tickets = [srv.submit(c, args.serve_tol, args.serve_max_steps, t_arrive=t0 + a) for c, a in zip(reqs, arrivals)]
        ok = srv.run(args.serve_timeout)
        st = srv.stats()
        res = [srv.poll(t) for t in tickets]
        srv.close()
        # latencies of converged requests first, then of step-limited ones (negated
        # so that they can be told apart after the ranks are merged)
        lat = [(r["t_done"] - r["t_arrive"]) * (1 if (r["state"] == lib.REQ_DONE and r["status"] == 0) else -1)
               for r in res]
        span = max(r["t_done"] for r in res) - t0
        conv = sum(1 for r in res if r["state"] == lib.REQ_DONE and r["status"] == 0)
        return ok, lat, span, st["total_cvu"], conv

    ok0, lat0, span0, cvu0, conv0 = run(np.zeros(len(reqs)))
    rate = 1.5 * len(reqs) / span0                 # offered load 1.5x the closed-run capacity
    arr = serving.poisson_arrivals(len(reqs), rate, seed=44 + rank)
    ok1, lat1, span1, cvu1, conv1 = run(arr)
    lat0, span0, cvu0, conv0 = _combine_serving(dist, lat0, span0, cvu0, conv0)
    lat1, span1, cvu1, conv1 = _combine_serving(dist, lat1, span1, cvu1, conv1)

    def pct(lat):
        ok = [x for x in lat if x >= 0]
        lim = [-x for x in lat if x < 0]
        allv = ok + lim
        return {"p50_s": float(np.percentile(allv, 50)), "p99_s": float(np.percentile(allv, 99)),
                "converged_p50_s": float(np.percentile(ok, 50)) if ok else None,
                "converged_p99_s": float(np.percentile(ok, 99)) if ok else None,
                "step_limited": len(lim)}

    p1, p0 = pct(lat1), pct(lat0)
    return {"requests": args.serve_n, "tol": args.serve_tol, "max_steps": args.serve_max_steps,
            "steps_per_tick": args.serve_tick, "slots": args.serve_slots, "budget_gb": args.serve_budget_gb,
            "arrival_rate_per_s": rate * ws, **p1, "aggregate_cvu_per_s": cvu1 / span1, "converged": conv1,
            "finished": bool(ok1),
            "closed_run": {"makespan_s": span0, "aggregate_cvu_per_s": cvu0 / span0, **p0, "converged": conv0},
            "workload": (f"seeded cavity/cylinder stream: cells {spec['c_lo']}-{spec['c_hi']}, N^2 velocities "
                         f"N in [{spec['n_lo']}, {spec['n_hi']}], Kn log-uniform [1e-3, 10], Mach [0.1, 6], "
                         "FP32 storage; latency = arrival to completion, quantised to ticks of "
                         f"{args.serve_tick} steps")}


def run_reference(args):
    """The oracle as it stands on the host cores: every timed step is one oracle
    step of the bench workload; cases above 3e8 cell-velocities step the local
    problem of a seeded sample of cells instead (one step of it gives the
    full-mesh step at the sample; about 5e7 cell-velocities, a second or two
    per step).  Rank 0 alone runs it."""
    dist_rank = int(os.environ.get("RANK", "0"))
    if dist_rank != 0:
        return 0
    import oracle
    from paper_2412_06546_gb300 import cases
    oracle.build()
    case = _workload(args.workload)
    cores = os.cpu_count() or 1
    mesh, C0, Nv0 = case["mesh"], len(case["mesh"]["cell_vol"]), len(case["vgrid"]["w"])
    if C0 * Nv0 <= 3e8:
        o = oracle.OracleCase(mesh, case["vgrid"], case["params"], case["init"], n_threads=cores)
        what = "full steps of the same case"
    else:
        n = max(48, min(C0 // 4, int(5e7 / Nv0 / 12)))
        sub, s2, _ = cases.local_problem(mesh, cases.pick_sample(mesh, n, 1))
        o = oracle.OracleCase(sub, case["vgrid"], case["params"], case["init"][s2], n_threads=cores)
        what = (f"steps of the local problem of {n} seeded cells of the same case "
                f"({len(s2)} of {C0} cells, all {Nv0} velocities)")
    o.step(args.ref_warmup)
    times = []
    for _ in range(args.ref_steps):
        t0 = time.perf_counter()
        o.step(1)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = o.C * o.Nv / (ms * 1e-3)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.ref_steps, "warmup": args.ref_warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "cells": C0, "nv": Nv0, "form": "fp64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_steps} {what} after {args.ref_warmup} warm-up, OpenMP"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _measure(torch, lib, name, case, args, dist, ws, local, steps, warmup, stream, e2e=False):
    """FP32-form steps of one workload: cell-velocity updates per second, the
    kernel-group times of the timed steps, the gather's HBM roofline and its
    FP32 ceiling, and (e2e) the same metric through the public API with host
    buffers."""
    import numpy as np
    tiling = (args.patch, args.vtile, args.threads, args.tile_group)
    if not any(tiling) and name in BENCH_TILING:
        tiling = BENCH_TILING[name]
    with torch.cuda.stream(stream):
        g = lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=lib.FP32,
                     stream=stream.cuda_stream, patch_cells=tiling[0], vtile=tiling[1],
                     threads=tiling[2], tile_group=tiling[3])
    info = g.info()
    C, Nv, nc = info["n_cells"], info["nv"], info["ncomp"]
    ms, groups, clocks = _time_steps(torch, g, steps, warmup, dist, local)
    g.check()
    ms = _max_over_ranks(torch, dist, ms)
    ms_step = ms / steps
    value = ws * C * Nv / (ms_step * 1e-3)
    # roofline of the dominant kernel (gather pass): 1 read + 1 write of f
    peak, peak_kind = _peaks()
    g_ms = groups.get("gather", 0.0) / max(steps, 1)
    alg_bytes = 2 * C * nc * Nv * 4
    achieved = alg_bytes / (g_ms * 1e-3) / 1e9 if g_ms > 0 else None
    share = {k: round(v / max(sum(groups.values()), 1e-12), 4) for k, v in groups.items()}
    # the second ceiling: FP32 arithmetic of the gather against the FP32 peak
    nf = float((np.asarray(case["mesh"]["face_cells"]) >= 0).sum()) / C
    flops_cvu = _gather_flops_per_cvu(info["dim"], nc, nf)
    alu_achieved = flops_cvu * C * Nv / (g_ms * 1e-3) / 1e12 if g_ms > 0 else None
    fp32_peak, n_sm, mhz = _fp32_peak(torch, clocks.get("sm_max_mhz"))
    out = {
        "value": value, "ms_per_step": ms_step, "steps": steps, "warmup": warmup, "clocks": clocks,
        "gpu_launches": info["kernel_launches_per_step"] * steps,
        "config": {"workload": name, "cells": C, "nv": Nv, "faces": info["n_faces"],
                   "form": "fp32 storage, fp64 moments", "patch_cells": info["patch_cells"],
                   "vtile": info["vtile"], "gather_threads": info["gather_threads"],
                   "gather_tile_group": info["gather_tile_group"],
                   "l2": f"inputs larger than L2 (f {info['f_bytes'] / 1e9:.2f} GB per copy)",
                   "w0": "analytic half-range moments" if args.w0_analytic else "discrete half-range sums",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "kernel": "k_gather", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": _gather_traffic(name, info["patch_cells"], info["vtile"],
                                                info["gather_threads"], info["gather_tile_group"]),
                     "peak_kind": peak_kind, "algorithmic_bytes_per_launch": alg_bytes,
                     "launch_ms": g_ms, "group_share": share},
        "alu_roofline": {"bound": "alu", "kernel": "k_gather", "achieved": alu_achieved, "peak": fp32_peak,
                         "unit": "TFLOP/s",
                         "frac": (alu_achieved / fp32_peak) if (alu_achieved and fp32_peak) else None,
                         "flops_per_cvu": round(flops_cvu, 1), "faces_per_cell": round(nf, 3),
                         "peak_kind": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {mhz} MHz"},
        "step_hbm_frac_1R1W": value / ws * 4 * nc * 2 / (peak * 1e9),
    }
    f_host_bytes = C * nc * Nv * 4
    if e2e:
        if args.no_e2e or args.e2e_steps < 1:
            out["e2e"] = {"skipped": "not requested"}
        elif f_host_bytes > E2E_MAX_BYTES:
            out["e2e"] = {"skipped": f"the host copy of f ({f_host_bytes / 1e9:.1f} GB) exceeds "
                                     f"{E2E_MAX_BYTES / 1e9:.0f} GB"}
        else:
            out["e2e"] = _e2e(torch, g, args, dist, ws, C, Nv, info)
    g.close()
    return out, info


def _fp64_plain(torch, lib, case, args, dist, ws, local, stream, steps, C, Nv):
    """The same step in the plain FP64 path (fixed tiling on large cases, where
    the autotuner's trial launches would take minutes)."""
    tiling = {"patch_cells": 16, "vtile": 32} if C * Nv > LARGE_CVU else {}
    with torch.cuda.stream(stream):
        g64 = lib.Case(case["mesh"], case["vgrid"], case["params"], case["init"], precision=lib.FP64,
                       stream=stream.cuda_stream, **tiling)
    ms64, _, _ = _time_steps(torch, g64, steps, 2, dist, local)
    g64.check()
    ms64 = _max_over_ranks(torch, dist, ms64) / steps
    g64.close()
    return {"value": ws * C * Nv / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "steps": steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ugks", choices=["ugks", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=3, help="steps of the FP64 plain path")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 leg")
    ap.add_argument("--secondary", default=CYLINDER,
                    help="workload reported beside the main one ('' for none)")
    ap.add_argument("--secondary-steps", type=int, default=100)
    ap.add_argument("--ref-steps", type=int, default=0)
    ap.add_argument("--ref-warmup", type=int, default=-1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-n", type=int, default=24)
    ap.add_argument("--serve-tol", type=float, default=1e-4)
    ap.add_argument("--serve-max-steps", type=int, default=6000)
    ap.add_argument("--serve-tick", type=int, default=25)
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=8.0)
    ap.add_argument("--serve-timeout", type=float, default=240.0)
    ap.add_argument("--serve-stream", default="small", choices=["small", "config"],
                    help="small: the fast default stream; config: cells 1k-40k, N up to 64")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--patch", type=int, default=0)
    ap.add_argument("--vtile", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0, help="gather CTA size, 256 or 512 (0: autotuned)")
    ap.add_argument("--tile-group", type=int, default=0,
                    help="velocity tiles per group of the gather grid order (0: autotuned)")
    ap.add_argument("--w0-analytic", action="store_true",
                    help="interface W0 from the analytic half-range moments (the variant of the N4 row)")
    args = ap.parse_args()
    if args.impl == "reference":
        args.ref_steps = args.ref_steps or args.steps
        args.ref_warmup = args.ref_warmup if args.ref_warmup >= 0 else args.warmup
        return run_reference(args)

    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (no CPU fallback)")
    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2412_06546_gb300 import build, _lib
    build.build()
    stream = torch.cuda.Stream()

    def load(name):
        c = _workload(name)
        if args.w0_analytic:
            c = dict(c, params=dict(c["params"], w0_analytic=1))
        return c

    case = load(args.workload)
    main_res, info = _measure(torch, _lib, args.workload, case, args, dist, ws, local, args.steps, args.warmup,
                              stream, e2e=True)
    C, Nv = info["n_cells"], info["nv"]
    fp64 = {"skipped": "not requested"}
    if not args.no_fp64:
        fp64 = _fp64_plain(torch, _lib, case, args, dist, ws, local, stream, args.fp64_steps, C, Nv)
        fp64["speedup_of_fp32_form"] = main_res["value"] / fp64["value"]
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = _cpu_baseline(case)
    del case

    secondary = None
    if args.secondary and args.secondary != args.workload:
        sc = load(args.secondary)
        sres, sinfo = _measure(torch, _lib, args.secondary, sc, args, dist, ws, local, args.secondary_steps,
                               args.warmup, stream)
        secondary = {k: sres[k] for k in ("value", "ms_per_step", "steps", "config", "roofline", "alu_roofline",
                                          "step_hbm_frac_1R1W")}
        if not args.no_fp64:
            s64 = _fp64_plain(torch, _lib, sc, args, dist, ws, local, stream, max(3, args.secondary_steps // 10),
                              sinfo["n_cells"], sinfo["nv"])
            s64["speedup_of_fp32_form"] = sres["value"] / s64["value"]
            secondary["fp64_plain"] = s64
        main_res["gpu_launches"] += sres["gpu_launches"]

    serving_res = None
    if not args.no_serving:
        serving_res = _serving(args, torch, _lib, dist, rank, ws)

    line = {
        "metric": METRIC, "value": main_res["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_res["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": main_res["config"], "roofline": main_res["roofline"], "alu_roofline": main_res["alu_roofline"],
        "fp64_plain": fp64, "e2e": main_res["e2e"], "clocks": main_res["clocks"],
        "gpu_launches": main_res["gpu_launches"], "step_hbm_frac_1R1W": main_res["step_hbm_frac_1R1W"],
    }
    if secondary:
        line["secondary"] = secondary
    if serving_res:
        line["serving"] = serving_res
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
