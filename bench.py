"""Benchmark: k-omega RANS finite-volume time steps on one GB300 (or N replicas).

Default workload: the mixed-precision indoor room, 512 x 256 x 128 cells
(16.8 M cells at 2 cm), seeded ceiling vents, floor outlet and heated boxes,
Boussinesq buoyancy, 7-level multigrid to a 1e-8 relative residual, FP32
field storage with BF16 multigrid corrections inside the FP64
defect-correction pressure solve (--precision bf16).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|f32|f64]
                    [--workload room|channel|channel2d|batched|served]
                    [--impl ours|reference]

Prints one JSON line.  value = cell-steps/s over all ranks (each rank steps
its own replica; no collective on the data path, weak scaling).  Timing: W
untimed steps, then K steps each bracketed by CUDA events on the case's
stream, with a 256 MB buffer written between steps (larger than the 129 MB
L2; the room's state is larger than L2 as well).
"""
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

from paper_2603_21869_gb300 import cases  # noqa: E402

PREC = {"f32": cases.FP32, "f64": cases.FP64, "bf16": cases.BF16_MIXED}


def workload(name, precision):
    if name == "channel":
        return cases.heated_channel_3d(256, 64, 64, mg_levels=6, precision=precision,
                                       mg_rel_tol=1e-8, max_vcycles=60), \
            "heated_channel_3d 256x64x64, 6-level V(3,3), rel tol 1e-8"
    if name == "room":
        return cases.room_3d(512, 256, 128, seed=0, mg_levels=7, precision=precision,
                             mg_rel_tol=1e-8, max_vcycles=60), \
            "room_3d 512x256x128 (16.8M cells), seeded vents/boxes, buoyancy"
    if name == "channel2d":
        return cases.channel_2d(), "channel_2d 128x32"
    raise SystemExit(f"unknown workload {name}")


NOMINAL_HBM_GBS = 7900.0   # GB300 HBM3e, nominal (the roofline's denominator is the measured copy)
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel,
# from one ncu capture, with the SHA-256 prefix of the source file that kernel was built from
# when the counters were taken: a changed source reports null until it is captured again.
TRAFFIC = {
    # fcg_L0 = FcgDotVK + FcgUpdVK on the room with BF16 corrections, one iteration with a kept
    # direction: ncu dram__bytes_read.sum + dram__bytes_write.sum of the two launches
    # (201.6 + 446.3 MB; the algorithmic 42 B per cell is 704.6 MB)
    ("room", "bf16", "fcg_L0"): {"bytes": 647.9e6, "src": "mg_kernels.cu", "sha": "78e46771d833774f"},
}
# the batched sweep launch covers every case's finest level: DRAM bytes per finest-level cell
TRAFFIC_PER_CELL = {}


def _src_sha(name):
    import hashlib
    with open(os.path.join(ROOT, "paper_2603_21869_gb300", "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_for(table, key):
    """Measured DRAM bytes for key, or None if absent or taken from an older source."""
    t = table.get(key)
    if not t:
        return None
    try:
        return t["bytes"] if _src_sha(t["src"]) == t["sha"] else None
    except OSError:
        return None


def time_projection_vjp(spec, stream, flush, peak, calls=3):
    """The projection adjoint (fvm_projection_vjp) on an FP64 copy of the case after one
    step: wall time per call (its V-cycles included) and, by the profiling hook, the two
    transposed stencil kernels."""
    import numpy as np
    import torch
    from paper_2603_21869_gb300 import binding
    sp = spec.replace(precision=cases.FP64)
    rng = np.random.default_rng(0)
    ybar = [rng.standard_normal((sp.nx, sp.ny, sp.nz)) for _ in range(4)]
    with binding.Case(sp, stream=stream.cuda_stream) as c:
        c.step(1, allow_not_converged=True)
        dt = c.info()["dt"]
        c.projection_vjp(dt, *ybar)
        c.profile(True)
        wall, rels = 0.0, []
        for _ in range(calls):
            with torch.cuda.stream(stream):
                flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, rel = c.projection_vjp(dt, *ybar)
            wall += time.perf_counter() - t0
            rels.append(rel)
        prof = c.profile_read()
        c.profile(False)
    out = {"ms_per_call_wall": wall / calls * 1e3, "rel_residual": max(rels),
           "note": "FP64; wall time includes the 4 N-double copy in, the 3 N-double copy out and the V-cycles"}
    for k in ("adj_grad", "adj_rhs"):
        if k in prof:
            d = prof[k]
            gbs = d["bytes"] / (d["ms"] / 1e3) / 1e9
            out[k] = {"ms": d["ms"] / d["launches"], "gbs": gbs, "frac": gbs / peak}
    vc = [v for k, v in prof.items() if k not in ("adj_grad", "adj_rhs")]
    out["solve_kernel_ms_per_call"] = sum(v["ms"] for v in vc) / calls
    return out


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    """Ranks of a torchrun launch (one per GPU, nccl); (0, 1, 0, None) alone."""
    from paper_2603_21869_gb300 import replicas
    rank, ws, local, on = replicas.setup()
    if not on:
        return 0, 1, 0, None
    import torch.distributed as dist
    return rank, ws, local, dist


# Above this many cells one oracle step takes minutes (about 6 minutes for the 16.8 M-cell
# room on one host thread): the oracle is then timed on the same workload scaled down.
ORACLE_FULL_CELLS = 1 << 21


def oracle_sample(spec, workload):
    """(spec, description) of the bounded sample the oracle is timed on: the workload itself when
    one step is short, else the same generator at a quarter of the cells along each axis and the
    same cell size (two multigrid levels fewer), whose per-cell-step rate stands in."""
    if spec.cells <= ORACLE_FULL_CELLS or workload != "room":
        return spec.replace(precision=cases.FP64), f"the full {spec.nx}x{spec.ny}x{spec.nz} workload"
    sp = cases.room_3d(spec.nx // 4, spec.ny // 4, spec.nz // 4, seed=spec.seed,
                       mg_levels=max(2, spec.mg_levels - 2), precision=cases.FP64,
                       mg_rel_tol=spec.mg_rel_tol, max_vcycles=spec.max_vcycles)
    return sp, (f"a {sp.nx}x{sp.ny}x{sp.nz} room from the same seeded generator at the same cell size "
                f"(1/64 of the cells; the oracle's per-cell-step rate falls by about a quarter from "
                f"0.26 M to 2.1 M cells)")


def run_reference(args, spec, label, rank, ws, workload="channel"):
    """The FP64 CPU oracle as it stands, on a bounded sample of the same workload."""
    if rank != 0:
        return
    from oracle.step import OracleCase
    sp, what = oracle_sample(spec, workload)
    c = OracleCase(sp)
    for _ in range(args.warmup):
        c.step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c.step()
    el = time.perf_counter() - t0
    v = sp.cells * args.steps / el
    # n_gpus: the launch's N (the --gpus value); the oracle itself runs on one host core
    line = {"impl": "reference", "metric": "cell-steps/s", "value": v, "unit": "cell-steps/s", "n_gpus": ws,
            "host_only": True,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": label, "cells": spec.cells},
            "cpu_baseline": {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.warmup} untimed + {args.steps} timed steps of {what} "
                                       "(numpy float64, one thread)"},
            "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def arith_dtype(precision):
    """The arithmetic type of a precision mode: FP64, or FP32 (fields and corrections computed
    in FP32, BF16 only storing the multigrid corrections; config.precision names the storage)."""
    return "f64" if precision == "f64" else "f32"


def parse_params(text):
    """PRE,POST,INNER,PLANES,KRYLOV[,COARSE[,SMOOTHER]] -> seven ints (COARSE, SMOOTHER default to 0)."""
    v = [int(x) for x in text.split(",")]
    if len(v) not in (5, 6, 7):
        raise SystemExit("--params wants PRE,POST,INNER,PLANES,KRYLOV[,COARSE[,SMOOTHER]]")
    return tuple(v + [0] * (7 - len(v)))


def breakdown(prof, nsteps, traffic=None):
    """Per-site table, dominant kernel roofline and V-cycle bandwidth from profile tallies
    (traffic: {site: DRAM bytes per launch} from an ncu capture)."""
    peak, peak_src = peaks()
    name, d = max(prof.items(), key=lambda kv: kv[1]["ms"])
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    mg = [k for k in prof if any(k.startswith(p) for p in ("sweep", "resid", "prolong", "coarse"))]
    mg_bytes = sum(prof[k]["bytes"] for k in mg)
    mg_ms = sum(prof[k]["ms"] for k in mg)
    return {
        "roofline": {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": (traffic or {}).get(name),
                     "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                     "bytes_per_launch": d["bytes"] / d["launches"], "ms_per_launch": d["ms"] / d["launches"],
                     "launches": d["launches"]},
        "vcycle": {"gbs": mg_bytes / (mg_ms / 1e3) / 1e9 if mg_ms else None,
                   "frac": (mg_bytes / (mg_ms / 1e3) / 1e9) / peak if mg_ms else None,
                   "ms_per_step": mg_ms / nsteps},
        "profiled_pass": {"steps": nsteps, "kernel_ms_per_step": sum(v["ms"] for v in prof.values()) / nsteps,
                          "mode": "launch by launch, CUDA events around every kernel"},
        "kernels": {k: {"ms_per_step": v["ms"] / nsteps, "launches_per_step": v["launches"] / nsteps,
                        "gbs": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] else None}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:12]},
    }


def field_errors(got, ref):
    """Per-field max |a - b| / max |b| (the parity tests' measure), and under "velocity" the
    largest velocity-component error against the largest component magnitude (a component
    that stays small, such as the cross-stream velocity of a channel, has no scale of its own)."""
    import numpy as np
    out = {}
    for f in cases.FIELDS:
        scale = float(np.max(np.abs(ref[f]))) or 1.0
        out[f] = float(np.max(np.abs(got[f] - ref[f]))) / scale
    vs = max(float(np.max(np.abs(ref[f]))) for f in ("u", "v", "w")) or 1.0
    out["velocity"] = max(float(np.max(np.abs(got[f] - ref[f]))) for f in ("u", "v", "w")) / vs
    return out


def run_batched(args, rank, ws, local, dist):
    """C4: uneven channel cases stepped as one batch (one CUDA graph per step,
    one launch per kernel site for all cases), against the same cases stepped
    one by one (FP32, and the plain FP64 form)."""
    import numpy as np
    import torch
    from paper_2603_21869_gb300 import binding, build, replicas
    build.ensure_built()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prec = PREC[args.precision]
    specs = cases.batched_channels(args.cases, seed=rank, precision=prec, mg_levels=5)
    tuning = None
    if args.params:
        pre, post, inner, _planes, kry, coarse, smoother = parse_params(args.params)
        specs = [sp.replace(pre_sweeps=pre, post_sweeps=post, inner_cycles=inner, krylov=kry, coarse_sweeps=coarse,
                            smoother=smoother) for sp in specs]
        tuning = {"pre_sweeps": pre, "post_sweeps": post, "inner_cycles": inner, "krylov": kry,
                  "coarse_sweeps": coarse, "smoother": smoother, "fixed": True}
    elif not args.no_autotune:
        # sweep counts, V-cycles per outer residual and planes per block, measured on the largest case
        _, tuning = binding.autotune(max(specs, key=lambda sp: sp.cells), steps=3)
        # (the planes per block are left to the batch rule: a batch has blocks to spare)
        specs = [sp.replace(pre_sweeps=tuning["pre_sweeps"], post_sweeps=tuning["post_sweeps"],
                            inner_cycles=tuning["inner_cycles"], krylov=tuning["krylov"],
                            coarse_sweeps=tuning["coarse_sweeps"], smoother=tuning["smoother"]) for sp in specs]
    N = sum(sp.cells for sp in specs)
    cs = [binding.Case(sp, stream=stream.cuda_stream) for sp in specs]
    batch = binding.Batch(cs, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        batch.step(1, allow_not_converged=True)
    torch.cuda.synchronize()
    l0 = batch.info()["kernel_launches"]
    clocks = Clocks(local)
    clocks.start()
    times, vc, rels = [], [], []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = batch.step(1, allow_not_converged=True)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        vc.append(statistics.mean(x["vcycles_last"] for x in st))
        rels.append(max(x["rel_residual"] for x in st))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = batch.info()["kernel_launches"] - l0
    total_ms = sum(times)
    if dist:
        total_ms = replicas.max_over_ranks(total_ms)
    value = ws * N * args.steps / (total_ms / 1e3)
    prof_steps = min(args.steps, 5)
    tpc = traffic_for(TRAFFIC_PER_CELL, ("batched", args.precision, "sweep_L0"))
    bd = breakdown(batch.profile(prof_steps), prof_steps, {"sweep_L0": tpc * N} if tpc else None)

    # end to end through the C-ABI with host buffers: write every case, one batched step, read back
    e2e = None
    if args.e2e_steps > 0:
        # pinned host buffers in the library's own layout, in the fields' storage precision (FP32
        # for FP32 fields: fvm_read_fields_f32); each step's output is the next input
        hdt = torch.float64 if args.precision == "f64" else torch.float32
        hosts = [torch.empty(7 * sp.cells, dtype=hdt, pin_memory=True).numpy() for sp in specs]
        for c, h in zip(cs, hosts):
            c.read_flat(h)
        te = 0.0
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            for c, h in zip(cs, hosts):
                c.write_flat(h)
            batch.step(1, allow_not_converged=True)
            for c, h in zip(cs, hosts):
                c.read_flat(h)
            te += time.perf_counter() - t0
        e2e = {"value": N * args.e2e_steps / te, "unit": "cell-steps/s",
               "h2d_bytes_per_step": 7 * N * hosts[0].itemsize, "d2h_bytes_per_step": 7 * N * hosts[0].itemsize}
        if dist:
            e2e["value"] = ws * N * args.e2e_steps / replicas.max_over_ranks(te)
    batch.close()

    # the same cases stepped one at a time (each its own graph per step), FP32 and plain FP64
    compare = None
    if ws == 1 and not args.no_compare:
        def one_by_one(case_list, rounds):
            for c in case_list:
                c.step(1, allow_not_converged=True)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(rounds):
                for c in case_list:
                    c.step(1, allow_not_converged=True)
            ev1.record(stream)
            ev1.synchronize()
            return N * rounds / (ev0.elapsed_time(ev1) / 1e3)
        per_case = one_by_one(cs, 2)
        for c in cs:
            c.close()
        plain = dict(precision=cases.FP64, pre_sweeps=3, post_sweeps=3, inner_cycles=0, sweep_planes=0)
        c64 = [binding.Case(sp.replace(**plain), stream=stream.cuda_stream) for sp in specs]
        per_case_fp64 = one_by_one(c64, 1)
        for c in c64:
            c.close()
        # accuracy at equal steps on a subset: the batched reduced-precision form vs the plain FP64 form
        sub = specs[:args.accuracy_cases]
        steps_acc = 5
        b_cs = [binding.Case(sp, stream=stream.cuda_stream) for sp in sub]
        with binding.Batch(b_cs, stream=stream.cuda_stream) as bb:
            sb = bb.step(steps_acc, allow_not_converged=True)
        got = [c.read() for c in b_cs]
        errs, rel64 = [], []
        for sp, g in zip(sub, got):
            with binding.Case(sp.replace(**plain), stream=stream.cuda_stream) as c:
                s64 = c.step(steps_acc, allow_not_converged=True)
                errs.append(field_errors(g, c.read()))
                rel64.append(s64["rel_residual"])
        for c in b_cs:
            c.close()
        compare = {"per_case_same_precision": {"value": per_case, "unit": "cell-steps/s"},
                   "per_case_fp64": {"value": per_case_fp64, "unit": "cell-steps/s"},
                   "speedup_vs_per_case_fp64": value / per_case_fp64,
                   "accuracy": {"cases": len(sub), "steps": steps_acc,
                                "max_rel_error_vs_fp64": {f: max(e[f] for e in errs) for f in cases.FIELDS + ("velocity",)},
                                "rel_residual_batched_max": max(x["rel_residual"] for x in sb),
                                "rel_residual_fp64_max": max(rel64)}}
    else:
        for c in cs:
            c.close()
    if rank == 0:
        sizes = sorted({(sp.nx, sp.ny, sp.nz) for sp in specs})
        line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": arith_dtype(args.precision),
                "data": "synthetic",
                "config": {"workload": f"batched_channels {len(specs)} cases, 64^3 .. 192x96x96, 5-level V-cycles, "
                                       "rel tol 1e-8, one batch per GPU",
                           "autotune": tuning,
                           "cells_per_gpu": N, "cases_per_gpu": len(specs), "sizes": [list(x) for x in sizes],
                           "precision": args.precision, "parallelism": f"replicas x{ws}",
                           "l2": "256 MB buffer written between timed steps (the batch's state is larger than L2)"},
                "vcycles_per_step": statistics.mean(vc), "rel_residual_max": max(rels),
                **bd, "gpu_launches": launches, "clocks": clk, "e2e": e2e, "compare": compare}
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(min(specs, key=lambda sp: sp.cells))
            line["cpu_baseline_all_cores"] = cpu_all_cores(min(specs, key=lambda sp: sp.cells))
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_served(args, rank, ws, local, dist):
    """C5: a Poisson stream of room and channel requests served with
    continuous batching under a device-memory budget: p50 / p99 latency
    (arrival to completion) and the aggregate cell-steps/s."""
    import torch
    from paper_2603_21869_gb300 import binding, build, replicas
    build.ensure_built()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    arrivals, specs = cases.served_rooms(args.requests, seed=rank, rate=args.rate)
    srv = binding.Server(budget_bytes=int(args.budget_gb * (1 << 30)), stream=stream.cuda_stream)
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = srv.now()
    nxt = 0
    done = []
    rid_of = {}   # request id -> index in the stream
    while len(done) < len(specs):
        now = srv.now() - t_start
        while nxt < len(specs) and arrivals[nxt] <= now:
            rid_of[srv.submit(specs[nxt], args.served_steps, t_arrive=t_start + float(arrivals[nxt]))] = nxt
            nxt += 1
        inf = srv.info()
        if inf["running"] == 0 and inf["queued"] == 0 and nxt < len(specs):
            time.sleep(max(0.0, min(0.05, arrivals[nxt] - (srv.now() - t_start))))
            continue
        done += srv.poll(chunk=args.chunk)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_end = srv.now()
    info = srv.info()
    srv.close()
    lat = sorted(d["t_done"] - d["t_arrive"] for d in done)
    q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
    makespan = t_end - t_start
    cell_steps = sum(d["cells"] * d["steps"] for d in done)
    bad = [d for d in done if d["status"] != 0]
    failures = []
    for d in bad[:20]:
        sp = specs[rid_of[d["id"]]]
        failures.append({"request": rid_of[d["id"]], "status": d["status"], "steps_done": d["steps"],
                         "kind": "channel" if not sp.boxes and not sp.vents else "room",
                         "shape": [sp.nx, sp.ny, sp.nz], "rel_residual": d["rel_residual"]})
    compare = served_vs_fp64(args, specs, stream) if (ws == 1 and not args.no_compare and rank == 0) else None
    if dist:
        makespan, cell_steps = replicas.max_over_ranks(makespan), replicas.sum_over_ranks(cell_steps)
    if rank == 0:
        line = {"metric": "cell-steps/s", "value": cell_steps / makespan, "unit": "cell-steps/s", "n_gpus": ws,
                "steps": args.served_steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"served: Poisson arrivals at {args.rate}/s of {len(specs)} requests per GPU "
                                       f"(rooms 64^3 .. 256x128x128 with seeded vents, boxes, heat; 20 % channels), "
                                       f"{args.served_steps} steps each, HBM budget {args.budget_gb} GB, "
                                       f"rounds of {args.chunk} steps",
                           "parallelism": f"replicas x{ws}", "l2": "not flushed (a serving loop)"},
                "latency_s": {"p50": q(0.50), "p99": q(0.99), "max": lat[-1], "mean": statistics.mean(lat)},
                "makespan_s": makespan, "requests": len(done), "failed": len(bad), "failures": failures,
                "server": info, "clocks": clk, "compare": compare,
                "e2e": {"value": cell_steps / makespan, "unit": "cell-steps/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0,
                        "note": "requests enter as case descriptions (fields initialised on the device)"}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def served_vs_fp64(args, specs, stream):
    """The target comparison of the served form: a seeded sample of the same requests, each
    (a) served (mixed precision, batched, one server) and (b) run alone in the plain FP64
    per-case form (FP64 fields and corrections, V(3,3), no Krylov acceleration, one graph
    per step), both for the full number of steps to the same 1e-8 relative residual: the
    cell-steps/s of each and the per-field error of (a) against (b)."""
    import numpy as np
    import torch
    from paper_2603_21869_gb300 import binding
    rng = np.random.default_rng(12345)
    pick = sorted(rng.choice(len(specs), size=min(args.compare_requests, len(specs)), replace=False).tolist())
    sample = [specs[i] for i in pick]
    cells = sum(sp.cells for sp in sample) * args.served_steps
    # (a) served together, all admitted at once
    with binding.Server(budget_bytes=int(args.budget_gb * (1 << 30)), stream=stream.cuda_stream,
                        keep_results=True) as srv:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids = [srv.submit(sp, args.served_steps, t_arrive=srv.now()) for sp in sample]
        done = []
        while len(done) < len(ids):
            done += srv.poll(chunk=args.chunk)
        t_served = time.perf_counter() - t0
        served = {i: srv.read(i) for i in ids}
        rel_served = max(d["rel_residual"] for d in done) if "rel_residual" in done[0] else None
    # (b) the plain FP64 per-case form, one request at a time
    # (the plain V-cycles need about 55 per step on a room with a small outlet: room to reach 1e-8)
    plain = dict(precision=cases.FP64, pre_sweeps=3, post_sweeps=3, inner_cycles=0, krylov=0, sweep_planes=0,
                 max_vcycles=200)
    errs, rels, t_fp64 = [], [], 0.0
    for i, sp in zip(ids, sample):
        with binding.Case(sp.replace(**plain), stream=stream.cuda_stream) as c:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = c.step(args.served_steps, allow_not_converged=True)
            torch.cuda.synchronize()
            t_fp64 += time.perf_counter() - t0
            errs.append(field_errors(served[i], c.read()))
            rels.append(st["rel_residual"])
    return {"requests": len(sample), "steps": args.served_steps,
            "served_mixed_batched": {"value": cells / t_served, "unit": "cell-steps/s",
                                     "rel_residual_max": rel_served},
            "per_case_fp64": {"value": cells / t_fp64, "unit": "cell-steps/s", "rel_residual_max": max(rels)},
            "speedup": t_fp64 / t_served,
            "max_rel_error_vs_fp64": {f: max(e[f] for e in errs) for f in cases.FIELDS + ("velocity",)},
            "note": "the same seeded sample of requests, wall time around each form on one GPU"}


def compare_variants(args):
    """The paper's multigrid scheme (Algorithm 1) against V(3,3) cycles on the
    default channel: device time per iteration (CUDA events) and residual
    contraction per iteration, in FP32 and FP64, from the same state."""
    import torch
    from paper_2603_21869_gb300 import binding, build
    build.ensure_built()
    out = {}
    for pname, prec in (("f32", cases.FP32), ("f64", cases.FP64)):
        for vname, variant in (("vcycle_V33", 0), ("paper_algorithm1", 1)):
            spec = cases.heated_channel_3d(256, 64, 64, mg_levels=6, precision=prec, fixed_vcycles=1,
                                           mg_variant=variant)
            with binding.Case(spec) as c:
                c.step(3)
                rels, ms = [], []
                for _ in range(20):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record()
                    rels.append(c.vcycle(1))
                    b.record()
                    b.synchronize()
                    ms.append(a.elapsed_time(b))
            out[f"{pname}/{vname}"] = {"ms_per_iteration": statistics.median(ms[2:]),
                                       "factor_per_iteration": (rels[-1] / rels[9]) ** (1 / 10),
                                       "rel_after_1_10_20": [rels[0], rels[9], rels[19]]}
    print(json.dumps({"comparison": "multigrid schemes on heated_channel_3d 256x64x64 (6 levels)",
                      "note": "one iteration per fvm_vcycle call (with its residual and a host read)",
                      "results": out}), flush=True)


def cpu_baseline(spec, workload="channel", budget_s=25.0):
    """Time the oracle (rank 0, N = 1) on a bounded sample: whole steps of the workload, or of
    its scaled-down copy when one full step would take minutes."""
    from oracle.step import OracleCase
    sp, what = oracle_sample(spec, workload)
    t0 = time.perf_counter()
    c = OracleCase(sp)
    n = 0
    ts = time.perf_counter()
    while n < 1 or (time.perf_counter() - t0 < budget_s and n < 3):
        c.step()
        n += 1
    el = time.perf_counter() - ts
    return {"value": sp.cells * n / el, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} step(s) of {what}, numpy float64 on one host thread "
                      f"({os.cpu_count()} cores present)"}


def _oracle_steps(job):
    """One worker of the all-cores oracle baseline: its own copy of the case, n whole steps."""
    spec, n = job
    from oracle.step import OracleCase
    c = OracleCase(spec)
    t = time.perf_counter()
    for _ in range(n):
        c.step()
    return time.perf_counter() - t


def cpu_all_cores(spec, n=1):
    """The oracle on every host core: one process per core, each stepping its own copy of the
    case (cases are independent, as in a batch); aggregate = cores x cells x steps / slowest.
    Spawned processes (the parent already holds a CUDA context)."""
    import multiprocessing as mp
    p = os.cpu_count() or 1
    # one thread per process (no BLAS thread pools competing for the cores)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with mp.get_context("spawn").Pool(p) as pool:
            ts = pool.map(_oracle_steps, [(spec.replace(precision=cases.FP64), n)] * p)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"value": p * spec.cells * n / max(ts), "unit": "cell-steps/s", "cores": p, "kind": "oracle",
            "sample": f"{p} processes, one copy of the {spec.nx}x{spec.ny}x{spec.nz} case each, {n} step(s); "
                      "aggregate over the slowest process"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=list(PREC))
    ap.add_argument("--workload", default="room")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cases", type=int, default=64, help="batched workload: cases per GPU")
    ap.add_argument("--accuracy-cases", type=int, default=8)
    ap.add_argument("--accuracy-steps", type=int, default=5, help="steps of the per-field comparison with FP64")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep V(3,3), the default grouping and plane rule")
    ap.add_argument("--params", default=None, metavar="PRE,POST,INNER,PLANES,KRYLOV[,COARSE[,SMOOTHER]]",
                    help="fixed multigrid parameters instead of the autotuner's (e.g. for profiling runs, where "
                         "the profiler's overhead would distort the autotuner's timings)")
    ap.add_argument("--krylov", default="auto", choices=["auto", "0", "1"],
                    help="flexible-CG acceleration of the pressure solve (auto: the autotuner's choice, else off)")
    ap.add_argument("--adjoint", action="store_true",
                    help="also time the projection adjoint (fvm_projection_vjp) on an FP64 copy of the workload")
    ap.add_argument("--rk-stages", type=int, default=1, choices=[1, 2, 3],
                    help="explicit stage: forward Euler (1) or the strong-stability-preserving Runge-Kutta "
                         "scheme of order 2 or 3")
    ap.add_argument("--requests", type=int, default=64, help="served workload: requests per GPU")
    ap.add_argument("--rate", type=float, default=20.0, help="served workload: arrivals per second")
    ap.add_argument("--served-steps", type=int, default=30, help="served workload: steps per request")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--chunk", type=int, default=10, help="served workload: steps per scheduling round")
    ap.add_argument("--compare-requests", type=int, default=8,
                    help="served workload: requests of the sample compared with the plain FP64 per-case form")
    ap.add_argument("--compare-variants", action="store_true",
                    help="time the paper's multigrid scheme against V-cycles and exit")
    args = ap.parse_args()
    if args.compare_variants:
        compare_variants(args)
        return
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.workload == "served":
        rank, ws, local, dist = dist_setup()
        if args.impl == "ours":
            run_served(args, rank, ws, local, dist)
            return
        args.steps, args.warmup = min(args.steps, 2), 0
        _, specs = cases.served_rooms(args.requests, seed=rank, rate=args.rate)
        run_reference(args, min(specs, key=lambda sp: sp.cells),
                      "served rooms: the smallest request (oracle, one request at a time)", rank, ws)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "batched":
        rank, ws, local, dist = dist_setup()
        if args.impl == "reference":
            args.steps, args.warmup = min(args.steps, 2), 0
            spec = min(cases.batched_channels(args.cases, seed=rank, mg_levels=5), key=lambda sp: sp.cells)
            run_reference(args, spec, "batched_channels: the smallest case (oracle, one case at a time)", rank, ws)
        else:
            run_batched(args, rank, ws, local, dist)
            return
        if dist:
            dist.destroy_process_group()
        return
    spec, label = workload(args.workload, PREC[args.precision])
    if args.rk_stages > 1:
        spec = spec.replace(rk_stages=args.rk_stages)
        label += f", SSP-RK{args.rk_stages} explicit stage"
    rank, ws, local, dist = dist_setup()
    tuning = None
    if args.params:
        pre, post, inner, planes, kry, coarse, smoother = parse_params(args.params)
        spec = spec.replace(pre_sweeps=pre, post_sweeps=post, inner_cycles=inner, sweep_planes=planes, krylov=kry,
                            coarse_sweeps=coarse, smoother=smoother)
        label = label.replace("V(3,3)", f"V({pre},{post})")
        tuning = {"pre_sweeps": pre, "post_sweeps": post, "inner_cycles": inner, "sweep_planes": planes,
                  "krylov": kry, "coarse_sweeps": coarse, "smoother": smoother, "fixed": True}
    elif args.impl == "ours" and not args.no_autotune and spec.nz > 1:
        # smoother sweeps, V-cycles per outer residual and planes per block, measured (fvm_autotune)
        from paper_2603_21869_gb300 import binding as _b, build as _bd
        _bd.ensure_built()
        import torch
        torch.cuda.set_device(local)
        spec, tuning = _b.autotune(spec, steps=3)
        label = label.replace("V(3,3)", f"V({spec.pre_sweeps},{spec.post_sweeps})")
    if args.krylov != "auto":
        spec = spec.replace(krylov=int(args.krylov))
    if args.impl == "reference":
        # each step is a bounded sample of the workload (the oracle on a room scaled to 1/64 of
        # the cells, about 2-5 s a step on one host thread); K and W as given
        run_reference(args, spec, label, rank, ws, args.workload)
        if dist:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2603_21869_gb300 import binding, build, replicas
    build.ensure_built()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    case = binding.Case(spec, stream=stream.cuda_stream)
    N = spec.cells
    vcycles = 0
    for _ in range(args.warmup):
        vcycles += case.step(1, allow_not_converged=True)["vcycles_last"]
    torch.cuda.synchronize()
    launches0 = case.info()["kernel_launches"]
    clocks = Clocks(local)
    clocks.start()
    times = []
    vc = []
    rels = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: each step is one CUDA graph (V-cycle loop on the device)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        st = case.step(1, allow_not_converged=True)
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        vc.append(st["vcycles_last"])
        rels.append(st["rel_residual"])
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = case.info()["kernel_launches"] - launches0
    total_ms = sum(times)
    if dist:
        total_ms = replicas.max_over_ranks(total_ms)
    value = ws * N * args.steps / (total_ms / 1e3)

    # per-kernel breakdown: the same steps again, launch by launch, each kernel
    # bracketed by CUDA events on the case's stream (the profiling hook)
    case.profile(True)
    prof_steps = min(args.steps, 10)
    for _ in range(prof_steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        case.step(1, allow_not_converged=True)
    prof = case.profile_read()
    case.profile(False)
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, d = dom
    peak, peak_src = peaks()
    achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
    mg_names = [k for k in prof if any(k.startswith(p) for p in ("sweep", "resid", "prolong", "coarse"))]
    mg_bytes = sum(prof[k]["bytes"] for k in mg_names)
    mg_ms = sum(prof[k]["ms"] for k in mg_names)
    kernel_ms = sum(v["ms"] for v in prof.values())

    # the lambda_2 vortex diagnostic (fvm_lambda2) on the current state, outside the step: its
    # kernel timed by the profiling hook, L2 flushed before each call
    case.profile(True)
    lam_out = np.empty(N)
    for _ in range(3):
        with torch.cuda.stream(stream):
            flush.zero_()
        case.lambda2(out=lam_out)
    lp = case.profile_read()["lambda2"]
    case.profile(False)
    lam_gbs = lp["bytes"] / (lp["ms"] / 1e3) / 1e9
    diagnostics = {"lambda2": {"ms_per_call": lp["ms"] / lp["launches"], "gbs": lam_gbs,
                               "frac": lam_gbs / peak, "bytes_per_cell": lp["bytes"] / lp["launches"] / N,
                               "vortex_cells": int(np.count_nonzero(lam_out < 0))}}
    if args.adjoint and rank == 0:
        diagnostics["projection_vjp"] = time_projection_vjp(spec, stream, flush, peak)

    # end to end through the C-ABI with host buffers: write state, one step, read state
    e2e = None
    if args.e2e_steps > 0:
        # a pinned host buffer in the library's own layout, in the fields' storage precision
        # (FP32 for FP32 fields: fvm_read_fields_f32); each step's output is the next input
        hdt = torch.float64 if args.precision == "f64" else torch.float32
        host = torch.empty(7 * N, dtype=hdt, pin_memory=True).numpy()
        case.read_flat(host)
        te = 0.0
        for _ in range(args.e2e_steps):
            t0 = time.perf_counter()
            case.write_flat(host)
            case.step(1, allow_not_converged=True)
            case.read_flat(host)
            te += time.perf_counter() - t0
        e2e = {"value": N * args.e2e_steps / te, "unit": "cell-steps/s",
               "h2d_bytes_per_step": 7 * N * host.itemsize, "d2h_bytes_per_step": 7 * N * host.itemsize}
        if dist:
            e2e["value"] = ws * N * args.e2e_steps / replicas.max_over_ranks(te)

    # per-field error of this precision against the FP64 path: the same case from its initial
    # state, a few steps each (not timed)
    accuracy = None
    if args.precision != "f64" and not args.no_compare and rank == 0:
        case.close()
        runs = {}
        for prec in (PREC[args.precision], cases.FP64):
            with binding.Case(spec.replace(precision=prec), stream=stream.cuda_stream) as c2:
                st2 = c2.step(args.accuracy_steps, allow_not_converged=True)
                runs[prec] = (c2.read(), st2)
        (got, s_got), (ref, s_ref) = runs[PREC[args.precision]], runs[cases.FP64]
        accuracy = {"steps": args.accuracy_steps, "max_rel_error_vs_fp64": field_errors(got, ref),
                    "rel_residual": s_got["rel_residual"], "rel_residual_fp64": s_ref["rel_residual"]}

    line = None
    if rank == 0:
        line = {"metric": "cell-steps/s", "value": value, "unit": "cell-steps/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": arith_dtype(args.precision), "data": "synthetic",
                "config": {"workload": label, "cells_per_gpu": N, "precision": args.precision,
                           "parallelism": f"replicas x{ws}", "l2": "256 MB buffer written between timed steps",
                           "autotune": tuning},
                "vcycles_per_step": statistics.mean(vc), "rel_residual_max": max(rels),
                "roofline": {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_source": peak_src,
                             "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
                             "traffic": traffic_for(TRAFFIC, (args.workload, args.precision, name)),
                             "bytes_per_launch": d["bytes"] / d["launches"],
                             "ms_per_launch": d["ms"] / d["launches"], "launches": d["launches"]},
                "vcycle": {"gbs": mg_bytes / (mg_ms / 1e3) / 1e9 if mg_ms else None,
                           "frac": (mg_bytes / (mg_ms / 1e3) / 1e9) / peak if mg_ms else None,
                           "ms_per_step": mg_ms / prof_steps},
                "profiled_pass": {"steps": prof_steps, "kernel_ms_per_step": kernel_ms / prof_steps,
                                  "mode": "launch by launch, CUDA events around every kernel"},
                "kernels": {k: {"ms_per_step": v["ms"] / prof_steps, "launches_per_step": v["launches"] / prof_steps,
                                "gbs": v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] else None}
                            for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])[:12]},
                "gpu_launches": launches, "clocks": clk, "e2e": e2e, "accuracy": accuracy,
                "diagnostics": diagnostics}
    case.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, args.workload)
        sp_all, _ = oracle_sample(spec, args.workload)
        if sp_all.cells <= (1 << 21):   # one copy per core must fit in host memory
            line["cpu_baseline_all_cores"] = cpu_all_cores(sp_all)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
