"""Benchmark: MPR gap site-updates/s of the whole gap-filling job on one GB300.

One step = the whole hot path on one batch (Alg. 2): map + hot start + e_s,
the specific-energy-matching temperature estimate, n_equil equilibration
sweeps, n_meas measurement sweeps and the prediction, for the workload
"4096 x 4096 lognormal GRF, 40% gaps, 32 realisations" (50 + 100 sweeps).
value = gap site-updates of the step's sweeps / step time (the temperature
estimate's lattice updates are not counted, its time is).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Several GPUs run independent replicas of the job (realisations are
independent; there is no collective): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MPR gap site-updates/s at 4096^2 (FP32, batched) and % HBM roofline vs plain path"
UNIT = "gap site-updates/s"
WORKLOAD = "lognormal4096_p40: 4096x4096 lognormal GRF (log-mean 5, log-std 1, exponential ell=16), 40% uniform gaps, 32 realisations, 50 equilibration + 100 measurement sweeps"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Sources that determine the colour-pass kernel; the DRAM traffic recorded
# from an ncu capture applies only while their hash is the recorded one.
KERNEL_SOURCES = ("mpr_tiled_kernel.cuh", "mpr_device.cuh", "mpr_async.cuh", "mpr_internal.h")
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "traffic.json")


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1710_03038_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic_per_update(key="dram_bytes_per_gap_update"):
    """A per-update figure of the sampling colour pass (DRAM bytes by default, or
    issued thread-instructions) from the committed record of an ncu capture, or
    None when the kernel sources changed since or the record lacks it."""
    if not os.path.exists(TRAFFIC_RECORD):
        return None
    with open(TRAFFIC_RECORD) as f:
        rec = json.load(f)
    if rec.get("kernel_sources_sha16") != kernel_sources_hash() or key not in rec:
        return None
    return float(rec[key])


def record_traffic(csv_path, size, command):
    """Writes the traffic record from `ncu --page raw --csv` output of one sampling
    launch of the colour pass (the kernel whose accumulation mode, its fifth
    template argument, is not 0)
    on the benchmark field at side `size`: DRAM bytes read + written per gap
    site-update, and the kernel sources' hash at the time of writing."""
    import csv
    import synthetic
    with open(csv_path) as f:
        rows = list(csv.reader(l for l in f if not l.startswith("==")))
    head, units = rows[0], rows[1]
    k = head.index("Kernel Name")
    import re
    pat = re.compile(r"tiled_pass_kernel<\d+, \d+, \d+, \d+, ([12]), \d+>")
    hit = [r for r in rows[2:] if pat.search(r[k])]
    if not hit:
        raise SystemExit("no sampling launch of the colour pass in " + csv_path)
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    tot = 0.0
    for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        i = head.index(m)
        tot += float(hit[0][i].replace(",", "")) * scale[units[i]]
    w = synthetic.workload("lognormal4096", L=size)
    updates = int(w.gap[0].sum()) * w.chains / 2.0
    extra = {}
    if "smsp__inst_executed.sum" in head:
        inst = float(hit[0][head.index("smsp__inst_executed.sum")].replace(",", ""))
        extra["thread_instructions_per_gap_update"] = round(inst * 32 / updates, 2)
    rec = {"dram_bytes_per_gap_update": round(tot / updates, 4), **extra,
           "kernel": hit[0][k], "field_side": size, "updates_per_launch": updates,
           "dram_bytes_per_launch": tot, "kernel_sources_sha16": kernel_sources_hash(),
           "command": command}
    with open(TRAFFIC_RECORD, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec))


def issue_ceiling(updates_per_s, clocks, dev):
    """Issued thread-instructions/s of the sampling pass (recorded instructions per
    update x its measured update rate) against the GPU's issue rate, or None
    without a current record."""
    import torch
    ipu = recorded_traffic_per_update("thread_instructions_per_gap_update")
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if ipu is None or not mhz:
        return None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sms * 4 * 32 * mhz * 1e6
    ach = ipu * updates_per_s
    return {"achieved": ach, "peak": peak, "unit": "thread-instructions/s", "frac": ach / peak,
            "thread_instructions_per_gap_update": ipu, "sms": sms, "sm_mhz": mhz}


def max_over_ranks(values, device):
    """Element-wise maximum of per-rank timings over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(units_per_rank_step, steps, world_size, ms_max):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank_step * steps * world_size / (ms_max / 1e3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------ oracle baseline

def _oracle_worker(args):
    path, chain, sweeps = args
    import numpy as np
    import oracle
    d = np.load(path)
    phi, g = d["phi"], d["gap"]
    phi = oracle.hot_start(phi, g, 1, 0, chain)
    P = int(g.sum())
    t0 = time.perf_counter()
    for s in range(sweeps):
        phi, _ = oracle.sweep(phi, g, T=3e-3, a=1.0 + s / 3.0, seed=1, chain=chain, sweep_index=s)
    return P * sweeps, time.perf_counter() - t0


def _crop(crop):
    import numpy as np
    import oracle
    import synthetic
    w = synthetic.workload("lognormal4096")
    z = w.z[0][:crop, :crop].astype(np.float64)
    g = w.gap[0][:crop, :crop]
    phi, _, _ = oracle.map_to_angles(z, g)
    return phi, g, int(w.gap[0].sum())


def host_cpu():
    """CPU model, logical cores and maximum clock of the host (lscpu, else /proc/cpuinfo)."""
    info = {"cores": os.cpu_count() or 1}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            v = v.strip()
            if k.strip() == "Model name" and "model" not in info:
                info["model"] = v
            elif k.strip() == "CPU max MHz":
                info["max_mhz"] = float(v)
    except (OSError, subprocess.SubprocessError, ValueError):
        pass
    if "model" not in info and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                info["model"] = line.split(":", 1)[1].strip()
                break
    return info


def cpu_baseline(workers=None, crop=2048, sweeps=1, data=None, single=True):
    """The FP64 oracle on the host cores: one sweep of a crop of the input per worker
    process on every core, and (single=True) the same work in one process alone."""
    import tempfile
    import numpy as np
    import oracle
    oracle.build()
    workers = workers or (os.cpu_count() or 1)
    phi, g, _ = data if data is not None else _crop(crop)
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "crop.npz")
        np.savez(path, phi=phi, gap=g)
        one = None
        if single:
            with ctx.Pool(1) as pool:
                u1, s1 = pool.map(_oracle_worker, [(path, 0, sweeps)])[0]
            one = u1 / s1
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.map(_oracle_worker, [(path, c, sweeps) for c in range(workers)])
        wall = time.perf_counter() - t0
    units = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    cpu = host_cpu()
    out = {"value": units / busy, "unit": UNIT, "cores": workers, "kind": "oracle",
           "sample": f"{sweeps} hybrid sweep(s) of a {phi.shape[0]}x{phi.shape[1]} crop of the "
                     f"4096^2 input, one realisation per worker, {workers} worker processes "
                     f"({units} gap site-updates, {wall:.1f} s wall)", "wall_s": wall,
           "cpu": cpu}
    if one is not None:
        out["single_thread"] = {"value": one, "unit": UNIT, "cores": 1}
    return out


# ------------------------------------------------------------ GPU arm

def run_gpu(args):
    import numpy as np
    import torch
    import synthetic
    import paper_1710_03038_gb300 as mpr
    from paper_1710_03038_gb300 import build

    ws, rank, local = _dist()
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    w = synthetic.workload("lognormal4096", L=args.size)
    z_h, g_h = w.z[0], w.gap[0]
    R, ne, nm = w.chains, w.n_equil, w.n_meas
    P = int(g_h.sum())
    N = g_h.size
    f = P / N
    z_d = torch.from_numpy(z_h).to(dev)
    g_d = torch.from_numpy(g_h).to(dev)
    z_pin = torch.from_numpy(z_h).pin_memory()
    g_pin = torch.from_numpy(g_h).pin_memory()
    params = mpr.Params(seed=12345 + rank, path=args.path, use_graphs=not args.no_graphs)
    topts = mpr.TOpts()
    # a stream of our own: runs of sweeps are captured into CUDA graphs and replayed
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    torch.cuda.set_stream(stream)

    sweep_events = []
    equil_events = []
    launches = []

    def step(z_in, g_in, host_out=None, timed=False):
        ctx = mpr.Context([z_in], [g_in], chains=R, params=params, topts=topts, device=dev)
        if args.T is None:
            ctx.estimate_T_async()
        else:
            ctx.set_T([args.T])
        # events around each run of sweeps (one graph replay each), the same
        # launches as an untimed step
        if timed:
            q0 = torch.cuda.Event(enable_timing=True)
            q1 = torch.cuda.Event(enable_timing=True)
            q0.record(stream)
        if not launches:
            launches.extend(ctx.sweep_launches())
        ctx.sweep(ne, "equil")
        if timed:
            q1.record(stream)
            equil_events.append((q0, q1))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        ctx.sweep(nm, "measure")
        if timed:
            e1.record(stream)
            sweep_events.append((e0, e1))
        if host_out is not None:
            ctx.predict_host(host_out)
            out = None
        else:
            out = ctx.predict()
        ctx.close()
        return out

    for _ in range(args.warmup):
        step(z_d, g_d)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clk = ClockSampler(local)
    clk.start()
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(z_d, g_d, timed=True)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = t0.elapsed_time(t1)
    clocks = clk.stop()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    ms_e2e = float("nan")
    if not args.no_e2e:
        zh_out = torch.empty(N, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step(z_pin, g_pin, host_out=zh_out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_e2e = e0.elapsed_time(e1)

    ms, ms_e2e = max_over_ranks([ms, ms_e2e], dev)

    units_step = (ne + nm) * P * R
    value = job_throughput(units_step, args.steps, ws, ms)
    e2e = job_throughput(units_step, args.steps, ws, ms_e2e)
    sweep_ms = [a.elapsed_time(b) / nm for a, b in sweep_events]
    equil_ms = [a.elapsed_time(b) / ne for a, b in equil_events]
    launch_ms = statistics.mean(sweep_ms) / 2.0  # two colour passes per sweep
    peak, peak_kind = _peaks()
    alg_bytes_per_update = 4.0 * (1.0 / f + 1.0)
    achieved = (P * R / 2.0) * alg_bytes_per_update / (launch_ms / 1e3) / 1e9
    # ncu DRAM bytes of one sampling launch, captured at 2048^2 and scaled by the
    # updates of one 4096^2 launch (the pass moves a fixed amount per update)
    tpu = recorded_traffic_per_update() if args.path == "tiled" else None
    traffic = None if tpu is None else tpu * P * R / 2.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": "gb300",
        "config": {"workload": WORKLOAD, "path": args.path, "image": [4096, 4096],
                   "gap_fraction": round(f, 6), "realisations": R, "n_equil": ne, "n_meas": nm,
                   "T_estimate": {"L": 256, "chains": topts.chains, "iters": topts.iters,
                                  "n_equil": topts.n_equil, "n_meas": topts.n_meas},
                   "l2": "inputs larger than L2 (state 2.1 GB)",
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "tiled_pass_kernel" if args.path == "tiled" else "plain_pass_kernel",
                     "alg_bytes_per_gap_update": alg_bytes_per_update,
                     "avg_launch_ms": launch_ms, "peak_kind": peak_kind},
        # the ceiling the pass actually meets: instruction issue (SMs x 4 schedulers x
        # 32 lanes x the sampled SM clock), with the recorded instructions per update
        "issue": issue_ceiling(P * R / 2.0 / (launch_ms / 1e3), clocks, dev),
        # gap site-updates/s of the sweeps alone, by phase (equilibration: the run of
        # sweeps as one graph replay; measurement: the 100 sweeps as one replay)
        "phases": {"equil": P * R / (statistics.mean(equil_ms) / 1e3),
                   "measure": P * R / (statistics.mean(sweep_ms) / 1e3), "unit": UNIT},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": N * 5,
                "d2h_bytes_per_step": N * 4},
        "clocks": clocks,
    }
    # kernel launches of one step: the library's per-sweep count for the realisations
    # and for the temperature lattices, the Newton steps (and their set-up), the 16
    # initialisation kernels of the two contexts (map, extremes, sample energy, tile
    # tables, hot starts, chain set-up) and the prediction
    t_sweeps = topts.iters * (topts.n_equil + topts.n_meas) + topts.n_equil
    line["gpu_launches"] = args.steps * (launches[0] * (ne + nm) + launches[1] * t_sweeps
                                         + topts.iters + 1 + 16 + 1)
    if not args.no_plain:
        # the plain single-image path on the same job (one warm-up, one timed step)
        plain = mpr.Params(seed=12345 + rank, path="plain")
        pctx = mpr.Context([z_d], [g_d], chains=R, params=plain, topts=topts, device=dev)
        pctx.close()
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        ctx_p = mpr.Context([z_d], [g_d], chains=R, params=plain, topts=topts, device=dev)
        if args.T is None:
            ctx_p.estimate_T_async()
        else:
            ctx_p.set_T([args.T])
        ctx_p.sweep(ne, "equil")
        ctx_p.sweep(nm, "measure")
        ctx_p.predict()
        q1.record(stream)
        torch.cuda.synchronize()
        ctx_p.close()
        plain_value = units_step / (q0.elapsed_time(q1) / 1e3)
        line["plain_path"] = {"value": plain_value, "unit": UNIT, "steps": 1,
                              "speedup_of_tiled": value / ws / plain_value}
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_baseline"].pop("wall_s", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return None
    data = _crop(1024)
    P = data[2]
    vals, walls = [], []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(crop=1024, data=data, single=False)
        if k >= args.warmup:
            vals.append(cb["value"])
            walls.append(cb["wall_s"])
    value = statistics.mean(vals)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(walls),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample": "oracle sweeps on crops of the input"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gap_sites": P,
    }
    print(json.dumps(line), flush=True)
    return line


def workload_rates(names):
    """Sweep rates of the named synthetic workloads (tiled path, default launch
    configuration, temperature from the estimate): one JSON line per workload with
    the gap site-updates/s of 20 equilibration and of 20 measurement sweeps (graph
    replays, CUDA events) and the HBM fraction at 4 (1/f + 1) bytes per update.
    These are the parity workloads' rates, not benchmark lines."""
    import torch
    import synthetic
    import paper_1710_03038_gb300 as mpr
    peak, peak_kind = _peaks()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    for name in names:
        w = synthetic.workload(name)
        zs = [torch.from_numpy(z).cuda() for z in w.z]
        gs = [torch.from_numpy(g).cuda() for g in w.gap]
        P = int(sum(int(g.sum()) for g in w.gap))
        N = int(sum(g.size for g in w.gap))
        f = P / N
        ctx = mpr.Context(zs, gs, chains=w.chains, params=mpr.Params(seed=3), device="cuda")
        ctx.estimate_T_async()
        ctx.sweep(10, "equil")
        torch.cuda.synchronize()
        out = {"workload": w.name, "images": len(w.z), "sites": N, "gap_fraction": round(f, 4),
               "realisations": w.chains, "unit": UNIT, "peak_gbs": peak, "peak_kind": peak_kind}
        for phase in ("equil", "measure"):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.sweep(20, phase)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
            rate = P * w.chains / (ms / 1e3)
            out[phase] = {"ms_per_sweep": round(ms, 4), "value": float(f"{rate:.4g}"),
                          "hbm_frac": round(rate * 4.0 * (1.0 / f + 1.0) / (peak * 1e9), 4)}
        ctx.close()
        print(json.dumps(out), flush=True)


def launch_ranks(n):
    """--gpus N without a launcher: N local ranks through torch.distributed.run (one
    process per GPU, RANK / LOCAL_RANK / WORLD_SIZE set for each), same arguments."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def dist_check(args):
    """Host-side plumbing of a multi-rank run without GPU work: every rank reports a
    timing, the slowest rank's counts, rank 0 prints one line (CPU ranks use gloo)."""
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("gloo")
    ms = 100.0 + 10.0 * rank
    ms_max = max_over_ranks([ms], torch.device("cpu"))[0]
    value = job_throughput(1000, args.steps, ws, ms_max)
    if ws > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps({"check": "dist", "n_gpus": ws, "ms": ms_max, "value": value}), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--path", default="tiled", choices=["tiled", "plain"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-graphs", action="store_true", help="launch sweeps without CUDA graphs")
    ap.add_argument("--size", type=int, default=4096,
                    help="image side (4096 is the benchmark; smaller sides are for profiler captures)")
    ap.add_argument("--T", type=float, default=None,
                    help="fixed temperature instead of the estimate (profiler captures)")
    ap.add_argument("--dist-check", action="store_true",
                    help="check the multi-rank host logic without GPU work")
    ap.add_argument("--record-traffic", default=None, metavar="NCU_RAW_CSV",
                    help="write the roofline traffic record from `ncu --page raw --csv` output of "
                         "one sampling launch captured on the field of side --size")
    ap.add_argument("--ncu-command", default="", help="the capture's command, kept in the record")
    ap.add_argument("--rates", nargs="*", default=None, metavar="WORKLOAD",
                    help="print the sweep rates of these synthetic workloads (all when none "
                         "is named) instead of the benchmark line")
    args = ap.parse_args()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_ranks(args.gpus))
    if args.record_traffic:
        record_traffic(args.record_traffic, args.size, args.ncu_command)
    elif args.dist_check:
        dist_check(args)
    elif args.rates is not None:
        import synthetic
        workload_rates(args.rates or [n for n in synthetic.WORKLOADS if n != "grf64"])
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
