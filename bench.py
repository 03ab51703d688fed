#!/usr/bin/env python3
"""Throughput benchmark of the fused D2Q9 BGK cylinder step (one JSON line).

Default workload: Re = 100 cylinder, D = 400, 16000 x 8000 lattice (128M
nodes), U = 0.04, tau = 0.98 (Eqs. 16-17), free-slip top/bottom, FP32
populations.  One step = one fused update of every node (pull-stream,
boundary rules, BGK collision, momentum-exchange force of the cylinder).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

value      = GLUPS over all ranks (nodes x steps / max-over-ranks device time),
             inputs resident in HBM (9.2 GB of populations, far above L2).
e2e        = the same metric through the C ABI with host buffers: upload of
             the initial fields from pinned memory, K steps each followed by a
             read of that step's Cd/Cl, read-back of the final fields.
roofline   = algorithmic bytes of one step (72 B/node FP32) over the step
             kernel's mean launch time (CUDA events on its stream), against
             the measured HBM copy bandwidth.
cpu_baseline / --impl reference = the FP64 test oracle on the host cores on a
             bounded sample of the same workload (a full-width strip).
Multi-GPU runs are independent replicas of the lattice (weak scaling).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GLUPS + % HBM roofline (D2Q9 BGK cylinder); wall time to periodic Cd/Cl/St"
UNIT = "GLUPS"

# dram__bytes_read.sum + dram__bytes_write.sum per launch of the step kernel,
# per node, per storage form, from one ncu capture each, with the
# kernel-source digest they were taken for; a figure is reported only while
# the step kernel source is unchanged.
# Taken on the 8000 x 4000 lattice of the same geometry (32M nodes, 2.3 GB of
# FP32 populations, far above L2) in the 768-node-tile shape the 16000 x 8000
# lattice uses; traffic per node does not depend on the lattice size.
NCU_TRAFFIC = {"digest": "749fa125f3d3d2f5",
               "bytes_per_node": {"f32": (1154348288 + 1102509824) / 32e6, "bf16sr": (593798144 + 532119808) / 32e6,
                                  "f16sr": (594534656 + 531918080) / 32e6}}

# The paper's own Re = 100 results (Table 2, "present work": MRT, D = 20,
# U = 0.02, 800 x 400), quoted as context; the paper states no hardware.
PAPER_TABLE2 = {"cd_mean": 1.4, "cl": 0.31, "st": 0.168,
                "source": "Table 2 (present work, Re = 100, MRT, D = 20, U = 0.02); no hardware or timing stated"}


# ----------------------------------------------------------------- helpers


def STORAGE_IDS(lbm):
    return {"f32": lbm.LBM_F32, "f16": lbm.LBM_F16_OFS, "bf16": lbm.LBM_BF16_OFS, "f64": lbm.LBM_F64,
            "f16sr": lbm.LBM_F16_SR, "bf16sr": lbm.LBM_BF16_SR}


def kernel_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2605_02185_gb300", "csrc")
    for name in ("lbm_device.cuh", "lbm_kernels.cuh"):
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def measured_bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed on its own."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        # let nvidia-smi finish starting up before anything is timed
        t0 = time.time()
        while not self.lines and time.time() - t0 < 10.0:
            time.sleep(0.05)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def dist_init(backend: str):
    import torch.distributed as dist
    rank, world, _ = dist_env()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if dist.get_backend() == "nccl" and device is not None:
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity when alone)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    dev = device if (device is not None and dist.get_backend() == "nccl") else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(nodes_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Weak scaling: every rank advances its own lattice replica."""
    return nodes_per_rank * steps * world / max_seconds / 1e9


# ------------------------------------------------------------ CPU oracle


def oracle_strip(workload, rows: int):
    """The FP64 oracle on a full-width strip of `rows` rows through the
    cylinder centre of `workload` (free-slip strip edges)."""
    import numpy as np
    from oracle import oracle as O
    y0 = max(0, workload.yc - rows // 2)
    mask = workload.mask()[y0:y0 + rows]
    o = O.Oracle(workload.nx, rows, workload.tau, workload.U, bc_y=O.Y_FREESLIP, mask=mask)
    rho = np.ones((rows, workload.nx))
    u = np.where(mask == 1, 0.0, workload.U)
    o.init_equilibrium(rho, u, np.zeros_like(rho))
    return o, O.max_threads()


def cpu_baseline(workload, target_s: float = 10.0, rows: int = 256):
    o, cores = oracle_strip(workload, rows)
    t0 = time.perf_counter()
    o.run(1)
    one = time.perf_counter() - t0
    n = max(2, int(target_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    o.run(n)
    dt = time.perf_counter() - t0
    cells = workload.nx * rows
    return {"value": cells * n / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, {workload.nx}x{rows} full-width strip through the cylinder of "
                      f"{workload.name}, {n} steps in {dt:.1f} s ({cells * n / dt / 1e6:.1f} MLUPS)"}


def run_reference(args, workload):
    rank, world = dist_init("gloo")
    if rank != 0:
        return 0
    rows = args.ref_rows
    o, cores = oracle_strip(workload, rows)
    o.run(args.warmup)
    t0 = time.perf_counter()
    o.run(args.steps)
    dt = time.perf_counter() - t0
    cells = workload.nx * rows
    val = cells * args.steps / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload.name, "nx": workload.nx, "ny": workload.ny, "D": workload.D,
                   "U": workload.U, "tau": workload.tau, "bc": "freeslip",
                   "sample_rows": rows, "parallelism": "host cores (OpenMP)"},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"FP64 oracle, {workload.nx}x{rows} full-width strip through the cylinder, "
                                   f"{args.steps} timed steps"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours


def run_ours(args, workload):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init("nccl")
    from paper_2605_02185_gb300 import lbm

    storage = STORAGE_IDS(lbm)[args.storage]
    shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
    nx, ny = workload.nx, workload.ny
    stream = torch.cuda.Stream(device)
    kernel = {"auto": lbm.LBM_KERNEL_AUTO, "tma": lbm.LBM_KERNEL_TMA, "direct": lbm.LBM_KERNEL_DIRECT,
              "wave": lbm.LBM_KERNEL_TMA_WAVE}[args.kernel]
    coll = lbm.LBM_COLLIDE_MRT if args.collision == "mrt" else lbm.LBM_COLLIDE_BGK
    lat = lbm.lattice_for(workload, storage=storage, kernel=kernel, shape=shape, ctas_per_sm=args.ctas_per_sm,
                          stream=stream, device=device, collision=coll)
    rho0, u0, v0 = workload.initial_fields()
    pin = [torch.from_numpy(a).pin_memory() for a in (rho0, u0, v0)]
    del rho0, u0, v0
    lat.init_fields(*(p.numpy() for p in pin))
    lat.step(args.warmup)
    lat.sync()

    # ---- device-resident timing
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(device)
    torch.cuda.synchronize(device)
    launches0 = lat.launch_count()
    ev0.record(stream)
    lat.step(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(device)
    barrier(device)
    clocks = sampler.stop()
    launches = lat.launch_count() - launches0
    lat.sync()
    t_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(t_ms / 1e3, device)
    value = whole_job_glups(nx * ny, args.steps, world, t_max)
    per_launch_s = (t_ms / 1e3) / args.steps
    bytes_step = lat.bytes_per_step()
    peak, peak_src = measured_peaks()
    achieved = bytes_step / per_launch_s / 1e9
    digest = kernel_digest()
    traffic = None
    if NCU_TRAFFIC["digest"] == digest and args.storage in NCU_TRAFFIC["bytes_per_node"]:
        traffic = NCU_TRAFFIC["bytes_per_node"][args.storage] * nx * ny
    info = lat.kernel_info()

    # ---- end to end through the C ABI with host buffers
    cd = torch.empty(1, dtype=torch.float64).pin_memory()
    cl = torch.empty(1, dtype=torch.float64).pin_memory()
    out = [torch.empty((ny, nx), dtype=torch.float32).pin_memory() for _ in range(3)]
    # a run's one-time transfers (initial fields in, final fields out) spread
    # over at least 200 steps, as in a real run of many steps
    e2e_steps = max(args.steps, 200)
    barrier(device)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    lbm.lbm_init_fields_ptr(lat.h, *(p.data_ptr() for p in pin))
    base = lat.force_count()
    for s in range(e2e_steps):
        lbm.lbm_step(lat.h, 1)
        lbm.lbm_forces_ptr(lat.h, base + s, 1, cd.data_ptr(), cl.data_ptr())
    lbm.lbm_fields_ptr(lat.h, 0, *(o.data_ptr() for o in out))
    t_e2e = time.perf_counter() - t0
    barrier(device)
    t_e2e = max_over_ranks(t_e2e, device)
    lat.sync()
    e2e = {"value": whole_job_glups(nx * ny, e2e_steps, world, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": int(3 * 8 * nx * ny / e2e_steps),
           "d2h_bytes_per_step": int(16 + 3 * 4 * nx * ny / e2e_steps),
           "steps": e2e_steps,
           "note": "per step: one lbm_step and one lbm_forces read of that step's Cd/Cl; "
                   "plus the initial-field upload (FP64 rho, u, v) and final-field read-back (FP32) "
                   "spread over the steps"}
    cdv, clv = float(cd[0]), float(cl[0])
    lat.close()

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": workload.name, "nx": nx, "ny": ny, "D": workload.D, "U": workload.U,
                   "tau": workload.tau, "Re": workload.Re, "bc": "freeslip", "storage": args.storage + " offsets",
                   "collision": args.collision,
                   "kernel": info, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "gpu": torch.cuda.get_device_name(device), "seed": workload.seed,
                   "l2": f"inputs {bytes_step / 2 / 1e9:.1f} GB of populations read per step, far above the "
                         "129 MB L2: no flush needed"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_step},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "last_cd_cl": [cdv, clv],
    }
    if not args.no_extras and world == 1:
        line["extra"] = extras(args, workload, device, stream)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(workload, target_s=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    return 0


def time_steps(step, steps: int, stream) -> float:
    """Seconds of `steps` steps (CUDA events on the launching stream)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def extras(args, workload, device, stream):
    """The rest of the headline metric in the same run: the 16-bit storage
    forms on the same lattice, the batch of 64 cases (MRT), the wall time of
    a cold start to periodic Cd/Cl/St on the 1600 x 800 grid, and the paper's
    Table 2 values as context."""
    import numpy as np
    import torch
    from paper_2605_02185_gb300 import lbm, postprocess
    from paper_2605_02185_gb300 import workloads as W
    out = {}
    peak, src = measured_peaks()
    steps = max(args.steps, 20)
    rho0, u0, v0 = workload.initial_fields()
    forms = {}
    for name, st in (("f16", lbm.LBM_F16_OFS), ("bf16", lbm.LBM_BF16_OFS), ("f16sr", lbm.LBM_F16_SR),
                     ("bf16sr", lbm.LBM_BF16_SR)):
        lat = lbm.lattice_for(workload, storage=st, stream=stream, device=device)
        lat.init_fields(rho0, u0, v0)
        lat.step(args.warmup)
        lat.sync()
        dt = time_steps(lat.step, steps, stream)
        lat.sync()
        b = lat.bytes_per_step()
        forms[name] = {"glups": workload.cells * steps / dt / 1e9, "bytes_per_node": b / workload.cells,
                       "roofline_frac": b * steps / dt / 1e9 / peak, "kernel": lat.kernel_info()}
        lat.close()
    del rho0, u0, v0
    torch.cuda.empty_cache()
    out["storage_forms"] = {"workload": workload.name, "steps": steps, "peak_gbs": peak, "peak_source": src, **forms}

    cases = W.batched_cases(64, seed=4)
    b = lbm.Batch(cases, stream=stream, device=device, collision=lbm.LBM_COLLIDE_MRT)
    b.init_all()
    b.step(args.warmup)
    torch.cuda.synchronize(device)
    nodes, bytes_step = b.nodes()
    dt = time_steps(b.step, steps, stream)
    out["batch"] = {"workload": "64 cylinder cases, Re log-uniform in [60, 200], D in {20, 30, 40, 60}, "
                                "40D x 20D, U = 0.05, free-slip, MRT (Eq. 6)",
                    "nodes": nodes, "steps": steps, "glups": nodes * steps / dt / 1e9,
                    "roofline_frac": bytes_step * steps / dt / 1e9 / peak, "kernel": b.kernel_info()}
    b.close()
    del b
    torch.cuda.empty_cache()

    # cold start to periodic lift: the seeded +-1e-3 U perturbation of the
    # resting-cylinder start, lift checked every `chunk` steps
    wl = W.cylinder_case(40, 0.05, 80.0, seed=5, perturb=1e-3, name="cyl_Re80_D40_1600x800")
    lat = lbm.lattice_for(wl, stream=stream, device=device, history_capacity=1 << 20)
    chunk, max_steps, n, at = 2000, 400_000, 0, None
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    lat.init_fields(*wl.initial_fields())
    cds, cls = [], []
    while n < max_steps and at is None:
        lat.step(chunk)
        have = sum(len(c) for c in cls)
        cd, cl = lat.forces(have, n + chunk + 1 - have)
        n += chunk
        cds.append(cd)
        cls.append(cl)
        at = postprocess.periodic_index(np.concatenate(cls), period_range=postprocess.shedding_periods(wl.D, wl.U))
    t_wall = time.perf_counter() - t0
    cd, cl = np.concatenate(cds), np.concatenate(cls)
    lat.close()
    row = {"workload": f"{wl.name}: Re = 80, D = 40, U = 0.05, tau = {wl.tau:.4f}, BGK, free-slip, "
                       "seeded +-1e-3 U start", "periodic_at_step": at, "steps_run": n,
           "wall_s": t_wall, "criterion": "lift amplitude >= 0.05 changing < 0.5 % per period, two periods, "
                                          "period within St 0.08-0.4"}
    if at is not None:
        row.update({k: v for k, v in postprocess.statistics(cd[:at + 1], cl[:at + 1], wl.D, wl.U, periods=2).items()
                    if k in ("cd_mean", "cl_amp", "st")})
    out["time_to_periodic"] = row
    out["paper_table2"] = PAPER_TABLE2
    return out


def run_batch(args):
    """64 independent cylinder cases (Re log-uniform in [60, 200], D in
    {20, 30, 40, 60}, 40D x 20D each) advanced by one launch per step, against
    the same cases run one after another as single graph-captured lattices."""
    import torch
    from paper_2605_02185_gb300 import autotune, lbm
    from paper_2605_02185_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist_init("nccl")
    cases = W.batched_cases(args.cases, seed=4)
    stream = torch.cuda.Stream(device)
    coll = lbm.LBM_COLLIDE_MRT if args.collision == "mrt" else lbm.LBM_COLLIDE_BGK
    b = lbm.Batch(cases, stream=stream, device=device, collision=coll)
    b.init_all()
    tuned = None
    if args.tune:
        tuned = autotune.tune(b, [(w.nx, w.ny) for w in cases], lbm.LBM_F32, stream, steps=10, warmup=3)
        for row in tuned.get("table", []):
            print(json.dumps(row), file=sys.stderr, flush=True)
        tuned = {k: v for k, v in tuned.items() if k != "table"}
    nodes, bytes_step = b.nodes()
    b.step(args.warmup)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(local)
    sampler.start()
    barrier(device)
    torch.cuda.synchronize(device)
    l0 = b.launch_count()
    e0.record(stream)
    b.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    clocks = sampler.stop()
    launches = b.launch_count() - l0
    torch.cuda.synchronize(device)
    # BGK at tau close to 1/2 (D = 20 at high Re) can diverge; the kernel does
    # the same work either way, so the timing stands and the cases are named.
    unstable = [w.name for c, w in enumerate(cases) if b.case_status(c) == lbm.LBM_ERR_UNSTABLE]
    t_batch = e0.elapsed_time(e1) / 1e3
    info = b.kernel_info()
    b.close()
    del b
    torch.cuda.empty_cache()
    # the same cases one after another, each a single graph-captured lattice
    t_seq = 0.0
    for w in cases:
        lat = lbm.lattice_for(w, stream=stream, device=device, collision=coll)
        lat.init_fields(*w.initial_fields())
        lat.step(args.warmup)
        torch.cuda.synchronize(device)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        lat.step(args.steps)
        a1.record(stream)
        a1.synchronize()
        t_seq += a0.elapsed_time(a1) / 1e3
        torch.cuda.synchronize(device)
        lat.close()
    t_max = max_over_ranks(t_batch, device)
    value = whole_job_glups(nodes, args.steps, world, t_max)
    seq = nodes * args.steps / t_seq / 1e9
    peak, src = measured_peaks()
    achieved = bytes_step / (t_batch / args.steps) / 1e9
    if rank == 0:
        print(json.dumps({
            "metric": "GLUPS, 64 independent cylinder cases in one launch per step", "value": value,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of {len(cases)} cylinder cases, Re in [60,200], D in {{20,30,40,60}}, "
                                   f"40D x 20D, U = 0.05, free-slip", "nodes": nodes, "kernel": info,
                       "collision": args.collision,
                       "tuned": tuned},
            "sequential": {"value": seq, "unit": UNIT, "note": "same cases one after another, each a "
                                                                "graph-captured single lattice"},
            "speedup_vs_sequential": value / seq / world,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_source": src, "algorithmic_bytes_per_launch": bytes_step},
            "unstable_cases": unstable, "gpu_launches": int(launches), "clocks": clocks}), flush=True)
    return 0


def run_warmstart(args):
    """Learned warm start (D = 40, 1600 x 800, Re in [60, 200]): train the
    network on snapshots from the batched solver, then compare time to
    periodic shedding of warm and cold starts on held-out Re."""
    import torch
    from paper_2605_02185_gb300 import warmstart as WS

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    cfg = WS.Config(snapshots=args.snapshots, train_cases=args.cases if args.cases != 64 else 32, iters=args.iters,
                    init_mode=args.ws_init)
    logs = []
    if args.ws_load:
        # a network trained by an earlier run (its state() saved with --ws-save)
        import numpy as np
        from paper_2605_02185_gb300 import nn
        net = nn.WarmStartNet(cfg.batch, 20 * cfg.D, 40 * cfg.D, device, seed=cfg.seed, zero_head=True)
        with np.load(args.ws_load) as z:
            net.load_state({k: z[k] for k in z.files})
        info = {"loaded": args.ws_load, "losses": [(0, float("nan")), (0, float("nan"))], "spinup_s": 0.0,
                "fill_s": 0.0, "train_s": 0.0, "snapshots": 0}
    else:
        net, info = WS.train(cfg, device, log=lambda m: logs.append(m) or print(m, file=sys.stderr, flush=True))
        if args.ws_save:
            import numpy as np
            np.savez(args.ws_save, **net.state())
    rows, summary = WS.evaluate(net, cfg, n_eval=args.eval_cases, device=device,
                                log=lambda m: logs.append(m) or print(m, file=sys.stderr, flush=True))
    if rank == 0:
        print(json.dumps({
            "metric": "wall time to periodic Cd/Cl/St, learned warm start vs cold start (median over all judged "
                      "cases; a rejected prediction costs its warm run plus the cold run)", "unit": "x faster",
            "value": summary["median_gain_all_judged"], "higher_is_better": True, "n_gpus": 1,
            "data": "synthetic", "dtype": "bf16 network, f32 lattice",
            "config": {"workload": f"cylinder D = {cfg.D}, {40 * cfg.D} x {20 * cfg.D}, U = {cfg.U}, "
                                   f"Re in [{cfg.re_lo}, {cfg.re_hi}], MRT collision", "train_cases": cfg.train_cases,
                       "snapshots": info["snapshots"], "batch": cfg.batch, "init_mode": cfg.init_mode},
            "summary": summary, "train": {k: v for k, v in info.items() if k != "losses"},
            "training_cost_s": info["spinup_s"] + info["fill_s"] + info["train_s"],
            "loss_first_last": [info["losses"][0], info["losses"][-1]], "cases": rows}), flush=True)
    return 0


def run_network(args):
    """The warm-start network's convolutions at the training shape (N = 4
    samples of 800 x 1600, D = 40): per layer, the forward, input-gradient
    and weight-gradient calls timed with CUDA events on their stream, as
    TFLOP/s against the dense BF16 peak, for the tensor-core (tcgen05) and
    the mma.sync kernels; and one whole training iteration."""
    import numpy as np
    import torch
    from paper_2605_02185_gb300 import nn

    _, _, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    N, H, W = args.net_batch, 800, 1600
    peak, src = measured_bf16_peak()
    net = nn.WarmStartNet(N, H, W, device, seed=0)
    rng = np.random.default_rng(0)
    with torch.no_grad():
        net.x0.copy_(torch.from_numpy(rng.standard_normal(net.x0.shape).astype(np.float32)).to(torch.bfloat16))
    stream = torch.cuda.current_stream(device)
    dims = {"c1": 0, "d1": 0, "he": 0, "c2": 1, "d2": 1, "c3": 2, "d3": 2, "c4": 3}
    rows = []
    reps = max(3, args.steps // 4)
    layers = set(args.layers.split(",")) if args.layers else None
    impls = [("tcgen05", nn.IMPL_AUTO), ("mma_sync", nn.IMPL_MMA_SYNC)]
    if args.conv_impl != "both":
        impls = [i for i in impls if i[0] == args.conv_impl]
    for name, c in net.layers.items():
        if layers is not None and name not in layers:
            continue
        h, w = net.dims[dims[name[:2]]]
        flops = 2.0 * N * h * w * 9 * c.cin * c.cout
        x = torch.from_numpy(rng.standard_normal((N, h, w, c.cin)).astype(np.float32)).to(device, torch.bfloat16)
        gy = torch.from_numpy(rng.standard_normal((N, h, w, c.cout)).astype(np.float32)).to(device, torch.bfloat16)
        y = torch.empty((N, h, w, c.cout), dtype=torch.bfloat16, device=device)
        gx = torch.empty((N, h, w, c.cin), dtype=torch.bfloat16, device=device)
        row = {"layer": name, "H": h, "W": w, "cin": c.cin, "cout": c.cout, "gflop": flops / 1e9}
        calls = {
            "fwd": lambda: nn.conv3x3_fwd(x, c.cin, c.w16, c.b, y, c.cout, N, h, w, c.cin, c.cout, 1),
            "dgrad": lambda: nn.conv3x3_dgrad(gy, c.cout, c.wf16, gx, c.cin, N, h, w, c.cin, c.cout),
            "wgrad": lambda: nn.conv3x3_wgrad(x, c.cin, gy, c.cout, c.gw, c.gb, N, h, w, c.cin, c.cout),
        }
        for impl_name, impl in impls:
            nn.set_conv_impl(impl)
            for kind, fn in calls.items():
                for _ in range(2):
                    fn()
                dt = time_steps(lambda k: [fn() for _ in range(k)], reps, stream) / reps
                row[f"{kind}_{impl_name}_tflops"] = flops / dt / 1e12
        nn.set_conv_impl(nn.IMPL_AUTO)
        rows.append(row)
        del x, gy, y, gx
    # one training iteration: forward, loss, backward, Adam
    tg = torch.zeros((N * H * W, 3), dtype=torch.float32, device=device)
    wg = torch.ones(N * H * W, dtype=torch.float32, device=device)

    def iteration(k):
        for _ in range(k):
            net.forward()
            net.loss_and_grad(tg, wg)
            net.backward()
            net.adam_step(1e-4)

    iters = {}
    for impl_name, impl in ([] if layers is not None else impls):
        nn.set_conv_impl(impl)
        iteration(2)
        iters[impl_name] = time_steps(iteration, reps, stream) / reps
    nn.set_conv_impl(nn.IMPL_AUTO)
    assert nn.status(reset=True) == 0
    fl = 3 * net.flops_per_sample() * N
    it = iters.get("tcgen05")
    print(json.dumps({
        "metric": "warm-start network training iteration (3x3 conv fwd + both gradients), BF16 tensor cores",
        "value": fl / it / 1e12 if it else None, "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1,
        "data": "synthetic", "dtype": "bf16 (FP32 accumulation)",
        "config": {"workload": f"warm-start U-Net, N = {N}, {H} x {W}", "reps": reps},
        "iteration_ms": {k: v * 1e3 for k, v in iters.items()},
        "roofline": {"bound": "tensor", "peak": peak, "unit": "TFLOP/s", "peak_source": src,
                     "frac": fl / it / 1e12 / peak if it else None},
        "layers": rows}), flush=True)
    return 0


def run_statistics(args):
    """Physics of the production case (Re = 100, D = 80, 3200 x 1600, U = 0.05,
    tau = 0.62, or the case --D/--U/--Re give): each (top/bottom rule,
    storage form) runs --stat-steps steps from the seeded perturbed start;
    mean Cd, Cl amplitude and Strouhal number over the last --window steps
    (Eq. 15, the lift spectrum), the step at which the lift turned periodic,
    and the relative errors of every storage form against the FP64 run of the
    same rule."""
    import dataclasses
    import numpy as np
    import torch
    from paper_2605_02185_gb300 import lbm, postprocess
    from paper_2605_02185_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    base = W.PRODUCTION_D80
    if args.D or args.U or args.Re:
        D, U, Re = args.D or base.D, args.U or base.U, args.Re or base.Re
        base = W.cylinder_case(D, U, Re, seed=base.seed, perturb=base.perturb, name=f"cyl_Re{Re:g}_D{D}_U{U:g}")
    bc_ids = {"freeslip": W.BC_FREESLIP, "periodic": W.BC_PERIODIC, "zouhe": W.BC_ZOUHE,
              "movingwall": W.BC_MOVINGWALL}
    st_ids = STORAGE_IDS(lbm)
    coll = lbm.LBM_COLLIDE_MRT if args.collision == "mrt" else lbm.LBM_COLLIDE_BGK
    runs = []
    for item in args.runs.split(","):
        bc, st = item.split(":")
        runs.append((bc, st))
    stream = torch.cuda.Stream(device)
    rows, total_nodes, total_s = [], 0, 0.0
    for bc, st in runs:
        wl = dataclasses.replace(base, bc=bc_ids[bc])
        bounce = lbm.LBM_BOUNCE_INTERPOLATED if args.bounce == "interpolated" else lbm.LBM_BOUNCE_HALFWAY
        lat = lbm.lattice_for(wl, storage=st_ids[st], stream=stream, device=device, collision=coll,
                              history_capacity=args.stat_steps + 16, bounce=bounce)
        lat.init_fields(*wl.initial_fields())
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        lat.step(args.stat_steps)
        lat.sync()
        dt = time.perf_counter() - t0
        cd, cl = lat.forces(0, args.stat_steps)
        lat.close()
        i0 = len(cl) - args.window
        stats = postprocess.statistics(cd[i0:], cl[i0:], wl.D, wl.U)
        per = postprocess.periodic_index(cl, period_range=postprocess.shedding_periods(wl.D, wl.U))
        row = {"bc": bc, "storage": st, "cd_mean": stats["cd_mean"], "cl_amp": stats["cl_amp"],
               "cl_amp_h1": stats["cl_amp_h1"], "st": stats["st"],
               "st_zero_crossings": stats["st_zc"], "periodic_at_step": per, "seconds": dt,
               "glups": wl.nx * wl.ny * args.stat_steps / dt / 1e9}
        rows.append(row)
        total_nodes += wl.nx * wl.ny * args.stat_steps
        total_s += dt
        print(json.dumps(row), file=sys.stderr, flush=True)
    errors = {}
    for r in rows:
        ref = next((q for q in rows if q["bc"] == r["bc"] and q["storage"] == "f64"), None)
        if ref is not None and r is not ref:
            errors[f"{r['bc']}:{r['storage']}"] = {k: abs(r[k] - ref[k]) / abs(ref[k])
                                                   for k in ("cd_mean", "cl_amp", "cl_amp_h1", "st")}
    if rank == 0:
        print(json.dumps({
            "metric": "mean Cd, Cl amplitude, Strouhal number (Eq. 15, lift spectrum)", "unit": "GLUPS",
            "value": total_nodes / total_s / 1e9, "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
            "dtype": ",".join(sorted({st for _, st in runs})), "steps": args.stat_steps,
            "config": {"workload": base.name, "nx": base.nx, "ny": base.ny, "D": base.D, "U": base.U,
                       "tau": base.tau, "Re": base.Re, "collision": args.collision, "window": args.window,
                       "bounce": args.bounce},
            "runs": rows, "errors_vs_f64": errors}), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=["f32", "f16", "bf16", "f64", "f16sr", "bf16sr"], default="f32")
    ap.add_argument("--kernel", choices=["auto", "tma", "direct", "wave"], default="auto",
                    help="wave: the multi-step TMA kernel (up to 64 steps per cooperative launch)")
    ap.add_argument("--collision", choices=["bgk", "mrt"], default="bgk",
                    help="bgk: Eq. 2 (the default hot path); mrt: the paper's Eq. 6 with its rates")
    ap.add_argument("--shape", default="", help="TMA shape: compute warps,cells per thread,stages")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="0: the library's tuned default")
    ap.add_argument("--workload", default="throughput",
                    choices=["throughput", "throughput_half", "production", "parity", "batch", "warmstart",
                             "statistics", "network"])
    ap.add_argument("--net-batch", type=int, default=4, help="network workload: samples per batch")
    ap.add_argument("--layers", default="", help="network workload: comma list of layers to time (default all, "
                                                 "and the whole training iteration)")
    ap.add_argument("--conv-impl", choices=["both", "tcgen05", "mma_sync"], default="both",
                    help="network workload: kernel families to time")
    ap.add_argument("--runs", default="freeslip:f64,freeslip:f32,freeslip:f16,freeslip:bf16,periodic:f32,"
                                      "zouhe:f32,movingwall:f32",
                    help="statistics workload: comma list of top/bottom rule:storage")
    ap.add_argument("--stat-steps", type=int, default=300_000, help="statistics workload: steps per run")
    ap.add_argument("--window", type=int, default=100_000, help="statistics workload: averaging window (steps)")
    ap.add_argument("--D", type=int, default=0, help="statistics workload: cylinder diameter (default 80)")
    ap.add_argument("--U", type=float, default=0.0, help="statistics workload: inlet speed (default 0.05)")
    ap.add_argument("--Re", type=float, default=0.0, help="statistics workload: Reynolds number (default 100)")
    ap.add_argument("--bounce", choices=["halfway", "interpolated"], default="halfway",
                    help="statistics workload: body bounce-back (interpolated runs on the direct kernel)")
    ap.add_argument("--snapshots", type=int, default=20000, help="warmstart workload: training snapshots")
    ap.add_argument("--eval-cases", type=int, default=16, help="warmstart workload: held-out Re values")
    ap.add_argument("--iters", type=int, default=0, help="warmstart workload: training iterations (0: snapshots/4)")
    ap.add_argument("--ws-save", default="", help="warmstart workload: save the trained weights (npz)")
    ap.add_argument("--ws-load", default="", help="warmstart workload: evaluate weights saved by --ws-save")
    ap.add_argument("--ws-init", choices=["noneq", "eq", "rho1"], default="noneq",
                    help="warmstart workload: how the prediction starts the lattice")
    ap.add_argument("--cases", type=int, default=64, help="batch workload: number of cases")
    ap.add_argument("--tune", action="store_true", help="batch workload: autotune the kernel shape first")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-rows", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 16-bit forms, batch and time-to-periodic measurements of the default line")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    from paper_2605_02185_gb300 import workloads as W
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "statistics":
        return run_statistics(args)
    if args.workload == "network":
        return run_network(args)
    wl = {"throughput": W.THROUGHPUT_D400, "throughput_half": W.THROUGHPUT_D200, "production": W.PRODUCTION_D80,
          "parity": W.PARITY_D10}[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
