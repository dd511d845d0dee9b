"""Benchmark: GCUPS of the 3D Yee update, systolic vs naive schedule, FP32 and
16-bit field storage, 1 GB300.

Workload (one bench "step" = one fdtd_step(2000) call of the whole hot path):
256^3 grid, seeded Si/SiO2 permittivity map (eps 2.1 background with 8-20
eps 12.1 slabs of 10x10 cross-section), PEC walls, sinusoidal point Jz dipole
(wavelength 20 cells) at the centre, Courant number 0.99/sqrt(3), 2000 steps.
GCUPS = cells * steps / seconds / 1e9.  The 470 MB of device state is larger
than L2 (129 MB), so no L2 flush is needed between timed calls.

The headline value is the FP32 systolic schedule; the line also carries the
naive schedule and both schedules with FP16 and BF16 field storage (FP32
arithmetic) on the same workload.
Prints ONE JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the reference arm), on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling; the
path has no data exchange between GPUs in this build).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

GRID = (256, 256, 256)
STEPS_PER_CALL = 2000
WAVELENGTH = 20.0
# Algorithmic bytes per cell-step: the streaming bound reads and writes the
# six fields once (12 x element bytes: 48 B FP32, 24 B 16-bit); the naive
# schedule and the systolic tiles are modelled in naive_bytes/systolic_bytes.
# Tiles: updated (tx, ty, tz), ring (tx+1, ty+1, tz+1); the library's default
# is 31 x 15 x 12.
TILE_SHAPES = {"31x15x15": (31, 15, 15), "31x7x15": (31, 7, 15), "31x15x12": (31, 15, 12), "31x15x8": (31, 15, 8)}
DEFAULT_TILE = "31x15x12"


# DRAM bytes per cell update from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum) of a 100-step, 256^3 launch of the same kernel, with
# the launch's fixed initial load and final flush (52 B per cell) taken out.
# This run does not measure them: the line scales them by its own cell
# updates and labels them as taken from the capture.  A kernel changed since
# its capture has no entry (its traffic is then reported as null).
CAPTURED_TRAFFIC = {"31x15x12": 10.70}
# Warp instructions issued per cell update (smsp__inst_executed.sum over the
# updates) in the same capture: with the bench's GCUPS it gives the SM
# sub-partitions' issue rate, the resource this kernel runs against.
CAPTURED_WARP_INST = {"31x15x12": 3.68}


STORAGE_BYTES = {"f32": 4, "f16": 2, "bf16": 2}


def systolic_bytes(tile, eb=4):
    """Algorithmic bytes per cell update of the systolic kernel: per tile step
    the lower shell is read (6 fields of eb bytes and the FP32 dt/eps) and
    the top faces are written (6 fields), divided by the updated cells."""
    tx, ty, tz = TILE_SHAPES[tile]
    upd = tx * ty * tz
    shell = (tx + 1) * (ty + 1) * (tz + 1) - upd
    top = upd - (tx - 1) * (ty - 1) * (tz - 1)
    return ((6 * eb + 4.0) * shell + 6.0 * eb * top) / upd


def naive_bytes(eb=4):
    """Two kernels per step: H reads 6 fields and writes 3; E reads 6 fields
    and dt/eps and writes 3."""
    return 6.0 * eb + 3.0 * eb + 6.0 * eb + 4.0 + 3.0 * eb


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def make_workload(shape):
    from paper_2502_20610_gb300 import workloads as wl
    eps = wl.si_sio2_eps(shape, 1)
    J = wl.sine_source(65536, wl.DT_DEFAULT, WAVELENGTH)
    src = (2, shape[2] // 2, shape[1] // 2, shape[0] // 2)  # Jz at the centre cell
    return eps, J, src


def cpu_model():
    """The host CPU's model string (from /proc/cpuinfo; Arm hosts give no
    'model name', so their implementer / part codes are reported)."""
    try:
        with open("/proc/cpuinfo") as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    for key in ("model name", "Model", "Hardware"):
        for ln in lines:
            if ln.split(":")[0].strip() == key:
                return ln.split(":", 1)[1].strip()
    impl = [ln.split(":", 1)[1].strip() for ln in lines if ln.startswith("CPU implementer")]
    part = [ln.split(":", 1)[1].strip() for ln in lines if ln.startswith("CPU part")]
    if impl and part:
        return f"CPU implementer {impl[0]}, part {part[0]}"
    return None


def _oracle_rate(shape, threads, budget_s):
    """Cell updates per second (in G) of the FP64 oracle with `threads` host
    threads on the bench workload's grid, geometry and source, for as many
    steps as fit in ~budget_s (at least 1); returns (gcups, steps, seconds)."""
    from oracle import YeeOracle
    from oracle.yee import set_threads
    from paper_2502_20610_gb300 import workloads as wl
    used = set_threads(threads)
    eps, J, (c, i, j, k) = make_workload(shape)
    o = YeeOracle(shape, wl.DT_DEFAULT, eps)
    o.add_source(c, i, j, k, J)
    o.step(1)  # first touch of the arrays
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(STEPS_PER_CALL, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    o.step(n)
    dt = time.perf_counter() - t0
    o.close()
    cells = shape[0] * shape[1] * shape[2]
    return cells * n / dt / 1e9, n, dt, used


def cpu_baseline(shape, budget_s=15.0, budget_1t_s=10.0):
    """The FP64 oracle as it stands, on this host's cores, on a bounded
    sample of the workload: the same grid and geometry for as many steps as
    fit in ~budget_s, with every core the process may use; and the same with
    one thread."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    v, n, dt, used = _oracle_rate(shape, cores, budget_s)
    v1, n1, dt1, _ = _oracle_rate(shape, 1, budget_1t_s)
    from oracle.yee import set_threads
    set_threads(cores)
    return {"value": v, "unit": "GCUPS", "cores": used, "kind": "oracle",
            "sample": f"{shape[2]}x{shape[1]}x{shape[0]} grid, same eps map and source, {n} steps "
                      f"(of {STEPS_PER_CALL}), FP64, {dt:.1f} s",
            "value_1_thread": v1, "sample_1_thread": f"{n1} steps, {dt1:.1f} s",
            "cpu_model": cpu_model()}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_reference(args, world, rank):
    """Reference arm: the FP64 CPU oracle as it stands, on this host's cores.
    Each of the W warm-up and K timed steps advances the same workload by a
    bounded number of oracle steps (the sample), so the run stays within a
    few minutes; the value is cell updates per second of the timed steps."""
    if rank != 0:
        return 0
    from oracle import YeeOracle
    from oracle.yee import set_threads
    from paper_2502_20610_gb300 import workloads as wl
    shape = GRID
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cores = set_threads(cores)
    eps, J, (c, i, j, k) = make_workload(shape)
    o = YeeOracle(shape, wl.DT_DEFAULT, eps)
    o.add_source(c, i, j, k, J)
    o.step(1)
    t0 = time.perf_counter()
    o.step(1)
    t1 = time.perf_counter() - t0
    budget = float(os.environ.get("BENCH_CPU_BUDGET_S", "60"))
    n = max(1, min(STEPS_PER_CALL, int(budget / max(args.steps + args.warmup, 1) / max(t1, 1e-6))))
    for _ in range(args.warmup):
        o.step(n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(n)
    el = time.perf_counter() - t0
    cells = shape[0] * shape[1] * shape[2]
    v = cells * n * args.steps / el / 1e9
    cb = {"value": v, "unit": "GCUPS", "cores": cores, "kind": "oracle",
          "sample": f"each step: {n} oracle steps (of {STEPS_PER_CALL}) of the same workload, FP64",
          "cpu_model": cpu_model()}
    line = {"impl": "reference", "metric": "GCUPS of 3D Yee update, systolic vs naive kernel, FP32 & FP16-stored, 1 GB300",
            "value": v, "unit": "GCUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(storage="f32"):
    return {"workload": f"{GRID[0]}^3 Si/SiO2 eps map (seed 1), PEC walls, Jz dipole lambda=20 at the "
                        f"centre, {STEPS_PER_CALL} steps per call, {storage.upper()} fields",
            "grid_xyz": list(GRID[::-1]), "steps_per_call": STEPS_PER_CALL,
            "l2": "inputs larger than L2 (470 MB device state), no flush",
            "parallelism": "replicas (one independent simulation per GPU)"}


def time_storage_variant(shape, eps, J, src, storage, device, stream, n_calls=1):
    """GCUPS of both schedules with 16-bit field storage on the same workload
    (one warm-up call, then n_calls timed calls each)."""
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import workloads as wl
    cells = shape[0] * shape[1] * shape[2]
    out = {"storage": storage, "unit": "GCUPS",
           "stream_bytes_per_cell_step": 12.0 * STORAGE_BYTES[storage]}
    for scheme in ("systolic", "naive"):
        sim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme=scheme, device=device, storage=storage,
                       steps_per_launch=STEPS_PER_CALL, max_source_steps=J.size)
        sim.add_source(*src, J)
        sim.step(STEPS_PER_CALL)
        sim.sync()
        t = time_calls(sim, n_calls, stream)
        sim.sync()
        sim.close()
        out[scheme] = cells * STEPS_PER_CALL * n_calls / t / 1e9
    peak, kind = load_peaks()
    bound = peak / out["stream_bytes_per_cell_step"]
    out["stream_bound_gcups"] = bound
    out["systolic_stream_frac"] = out["systolic"] / bound
    out["peak_kind"] = kind
    return out


def naive_threads(shape):
    """Threads the library's naive scheme launches on a (nz, ny, nx) grid: one
    per cell in a single CTA up to 1024 cells, else 32 x 8 CTAs in x-y with
    each thread marching 8 cells in z."""
    nz, ny, nx = shape
    cells = nx * ny * nz
    if cells <= 1024:
        return (cells + 31) // 32 * 32
    return -(-nx // 32) * -(-ny // 8) * -(-nz // 8) * 256


def sweep_shapes(min_cells=32, max_cells=1 << 28):
    """Grids whose cell counts double from min_cells to max_cells, as
    balanced as powers of two allow (x >= y >= z)."""
    out = []
    m = int(math.log2(min_cells))
    while (1 << m) <= max_cells:
        a = [m // 3 + (1 if r < m % 3 else 0) for r in range(3)]  # x, y, z exponents
        out.append((1 << a[2], 1 << a[1], 1 << a[0]))
        m += 1
    return out


def run_sweep(args):
    """Size sweeps through the C ABI, one JSON line per measurement.
    fig1: the naive schedule (FP32) on grids from ~1 KB to a few GB of field
    state, per-thread and total throughput (Fig. 1), with the systolic
    schedule beside it.  sizes: 128^3 .. 1024^3 of the Si/SiO2 workload with
    FP32, FP16 and BF16 field storage, both schedules, 1000 steps each."""
    import torch
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import workloads as wl
    device = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(device)
    props = torch.cuda.get_device_properties(device)
    info = {"sm_count": props.multi_processor_count,
            "l2_bytes": getattr(props, "L2_cache_size", None),
            "smem_per_block_optin": getattr(props, "shared_memory_per_block_optin", None)}
    print(json.dumps({"sweep": args.sweep, "device": props.name, **info}), flush=True)

    def measure(shape, scheme, storage, steps, eps, src=None, J=None):
        cells = shape[0] * shape[1] * shape[2]
        sim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme=scheme, device=device, storage=storage,
                       steps_per_launch=min(steps, 1024), max_source_steps=max(steps, 1) if J is not None else 0)
        if src is not None:
            sim.add_source(*src, J[:steps])
        warm = max(1, steps // 20)
        sim.step(warm)
        sim.sync()
        sim.set_current_step(0)
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        l0 = sim.launch_count
        start.record(stream)
        sim.step(steps)
        end.record(stream)
        end.synchronize()
        sim.sync()
        t = start.elapsed_time(end) / 1e3
        launches = sim.launch_count - l0
        sim.close()
        return cells * steps / t / 1e9, t, launches

    if args.sweep == "fig1":
        for shape in sweep_shapes(32, 1 << args.sweep_max_log2):
            cells = shape[0] * shape[1] * shape[2]
            steps = int(min(20000, max(200, 4e9 / cells / 10)))
            eps = np.ones(shape)
            row = {"grid_xyz": list(shape[::-1]), "cells": cells, "bytes_fields": 24 * cells, "steps": steps}
            g, t, nl = measure(shape, "naive", "f32", steps, eps)
            thr = naive_threads(shape)
            resident = min(thr, info["sm_count"] * 2048)  # at most 2048 resident threads per SM
            row.update({"naive_gcups": g, "naive_threads": thr, "naive_launches": nl,
                        "naive_updates_per_us_per_thread": g * 1e3 / thr,
                        "naive_resident_threads": resident,
                        "naive_updates_per_us_per_resident_thread": g * 1e3 / resident})
            if cells >= 1024:
                row["systolic_gcups"] = measure(shape, "systolic", "f32", steps, eps)[0]
            print(json.dumps(row), flush=True)
        return 0
    if args.sweep == "config4":
        return run_config4(device, stream, measure)
    if args.sweep == "config5":
        return run_config5(device)
    if args.sweep == "errors":
        return run_errors(device)
    # sizes: the Si/SiO2 workload at 128^3 .. 1024^3, three storage formats
    steps = args.steps_per_call if args.steps_per_call != STEPS_PER_CALL else 1000
    for n in (128, 256, 512, 768, 1024):
        shape = (n, n, n)
        eps = wl.si_sio2_eps(shape, 1)
        J = wl.sine_source(steps, wl.DT_DEFAULT, WAVELENGTH)
        src = (2, n // 2, n // 2, n // 2)
        for storage in ("f32", "f16", "bf16"):
            eb = STORAGE_BYTES[storage]
            for scheme in ("systolic", "naive"):
                g, t, nl = measure(shape, scheme, storage, steps, eps, src, J)
                b = systolic_bytes(DEFAULT_TILE, eb) if scheme == "systolic" else naive_bytes(eb)
                print(json.dumps({"grid": n, "storage": storage, "scheme": scheme, "steps": steps, "gcups": g,
                                  "seconds": t, "launches": nl, "algorithmic_bytes_per_cell_step": round(b, 3),
                                  "stream_bound_gcups": load_peaks()[0] / (12.0 * eb),
                                  "stream_frac": g / (load_peaks()[0] / (12.0 * eb))}), flush=True)
            torch.cuda.empty_cache()
    return 0


def run_errors(device, sizes=(128, 256), steps=1000):
    """Per-field relative L2 error against the FP64 oracle of the size
    sweep's workload (Si/SiO2 seed 1, Jz dipole at the centre, 1000 steps) at
    the sizes the oracle can follow: the systolic schedule with FP32, FP16 and
    BF16 field storage, and beside each 16-bit format the error of the
    oracle's own emulation of that storage rounding (FP64 arithmetic, the
    same rounding points)."""
    from oracle import YeeOracle
    from oracle.yee import set_threads
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import workloads as wl
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    set_threads(cores)
    names = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")

    def rel(got, ref):
        total = np.sqrt((ref ** 2).sum())
        out = {}
        for c in range(6):
            nb = np.sqrt((ref[c] ** 2).sum())
            out[names[c]] = float(np.sqrt(((got[c] - ref[c]) ** 2).sum()) / (nb if nb >= 1e-6 * total else total))
        return out

    def oracle(shape, eps, src, storage, quantize):
        o = YeeOracle(shape, wl.DT_DEFAULT, eps, quantize_ce_f32=quantize)
        o.set_fields(np.zeros((6,) + shape))
        if storage is not None:
            o.set_storage(storage, [1.0] * 6)
        o.add_source(*src)
        o.step(steps)
        f = o.fields()
        o.close()
        return f

    for n in sizes:
        shape = (n, n, n)
        eps = wl.si_sio2_eps(shape, 1)
        src = (2, n // 2, n // 2, n // 2, wl.sine_source(steps, wl.DT_DEFAULT, WAVELENGTH))
        t0 = time.perf_counter()
        ref = oracle(shape, eps, src, None, False)
        t_or = time.perf_counter() - t0
        refq = oracle(shape, eps, src, None, True)
        for storage in ("f32", "f16", "bf16"):
            sim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme="systolic", device=device, storage=storage,
                           steps_per_launch=steps, max_source_steps=steps)
            sim.add_source(*src)
            sim.step(steps)
            got = sim.read_fields().cpu().numpy().astype(np.float64)
            sim.close()
            row = {"sweep": "errors", "grid": n, "steps": steps, "storage": storage, "scheme": "systolic",
                   "rel_l2_vs_fp64": rel(got, ref), "oracle_seconds": t_or, "oracle_threads": cores}
            if storage == "f32":
                row["rel_l2_vs_fp64_fp32_coefficients"] = rel(got, refq)
            else:
                row["emulation_rel_l2_vs_fp64"] = rel(oracle(shape, eps, src, storage, True), ref)
            print(json.dumps(row), flush=True)
            del got
        del ref, refq
    return 0


def run_config4(device, stream, measure):
    """384^3 Si/SiO2 with a Gaussian-modulated pulse (centre wavelength 20,
    50% bandwidth): the 32-cell graded absorber (sigma_max 0.5, order 3) with
    both schedules, against the 4-cell learned boundary (graded base 0.3 and
    a network trained here, on the GPU, on 48^3 thick-absorber runs) for the
    same physical interior (328^3 = 320^3 + 2 x 4 layer cells); then the
    reflection errors of the 48^3 experiment against the thick absorber."""
    import torch
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import learned
    from paper_2502_20610_gb300 import workloads as wl
    t0 = time.time()
    setup = learned.Setup(n=48, thickness=4, pad=32, absorber=(32, 0.5, 3), base_sigma=0.3)
    x, y = learned.record(setup, seed=1, runs=4, sources_per_run=3, steps=250, per_step=1000, noise=0.05)  # 10^6 pairs
    t_record = time.time() - t0
    # the reflection of a trained network varies with the training seed (the
    # one-step loss barely does): train three, report each and their mean
    nets = []
    for seed, init in ((0, 0), (1, 0), (0, 1)):
        t1 = time.time()
        params, loss = learned.train(x, y, epochs=30, batch=4096, lr=1e-3, seed=seed, init_seed=init)
        nets.append((params.cpu().numpy(), loss, time.time() - t1, seed, init))
    theta = nets[0][0]
    del x, y, params
    torch.cuda.empty_cache()
    e_b, trace = learned.reflection(setup, "thin", seed=99, steps=300)
    e_ls = [learned.reflection(setup, "learned", th, seed=99, steps=300, ref_fields=trace)[0] for th, *_ in nets]
    e_t, _ = learned.reflection(setup, "thin", seed=99, steps=300, ref_fields=trace, sigma=0.5)
    e_p, _ = learned.reflection(setup, "pec", seed=99, steps=300, ref_fields=trace)
    del trace
    torch.cuda.empty_cache()
    # the same comparison on config 4's own grid: the yardstick is 384^3 with
    # the 32-cell absorber (320^3 interior); the other domains are that
    # interior plus a 4-cell layer (328^3); a Gaussian-modulated Jz pulse
    # (wavelength 20) at a seeded position, every domain stepped together
    big = learned.Setup(n=328, thickness=4, pad=28, absorber=(32, 0.5, 3), base_sigma=0.3)
    bsteps = 700
    u = wl.uniform_pm1(4242, 3)
    pos = [int(40 + 248 * (0.5 + 0.5 * float(v))) for v in u]  # 40 .. 288 in each axis
    bsrc = (2, pos[0], pos[1], pos[2], wl.gaussian_pulse_source(bsteps, wl.DT_DEFAULT, wavelength=WAVELENGTH))
    t_big = time.time()
    big_err = learned.reflection_lockstep(big, {
        "learned_4cell": ("learned", nets[2][0], None), "base_layer_alone": ("thin", None, None),
        "graded_4cell_sigma0.5": ("thin", None, 0.5), "pec": ("pec", None, None)}, bsrc, bsteps)
    t_big = time.time() - t_big
    torch.cuda.empty_cache()
    out = {"config": "config4", "record_seconds": t_record, "train_pairs": 1000000,
           "reflection_384cube": {"errors": big_err, "steps": bsteps, "source_xyz": pos,
                                  "network": "training seeds (shuffle 0, init 1)",
                                  "domain": "yardstick 384^3 with the 32-cell absorber; 328^3 = its 320^3 "
                                            "interior + 4-cell layer; eps 2.1", "seconds": t_big},
           "trainings": [{"shuffle_seed": sd, "init_seed": ini, "train_seconds": ts, "train_loss": ls,
                          "reflection": e} for (_, ls, ts, sd, ini), e in zip(nets, e_ls)],
           "reflection_error_vs_32cell_absorber": {"learned_4cell_mean": float(np.mean(e_ls)),
                                                   "learned_4cell_min": float(np.min(e_ls)),
                                                   "learned_4cell_max": float(np.max(e_ls)),
                                                   "base_layer_alone": e_b,
                                                   "graded_4cell_sigma0.5": e_t, "pec": e_p,
                                                   "domain": "48^3 + 2x32 pad, eps 2.1, 300 steps"}}
    steps = 500
    for n, kind in ((384, "absorber32"), (328, "learned4")):
        shape = (n, n, n)
        eps = wl.si_sio2_eps(shape, 1)
        J = wl.gaussian_pulse_source(steps, wl.DT_DEFAULT, wavelength=WAVELENGTH)
        src = (2, n // 2, n // 2, n // 2)
        schemes = ("systolic", "naive") if kind == "absorber32" else ("naive",)
        for scheme in schemes:
            kw = dict(boundary="graded", absorber=(32, 0.5, 3)) if kind == "absorber32" else \
                dict(boundary="learned", learned=(4, theta, 0.3, 3))
            sim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme=scheme, device=device, max_source_steps=steps,
                           steps_per_launch=min(steps, 1024), **kw)
            sim.add_source(*src, J)
            sim.step(20)
            sim.sync()
            sim.set_current_step(0)
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            sim.step(steps)
            end.record(stream)
            end.synchronize()
            sim.sync()
            t = start.elapsed_time(end) / 1e3
            finite = bool(torch.isfinite(sim.read_fields()).all())
            sim.close()
            interior = 320 ** 3
            out[f"{kind}_{scheme}"] = {"grid": n, "gcups": n ** 3 * steps / t / 1e9,
                                       "interior_gcups_320cube": interior * steps / t / 1e9,
                                       "seconds": t, "steps": steps, "finite": finite}
            torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def config5_problem(scheme="systolic"):
    """200 x 200 x 100 grid (eps 2.1), a 64 x 64 x 20 design box of seeded
    uniform eps in [2.1, 12.1] at the centre, a CW Jz dipole (wavelength 20)
    below it, the overlap of Ez on the plane z = 80 with a seeded Gaussian
    mode profile over the last 350 steps of 4000, checkpoints every 100."""
    from paper_2502_20610_gb300 import adjoint as gadj
    from paper_2502_20610_gb300 import workloads as wl
    nx, ny, nz = 200, 200, 100
    lo, hi = (68, 68, 40), (132, 132, 60)
    steps = 4000
    u = np.asarray(wl.uniform_pm1(11, 64 * 64 * 20)).reshape(20, 64, 64)
    eps_box = 2.1 + 10.0 * (0.5 + 0.5 * u)
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    noise = np.asarray(wl.uniform_pm1(12, nx * ny)).reshape(ny, nx)
    mode = np.exp(-((ii - 100.0) ** 2 + (jj - 100.0) ** 2) / (2 * 10.0 ** 2)) * (1.0 + 0.2 * noise)
    src = (2, 100, 100, 15, wl.sine_source(steps, wl.DT_DEFAULT, WAVELENGTH))
    p = gadj.Problem((nz, ny, nx), 2.1, lo, hi, src, k0=80, mode=mode, n_steps=steps, window=350,
                     checkpoint_every=100, scheme=scheme)
    return p, eps_box


def run_config5(device):
    """Config 5 at full size: the adjoint gradient's cost, and its
    directional derivative against a central difference of the objective
    along a seeded +-1 direction over the whole design box."""
    import torch
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import workloads as wl
    p, eps_box = config5_problem()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L, g = p.run(eps_box)
    t_adj = time.perf_counter() - t0
    # forward alone, same schedule
    sim = fdtd.Sim(p.shape, p.eps_with(eps_box), wl.DT_DEFAULT, scheme="systolic", max_source_steps=p.n_steps,
                   steps_per_launch=1024)
    sim.add_source(*p.source)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(p.n_steps)
    sim.sync()
    t_fwd = time.perf_counter() - t0
    sim.close()
    v = np.sign(np.asarray(wl.uniform_pm1(13, eps_box.size)).reshape(eps_box.shape))
    # the same gradient with checkpoints every step would need no recompute:
    # not affordable at this size, so instead time a second run to check
    # the first was not a warm-up outlier
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    p.run(eps_box)
    t_adj2 = time.perf_counter() - t0
    out = {"config": "config5", "grid_xyz": [200, 200, 100], "design_box": [64, 64, 20], "steps": p.n_steps,
           "seconds_gradient_second_run": t_adj2,
           "checkpoint_every": p.checkpoint_every, "L": L, "seconds_gradient": t_adj, "seconds_forward": t_fwd,
           "gradient_over_forward": t_adj / t_fwd,
           "forward_gcups": 200 * 200 * 100 * p.n_steps / t_fwd / 1e9,
           "grad_abs_max": float(g.abs().max()), "grad_norm": float(g.norm())}
    dd = float((g.cpu().numpy() * v).sum())
    for h in (0.2, 0.05):
        lp, _ = p.run(eps_box + h * v)
        lm, _ = p.run(eps_box - h * v)
        fd = (lp - lm) / (2 * h)
        out[f"directional_fd_h{h}"] = fd
        out[f"directional_rel_err_h{h}"] = abs(fd - dd) / abs(dd)
    out["directional_adjoint"] = dd
    print(json.dumps(out), flush=True)
    return 0


def time_calls(sim, n_calls, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(n_calls):
        sim.step(STEPS_PER_CALL)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3


def main():
    global GRID, STEPS_PER_CALL
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--naive-calls", type=int, default=1, help="timed naive calls (context)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", type=int, default=GRID[0], help="cubic grid edge (profiling runs)")
    ap.add_argument("--steps-per-call", type=int, default=STEPS_PER_CALL)
    ap.add_argument("--scheme", default="systolic", choices=["systolic", "naive"])
    ap.add_argument("--tile", default=None, help="systolic tile shape, e.g. 31x15x15 (default: library's)")
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "bf16"], help="field storage format")
    ap.add_argument("--no-16bit", action="store_true", help="skip the FP16/BF16 storage context lines")
    ap.add_argument("--no-1024", action="store_true", help="skip the 1024^3 context measurement")
    ap.add_argument("--sweep", default=None, choices=["fig1", "sizes", "errors", "config4", "config5"],
                    help="print size-sweep lines instead of the benchmark line")
    ap.add_argument("--sweep-max-log2", type=int, default=28, help="fig1: largest grid, log2 of cells")
    args = ap.parse_args()
    GRID = (args.grid,) * 3
    STEPS_PER_CALL = args.steps_per_call
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.sweep:
        return run_sweep(args)

    import torch
    from paper_2502_20610_gb300 import fdtd
    from paper_2502_20610_gb300 import workloads as wl

    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    shape = GRID
    cells = shape[0] * shape[1] * shape[2]
    eps, J, (c, i, j, k) = make_workload(shape)

    sim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme=args.scheme, device=device,
                   steps_per_launch=STEPS_PER_CALL, max_source_steps=J.size, tile=args.tile,
                   storage=args.storage)
    sim.add_source(c, i, j, k, J)
    for _ in range(args.warmup):
        sim.step(STEPS_PER_CALL)
    sim.sync()
    barrier(world)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = sim.launch_count
    elapsed = time_calls(sim, args.steps, stream)
    launches = sim.launch_count - l0
    sim.sync()
    clk = clocks.stop()
    barrier(world)
    elapsed = max_over_ranks(elapsed, world, device)
    gcups = world * cells * STEPS_PER_CALL * args.steps / elapsed / 1e9

    # naive schedule on the same workload (context for "systolic vs naive")
    naive = None
    if args.naive_calls > 0:
        nsim = fdtd.Sim(shape, eps, wl.DT_DEFAULT, scheme="naive", device=device, max_source_steps=J.size,
                        storage=args.storage)
        nsim.add_source(c, i, j, k, J)
        nsim.step(STEPS_PER_CALL)
        nsim.sync()
        t = time_calls(nsim, args.naive_calls, stream)
        nsim.sync()
        naive_gcups = cells * STEPS_PER_CALL * args.naive_calls / t / 1e9
        naive = {"value": naive_gcups, "unit": "GCUPS", "ms_per_step": 1e3 * t / args.naive_calls,
                 "kernels_per_step": 2 * STEPS_PER_CALL,
                 "algorithmic_bytes_per_cell_step": naive_bytes(STORAGE_BYTES[args.storage]),
                 "hbm_gbs_algorithmic": naive_gcups * naive_bytes(STORAGE_BYTES[args.storage]),
                 "speedup_systolic": gcups / world / naive_gcups}
        nsim.close()

    # end to end through the public API with host buffers: H2D of the initial
    # fields from pinned memory, the 2000 steps, D2H of the result
    e2e = None
    if not args.no_e2e:
        host_in = torch.from_numpy(wl.random_fields(shape, 0)).pin_memory()
        host_out = torch.empty((6,) + shape, dtype=torch.float32).pin_memory()
        nb = 6 * cells * 4  # the API exchanges FP32 fields whatever the storage
        sim.write_fields(host_in)
        sim.step(STEPS_PER_CALL)
        sim.read_fields(out=host_out)
        barrier(world)
        # device time of the steps inside the loop (CUDA events around each
        # call's launches) and clocks, so the line shows what the copies add
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        eclk = ClockSampler(local)
        eclk.start()
        t0 = time.perf_counter()
        for q in range(args.steps):
            sim.write_fields_ptr(host_in.data_ptr())
            ev[q][0].record(stream)
            sim.step(STEPS_PER_CALL)
            ev[q][1].record(stream)
            sim.read_fields_ptr(0x3F, host_out.data_ptr())
        te = time.perf_counter() - t0
        e_clk = eclk.stop()
        dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        te = max_over_ranks(te, world, device)
        e2e = {"value": world * cells * STEPS_PER_CALL * args.steps / te / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
               "ms_per_step": 1e3 * te / args.steps, "device_ms_per_step": 1e3 * dev_s / args.steps,
               "clocks": e_clk}
    sim.close()

    # the same workload with 16-bit field storage (FP32 arithmetic), both schedules
    narrow = None
    if not args.no_16bit and args.storage == "f32" and args.scheme == "systolic":
        narrow = [time_storage_variant(shape, eps, J, (c, i, j, k), st, device, stream) for st in ("f16", "bf16")]

    # the systolic kernel at 1024^3 (same generator, 1000 steps), where the
    # target of the metric's streaming roofline is quoted; FP32 fields, then
    # FP16 and BF16 storage (FP32 arithmetic)
    big = None
    if not args.no_1024 and args.storage == "f32" and args.scheme == "systolic" and GRID[0] == 256:
        n, steps = 1024, 1000
        bshape = (n, n, n)
        beps, bJ, (bc, bi, bj, bk) = make_workload(bshape)

        def time_big(storage):
            bsim = fdtd.Sim(bshape, beps, wl.DT_DEFAULT, scheme="systolic", device=device, storage=storage,
                            steps_per_launch=steps, max_source_steps=bJ.size)
            bsim.add_source(bc, bi, bj, bk, bJ)
            bsim.step(steps)
            bsim.sync()
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            bsim.step(steps)
            end.record(stream)
            end.synchronize()
            bsim.sync()
            bsim.close()
            torch.cuda.empty_cache()
            return start.elapsed_time(end) / 1e3

        tb = time_big("f32")
        peak_b, kind_b = load_peaks()
        g = n ** 3 * steps / tb / 1e9
        big = {"grid_xyz": [n, n, n], "steps": steps, "gcups": g, "seconds": tb,
               "stream_frac": g / (peak_b / 48.0), "peak_kind": kind_b, "storage_16bit": []}
        if not args.no_16bit:
            for st in ("f16", "bf16"):
                g16 = n ** 3 * steps / time_big(st) / 1e9
                big["storage_16bit"].append({"storage": st, "gcups": g16, "vs_f32": g16 / g})
        del beps

    if rank != 0:
        return 0
    peak, peak_kind = load_peaks()
    per_launch_s = elapsed / max(launches, 1)
    cell_steps_per_launch = cells * STEPS_PER_CALL * args.steps / max(launches, 1)
    tile = args.tile or DEFAULT_TILE
    eb = STORAGE_BYTES[args.storage]
    sys_bytes = systolic_bytes(tile, eb) if args.scheme == "systolic" else naive_bytes(eb)
    per_update = CAPTURED_TRAFFIC.get(tile) if args.scheme == "systolic" and args.storage == "f32" else None
    traffic = per_update * cell_steps_per_launch + 52.0 * cells if per_update else None
    achieved = sys_bytes * cell_steps_per_launch / per_launch_s / 1e9
    # issue roofline: one warp instruction per clock per SM sub-partition
    wi = CAPTURED_WARP_INST.get(tile) if args.scheme == "systolic" and args.storage == "f32" else None
    issue = None
    if wi and clk and clk.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        peak_i = sms * 4 * clk["sm_mhz"] * 1e6 / 1e12
        ach_i = gcups / world * 1e9 * wi / 1e12
        issue = {"warp_instructions_per_cell_update": wi, "warp_instructions_source": "ncu capture (256^3, 100 steps)",
                 "achieved": ach_i, "peak": peak_i,
                 "unit": "T warp instructions/s", "frac": ach_i / peak_i,
                 "peak_from": f"{sms} SMs x 4 sub-partitions x 1 instruction/clock x sampled SM clock"}
    line = {
        "metric": "GCUPS of 3D Yee update, systolic vs naive kernel, FP32 & FP16-stored, 1 GB300",
        "value": gcups, "unit": "GCUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args.storage),
        "scheme": args.scheme, "storage": args.storage,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "traffic_source": ("ncu capture of the same kernel (256^3, 100 steps), bytes per update "
                                        "scaled to this launch" if traffic else None),
                     "kernel": "systolic_reg_kernel" if args.scheme == "systolic" else "naive_h/e",
                     "tile": tile, "algorithmic_bytes_per_cell_step": round(sys_bytes, 3)},
        "stream_roofline": {"bytes_per_cell_step": 12.0 * eb,
                            "bound_gcups": peak / (12.0 * eb),
                            "frac": gcups / world / (peak / (12.0 * eb)), "peak_kind": peak_kind},
        "dram_gbs_from_capture": (per_update * cells * STEPS_PER_CALL * args.steps / elapsed / 1e9) if per_update else None,
        "issue_roofline": issue,
        "paper_context": {"tcups_abstract": 0.15, "tcups_introduction": 0.18, "hardware": "1x H100",
                          "conditions": "16-bit fields, eps and sigma, no sources, domain size not stated",
                          "note": "context only, not this workload"},
        "naive": naive,
        "storage_16bit": narrow,
        "systolic_1024": big,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(shape, budget_s=float(os.environ.get("BENCH_CPU_BUDGET_S", "15")))
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
