#!/usr/bin/env python
"""Throughput benchmark of the open-pipe Poisson solve on GB300.

Workload: one 128x128x1024 IGF solve (padded 256x256x2048), a = b = 1,
sigma_perp = 0.15, sigma_z = 3 (sigma_z/sigma_x = 20), Lz = 8 sigma_z, M = 20,
FP32 path; a step is one full solve of a synthetic Gaussian bunch resident in
HBM, in the handle's default form (the mode-space form at this size: the
transverse transforms pruned to the 20 x 20 modes, the zero-padded z
convolution per mode, the back-projection); the padded-transform form (z
transform, transverse stage with the four-term Green product, inverse z
transform) is timed beside it.  L2 (129 MB) is flushed by a 256 MB write
between steps and the flush is outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the solve does not shard; N ranks run N independent replicas
(weak scaling), value = total solves / max-over-ranks time.
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

METRIC = "pipe-Poisson solves/s at 128^2x1024 (FP32 vs FP64 at stated err); % HBM roofline"
WORKLOAD = "pipe128x128x1024_igf"


# kernel sources whose ncu counters are summarised under profiles/; the
# recorded DRAM traffic is reported only while these files hash to the value
# written next to it (a changed kernel reports traffic null)
KERNEL_SOURCES = {
    "transverse": ["tdst_impl.cuh", "transverse_sym.cu", "fft_common.cuh", "solver.cuh"],
    "z_forward": ["zfft_impl.cuh", "zfft.cu", "fft_common.cuh", "solver.cuh"],
    "z_inverse": ["zfft_impl.cuh", "zfft.cu", "fft_common.cuh", "solver.cuh"],
    "mode_project": ["modes_fast.cu", "modes_impl.cuh", "modes.cuh", "zfft_impl.cuh"],
    "mode_z": ["modes_z.cu", "modes_impl.cuh", "modes.cuh", "zfft_impl.cuh", "fft_common.cuh"],
    "mode_back": ["modes_fast.cu", "modes_impl.cuh", "modes.cuh", "zfft_impl.cuh"],
}
PROFILE_FILES = {
    "transverse": "transverse_dsts_pipe128x128x1024_igf_f32.md",
    "z_forward": "zfft_pipe128x128x1024_igf_f32.md",
    "z_inverse": "zfft_pipe128x128x1024_igf_f32.md",
    "mode_project": "modes_pipe128x128x1024_igf_f32.md",
    "mode_z": "modes_pipe128x128x1024_igf_f32.md",
    "mode_back": "modes_pipe128x128x1024_igf_f32.md",
}


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1111_4971_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def memory_floors(rho, phi, flush, steps, stream):
    """Yardsticks for the field's bytes under the same flush as the solves: a
    plain read of rho (torch.sum) and a plain write of phi (fill_), each after
    the 256 MB flush, timed with CUDA events (library kernels, not the path)."""
    import torch
    out = {}
    for name, fn in (("read_field_ms", lambda: rho.sum()), ("write_field_ms", lambda: phi.fill_(0.0))):
        ts = []
        for i in range(steps + 2):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        out[name] = statistics.median(ts)
    return out


def bench_config(nx, ny, nz, world):
    """The workload description both arms print."""
    return {"workload": WORKLOAD, "grid": [nx, ny, nz], "padded": [2 * nx, 2 * ny, 2 * nz],
            "green": "igf", "modes": 20, "sigma": [0.15, 0.15, 3.0], "parallelism": f"replicas{world}",
            "l2": "flushed between steps (256 MB write, outside the timed events)"}


def transform_alg_bytes(nx, ny, nz, esz=4):
    """Algorithmic bytes per launch of the padded-transform form's kernels:
    z forward reads rho and writes the (nz+1) x nx x ny half spectrum, the
    transverse stage reads and writes every kz plane and reads the Green octant
    plane, z inverse reads the spectrum and writes phi."""
    plane = nx * ny * 2 * esz
    green_plane = (nx + 1) * (ny + 1) * esz
    return {"z_forward": nx * ny * nz * esz + (nz + 1) * plane,
            "transverse": (nz + 1) * (2 * plane + green_plane),
            "z_inverse": (nz + 1) * plane + nx * ny * nz * esz}


def mode_alg_bytes(nx, ny, nz, mc, groups, esz=4):
    """Algorithmic bytes per launch of the mode-space form's kernels: the
    projection reads rho and writes one partial projection per group of x
    rows, the z kernel reads the partials and the kernel spectra and writes
    the convolved mode columns, the back-projection reads those (once per z
    chunk) and writes phi."""
    field = nx * ny * nz * esz
    part = groups * mc * nz * esz
    psi = mc * nz * esz
    return {"mode_project": field + part, "mode_z": part + mc * (nz + 1) * esz + psi,
            "mode_back": psi + field}


def mode_flops(nx, ny, nz, mx, mxp, myp, fold, mc):
    """Floating-point operations per launch of the mode-space kernels, counted
    from their sums (an FMA is 2): the projection's y sums (over ny/2 folded
    pairs, or ny rows) and x sums, the back-projection's x sums and y sums, and
    for the z kernel two complex L = nz point FFTs per column at 5 L log2 L
    plus the spectral product (about 40 flops per point)."""
    import math
    yrows = ny // 2 if fold else ny
    proj = 2 * nx * nz * myp * (yrows + mxp) + (2 * nx * nz * yrows if fold else 0)
    back = 2 * nx * nz * myp * (mx + yrows) + (2 * nx * nz * yrows if fold else 0)
    zc = mc * (2 * 5 * nz * int(math.log2(nz)) + 40 * nz)
    return {"mode_project": proj, "mode_z": zc, "mode_back": back}


def dgemm_tflops(n=4096, reps=3):
    """Measured dense FP64 rate of this GPU: a cuBLAS DGEMM (torch.matmul on
    float64), as the yardstick of the FP64 path's arithmetic rate."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return 2.0 * n ** 3 / (min(ts) * 1e-3) / 1e12


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", PROFILE_FILES[kernel])
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                line = line.strip().lstrip("-").strip()
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get(f"{kernel}_source_sha256") != source_hash(kernel):
            return None
        return float(fields[f"{kernel}_dram_bytes_per_launch"])
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend="nccl"):
    """Replica setup from the launcher's environment: one process per GPU
    (RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR/PORT).  backend "gloo" (CPU)
    serves the host-side tests of the N > 1 path."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cuda = backend == "nccl"
    if cuda:
        import torch
        torch.cuda.set_device(local)
    if world > 1:
        import torch
        import torch.distributed as dist
        if cuda:
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world, cuda=True):
    """All ranks here, and (on GPUs) this rank's device idle."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if cuda:
        import torch
        torch.cuda.synchronize()


def max_over_ranks(world, value, device="cuda"):
    """The slowest rank's value (the job's wall time is set by it)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps_per_rank, max_total_ms):
    """Units of all ranks per second: replicas each run `steps_per_rank` solves,
    the job takes the slowest rank's time."""
    return world * steps_per_rank / (max_total_ms / 1e3)


def cpu_oracle_baseline(w, steps=1, budget_s=None, warmup=0):
    """The FP64 oracle (scipy.fft, literal four-term Eq. 10) on the host cores:
    `warmup` untimed solves, then `steps` timed full solves, or fewer (at least
    one) once `budget_s` seconds of timed solves have run."""
    from oracle import pipe
    cores = os.cpu_count() or 1
    geom, grid, rho = w["geom"], w["grid"], w["rho"][0]
    spectra = pipe.green_spectra(geom, grid, 1, workers=cores)     # setup, untimed
    for _ in range(warmup):
        pipe.fft_solve(rho, geom, grid, 1, spectra=spectra, workers=cores)
    times = []
    phi = None
    for _ in range(steps):
        t0 = time.perf_counter()
        phi = pipe.fft_solve(rho, geom, grid, 1, spectra=spectra, workers=cores)
        times.append(time.perf_counter() - t0)
        if budget_s is not None and sum(times) >= budget_s:
            break
    del spectra
    return times, cores, phi


# The reference arm's run is bounded: one full oracle solve takes about 9 s on
# 16 cores, so at most REF_WARMUP warm-up solves and as many of the K timed
# steps as fit in REF_BUDGET_S seconds are run (at least one).
REF_WARMUP = 1
REF_BUDGET_S = 120.0


def run_reference(args):
    """--impl reference: the FP64 CPU oracle as it stands, timed per step."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from inputs import bunches
    w = bunches.workload_throughput_128()
    warm = min(args.warmup, REF_WARMUP)
    timed, cores, _ = cpu_oracle_baseline(w, steps=args.steps, budget_s=REF_BUDGET_S, warmup=warm)
    total = sum(timed)
    value = len(timed) / total
    nx, ny, nz = w["grid"].shape
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": len(timed), "steps_requested": args.steps, "warmup": warm,
        "ms_per_step": 1e3 * total / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(nx, ny, nz, world),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "sample": f"{len(timed)} of the {args.steps} requested steps timed "
                                   f"({REF_BUDGET_S:.0f} s budget, {warm} warm-up solve), each one "
                                   "full 128x128x1024 solve (Green spectra precomputed, untimed), "
                                   "scipy.fft with workers=cores"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def time_stages(stages, names, steps, flush, stream):
    """Each stage of `steps` solves timed with CUDA events on `stream`, L2
    flushed before each solve (outside the events)."""
    import torch
    kev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        e = kev[i]
        e[0].record(stream)
        for k, fn in enumerate(stages):
            fn()
            e[k + 1].record(stream)
    torch.cuda.synchronize()
    return {n: [e[k].elapsed_time(e[k + 1]) for e in kev] for k, n in enumerate(names)}


def bench_batched(args, count=96):
    """96 independent IGF solves on mixed grids / aspect ratios: the batched
    call (persistent launch, grouped mode-form launches and the single-solve
    launches its tuner picks) replayed from a CUDA graph, against a loop of
    single solves.  Each arm runs its own handles in its best configuration:
    the loop with every handle autotuned for its single solve (which puts the
    64^2 solves in the transform form), the batched call with the default
    plans (the mode form wherever the modes are at most half the mesh),
    which lets it group those solves as well."""
    import torch

    from inputs import bunches
    from paper_1111_4971_gb300 import (PipeSolver, batch_grouped, batch_plan_info, batch_side_streams, batch_status,
                                       solve_batched)
    items = bunches.workload_batched_96(count=count)
    solvers, loop_solvers, rhos = [], [], []
    for it in items:
        solvers.append(PipeSolver(it["geom"], it["grid"], igf=True, dtype=torch.float32))
        loop_solvers.append(PipeSolver(it["geom"], it["grid"], igf=True, dtype=torch.float32))
        rhos.append(torch.tensor(it["rho"], dtype=torch.float32, device="cuda"))
    phis = [s.empty() for s in solvers]
    loop_phis = [s.empty() for s in loop_solvers]
    grids = sorted({(it["grid"].nx, it["grid"].nz) for it in items})
    for s in loop_solvers:              # autotuned plans for the loop of single solves
        s.autotune()
    stream = torch.cuda.Stream()
    reps = max(5, args.steps // 4)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    with torch.cuda.stream(stream):
        loop_ms = timed(lambda: [s.solve(r, p, stream=stream) for s, r, p in zip(loop_solvers, rhos, loop_phis)])
        solve_batched(solvers, rhos, phis, stream=stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            solve_batched(solvers, rhos, phis, stream=stream)
        batch_ms = timed(g.replay)
    ok = batch_status(solvers) == 0
    persistent, order = batch_plan_info(solvers)
    grouped, ngroups = batch_grouped(solvers, with_groups=True)
    # the two arms compute the same operator in their own forms: they agree to FP32 rounding
    agree = max(float((a - b).norm() / b.norm()) for a, b in zip(phis, loop_phis))
    forms = {"batched": sum(1 for s in solvers if s.plan["t_kind"] == 3),
             "loop": sum(1 for s in loop_solvers if s.plan["t_kind"] == 3)}
    return {"solves": count, "grids": grids, "batched_ms": batch_ms, "loop_ms": loop_ms,
            "plans": {"batched": "default", "loop": "autotuned per handle"},
            "mode_form_solves": forms, "max_rel_l2_batched_vs_loop": agree,
            "batched_solves_per_s": count / (batch_ms * 1e-3),
            "loop_solves_per_s": count / (loop_ms * 1e-3), "speedup": loop_ms / batch_ms,
            "status_ok": ok, "persistent_solves": persistent,
            "order": ["stage-major", "pipelined", "L2-local"][order],
            "launches_per_batch": (1 if persistent else 0) + 3 * (count - persistent - grouped) + 3 * ngroups,
            "side_streams": batch_side_streams(solvers),
            # mode-form solves of one shape run as one launch per stage
            "grouped_solves": grouped, "groups": ngroups}


def bench_banded(args):
    """Banded reduction (Sec. 5, Eq. 17-18) against the full solve on a bunch
    30 pipe widths long, 128^2 x 1024 cell-centred, FP32: solves/s and the
    relative difference to the full solve for a few band widths."""
    import torch

    from inputs.bunches import cell_centred, gaussian_bunch
    from paper_1111_4971_gb300 import PipeSolver
    geom, grid = cell_centred(1.0, 1.0, 128, 128, 1024, 240.0 / 1024, modes=20)
    rho = torch.tensor(gaussian_bunch(geom, grid, (0.5, 0.5, 120.0), (0.15, 0.15, 30.0)),
                       dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def timed(s, out, reps=10):
        for _ in range(3):
            s.solve(rho, out)
        ts = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.solve(rho, out)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    full = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    pf = full.empty()
    t_full = timed(full, pf)
    ref = pf.double()
    out = {"workload": "pipe128x128x1024_igf_sigmaz30a", "full_ms": t_full, "bands": []}
    for nb in (0, 2, 8, 10, 16):
        s = PipeSolver(geom, grid, igf=True, dtype=torch.float32, banded=nb)
        p = s.empty()
        t = timed(s, p)
        err = float((p.double() - ref).norm() / ref.norm())
        out["bands"].append({"n_neighbors": nb, "ms": t, "speedup_vs_full": t_full / t,
                             "rel_l2_vs_full": err})
    return out


def run_ours(args):
    import numpy as np
    import torch

    from inputs import bunches
    from paper_1111_4971_gb300 import PipeSolver

    world, rank, local = dist_setup()
    w = bunches.workload_throughput_128()
    geom, grid, rho_np = w["geom"], w["grid"], w["rho"][0]
    nx, ny, nz = grid.shape
    dev = torch.device("cuda", local)

    s32 = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
    if args.form == "transforms":              # the padded-transform form as the headline
        s32.set_plan(z_warps=4, z_pipe=0, t_h=1, t_threads=256, t_kind=2)
    if args.autotune:
        s32.autotune()
    rho = torch.tensor(rho_np, dtype=torch.float32, device=dev)
    phi = s32.empty()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()
    modes_form = s32.plan["t_kind"] == 3
    if modes_form:
        mx, mxp, myp, fold, groups = s32.mode_layout()
        part, psi = s32.mode_buffers()
        stage_names = ["mode_project", "mode_z", "mode_back"]
        stages = [lambda: s32.stage_modes(0, rho, part), lambda: s32.stage_modes(1, part, psi),
                  lambda: s32.stage_modes(2, psi, phi)]
        alg_bytes = mode_alg_bytes(nx, ny, nz, mxp * myp, groups)
    else:
        spec = s32.spectrum_buffer()
        stage_names = ["z_forward", "transverse", "z_inverse"]
        stages = [lambda: s32.stage_z_forward(rho, spec), lambda: s32.stage_transverse(spec),
                  lambda: s32.stage_z_inverse(spec, phi)]
        alg_bytes = transform_alg_bytes(nx, ny, nz)

    for _ in range(args.warmup):
        s32.solve(rho, phi)
    barrier(world)
    if args.solves_only:                       # profiling target: K plain solves
        sp, rp, pp_ = s32, rho, phi
        if args.dtype == "f64":
            sp = PipeSolver(geom, grid, igf=True, dtype=torch.float64)
            rp = rho.double()
            pp_ = sp.empty()
            for _ in range(args.warmup):
                sp.solve(rp, pp_)
        for _ in range(args.steps):
            if args.flush:
                flush.fill_(0.0)
            sp.solve(rp, pp_)
        barrier(world)
        if rank == 0:
            print(json.dumps({"solves_only": args.steps, "plan": sp.plan, "dtype": args.dtype}))
        return 0

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    # ---- timed region: K solves ------------------------------------------
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        s32.solve(rho, phi)
        ev[i][1].record(stream)
    barrier(world)
    t_wall = time.perf_counter() - t_wall
    solve_ms = [a.elapsed_time(b) for a, b in ev]
    # ---- the same K steps through the stage entry points, per kernel -------
    k_ms = time_stages(stages, stage_names, args.steps, flush, stream)
    floors = memory_floors(rho, phi, flush, min(args.steps, 20), stream)
    barrier(world)
    clocks = sampler.stop()
    total_ms = max_over_ranks(world, sum(solve_ms))
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, args.steps, total_ms)

    # ---- end to end through host buffers (copies inside the timed region) --
    # The public host API for a sequence of solves: every step copies its
    # input in from pinned host memory and its result out, overlapped with
    # the neighbouring steps' compute (pipe_poisson_solve_host_stream).
    nbuf = 4
    rho_h = [torch.tensor(rho_np, dtype=torch.float32).pin_memory() for _ in range(nbuf)]
    phi_h = [torch.empty((nx, ny, nz), dtype=torch.float32).pin_memory() for _ in range(nbuf)]
    ins = [rho_h[k % nbuf] for k in range(args.steps)]
    outs = [phi_h[k % nbuf] for k in range(args.steps)]
    s32.solve_host_stream(ins[:3], outs[:3])            # warm-up: creates the staging ring
    flush.fill_(0.0)
    barrier(world)
    t0 = time.perf_counter()
    s32.solve_host_stream(ins, outs)
    e2e_total = max_over_ranks(world, 1e3 * (time.perf_counter() - t0))
    e2e_value = whole_job_rate(world, args.steps, e2e_total)
    # the same, one blocking call per step (pipe_poisson_solve_host), for reference
    for _ in range(2):
        s32.solve_host(rho_h[0], phi_h[0])
    barrier(world)
    serial_ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s32.solve_host(rho_h[0], phi_h[0])
        serial_ms.append(1e3 * (time.perf_counter() - t0))
    serial_value = whole_job_rate(world, args.steps, max_over_ranks(world, sum(serial_ms)))
    nbytes = nx * ny * nz * 4

    # ---- roofline of the dominant kernel and of the whole solve ----------
    peak, peak_kind = peaks()
    means = {k: statistics.mean(v) for k, v in k_ms.items()}
    dom = max(means, key=means.get)
    achieved = {k: alg_bytes[k] / (means[k] * 1e-3) / 1e9 for k in means}
    solve_bytes = sum(alg_bytes.values())
    b_pad = 4 * (2 * nx) * (2 * ny) * (nz + 1) * 8
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(nx, ny, nz, world),
        "form": "modes" if modes_form else "transforms",
        "plan": s32.plan,
        "gpu_launches": 3 * args.steps,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved[dom], "peak": peak,
                     "unit": "GB/s", "frac": achieved[dom] / peak, "traffic": recorded_traffic(dom),
                     "peak_kind": peak_kind,
                     "alg_bytes_per_launch": alg_bytes[dom], "kernel_ms": means[dom]},
        "kernels_ms": means,
        "kernels_gbs": achieved,
        # what the memory delivers for the field's 64 MB under the same flush
        # (plain read / write, library kernels): the floors of the projection
        # and the back-projection, and each kernel's time against its floor
        "memory_floors": dict(floors, **({
            "mode_project_floor_over_kernel": floors["read_field_ms"] / means["mode_project"],
            "mode_back_floor_over_kernel": floors["write_field_ms"] / means["mode_back"]} if modes_form else {})),
        "kernels_source_sha256": {k: source_hash(k) for k in KERNEL_SOURCES},
        # the whole solve against its own algorithmic bytes (the sum over its kernels)
        "solve_alg_bytes": solve_bytes,
        "solve_gbs": solve_bytes / (ms_per_step * 1e-3) / 1e9,
        "solve_frac": solve_bytes / (ms_per_step * 1e-3) / 1e9 / peak,
        # the metric's nominal bytes: the padded transforms' half spectra read and
        # written twice (4 |S|); neither form moves them, so this is not a traffic
        "b_pad": {"bytes": b_pad, "gbs": b_pad / (ms_per_step * 1e-3) / 1e9,
                  "frac_of_measured": b_pad / (ms_per_step * 1e-3) / 1e9 / peak,
                  "frac_of_8tbs": b_pad / (ms_per_step * 1e-3) / 1e9 / 8000.0},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": nbytes,
                "d2h_bytes_per_step": nbytes,
                "api": "pipe_poisson_solve_host_stream (pinned host buffers, copies of "
                       "neighbouring steps overlapped with the compute)",
                "serial_one_call_per_step": serial_value},
        "wall_s_timed_loop": t_wall,
        # the handle's device error word after the timed steps (0: no bounded
        # wait of the staged transverse kernel gave up)
        "device_status": s32.status(),
    }

    # ---- the padded-transform form of the same solve, same steps ---------
    if modes_form and not args.quick:
        st32 = PipeSolver(geom, grid, igf=True, dtype=torch.float32)
        st32.set_plan(z_warps=4, z_pipe=0, t_h=1, t_threads=256, t_kind=2)
        spec = st32.spectrum_buffer()
        for _ in range(args.warmup):
            st32.solve(rho, phi)
        tms = []
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st32.solve(rho, phi)
            b.record(stream)
            tms.append((a, b))
        torch.cuda.synchronize()
        t_ms = statistics.mean(a.elapsed_time(b) for a, b in tms)
        tk = time_stages([lambda: st32.stage_z_forward(rho, spec), lambda: st32.stage_transverse(spec),
                          lambda: st32.stage_z_inverse(spec, phi)], ["z_forward", "transverse", "z_inverse"],
                         args.steps, flush, stream)
        tmeans = {k: statistics.mean(v) for k, v in tk.items()}
        tbytes = transform_alg_bytes(nx, ny, nz)
        tdom = max(tmeans, key=tmeans.get)
        tach = {k: tbytes[k] / (tmeans[k] * 1e-3) / 1e9 for k in tmeans}
        line["transform_form"] = {
            "plan": st32.plan, "solves_per_s": 1e3 / t_ms, "ms": t_ms, "kernels_ms": tmeans,
            "kernels_gbs": tach, "solve_alg_bytes": sum(tbytes.values()),
            "solve_frac": sum(tbytes.values()) / (t_ms * 1e-3) / 1e9 / peak,
            "roofline": {"bound": "hbm", "kernel": tdom, "achieved": tach[tdom], "peak": peak, "unit": "GB/s",
                         "frac": tach[tdom] / peak, "traffic": recorded_traffic(tdom),
                         "alg_bytes_per_launch": tbytes[tdom], "kernel_ms": tmeans[tdom]}}
        st32.close()

    # ---- FP64 path, free-space (Hockney) comparison, accuracy -------------
    if rank == 0 and not args.quick:
        s64 = PipeSolver(geom, grid, igf=True, dtype=torch.float64)
        rho64 = torch.tensor(rho_np, dtype=torch.float64, device=dev)
        phi64 = s64.empty()
        for _ in range(2):
            s64.solve(rho64, phi64)
        t64 = []
        for i in range(5):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64.solve(rho64, phi64)
            b.record(stream)
            torch.cuda.synchronize()
            t64.append(a.elapsed_time(b))
        s32.solve(rho, phi)
        torch.cuda.synchronize()
        p32 = phi.double().cpu().numpy()
        p64 = phi64.cpu().numpy()
        err = float(np.linalg.norm(p32 - p64) / np.linalg.norm(p64))
        sh = PipeSolver(None, grid, dtype=torch.float32, free_space=True)
        phih = sh.empty()
        for _ in range(2):
            sh.solve(rho, phih)
        th = []
        for i in range(10):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sh.solve(rho, phih)
            b.record(stream)
            torch.cuda.synchronize()
            th.append(a.elapsed_time(b))
        # complex-FP16 spectra with per-slab scales (optional variant)
        s16 = PipeSolver(geom, grid, igf=True, dtype=torch.float32, fp16_spectra=True)
        phi16 = s16.empty()
        for _ in range(2):
            s16.solve(rho, phi16)
        t16 = []
        for i in range(10):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s16.solve(rho, phi16)
            b.record(stream)
            torch.cuda.synchronize()
            t16.append(a.elapsed_time(b))
        p16 = phi16.double().cpu().numpy()
        line["fp16_spectra"] = {"solves_per_s": 1e3 / statistics.median(t16), "ms": statistics.median(t16),
                                "rel_l2_vs_fp64": float(np.linalg.norm(p16 - p64) / np.linalg.norm(p64))}
        line["fp64"] = {"solves_per_s": 1e3 / statistics.median(t64), "ms": statistics.median(t64),
                        "plan": s64.plan}
        if s64.plan["t_kind"] == 3:
            # the FP64 mode kernels against the measured FP64 rate: they run
            # on the FP64 FMA units, so their bound is arithmetic, not HBM
            m64 = s64.mode_layout()
            part64, psi64 = s64.mode_buffers()
            st64 = [lambda: s64.stage_modes(0, rho64, part64), lambda: s64.stage_modes(1, part64, psi64),
                    lambda: s64.stage_modes(2, psi64, phi64)]
            k64 = time_stages(st64, stage_names, 5, flush, stream)
            k64 = {k: statistics.median(v) for k, v in k64.items()}
            fl = mode_flops(nx, ny, nz, m64[0], m64[1], m64[2], m64[3], m64[1] * m64[2])
            peak64 = dgemm_tflops()
            rate = {k: fl[k] / (k64[k] * 1e-3) / 1e12 for k in k64}
            dom64 = max(k64, key=k64.get)
            line["fp64"].update({
                "kernels_ms": k64, "kernels_flops": fl, "kernels_tflops": rate,
                "peak_tflops": peak64, "peak_kind": "measured: cuBLAS DGEMM 4096^3 (torch.matmul)",
                "roofline": {"bound": "fp64", "kernel": dom64, "achieved": rate[dom64], "peak": peak64,
                             "unit": "TFLOP/s", "frac": rate[dom64] / peak64},
                "solve_tflops": sum(fl.values()) / (statistics.median(t64) * 1e-3) / 1e12,
                "solve_frac": sum(fl.values()) / (statistics.median(t64) * 1e-3) / 1e12 / peak64})
        # the FP64 padded-transform form (n-point transverse routine, global scratch planes)
        s64t = PipeSolver(geom, grid, igf=True, dtype=torch.float64)
        s64t.set_plan(z_warps=8, z_pipe=0, t_h=1, t_threads=256, t_kind=1)
        s64t.solve(rho64, phi64)
        t64t = []
        for i in range(3):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s64t.solve(rho64, phi64)
            b.record(stream)
            torch.cuda.synchronize()
            t64t.append(a.elapsed_time(b))
        line["fp64_transform_form"] = {"solves_per_s": 1e3 / statistics.median(t64t),
                                       "ms": statistics.median(t64t), "plan": s64t.plan}
        s64t.close()
        line["fp32_rel_l2_vs_fp64"] = err
        line["hockney_fp32"] = {"solves_per_s": 1e3 / statistics.median(th), "ms": statistics.median(th)}
        if args.check_oracle:
            from oracle import pipe
            nodes = [(64, 64, 512), (0, 0, 0), (127, 127, 1023), (5, 100, 300), (90, 30, 700)]
            want = pipe.direct_sum_at(rho_np, geom, grid, 1, nodes)
            got = np.array([p64[n] for n in nodes])
            line["fp64_sampled_max_err_vs_direct_sum"] = float(np.abs(got - want).max()
                                                               / np.abs(p64).max())

    if rank == 0 and not args.quick:
        line["batched"] = bench_batched(args)
        line["banded"] = bench_banded(args)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, cores, _ = cpu_oracle_baseline(w, steps=1)
        line["cpu_baseline"] = {"value": 1.0 / times[0], "unit": "solves/s", "cores": cores,
                                "kind": "oracle",
                                "sample": "one full 128x128x1024 FP64 solve of the same bunch "
                                          "(scipy.fft four-term Eq. 10, Green spectra "
                                          "precomputed and untimed)"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the FP64 / Hockney extras")
    ap.add_argument("--check-oracle", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"],
                    help="with --solves-only: the solves' dtype (profiling of the FP64 kernels)")
    ap.add_argument("--form", default="default", choices=["default", "transforms"],
                    help="transforms: time the padded-transform form (profiling of its kernels)")
    ap.add_argument("--solves-only", action="store_true",
                    help="setup, warm-up and K plain solves only (profiling target)")
    ap.add_argument("--flush", action="store_true",
                    help="with --solves-only: flush L2 before every solve, as the timed steps do")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    how, what = replica_launch(args.gpus, os.environ)
    if how == "error":
        print(what, file=sys.stderr)
        return 2
    if how == "spawn":
        return subprocess.call(what)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


def replica_launch(gpus, env):
    """How to run N replicas: ("run", None) in this process when the launcher's
    WORLD_SIZE matches --gpus (or N = 1 with no launcher); ("spawn", command)
    to start N processes, one per GPU, through torch.distributed.run when N > 1
    and no launcher did; ("error", message) when WORLD_SIZE and --gpus differ."""
    world = env.get("WORLD_SIZE")
    if world is None:
        if gpus <= 1:
            return "run", None
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={gpus}",
               "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)]
        return "spawn", cmd + sys.argv[1:]
    if int(world) != gpus:
        return "error", f"bench.py: --gpus {gpus} but WORLD_SIZE={world} processes were launched"
    return "run", None


if __name__ == "__main__":
    sys.exit(main())
