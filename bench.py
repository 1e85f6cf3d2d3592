#!/usr/bin/env python
"""Benchmark of the LFD propagation hot path on one GB300 (or N replicas).

Headline workload (c2, the largest single domain): 64^3 periodic grid,
h = 0.35 bohr, 1024 complex64 Kohn-Sham orbitals, 4th-order finite
differences, 128 Gaussian wells and 128 atoms x 8 projectors on a perturbed
4x4x4 two-site lattice, Gaussian-envelope vector potential, f_n = 2, Gram
and update GEMMs in BF16x3 split precision on the tensor cores, FP64
Cholesky re-orthonormalisation every 10 steps.  One benchmark step is one
mlmd_propagate call of 10 full-scheme Taylor-4 steps with per-step
observables (electron count, energy, current), which ends with one
re-orthonormalisation, plus the density/current fields of the final state.

The same run also measures, each as an object inside the one JSON line:
  c1  48^3 x 256 orbitals, 64 atoms x 4 projectors, 1000 Taylor steps per
      benchmark step;
  c3  216 uneven domains (N ~ U{24..40}^3, N_o ~ U{32..192}, about 41
      projector spheres over every grid point) stepped together, one Taylor
      step of every domain per benchmark step (one CUDA graph launch).
Metric: orbital*gridpoint*steps per second (units = N_o * N_g * Taylor
steps, summed over domains); also seconds per (electron * step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--headline-only]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "orbital·gridpoint·steps/s per GB300"
UNIT = "orbital·gridpoint·steps/s"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# algorithmic HBM bytes per orbital*gridpoint*step of the four staged
# full-scheme passes in complex64: the first reads psi and writes w (16 B),
# the other three read w and psi and write w or psi (24 B each)
STAGE_BYTES_PER_UNIT = 16 + 3 * 24
C2_QD_PER_STEP = 10          # Taylor steps per c2 benchmark step (one re-orthonormalisation period)
STAGE_SRC = os.path.join(ROOT, "paper_2509_00966_gb300", "csrc", "k_stage_tma.cu")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per stage launch,
# the mean over the four stage launches of one Taylor step, from one ncu
# capture per workload, keyed by the SHA-256 (first 16 hex digits) of the
# stage kernel's source at the time of the capture; a different source
# reports no traffic.  Per orbital*gridpoint, so that a capture on fewer
# orbitals scales to the benchmark's orbital count.
STAGE_TRAFFIC = {
    # (313.2 + 184.1) + (547.1 + 194.8) + (547.1 + 194.4) + (544.8 + 185.2) MB over
    # the four launches, 48^3 x 256 orbitals
    "c1": {"src_sha16": "5a382b1bf69fc774", "bytes_per_unit": 677.7e6 / (48 ** 3 * 256)},
    # (793.8 + 496.7) + (1332.3 + 506.4) + (1333.4 + 506.9) + (1330.4 + 497.9) MB over
    # the four launches, the c2 grid and projectors on 256 of its 1024 orbitals
    "c2": {"src_sha16": "5a382b1bf69fc774", "bytes_per_unit": 1699.5e6 / (64 ** 3 * 256)},
}


def _sha16(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--headline-only", action="store_true", help="measure c2 only (no c1 / c3 objects)")
    p.add_argument("--c1-qd-steps", type=int, default=1000, help="Taylor steps per c1 benchmark step")
    p.add_argument("--c1-steps", type=int, default=5, help="timed c1 benchmark steps")
    p.add_argument("--c3-steps", type=int, default=10, help="timed c3 benchmark steps")
    p.add_argument("--e2e-steps", type=int, default=4)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU work of each oracle sample")
    p.add_argument("--ks", nargs=3, metavar=("N", "N_ORB", "MODE"),
                   help="time the Eq. 5 KS-space nonlocal correction on an N^3 x N_ORB complex64 domain in gemm MODE")
    p.add_argument("--occ", nargs=3, metavar=("N", "N_ORB", "MODE"),
                   help="time the shadow-dynamics occupations (overlap with Psi(0) and the f_s sums) on an "
                        "N^3 x N_ORB complex64 domain in gemm MODE")
    p.add_argument("--reorth", nargs=3, metavar=("N", "N_ORB", "MODE"),
                   help="time Cholesky re-orthonormalisations of an N^3 x N_ORB complex64 domain in gemm MODE")
    p.add_argument("--gram", nargs=3, metavar=("N", "N_ORB", "MODE"),
                   help="time the overlap (Gram) GEMM of an N^3 x N_ORB complex64 domain in gemm MODE")
    p.add_argument("--suite", action="store_true",
                   help="time the remaining workloads (c0, c4), one JSON line each")
    p.add_argument("--stage-case", nargs=4, metavar=("CFG", "N_ORB", "QD_STEPS", "REPS"),
                   help="run only stage launches of workload CFG (c1 or c2) on N_ORB orbitals, REPS propagate "
                        "calls of QD_STEPS steps (a small case for ncu captures)")
    p.add_argument("--sweep-case", nargs=4, metavar=("CFG", "N_ORB", "QD_STEPS", "REPS"),
                   help="time the one-sweep local Taylor-4 against the four staged passes on a "
                        "projector-free domain of config CFG's grid")
    p.add_argument("--gauge-case", nargs=4, metavar=("CFG", "N_ORB", "QD_STEPS", "REPS"),
                   help="time workload CFG on N_ORB orbitals with real and with velocity-gauge projectors")
    p.add_argument("--nl-case", nargs=4, metavar=("N", "N_ORB", "QD_STEPS", "REPS"),
                   help="one domain of the batched workload's kind (N^3 grid, h = 0.35, round(N^3/64) atoms x 4 "
                        "projectors): REPS propagate calls of QD_STEPS steps; per-kernel times")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), "src": "measured"}
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS,
                "bf16_tflops_sustained": 1700.0, "src": "fallback"}


class Clocks:
    """nvidia-smi samples (200 ms) of one GPU while the timed region runs."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                smax.append(float(c[2]))
            except ValueError:
                continue
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _max_over_ranks(x, ws):
    """The largest x over the ranks (the slowest replica's time); x itself
    on one rank.  Uses the process group's own device: CUDA under NCCL, the
    host under gloo."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(ws, units_per_rank, t_s):
    """Whole-job throughput of ws independent replicas (no data exchanged
    between them): every rank processed units_per_rank, in at most the
    slowest rank's time t_s."""
    return ws * units_per_rank / t_s


def _physical_gpu(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local < len(ids):
            return ids[local]
    return str(local)


def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def _c2_spec():
    from paper_2509_00966_gb300 import inputs
    return inputs.config("c2")


def _c2_name(spec):
    return (f"c2: {spec.n[0]}^3 grid h={spec.h} bohr, {spec.n_orb} complex64 orbitals, {spec.fd_order}th-order FD, "
            f"{len(spec.atoms)} atoms x {spec.n_proj} projectors, Gaussian-envelope A(t), BF16x3 tensor-core Gram "
            f"and update GEMMs, FP64 Cholesky re-orthonormalisation every {spec.ortho_every} steps; "
            f"{C2_QD_PER_STEP} full-scheme Taylor-4 steps + per-step norm/energy/current + one "
            f"re-orthonormalisation + density/current fields per bench step")


def _c1_workload(qd_steps):
    from paper_2509_00966_gb300 import inputs
    spec = inputs.config("c1")
    A = inputs.envelope_pulse(1000, spec.dt)
    reps = (qd_steps + 999) // 1000
    spec.A = np.tile(A, (reps, 1))[:qd_steps]
    spec.n_steps = qd_steps
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    psi = inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed)
    return spec, V, psi


def _device_orbitals(n_grid, n_orb, dV, seed, dtype):
    """Seeded random orbitals generated on the device (normalised; the
    library's own Cholesky re-orthonormalisation makes them orthonormal)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    rdt = torch.float32 if dtype == torch.complex64 else torch.float64
    re = torch.randn(n_grid, n_orb, generator=g, device="cuda", dtype=rdt)
    im = torch.randn(n_grid, n_orb, generator=g, device="cuda", dtype=rdt)
    # E|re + i im|^2 = 2 per point
    return (torch.complex(re, im) / float(np.sqrt(2.0 * n_grid * dV))).contiguous()


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_steps(spec, V, psi, A, target_s, max_steps, ortho_every=0):
    """Time the FP64 oracle as it stands: one warm step, then as many Taylor
    steps (+ observables) as fill about target_s.  Returns (units/s, n, dt)."""
    import oracle
    od = oracle.Domain(spec.n, spec.h, psi.shape[1], spec.fd_order, V, spec.atoms, spec.n_proj, spec.r_c,
                       spec.r_cut, spec.D)
    f = np.full(psi.shape[1], 2.0)
    p = np.ascontiguousarray(psi, np.complex128)
    t0 = time.perf_counter()
    p, _ = oracle.propagate(od, p, A[:1], spec.dt, f)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_steps, round(target_s / max(t1, 1e-3)) - 1)))
    t0 = time.perf_counter()
    p, _ = oracle.propagate(od, p, A[1:1 + n], spec.dt, f, ortho_every=ortho_every, step0=1)
    dt = time.perf_counter() - t0
    return spec.n_grid * psi.shape[1] * n / dt, n, dt


def cpu_baseline_c2(spec, V, psi_sample, target_s):
    v, n, dt = _oracle_steps(spec, V, psi_sample, spec.A, target_s, 20)
    return {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{n} Taylor-4 steps (+observables) of the c2 domain (full grid, all {len(spec.atoms)}x"
                      f"{spec.n_proj} projectors) on {psi_sample.shape[1]} of its {spec.n_orb} orbitals, FP64 "
                      f"C/OpenMP oracle, {dt:.1f} s; the re-orthonormalisation every 10 steps is not in the sample"}


def cpu_baseline_c1(spec, V, psi, target_s):
    v, n, dt = _oracle_steps(spec, V, psi, spec.A, target_s, 20)
    return {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"{n} Taylor-4 steps (+observables) of the full c1 workload, all {spec.n_orb} orbitals, "
                      f"FP64 C/OpenMP oracle, {dt:.1f} s"}


def cpu_baseline_c3(specs, target_s):
    """One Taylor step (+ observables) of the first few c3 domains, all their
    orbitals, until about target_s of CPU work; the rate is their units over
    their summed time."""
    from paper_2509_00966_gb300 import inputs
    import oracle
    units, spent, used = 0, 0.0, 0
    for i, sp in enumerate(specs):
        V = inputs.gaussian_wells(sp.n, sp.h, sp.wells, sp.well_depth, sp.well_width)
        psi = inputs.random_orbitals(sp.n_grid, sp.n_orb, sp.dV, 1000 + i)
        od = oracle.Domain(sp.n, sp.h, sp.n_orb, sp.fd_order, V, sp.atoms, sp.n_proj, sp.r_c, sp.r_cut, sp.D)
        t0 = time.perf_counter()
        oracle.propagate(od, psi, sp.A[:1], sp.dt, np.full(sp.n_orb, 2.0))
        spent += time.perf_counter() - t0
        units += sp.n_grid * sp.n_orb
        used += 1
        if spent >= target_s:
            break
    return {"value": units / spent, "unit": UNIT, "cores": _cores(), "kind": "oracle",
            "sample": f"1 Taylor-4 step (+observables) of each of the first {used} of the {len(specs)} c3 domains, "
                      f"all their orbitals, FP64 C/OpenMP oracle, {spent:.1f} s"}


def run_reference(args):
    """The oracle as the reference arm, on the headline workload's domain:
    each step is one Taylor step (+ observables) of the c2 domain on 64 of
    its 1024 orbitals (host cores, rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_2509_00966_gb300 import inputs
    spec = _c2_spec()
    n_orb = 64
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    psi = inputs.random_orbitals(spec.n_grid, n_orb, spec.dV, spec.seed)
    od = oracle.Domain(spec.n, spec.h, n_orb, spec.fd_order, V, spec.atoms, spec.n_proj, spec.r_c, spec.r_cut,
                       spec.D)
    f = np.full(n_orb, 2.0)
    p = psi
    A = spec.A
    for k in range(args.warmup):
        p, _ = oracle.propagate(od, p, A[k % len(A):k % len(A) + 1], spec.dt, f)
    t0 = time.perf_counter()
    for k in range(args.steps):
        j = (args.warmup + k) % len(A)
        p, _ = oracle.propagate(od, p, A[j:j + 1], spec.dt, f)
    dt = time.perf_counter() - t0
    units = spec.n_grid * n_orb * args.steps
    v = units / dt
    sample = (f"{args.steps} Taylor-4 steps (+observables) of the c2 domain (full grid, all 128x8 projectors) on "
              f"{n_orb} of its 1024 orbitals, FP64 C/OpenMP oracle")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PbTiO3-like domain)",
            "config": {"workload": _c2_name(spec), "reference_step": f"1 Taylor-4 step with observables on {n_orb} "
                                                                     f"orbitals", "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _stage_roofline(peaks, units_per_launch, st_ms, st_n, total_ms, pr_ms, traffic_key, n_grid, n_orb):
    """Roofline of the stage kernel: algorithmic bytes per launch (88 B/unit
    over four launches of a Taylor step) over its mean launch time."""
    avg_s = st_ms * 1e-3 / max(st_n, 1)
    achieved = (STAGE_BYTES_PER_UNIT / 4.0) * units_per_launch / avg_s / 1e9 if st_ms > 0 else None
    tr = STAGE_TRAFFIC.get(traffic_key)
    traffic = None
    if tr and tr["src_sha16"] == _sha16(STAGE_SRC):
        traffic = tr["bytes_per_unit"] * n_grid * n_orb
    return {"bound": "hbm", "kernel": "k_stage_tma (fused stencil + V + A + nonlocal scatter + Taylor combine)",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
            "peak_source": f"{peaks['src']} hbm_gbs",
            "algorithmic_bytes_per_launch": (STAGE_BYTES_PER_UNIT / 4.0) * units_per_launch,
            "traffic": traffic,
            "traffic_unit": "DRAM bytes read + written per stage launch (ncu, mean of the four stage launches of a "
                            "Taylor step), null when the kernel source differs from the captured one",
            "mean_launch_us": avg_s * 1e6,
            "kernel_share": {"stage": st_ms / total_ms, "project": pr_ms / total_ms},
            "launches": {"stage": st_n, "project": None}}


def run_c2(args, peaks, ws, rank, local):
    """The headline: c2, one benchmark step = 10 Taylor steps + observables,
    one Cholesky re-orthonormalisation, density/current fields."""
    import torch
    from paper_2509_00966_gb300 import inputs, mlmd
    spec = _c2_spec()
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    dom = mlmd.Domain.from_spec(spec, V=V, gemm_mode="bf16x3")
    dom.set_orbitals(_device_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed, torch.complex64))
    dom.reorthonormalize("chol")
    psi0 = dom.get_orbitals()                      # orthonormal start, kept for the e2e leg
    dom.set_orbitals(psi0)
    A_all = spec.A
    blocks = [A_all[(k * C2_QD_PER_STEP) % len(A_all):(k * C2_QD_PER_STEP) % len(A_all) + C2_QD_PER_STEP]
              for k in range(len(A_all) // C2_QD_PER_STEP)]
    counter = [0]

    def one_step():
        A = blocks[counter[0] % len(blocks)]
        counter[0] += 1
        obs = dom.propagate(A, obs=True)
        dom.density_current(A[-1])
        return obs

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        sample = psi0[:, :128].cpu().numpy().astype(np.complex128)
        cpu = cpu_baseline_c2(spec, V, sample, args.cpu_seconds)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(_physical_gpu(local))
    clocks.start()
    time.sleep(0.3)
    l0 = dom.launches
    stream = torch.cuda.current_stream()
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = dom.launches - l0
    ck = clocks.stop()
    t_ms = _max_over_ranks(t_ms, ws)
    if ws > 1:
        torch.distributed.barrier()

    # a second, shorter pass with per-launch CUDA events on the library's
    # stream: the stage kernel's mean launch time and the kernel shares
    prof_steps = max(2, min(args.steps, 5))
    mlmd.profile_enable(dom.handle, True)
    p0, p1 = _events()
    p0.record(stream)
    for _ in range(prof_steps):
        one_step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    st_ms, st_n = mlmd.profile_read(dom.handle, "stage")
    pr_ms, pr_n = mlmd.profile_read(dom.handle, "project")
    mlmd.profile_enable(dom.handle, False)

    # end to end through the C ABI with host buffers: h2d of the orbitals,
    # the propagation, d2h of the orbitals and observables, every step
    pinned_in = psi0.cpu().pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    e2e_t = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dom.set_orbitals(pinned_in)
        dom.propagate(blocks[0], obs=True)
        mlmd.get_orbitals(dom.handle, pinned_out)
        torch.cuda.synchronize()
        if k > 0:
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = _max_over_ranks(float(np.mean(e2e_t)) if e2e_t else float("nan"), ws)
    dom.close()
    del psi0, pinned_in, pinned_out
    torch.cuda.empty_cache()

    units_step = spec.n_grid * spec.n_orb * C2_QD_PER_STEP
    value = _job_value(ws, units_step * args.steps, t_ms * 1e-3)
    electrons = float(np.sum(spec.occ))
    roof = _stage_roofline(peaks, spec.n_grid * spec.n_orb, st_ms, st_n, prof_ms, pr_ms, "c2", spec.n_grid,
                           spec.n_orb)
    roof["launches"]["project"] = pr_n
    roof["profiled_pass"] = {"steps": prof_steps, "ms_per_step": prof_ms / prof_steps,
                             "note": "per-launch events on; the timed region above ran without them"}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded PbTiO3-like domain; orbitals drawn from a seeded device "
                                "generator and Cholesky-orthonormalised by the library)",
        "config": {"workload": _c2_name(spec), "n_grid": spec.n_grid, "n_orb": spec.n_orb,
                   "qd_steps_per_step": C2_QD_PER_STEP, "scheme": "full (v_nl inside Taylor-4)",
                   "gemm_mode": "bf16x3", "l2": "inputs larger than L2 (psi 2.1 GB per state), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "t2s_s_per_electron_step": (t_ms * 1e-3) / (args.steps * C2_QD_PER_STEP * electrons),
        "t2s_paper_context": "1.11e-7 s/(electron*step) on 120,000 PVC tiles (paper, other hardware; context only)",
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": _job_value(ws, units_step, e2e_s), "unit": UNIT,
                "ms_per_call": [round(t * 1e3, 1) for t in e2e_t],
                "h2d_bytes_per_step": int(spec.n_grid * spec.n_orb * 8 + C2_QD_PER_STEP * 3 * 8),
                "d2h_bytes_per_step": int(spec.n_grid * spec.n_orb * 8 + C2_QD_PER_STEP * 5 * 8)},
        "gpu_launches": int(launches),
        "clocks": ck,
    }


def run_c1(args, peaks, want_cpu):
    import torch
    from paper_2509_00966_gb300 import mlmd
    qd = args.c1_qd_steps
    spec, V, psi = _c1_workload(qd)
    cpu = cpu_baseline_c1(spec, V, psi, args.cpu_seconds) if want_cpu else None
    dom = mlmd.Domain.from_spec(spec, V=V)
    dom.set_orbitals(torch.from_numpy(psi).to(torch.complex64).cuda())
    A = spec.A

    def one_step():
        obs = dom.propagate(A, obs=True)
        dom.density_current(A[-1])
        return obs

    for _ in range(2):
        one_step()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    l0 = dom.launches
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(args.c1_steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = dom.launches - l0
    mlmd.profile_enable(dom.handle, True)
    p0, p1 = _events()
    p0.record(stream)
    one_step()
    p1.record(stream)
    torch.cuda.synchronize()
    prof_ms = p0.elapsed_time(p1)
    st_ms, st_n = mlmd.profile_read(dom.handle, "stage")
    pr_ms, pr_n = mlmd.profile_read(dom.handle, "project")
    mlmd.profile_enable(dom.handle, False)
    pinned_in = torch.from_numpy(psi.astype(np.complex64)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dom.set_orbitals(pinned_in)
    dom.propagate(A, obs=True)
    mlmd.get_orbitals(dom.handle, pinned_out)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    dom.close()
    units_step = spec.n_grid * spec.n_orb * qd
    roof = _stage_roofline(peaks, spec.n_grid * spec.n_orb, st_ms, st_n, prof_ms, pr_ms, "c1", spec.n_grid,
                           spec.n_orb)
    roof["launches"]["project"] = pr_n
    return {"workload": (f"c1: 48^3 grid h=0.35 bohr, 256 complex64 orbitals, 4th-order FD, 64 atoms x 4 "
                         f"projectors, Gaussian-envelope A(t), {qd} full-scheme Taylor-4 steps + per-step "
                         f"observables + density/current fields per bench step"),
            "value": units_step * args.c1_steps / (t_ms * 1e-3), "unit": UNIT, "steps": args.c1_steps,
            "ms_per_step": t_ms / args.c1_steps,
            "t2s_s_per_electron_step": (t_ms * 1e-3) / (args.c1_steps * qd * float(np.sum(spec.occ))),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": units_step / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(psi.size * 8 + A.size * 8),
                    "d2h_bytes_per_step": int(psi.size * 8 + qd * 5 * 8)},
            "gpu_launches": int(launches)}


def run_c3(args, peaks, want_cpu):
    """216 uneven domains stepped together (one CUDA graph launch per Taylor
    step of all domains)."""
    import torch
    from paper_2509_00966_gb300 import inputs, mlmd
    specs = inputs.batched_specs(n_steps=200)
    cpu = cpu_baseline_c3(specs, args.cpu_seconds) if want_cpu else None
    doms, host_psi = [], []
    for i, sp in enumerate(specs):
        dd = mlmd.Domain.from_spec(sp)
        p = _device_orbitals(sp.n_grid, sp.n_orb, sp.dV, 1000 + i, torch.complex64)
        dd.set_orbitals(p)
        doms.append(dd)
    b = mlmd.batch_create([dd.handle for dd in doms])
    A = np.stack([sp.A for sp in specs])            # [216, 200, 3]
    units = sum(sp.units_per_step for sp in specs)
    k = [0]

    def one_step():
        j = k[0] % A.shape[1]
        k[0] += 1
        return mlmd.batch_propagate(b, A[:, j:j + 1], first_handle=doms[0].handle)

    for _ in range(2):
        one_step()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    l0 = sum(dd.launches for dd in doms)
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(args.c3_steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = sum(dd.launches for dd in doms) - l0
    # per-kernel times: one Taylor step of every domain outside the graph
    # with per-launch CUDA events (the graph carries no timing events)
    kinds = ("stage", "scatter", "project")
    ktot = {kind: 0.0 for kind in kinds}
    kcnt = {kind: 0 for kind in kinds}
    n_list = 0
    for dd, sp in zip(doms, specs):
        mlmd.profile_enable(dd.handle, True)
        dd.propagate(sp.A[:1], obs=True)
        for kind in kinds:
            t, c = mlmd.profile_read(dd.handle, kind)
            ktot[kind] += t
            kcnt[kind] += c
        mlmd.profile_enable(dd.handle, False)
        n_list += dd.projector_list_length() * sp.n_orb
    # the same Taylor step with the domains one at a time (no graph; each
    # propagate returns its observables to the host), against the batched step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for dd, sp in zip(doms, specs):
        dd.propagate(sp.A[:1], obs=True)
    torch.cuda.synchronize()
    seq_ms = (time.perf_counter() - t0) * 1e3
    # algorithmic nonlocal work of a Taylor step: per stage one projection and
    # one scatter, 4 real flops per (list entry, projector, orbital)
    nl_flops = 4 * 2 * 4 * 4.0 * n_list
    nl_ms = ktot["scatter"] + ktot["project"]
    nl_tf = nl_flops / (nl_ms * 1e-3) / 1e12 if nl_ms > 0 else None
    roof = {"bound": "tensor", "kernel": "k_nl_scatter_tc + k_nl_project_tc (BF16x3 brick GEMMs on tcgen05)",
            "achieved": nl_tf, "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s",
            "frac": (nl_tf / peaks["bf16_tflops_sustained"]) if nl_tf else None,
            "peak_source": f"{peaks['src']} bf16_tflops_sustained",
            "algorithmic_flops_per_step": nl_flops,
            "note": "achieved counts only the algorithmic (list-entry) nonlocal flops, not the six split products "
                    "nor the zeros of the dense brick tiles",
            "traffic": None,
            "kernel_ms_per_step": dict(ktot), "launches_per_step": kcnt}
    # end to end: every domain's orbitals from pinned host memory, one batched
    # step, every domain's orbitals back
    pin_in = [dd.get_orbitals(device=False).pin_memory() for dd in doms]
    pin_out = [torch.empty_like(p).pin_memory() for p in pin_in]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for dd, p in zip(doms, pin_in):
        dd.set_orbitals(p)
    one_step()
    for dd, p in zip(doms, pin_out):
        mlmd.get_orbitals(dd.handle, p)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    mlmd.batch_destroy(b)
    for dd in doms:
        dd.close()
    electrons = float(sum(sp.occ.sum() for sp in specs))
    # nonlocal work of the step, counted on the projector lists: per Taylor
    # stage a projection and a scatter-back of 4 real flops (one complex
    # times real multiply-add) per (list entry, projector, orbital), 4 stages
    return {"workload": (f"c3: {len(specs)} domains N~U{{24..40}}^3, N_o~U{{32..192}}, h=0.35, round(N^3/64) "
                         f"atoms x 4 projectors per domain, complex64, one full-scheme Taylor-4 step of every "
                         f"domain per bench step (one CUDA graph launch)"),
            "value": units * args.c3_steps / (t_ms * 1e-3), "unit": UNIT, "steps": args.c3_steps,
            "ms_per_step": t_ms / args.c3_steps, "units_per_step": units, "electrons": electrons,
            "one_by_one_ms_per_step": seq_ms, "batched_speedup": seq_ms / (t_ms / args.c3_steps),
            "t2s_s_per_electron_step": (t_ms * 1e-3) / (args.c3_steps * electrons),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": units / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": int(units * 8 + len(specs) * 3 * 8),
                    "d2h_bytes_per_step": int(units * 8 + len(specs) * 5 * 8)},
            "gpu_launches": int(launches)}


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2509_00966_gb300 import build
    build.build()
    peaks = _peaks()
    line = run_c2(args, peaks, ws, rank, local)
    if not args.headline_only:
        want_cpu = rank == 0 and ws == 1 and not args.no_cpu_baseline
        line["c1"] = run_c1(args, peaks, want_cpu)
        torch.cuda.empty_cache()
        line["c3"] = run_c3(args, peaks, want_cpu)
        torch.cuda.empty_cache()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# single-kernel and component timings (not the benchmark line)
# ---------------------------------------------------------------------------

def _timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0, e1 = _events()
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def run_stage_case(args):
    """A small case for ncu captures: REPS propagate calls of QD_STEPS Taylor
    steps of workload c1 or c2 (grid, atoms and projectors as configured) on
    N_ORB orbitals; prints the stage kernel's mean launch time."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    cfg, no, qd, reps = args.stage_case[0], int(args.stage_case[1]), int(args.stage_case[2]), int(args.stage_case[3])
    spec = inputs.config(cfg, n_orb=no)
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    d = mlmd.Domain.from_spec(spec, V=V, ortho_every=0)
    d.set_orbitals(_device_orbitals(spec.n_grid, no, spec.dV, spec.seed, torch.complex64))
    A = spec.A[:qd]
    d.propagate(A)
    mlmd.profile_enable(d.handle, True)
    for _ in range(reps):
        d.propagate(A)
    st, n = mlmd.profile_read(d.handle, "stage")
    pr, npj = mlmd.profile_read(d.handle, "project")
    print(json.dumps({"case": f"{cfg} on {no} orbitals", "stage_us_per_launch": 1e3 * st / max(n, 1),
                      "project_us_per_launch": 1e3 * pr / max(npj, 1), "stage_launches": n,
                      "stage_src_sha16": _sha16(STAGE_SRC)}), flush=True)
    d.close()


# Real flops of one h_loc application per complex value (4th-order stencil):
# neighbour sums 20, Laplacian 10, gradients 30, A.grad 10, diagonal 7; and
# of one Taylor term (complex multiply-add) 8.
SWEEP_FLOPS_PER_UNIT = {4: 4 * (77 + 8), 2: 4 * (41 + 8)}
SMS, FP32_LANES = 152, 128


def run_sweep_case(args):
    """The one-sweep local Taylor-4 against the staged form on config CFG's
    grid without projectors: N_ORB orbitals, REPS propagate calls of QD_STEPS
    steps each, timed with CUDA events; orbital-gridpoint-steps per second
    for both and the sweep's FP32 rate against the ALU peak."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    cfg, no, qd, reps = args.sweep_case[0], int(args.sweep_case[1]), int(args.sweep_case[2]), int(args.sweep_case[3])
    spec = inputs.config(cfg, n_orb=no)
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    A = spec.A[:qd]
    out = {"case": f"{cfg} grid {spec.n} x {no} orbitals ({spec.precision}), no projectors, {qd} steps per call"}
    for mode in ("sweep", "staged"):
        os.environ["MLMD_SWEEP"] = "1" if mode == "sweep" else "0"
        d = mlmd.Domain(spec.n, spec.h, no, spec.fd_order, spec.precision, "fp32", "full", spec.dt, 0)
        d.set_potential(V)
        d.set_orbitals(_device_orbitals(spec.n_grid, no, spec.dV, spec.seed,
                                        torch.complex64 if spec.precision == "c64" else torch.complex128))
        d.propagate(A, obs=False)
        mlmd.profile_enable(d.handle, True)
        ms, _ = _timed(lambda: d.propagate(A, obs=False), reps=reps)
        t, c = mlmd.profile_read(d.handle, "stage")
        units = spec.n_grid * no * qd
        out[mode] = {"ms_per_step": ms / qd, "units_per_s": units / (ms * 1e-3),
                     "stage_launches_per_step": c / max(reps * qd, 1), "stage_us_per_launch": 1e3 * t / max(c, 1)}
        d.close()
    os.environ.pop("MLMD_SWEEP", None)
    fl = SWEEP_FLOPS_PER_UNIT[spec.fd_order] * out["sweep"]["units_per_s"]
    out["sweep"]["flops_per_unit"] = SWEEP_FLOPS_PER_UNIT[spec.fd_order]
    out["sweep"]["tflops"] = fl / 1e12
    out["sweep"]["alu_peak_tflops_at_2070mhz"] = SMS * FP32_LANES * 2 * 2070e6 / 1e12
    out["sweep"]["hbm_gbs_at_16B_per_unit"] = 2 * (8 if spec.precision == "c64" else 16) * out["sweep"]["units_per_s"] / 1e9
    out["speedup"] = out["sweep"]["units_per_s"] / out["staged"]["units_per_s"]
    print(json.dumps(out), flush=True)


def run_gauge_case(args):
    """Workload CFG (grid, atoms, projectors) on N_ORB orbitals: propagate
    with observables every step, real projectors against velocity-gauge
    projectors (per-step phases, per-point projection and scatter kernels,
    three moment projections per step for the commutator current)."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    cfg, no, qd, reps = args.gauge_case[0], int(args.gauge_case[1]), int(args.gauge_case[2]), int(args.gauge_case[3])
    spec = inputs.config(cfg, n_orb=no)
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    A = spec.A[:qd]
    out = {"case": f"{cfg} on {no} orbitals, {qd} steps per call with observables"}
    for gauge in ("real", "velocity"):
        d = mlmd.Domain.from_spec(spec, V=V, ortho_every=0)
        d.set_nonlocal_gauge(gauge)
        d.set_orbitals(_device_orbitals(spec.n_grid, no, spec.dV, spec.seed, torch.complex64))
        d.propagate(A)
        ms, obs = _timed(lambda: d.propagate(A), reps=reps)
        units = spec.n_grid * no * qd
        out[gauge] = {"ms_per_step": ms / qd, "units_per_s": units / (ms * 1e-3), "J_last": [float(v) for v in obs[-1, 2:]]}
        d.close()
    out["velocity_over_real_time"] = out["velocity"]["ms_per_step"] / out["real"]["ms_per_step"]
    print(json.dumps(out), flush=True)


def run_nl_case(args):
    """One c3-kind domain (dense projector spheres, tensor-core nonlocal
    path): per-kernel mean launch times of the stage, scatter and projection
    kernels, and the nonlocal algorithmic FLOP rate."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    n, no, qd, reps = (int(v) for v in args.nl_case)
    rng = np.random.Generator(np.random.PCG64(4242))
    h = 0.35
    na = int(round(n ** 3 / 64))
    L = n * h
    sites = rng.uniform(0.0, 1.0, (na, 3)) * L
    spec = inputs.make_domain(n, h, no, 4, "c64", 0.02, qd, seed=4242, geo_seed=4243, wells=sites,
                              well_depth=rng.uniform(0.5, 2.0, na), atoms=sites, n_proj=4,
                              D=rng.uniform(-1.0, 1.0, (na, 4)), A=inputs.envelope_pulse(1000, 0.02)[:qd])
    d = mlmd.Domain.from_spec(spec)
    d.set_orbitals(_device_orbitals(spec.n_grid, no, spec.dV, 5, torch.complex64))
    d.propagate(spec.A)
    n_list = d.projector_list_length()
    mlmd.profile_enable(d.handle, True)
    ms, _ = _timed(lambda: d.propagate(spec.A), reps=reps)
    out = {"case": f"{n}^3 x {no} orbitals, {na} atoms x 4 projectors", "ms_per_propagate": ms}
    tot = 0.0
    for k in ("stage", "scatter", "project"):
        t, c = mlmd.profile_read(d.handle, k)
        out[f"{k}_us_per_launch"] = 1e3 * t / max(c, 1)
        out[f"{k}_launches"] = c
        if k != "stage":
            tot += t
    # algorithmic nonlocal work: per Taylor stage one projection and one
    # scatter of 4 real flops per (list entry, projector, orbital)
    flops = 4 * qd * reps * 2 * n_list * 4 * 4.0 * no
    out["list_entries_per_point"] = n_list / spec.n_grid
    out["nonlocal_tflops_algorithmic"] = flops / (tot * 1e-3) / 1e12 if tot > 0 else None
    print(json.dumps(out), flush=True)
    d.close()


def run_suite(args):
    """Time the workloads outside the benchmark line (c0, c4) through the C ABI."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    lines = []
    spec = inputs.config("c0")
    d = mlmd.Domain.from_spec(spec)
    d.set_orbitals(torch.from_numpy(inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed)).cuda())
    d.propagate(spec.A[:10])
    ms, _ = _timed(lambda: d.propagate(spec.A), reps=3)
    lines.append({"workload": "c0 16^3 x 32 complex128, 100 steps", "ms_per_run": ms,
                  "value": spec.units_per_step * 100 / (ms * 1e-3), "unit": UNIT})
    d.close()
    spec = inputs.config("c4")
    d = mlmd.Domain.from_spec(spec)
    d.set_orbitals(torch.from_numpy(inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV,
                                                           spec.seed).astype(np.complex64)).cuda())
    ms, out = _timed(lambda: d.propagate_adjoint(spec.A, spec.ckpt_every), reps=1)
    lines.append({"workload": "c4 32^3 x 128 complex64, 32x4 projectors, 500 steps forward + adjoint, K=50",
                  "ms_per_run": ms, "value": spec.units_per_step * 500 / (ms * 1e-3), "unit": UNIT,
                  "loss": out[0]})
    d.close()
    for l in lines:
        print(json.dumps(l), flush=True)


def _nprod(mode):
    return {"bf16": 1, "bf16x2": 3, "bf16x3": 6, "fp16": 1, "fp32": 1}[mode]


def run_gram(args):
    """Time mlmd_overlap (Gram S = dV Psi^H Psi) for an N^3 x N_ORB complex64
    domain in the given gemm mode; reports tensor FLOP/s of the real product
    (2 (2 ld)^2 N_g per 16-bit product, upper triangle only)."""
    import torch
    from paper_2509_00966_gb300 import build, mlmd
    build.build()
    n, no, mode = int(args.gram[0]), int(args.gram[1]), args.gram[2]
    h = 0.35
    d = mlmd.Domain((n, n, n), h, no, 4, "c64", gemm_mode=mode)
    d.set_orbitals(_device_orbitals(n ** 3, no, h ** 3, 2, torch.complex64))
    d.overlap()
    mlmd.profile_enable(d.handle, True)
    ms, _ = _timed(lambda: d.overlap(), reps=3)
    gms, gn = mlmd.profile_read(d.handle, "gemm")
    mlmd.profile_enable(d.handle, False)
    dev_ms = gms / max(gn, 1)
    ld = (no + 7) // 8 * 8
    nmt = (2 * ld + 127) // 128
    tri = nmt * (nmt + 1) / 2 / (nmt * nmt)
    flops = 2.0 * (2 * ld) ** 2 * n ** 3 * tri * _nprod(mode)
    peak = _peaks()["bf16_tflops"]
    # ms: the whole API call (S copied to a host array); device_ms: the GEMM on
    # the device (operand split, tensor-core Gram, K-slice reduction)
    print(json.dumps({"kernel": "overlap", "grid": n, "n_orb": no, "mode": mode, "ms": ms,
                      "tensor_tflops": flops / (ms * 1e-3) / 1e12, "peak_bf16_tflops": peak,
                      "frac": flops / (ms * 1e-3) / 1e12 / peak, "device_ms": dev_ms,
                      "device_frac": flops / (dev_ms * 1e-3) / 1e12 / peak}), flush=True)
    d.close()


def run_ks(args):
    """Time mlmd_ks_correction (Eq. 5: C = dV Psi(0)^H Psi(t), then
    Psi(t) - delta Psi(0) C) on an N^3 x N_ORB complex64 domain; reports ms
    per call and the tensor FLOP/s of the two real-embedded GEMMs
    (2 (2 ld)^2 N_g each, times the split mode's products)."""
    import torch
    from paper_2509_00966_gb300 import build, mlmd
    build.build()
    n, no, mode = int(args.ks[0]), int(args.ks[1]), args.ks[2]
    h = 0.35
    d = mlmd.Domain((n, n, n), h, no, 4, "c64", gemm_mode=mode)
    d.set_orbitals(_device_orbitals(n ** 3, no, h ** 3, 2, torch.complex64))
    d.ks_correction(0.01 - 0.005j)
    ms, _ = _timed(lambda: d.ks_correction(0.01 - 0.005j), reps=3)
    ld = (no + 7) // 8 * 8
    flops = 2 * 2.0 * (2 * ld) ** 2 * n ** 3 * _nprod(mode)
    peak = _peaks()["bf16_tflops"]
    print(json.dumps({"kernel": "ks_correction (Eq. 5)", "grid": n, "n_orb": no, "mode": mode, "ms": ms,
                      "tensor_tflops": flops / (ms * 1e-3) / 1e12, "peak_bf16_tflops": peak,
                      "frac": flops / (ms * 1e-3) / 1e12 / peak}), flush=True)
    d.close()


def run_occ(args):
    """Time mlmd_occupations (C = dV Psi(0)^H Psi(t) as one real-embedded
    GEMM of 2 (2 ld)^2 N_g flops times the split mode's products, then the
    FP64 occupation sums on the device) on an N^3 x N_ORB complex64 domain."""
    import torch
    from paper_2509_00966_gb300 import build, mlmd
    build.build()
    n, no, mode = int(args.occ[0]), int(args.occ[1]), args.occ[2]
    h = 0.35
    d = mlmd.Domain((n, n, n), h, no, 4, "c64", gemm_mode=mode)
    d.set_occupations(np.full(no, 2.0))
    d.set_orbitals(_device_orbitals(n ** 3, no, h ** 3, 2, torch.complex64))
    d.reorthonormalize("chol")
    d.set_orbitals(d.get_orbitals())             # orthonormal reference Psi(0)
    d.ks_correction(0.01 - 0.005j)               # Psi(t) = (1 - delta) Psi(0): n_exc = 2 N_o (1 - |1 - delta|^2)
    d.occupations()
    ms, (fs, nx) = _timed(lambda: d.occupations(), reps=5)
    ld = (no + 7) // 8 * 8
    flops = 2.0 * (2 * ld) ** 2 * n ** 3 * _nprod(mode)
    peak = _peaks()["bf16_tflops"]
    print(json.dumps({"kernel": "occupations (overlap GEMM + FP64 sums)", "grid": n, "n_orb": no, "mode": mode,
                      "ms": ms, "tensor_tflops": flops / (ms * 1e-3) / 1e12, "peak_bf16_tflops": peak,
                      "frac": flops / (ms * 1e-3) / 1e12 / peak, "n_exc": nx}), flush=True)
    d.close()


def run_reorth(args):
    """Time mlmd_reorthonormalize (FP64 Cholesky on the device, Gram and
    update GEMMs in the given gemm mode) on an N^3 x N_ORB complex64 domain
    of seeded random orbitals; reports ms per call and max |S - I| after."""
    import torch
    from paper_2509_00966_gb300 import build, mlmd
    build.build()
    n, no, mode = int(args.reorth[0]), int(args.reorth[1]), args.reorth[2]
    h = 0.35
    d = mlmd.Domain((n, n, n), h, no, 4, "c64", gemm_mode=mode)
    d.set_orbitals(_device_orbitals(n ** 3, no, h ** 3, 2, torch.complex64))
    d.reorthonormalize("chol")
    ms, _ = _timed(lambda: d.reorthonormalize("chol"), reps=3)
    S = d.overlap()
    print(json.dumps({"kernel": "reorthonormalize(chol)", "grid": n, "n_orb": no, "mode": mode, "ms": ms,
                      "max_abs_S_minus_I": float(np.abs(S - np.eye(no)).max())}), flush=True)
    d.close()


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.gram:
        run_gram(args)
    elif args.reorth:
        run_reorth(args)
    elif args.ks:
        run_ks(args)
    elif args.occ:
        run_occ(args)
    elif args.suite:
        run_suite(args)
    elif args.stage_case:
        run_stage_case(args)
    elif args.sweep_case:
        run_sweep_case(args)
    elif args.gauge_case:
        run_gauge_case(args)
    elif args.nl_case:
        run_nl_case(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
