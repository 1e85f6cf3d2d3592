#!/usr/bin/env python
"""Benchmark of the LFD propagation hot path on one GB300 (or N replicas).

Workload (the c1 domain): 48^3 periodic grid, h = 0.35 bohr, 256 complex64
Kohn-Sham orbitals, 4th-order finite differences, 64 Gaussian wells on a
perturbed 4x4x4 lattice, 64 atoms x 4 projectors (r_c = 1.2, r_cut = 3),
Gaussian-envelope vector potential, f_n = 2.  One benchmark step is one
mlmd_propagate call of 1000 full-scheme Taylor-4 steps with per-step
observables (electron count, energy, current), plus the density/current
fields of the final state.  Metric: orbital*gridpoint*steps per second
(units = N_o * N_g * Taylor steps); also seconds per (electron * step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
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
# algorithmic HBM bytes per orbital*gridpoint*step of the four staged
# full-scheme passes in complex64: the first reads psi and writes w (16 B),
# the other three read w and psi and write w or psi (24 B each)
STAGE_BYTES_PER_UNIT = 16 + 3 * 24
# DRAM bytes (read + write) per stage launch on this workload, the mean over
# the four stage launches of one Taylor step (490 + 759 + 759 + 724 MB), from
# one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum of the
# current stage kernel in the tile shape the autotuner picks (128-byte
# orbital chunks, 4 threads per point); the command is in
# profiles/k_stage_tma_c1.md.  The algorithmic mean is 88 / 4 B x N_g N_o =
# 622.9 MB: the 1.10x are the z halo planes and the scatter entry blocks.
STAGE_TRAFFIC_BYTES_PER_LAUNCH = 683.1e6


def _is_bench_workload(spec):
    """The traffic figure was measured on the 48^3 x 256 domain with 64 x 4
    projectors; other sizes report none."""
    return spec.n == (48, 48, 48) and spec.n_orb == 256 and spec.n_proj == 4 and len(spec.atoms) == 64


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--qd-steps", type=int, default=1000, help="Taylor steps per benchmark step")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
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
                   help="also time the other workloads (c0, c2, c3, c4), one JSON line each")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


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


def _workload(qd_steps):
    from paper_2509_00966_gb300 import inputs
    spec = inputs.config("c1")
    A = inputs.envelope_pulse(1000, spec.dt)
    reps = (qd_steps + 999) // 1000
    spec.A = np.tile(A, (reps, 1))[:qd_steps]
    spec.n_steps = qd_steps
    V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
    psi = inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed)
    return spec, V, psi


def _workload_name(spec, qd):
    return (f"c1: {spec.n[0]}^3 grid h={spec.h} bohr, {spec.n_orb} complex64 orbitals, {spec.fd_order}th-order FD, "
            f"{len(spec.atoms)} atoms x {spec.n_proj} projectors, Gaussian-envelope A(t), {qd} full-scheme "
            f"Taylor-4 steps + per-step norm/energy/current per bench step")


def oracle_sample(spec, V, psi, target_s, max_steps=20):
    """Time the FP64 oracle (as it stands) on the benchmark workload: all
    orbitals, the full grid, a few Taylor steps with observables."""
    import oracle
    od = oracle.Domain(spec.n, spec.h, spec.n_orb, spec.fd_order, V, spec.atoms, spec.n_proj, spec.r_c, spec.r_cut,
                       spec.D)
    f = np.full(spec.n_orb, 2.0)
    p = psi.astype(np.complex128)
    t0 = time.perf_counter()
    p, _ = oracle.propagate(od, p, spec.A[:1], spec.dt, f)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(max_steps, round(target_s / max(t1, 1e-3)) - 1)))
    t0 = time.perf_counter()
    p, _ = oracle.propagate(od, p, spec.A[1:1 + n], spec.dt, f)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    units = spec.n_grid * spec.n_orb * n
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} Taylor-4 steps (+observables) of the full workload, all {spec.n_orb} orbitals, "
                      f"FP64 C/OpenMP oracle, {dt:.1f} s"}


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


def run_reference(args):
    """The oracle as the reference arm: each step is one Taylor step of the
    same workload on the host cores (rank 0 only)."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    spec, V, psi = _workload(max(args.steps + args.warmup, 1))
    od = oracle.Domain(spec.n, spec.h, spec.n_orb, spec.fd_order, V, spec.atoms, spec.n_proj, spec.r_c, spec.r_cut,
                       spec.D)
    f = np.full(spec.n_orb, 2.0)
    p = psi.astype(np.complex128)
    for k in range(args.warmup):
        p, _ = oracle.propagate(od, p, spec.A[k:k + 1], spec.dt, f)
    t0 = time.perf_counter()
    for k in range(args.steps):
        p, _ = oracle.propagate(od, p, spec.A[k:k + 1], spec.dt, f)
    dt = time.perf_counter() - t0
    units = spec.n_grid * spec.n_orb * args.steps
    v = units / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded PbTiO3-like domain)",
            "config": {"workload": _workload_name(spec, 1), "reference_step": "1 Taylor-4 step with observables",
                       "parallelism": "host cores (OpenMP)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} Taylor steps of the full workload, FP64 C/OpenMP oracle"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2509_00966_gb300 import build, mlmd
    build.build()
    spec, V, psi = _workload(args.qd_steps)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(spec, V, psi, args.cpu_seconds)

    dom = mlmd.Domain.from_spec(spec, V=V)
    psi_dev = torch.from_numpy(psi).to(torch.complex64).cuda()
    dom.set_orbitals(psi_dev)
    A = spec.A
    A_last = A[-1]

    def one_step():
        obs = dom.propagate(A, obs=True)
        dom.density_current(A_last)
        return obs

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(_physical_gpu(local))
    clocks.start()
    time.sleep(0.3)
    mlmd.profile_enable(dom.handle, True)
    l0 = dom.launches
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        obs = one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = dom.launches - l0
    st_ms, st_n = mlmd.profile_read(dom.handle, "stage")
    pr_ms, pr_n = mlmd.profile_read(dom.handle, "project")
    mlmd.profile_enable(dom.handle, False)
    ck = clocks.stop()
    t_ms = _max_over_ranks(t_ms, ws)
    if ws > 1:
        torch.distributed.barrier()

    # end to end through the C ABI with host buffers: h2d of the orbitals,
    # the propagation, d2h of the orbitals and observables, every step
    pinned_in = torch.from_numpy(psi.astype(np.complex64)).pin_memory()
    pinned_out = torch.empty_like(pinned_in).pin_memory()
    e2e_t = []
    for k in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dom.set_orbitals(pinned_in)
        dom.propagate(A, obs=True)
        mlmd.get_orbitals(dom.handle, pinned_out)
        torch.cuda.synchronize()
        if k > 0:
            e2e_t.append(time.perf_counter() - t0)
    e2e_s = float(np.mean(e2e_t)) if e2e_t else float("nan")
    e2e_s = _max_over_ranks(e2e_s, ws)

    units_step = spec.n_grid * spec.n_orb * args.qd_steps
    value = _job_value(ws, units_step * args.steps, t_ms * 1e-3)
    electrons = float(np.sum(spec.occ))
    t2s = (t_ms * 1e-3) / (args.steps * args.qd_steps * electrons)
    peak, peak_src = _peaks()
    stage_units = st_n / 4 * spec.n_grid * spec.n_orb   # four stage launches per Taylor step
    achieved = STAGE_BYTES_PER_UNIT * stage_units / (st_ms * 1e-3) / 1e9 if st_ms > 0 else None
    dom.close()
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded PbTiO3-like domain, random orthonormal orbitals)",
        "config": {"workload": _workload_name(spec, args.qd_steps), "n_grid": spec.n_grid, "n_orb": spec.n_orb,
                   "qd_steps_per_step": args.qd_steps, "scheme": "full (v_nl inside Taylor-4)",
                   "l2": "inputs larger than L2 (psi 226 MB + two work states > 129 MB), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "t2s_s_per_electron_step": t2s,
        "t2s_paper_context": "1.11e-7 s/(electron*step) on 120,000 PVC tiles (paper, other hardware; context only)",
        "roofline": {"bound": "hbm", "kernel": "k_stage (fused stencil + V + A + scatter + Taylor combine)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": (achieved / peak) if achieved else None, "peak_source": f"{peak_src} hbm_gbs",
                     "bytes_per_unit_step": STAGE_BYTES_PER_UNIT,
                     "traffic": STAGE_TRAFFIC_BYTES_PER_LAUNCH if _is_bench_workload(spec) else None,
                     "traffic_unit": "bytes per stage launch (ncu, mean of the four stage launches of a step)",
                     "kernel_share": {"stage": st_ms / t_ms, "project": pr_ms / t_ms},
                     "launches": {"stage": st_n, "project": pr_n}},
        "cpu_baseline": cpu,
        "e2e": {"value": _job_value(ws, units_step, e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": int(psi.size * 8 + A.size * 8),
                "d2h_bytes_per_step": int(psi.size * 8 + args.qd_steps * 5 * 8)},
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def _timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


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


def run_suite(args):
    """Time each of the other workloads through the C ABI (kernel time from the
    library's CUDA-event hooks); one JSON line per workload."""
    import torch
    from paper_2509_00966_gb300 import build, inputs, mlmd
    build.build()
    torch.cuda.set_device(0)
    peak, src = _peaks()
    lines = []

    def stage_report(d, units_per_step, bytes_per_unit):
        st, n = mlmd.profile_read(d.handle, "stage")
        pr, npj = mlmd.profile_read(d.handle, "project")
        ach = bytes_per_unit * units_per_step * (n / 4) / (st * 1e-3) / 1e9 if st > 0 else None
        return {"stage_ms_per_launch": st / max(n, 1), "project_ms_total": pr, "stage_achieved_gbs": ach,
                "stage_frac_of_measured_hbm": ach / peak if ach else None}

    # c0: complex128, local only, 100 steps
    spec = inputs.config("c0")
    d = mlmd.Domain.from_spec(spec)
    d.set_orbitals(torch.from_numpy(inputs.random_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed)).cuda())
    d.propagate(spec.A[:10])
    mlmd.profile_enable(d.handle, True)
    ms, _ = _timed(lambda: d.propagate(spec.A), reps=3)
    r = stage_report(d, spec.units_per_step, 16 * 11)
    lines.append({"workload": "c0 16^3 x 32 complex128, 100 steps", "ms_per_run": ms,
                  "value": spec.units_per_step * 100 / (ms * 1e-3), "unit": UNIT, **r})
    d.close()

    # c2: 64^3 x 1024 complex64, 128 x 8 projectors, Cholesky every 10 steps, BF16X3 Gram
    spec = inputs.config("c2", n_steps=20)
    for mode in ["bf16x3", "fp32"]:
        V = inputs.gaussian_wells(spec.n, spec.h, spec.wells, spec.well_depth, spec.well_width)
        d = mlmd.Domain.from_spec(spec, V=V, gemm_mode=mode)
        d.set_orbitals(_device_orbitals(spec.n_grid, spec.n_orb, spec.dV, spec.seed, torch.complex64))
        d.reorthonormalize("chol")
        d.propagate(spec.A[:2])
        mlmd.profile_enable(d.handle, True)
        ms, obs = _timed(lambda: d.propagate(spec.A), reps=1)
        r = stage_report(d, spec.units_per_step, 88)
        g_ms, _ = _timed(lambda: d.overlap(), reps=2)
        lines.append({"workload": f"c2 64^3 x 1024 complex64, 128x8 projectors, 20 steps incl. 2 Cholesky "
                                  f"re-orthonormalisations, gemm_mode={mode}", "ms_per_run": ms,
                      "value": spec.units_per_step * 20 / (ms * 1e-3), "unit": UNIT, "overlap_ms": g_ms,
                      "overlap_tflops_complex_equiv": 8.0 * spec.n_orb ** 2 * spec.n_grid / (g_ms * 1e-3) / 1e12,
                      **r})
        d.close()

    # c3: 216 uneven domains in one batch, per-step CUDA graph
    specs = inputs.batched_specs(n_steps=20)
    doms = []
    for i, sp in enumerate(specs):
        dd = mlmd.Domain.from_spec(sp)
        dd.set_orbitals(_device_orbitals(sp.n_grid, sp.n_orb, sp.dV, 1000 + i, torch.complex64))
        doms.append(dd)
    b = mlmd.batch_create([dd.handle for dd in doms])
    A = np.stack([sp.A for sp in specs])
    mlmd.batch_propagate(b, A[:, :2], first_handle=doms[0].handle)
    ms, _ = _timed(lambda: mlmd.batch_propagate(b, A, first_handle=doms[0].handle), reps=1)
    units = sum(sp.units_per_step for sp in specs)

    def one_by_one():
        for dd, sp in zip(doms, specs):
            dd.propagate(sp.A, obs=True)
    one_by_one()
    ms_seq, _ = _timed(one_by_one, reps=1)
    lines.append({"workload": f"c3 {len(specs)} domains N~U{{24..40}}^3, N_o~U{{32..192}}, 20 steps, batched graph",
                  "ms_per_run": ms, "value": units * 20 / (ms * 1e-3), "unit": UNIT,
                  "electrons": float(sum(sp.occ.sum() for sp in specs)),
                  "one_by_one_ms": ms_seq, "one_by_one_value": units * 20 / (ms_seq * 1e-3),
                  "batched_speedup": ms_seq / ms})
    mlmd.batch_destroy(b)
    for dd in doms:
        dd.close()

    # c4: 32^3 x 128 complex64, 500-step forward + checkpointed adjoint (K = 50)
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
        l["peak_hbm_gbs"] = peak
        l["peak_source"] = src
        print(json.dumps(l), flush=True)


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
    ms, _ = _timed(lambda: d.overlap(), reps=3)
    ld = (no + 7) // 8 * 8
    nmt = (2 * ld + 127) // 128
    tri = nmt * (nmt + 1) / 2 / (nmt * nmt)
    nprod = {"bf16": 1, "bf16x2": 3, "bf16x3": 6, "fp16": 1, "fp32": 1}[mode]
    flops = 2.0 * (2 * ld) ** 2 * n ** 3 * tri * nprod
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        peak = 1900.0
    print(json.dumps({"kernel": "overlap", "grid": n, "n_orb": no, "mode": mode, "ms": ms,
                      "tensor_tflops": flops / (ms * 1e-3) / 1e12, "peak_bf16_tflops": peak,
                      "frac": flops / (ms * 1e-3) / 1e12 / peak}), flush=True)
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
    nprod = {"bf16": 1, "bf16x2": 3, "bf16x3": 6, "fp16": 1, "fp32": 1}[mode]
    flops = 2 * 2.0 * (2 * ld) ** 2 * n ** 3 * nprod
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        peak = 1900.0
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
    nprod = {"bf16": 1, "bf16x2": 3, "bf16x3": 6, "fp16": 1, "fp32": 1}[mode]
    flops = 2.0 * (2 * ld) ** 2 * n ** 3 * nprod
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        peak = 1900.0
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
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
