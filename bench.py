#!/usr/bin/env python3
"""Throughput of Pauli-rotation time evolution on one GB300 (or N replicas).

Workload (the n = 30 qDRIFT configuration): a synthetic Jordan-Wigner-like
Hamiltonian with 10^4 terms on 30 qubits (one-norm 7.5), qDRIFT with
N = 10^5 samples at t = 1, applied to a complex64 state that starts as an
8-determinant superposition.  The run is split into 10 segments of 10^4
rotations; one benchmark step applies one segment and reads the overlap
<psi0|psi> (FP64) back to the host, so 10 timed steps are one complete
qDRIFT run.  Every state is 8 GiB, far larger than the 129 MB L2, so no L2
flush is needed between steps.

Reported beside the headline (complex64, fused windows): the FP64
(complex128) path on a 1000-rotation prefix of the same stream and its
distance to the complex64 result; the CPU oracle on a bounded prefix.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pauli rotations/sec and HBM GB/s at n=30, complex64 fused vs FP64 at stated error"
UNIT = "rotations/s"
N_QUBITS = 30
N_TERMS = 10_000
HAM_SEED = 3
N_SAMPLES = 100_000
T_TOTAL = 1.0
QDRIFT_SEED = 4
PSI0_SEED = 11
SEGMENTS = 10
SEG_LEN = N_SAMPLES // SEGMENTS
FP64_PREFIX = SEG_LEN
CPU_ROTATIONS_1T = 2      # oracle sample, one thread
CPU_ROTATIONS_MT = 8      # oracle sample, all host cores
REF_ROTATIONS_PER_STEP = 4
FALLBACK_HBM_GBS = 6800.0
BATCH_RUNS = 512
BATCH_SEED = 5
LEARNED_TIMES = (0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0)  # the n = 32 step-choice queries


def workload_name():
    return (f"qdrift n={N_QUBITS} complex64: JW-like H with {N_TERMS} terms (lambda 7.5), "
            f"N={N_SAMPLES} samples at t={T_TOTAL}, {SEGMENTS} segments of {SEG_LEN} rotations "
            f"+ FP64 overlap per step, 8-determinant initial state")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=SEGMENTS)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-rotations", type=int, default=SEG_LEN,
                    help="rotations of the stream run in complex128 and complex64 for the error report "
                         "(default one segment; 100000 for the whole run)")
    ap.add_argument("--workload", choices=["qdrift30", "batched", "learned", "trotter26", "kernels"], default="qdrift30",
                    help="batched: 512 independent qDRIFT / partially randomised runs, n 14..22, in one "
                         "persistent launch (reported on its own JSON line)")
    ap.add_argument("--batch-runs", type=int, default=BATCH_RUNS)
    ap.add_argument("--no-sequential", action="store_true", help="batched: skip the one-run-at-a-time comparison")
    ap.add_argument("--no-autotune", action="store_true", help="batched: default lane size and tile bits")
    ap.add_argument("--no-c128", action="store_true", help="batched: skip the complex128 comparison batch")
    ap.add_argument("--batch-n", type=int, default=None, help="batched: every run at this n (default 14..22)")
    ap.add_argument("--batch-rotations", type=int, default=None,
                    help="batched: every run with this many rotations (default 2000..20000)")
    ap.add_argument("--train-problems", type=int, default=128, help="learned: training Hamiltonians")
    ap.add_argument("--train-times", type=int, choices=[8, 16], default=8,
                    help="learned: times per Hamiltonian (8: every second of the 16 of the configuration)")
    ap.add_argument("--train-nmax", type=int, default=18, help="learned: largest n of the training Hamiltonians")
    ap.add_argument("--use-qubits", type=int, default=32, help="learned: qubits of the step-choice queries")
    ap.add_argument("--qubits", type=int, default=30,
                    help="state size; values other than 30 are for profiling captures only")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------ peaks, clocks

def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.splitlines():
            f = [p.strip() for p in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def tile_kernel_sha256():
    """Hash of the tile kernel's device sources (the pass body and its launch)."""
    h = hashlib.sha256()
    for f in ("ps_device.cuh", "ps_tile.cuh", "ps_tile.cu"):
        h.update(open(os.path.join(ROOT, "paper_2504_17881_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic():
    """Per-launch DRAM bytes of the tile kernel from the committed ncu summary, if the
    kernel source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_tile_c64_n30.txt")
    try:
        text = open(path).read()
        sha = tile_kernel_sha256()
    except OSError:
        return None
    fields = dict(ln.split(":", 1) for ln in text.splitlines() if ":" in ln and not ln.startswith(" "))
    if fields.get("kernel_source_sha256", "").strip() != sha:
        return None
    try:
        return float(fields["traffic_bytes_per_launch_full"].strip())
    except (KeyError, ValueError):
        return None


# --------------------------------------------------------------- workload

def aggregate_ranks(dist, device, elapsed_ms: float, units: int, launches: int):
    """Whole-job numbers of a replica run: the slowest rank's time, and the
    units and kernel launches summed over ranks (identity without dist)."""
    if dist is None:
        return elapsed_ms, units, launches
    import torch
    tt = torch.tensor([elapsed_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    tr = torch.tensor([units, launches], device=device, dtype=torch.float64)
    dist.all_reduce(tr)
    return float(tt.item()), int(tr[0].item()), int(tr[1].item())


def make_workload(rank: int):
    inputs = load_inputs()
    x, z, h = inputs.jw_hamiltonian(N_QUBITS, N_TERMS, seed=HAM_SEED)
    idx, amp = inputs.determinant_state(N_QUBITS, seed=PSI0_SEED)
    return x, z, h, idx, amp, QDRIFT_SEED + rank


def load_inputs():
    """The seeded input generators, loaded by file path: the oracle legs must
    not import the package (its __init__ opens libps)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_ps_inputs", os.path.join(ROOT, "paper_2504_17881_gb300", "inputs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


class OracleRun:
    """The oracle (complex128 scatter form) walking the benchmark's qDRIFT
    stream from the 8-determinant state, with its own sampler."""

    def __init__(self, total_rotations: int):
        import oracle
        inputs = load_inputs()
        self.oracle = oracle
        x, z, h = inputs.jw_hamiltonian(N_QUBITS, N_TERMS, seed=HAM_SEED)
        idx = oracle.qdrift_indices(h, QDRIFT_SEED, 0, total_rotations).astype(np.int64)
        lam = 0.0
        for v in h:
            lam += abs(float(v))
        tau = lam * T_TOTAL / N_SAMPLES
        self.xs, self.zs = x[idx], z[idx]
        self.ph = np.where(h[idx] > 0, tau, -tau)
        self.sidx, self.samp = inputs.determinant_state(N_QUBITS, seed=PSI0_SEED)
        self.psi0 = np.zeros(1 << N_QUBITS, dtype=np.complex128)
        self.psi0[self.sidx.astype(np.int64)] = self.samp
        self.psi = self.psi0.copy()
        self.tmp = np.empty_like(self.psi)
        self.tmp.fill(0)  # touch every page before any timing

    def reset(self):
        np.copyto(self.psi, self.psi0)

    def apply(self, first: int, count: int, threads: int) -> float:
        """Rotations [first, first + count) on the current state; seconds taken."""
        self.oracle.set_threads(threads)
        try:
            t0 = time.perf_counter()
            self.oracle.apply_inplace(self.psi, self.tmp, self.xs[first:first + count],
                                      self.zs[first:first + count], self.ph[first:first + count])
            return time.perf_counter() - t0
        finally:
            self.oracle.set_threads(1)

    def overlap(self, threads: int) -> complex:
        self.oracle.set_threads(threads)
        try:
            return self.oracle.overlap(self.psi0, self.psi)
        finally:
            self.oracle.set_threads(1)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def cpu_baseline_leg():
    """The oracle as it stands on this host: the first rotations of the same
    stream at n = 30, once on one thread and once on every host core."""
    cores = host_cores()
    try:
        import oracle
        run = OracleRun(max(CPU_ROTATIONS_1T, CPU_ROTATIONS_MT))
        dt1 = run.apply(0, CPU_ROTATIONS_1T, 1)
        run.reset()
        dtm = run.apply(0, CPU_ROTATIONS_MT, cores)
        threads = cores if oracle.has_openmp() else 1
        del run
    except Exception as e:  # noqa: BLE001
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(e)}
    return {"value": CPU_ROTATIONS_MT / dtm, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {CPU_ROTATIONS_MT} rotations of the same qDRIFT stream at n={N_QUBITS} "
                      f"(complex128 scatter-form oracle, OpenMP over {threads} threads, {dtm:.1f} s)",
            "single_thread": {"value": CPU_ROTATIONS_1T / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"first {CPU_ROTATIONS_1T} rotations, 1 thread ({dt1:.1f} s)"},
            "host_cores_available": cores}


# ------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import paper_2504_17881_gb300 as ps

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    x, z, h, idx, amp, seed = make_workload(rank)
    H = ps.Hamiltonian(N_QUBITS, x, z, h)
    segs = [H.qdrift_stream(T_TOTAL, N_SAMPLES, seed, first=s * SEG_LEN, count=SEG_LEN) for s in range(SEGMENTS)]
    plans = [ps.Plan(N_QUBITS, ps.PS_C64, *sg) for sg in segs]
    rot_per_pass = sum(p.info["rotations"] for p in plans) / sum(p.info["windows"] for p in plans)

    def init_state(t):
        t.zero_()
        t[torch.as_tensor(idx.astype(np.int64), device=dev)] = torch.as_tensor(amp, device=dev).to(t.dtype)

    psi0 = ps.StateVector(N_QUBITS, dtype=torch.complex64, device=dev)
    init_state(psi0.tensor)
    psi = ps.StateVector(N_QUBITS, dtype=torch.complex64, device=dev)
    psi.set_tuning(kernel_timing=1)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    psi.copy_from(psi0)
    for s in range(args.warmup):
        psi.apply_plan(plans[s % SEGMENTS])
        psi.overlap(psi0)
    psi.copy_from(psi0)
    torch.cuda.synchronize(dev)
    ps.ps_reset_stats(psi.handle)

    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    overlaps = []
    for s in range(args.steps):
        psi.apply_plan(plans[s % SEGMENTS])
        overlaps.append(psi.overlap(psi0))
    ev1.record(stream)
    barrier()
    clock_info = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    stats = psi.stats()
    rotations = args.steps * SEG_LEN

    t_max, tot_rot, launches = aggregate_ranks(dist, dev, elapsed_ms, rotations, sum(stats["launches"].values()))
    value = tot_rot / (t_max / 1e3)

    # roofline of the dominant kernel (fused tile kernel), timed live with events
    tile_ms = stats["kernel_ms"]["tile"]
    tile_n = max(stats["launches"]["tile"], 1)
    bytes_per_launch = 2.0 * 8.0 * (1 << N_QUBITS)
    achieved = bytes_per_launch / (tile_ms / tile_n / 1e3) / 1e9 if tile_ms > 0 else None
    peak, peak_kind = hbm_peak()
    roofline = {"bound": "hbm", "kernel": "k_tile<float,3,4>", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": kernel_traffic(),
                "peak_source": f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": bytes_per_launch,
                "avg_launch_ms": tile_ms / tile_n}
    step_gbs = stats["bytes"]["tile"] + stats["bytes"]["pair"] + stats["bytes"]["reduce"]
    step_gbs = step_gbs / (elapsed_ms / 1e3) / 1e9

    # ------------------------------------------------------------- FP64 path
    fp64 = None
    if not args.no_fp64:
        nrot = max(1, min(args.fp64_rotations, N_SAMPLES))
        nseg = (nrot + SEG_LEN - 1) // SEG_LEN
        parts = []
        for sidx in range(nseg):
            cnt = min(SEG_LEN, nrot - sidx * SEG_LEN)
            sg = segs[sidx] if sidx < len(segs) else H.qdrift_stream(T_TOTAL, N_SAMPLES, seed, first=sidx * SEG_LEN,
                                                                     count=SEG_LEN)
            parts.append((sg[0][:cnt], sg[1][:cnt], sg[2][:cnt]))
        plans64 = [ps.Plan(N_QUBITS, ps.PS_C128, *pt) for pt in parts]
        plans32 = [ps.Plan(N_QUBITS, ps.PS_C64, *pt) for pt in parts]
        p64 = ps.StateVector(N_QUBITS, dtype=torch.complex128, device=dev)
        p64_0 = ps.StateVector(N_QUBITS, dtype=torch.complex128, device=dev)
        init_state(p64.tensor)
        init_state(p64_0.tensor)
        p64.set_tuning(kernel_timing=1)
        p64.apply_plan(plans64[0])  # warm-up on a throwaway state
        init_state(p64.tensor)
        torch.cuda.synchronize(dev)
        ps.ps_reset_stats(p64.handle)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for pl in plans64:
            p64.apply_plan(pl)
        g64 = p64.overlap(p64_0)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1)
        st64 = p64.stats()
        # complex64 on the same rotations, compared with the FP64 state
        psi.copy_from(psi0)
        for pl in plans32:
            psi.apply_plan(pl)
        g32 = psi.overlap(psi0)
        diff = torch.linalg.vector_norm(psi.tensor.to(torch.complex128) * psi.scale() - p64.tensor * p64.scale()).item()
        ref = torch.linalg.vector_norm(p64.tensor * p64.scale()).item()
        tile64 = st64["kernel_ms"]["tile"] / max(st64["launches"]["tile"], 1)
        # ALU roofline of the complex128 pass: two FP64 FMAs (4 flops) per amplitude and
        # rotation (the stored-scale FMA pair is applied on a few passes only and not counted)
        rpp64 = sum(pl.info["rotations"] for pl in plans64) / max(1, sum(pl.info["windows"] for pl in plans64))
        fma_peak = ps.ps_measure_fma_rate(ps.PS_C128)
        flops_pass = 4.0 * rpp64 * (1 << N_QUBITS)
        ach_tf = flops_pass / (tile64 / 1e3) / 1e12 if tile64 > 0 else None
        fp64_roof = {"bound": "alu", "kernel": "k_tile<double,3,2>", "achieved": ach_tf, "peak": fma_peak,
                     "unit": "TFLOP/s", "frac": ach_tf / fma_peak if ach_tf else None,
                     "peak_source": "measured FP64 FMA throughput (ps_measure_fma_rate, this run)",
                     "flops_per_launch": flops_pass}
        fp64 = {"value": nrot / (ms64 / 1e3), "unit": UNIT, "dtype": "f64", "rotations": nrot, "roofline": fp64_roof,
                "rot_per_pass": rpp64,
                "tile_avg_launch_ms": tile64,
                "tile_achieved_gbs": 2.0 * 16.0 * (1 << N_QUBITS) / (tile64 / 1e3) / 1e9 if tile64 > 0 else None,
                "bound": "alu (FP64 pipe)",
                "c64_vs_fp64": {"state_rel_l2": diff / ref, "overlap_abs": abs(g32 - g64),
                                "overlap_rel": abs(g32 - g64) / abs(g64), "overlap_fp64": [g64.real, g64.imag],
                                "after_rotations": nrot}}
        del p64, p64_0, plans64, plans32
        torch.cuda.empty_cache()

    # ------------------------------------------------------------- end to end
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(ps, torch, dev, segs, idx, amp, args.steps)

    if dist is not None:
        dist.barrier()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(), "n": N_QUBITS, "terms": N_TERMS, "samples": N_SAMPLES,
                   "rotations_per_step": SEG_LEN, "state": "complex64 (FP64 trig, norm and overlap)",
                   "l2": "inputs larger than L2 (8 GiB state vs 129 MB L2), no flush",
                   "parallelism": f"replicas x{world} (independent qDRIFT seeds)"},
        "hbm_gbs": step_gbs, "rot_per_pass": rot_per_pass, "overlap_final": [overlaps[-1].real, overlaps[-1].imag],
        "roofline": roofline, "fp64": fp64, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_e2e(ps, torch, dev, segs, idx, amp, steps):
    """Same metric through the public API from host buffers: the initial state
    is uploaded from pinned host memory, each step passes the segment's
    rotations as host arrays (scheduling and upload inside the library) and
    reads the overlap back."""
    nbytes = 8 << N_QUBITS
    host0 = torch.zeros(1 << N_QUBITS, dtype=torch.complex64).pin_memory()
    host0[torch.as_tensor(idx.astype(np.int64))] = torch.as_tensor(amp).to(torch.complex64)
    psi = ps.StateVector(N_QUBITS, dtype=torch.complex64, device=dev)
    psi0 = ps.StateVector(N_QUBITS, dtype=torch.complex64, device=dev)
    h2d = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ps.ps_set_state(psi0.handle, host0.data_ptr())
    ps.ps_set_state(psi.handle, host0.data_ptr())
    h2d += 2 * nbytes
    for s in range(steps):
        xs, zs, ph = segs[s % SEGMENTS]
        psi.apply_rotations(xs, zs, ph)
        h2d += xs.nbytes + zs.nbytes + ph.nbytes
        psi.overlap(psi0)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    del psi, psi0
    torch.cuda.empty_cache()
    return {"value": steps * SEG_LEN / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": 16, "note": "wall clock; includes 2 x 8 GiB state upload, host scheduling, "
                                              "per-step rotation upload and overlap readback"}


# ---------------------------------------------------------------- batched

def batched_workload(nruns: int, seed: int = BATCH_SEED, n_fixed: int | None = None, rot_fixed: int | None = None):
    """Independent runs of uneven size: n uniform in 14..22, 200-2000 JW-like
    terms per Hamiltonian, 2000-20000 rotations; even runs qDRIFT, odd runs
    partially randomised (L_D = 10% of the terms, r = 4 steps).  n_fixed /
    rot_fixed give every run that n / rotation count (profiling workloads)."""
    import paper_2504_17881_gb300 as ps
    from paper_2504_17881_gb300 import inputs
    rng = np.random.default_rng(seed)
    runs = []
    for i in range(nruns):
        n = int(rng.integers(14, 23))
        L = int(rng.integers(200, 2001))
        cnt = int(rng.integers(2000, 20001))
        n = n_fixed if n_fixed else n
        cnt = rot_fixed if rot_fixed else cnt
        x, z, h = inputs.jw_hamiltonian(n, L, seed=seed * 100000 + i)
        H = ps.Hamiltonian(n, x, z, h)
        if i % 2 == 0:
            xs, zs, ph = H.qdrift_stream(T_TOTAL, cnt, seed * 100000 + i)
            kind = "qdrift"
        else:
            LD = max(1, L // 10)
            xs, zs, ph = H.partial_stream(LD, T_TOTAL, 4, max(1, cnt // 4 - LD), seed * 100000 + i)
            kind = "partial"
        H.close()
        runs.append(dict(n=n, x=xs, z=zs, phi=ph, kind=kind, det_seed=seed * 100000 + i))
    return runs


def run_batched(args):
    import torch
    import paper_2504_17881_gb300 as ps
    from paper_2504_17881_gb300 import autotune, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    t_host = time.perf_counter()
    runs = batched_workload(args.batch_runs, BATCH_SEED + 1000 * rank, args.batch_n, args.batch_rotations)
    host_gen_s = time.perf_counter() - t_host

    def psi0_for(r, dtype):
        idx, amp = inputs.determinant_state(r["n"], seed=r["det_seed"])
        t = torch.zeros(1 << r["n"], dtype=dtype, device=dev)
        t[torch.as_tensor(idx.astype(np.int64), device=dev)] = torch.as_tensor(amp, device=dev).to(dtype)
        return t

    for r in runs:
        r["psi0"] = psi0_for(r, torch.complex64)
    tune = None
    cfg = None
    if not args.no_autotune:
        tune = autotune.tune_batch(runs, torch.complex64)
        cfg = {k: tune[k] for k in ("lane_size", "tile_bits", "single_bits") if k in tune}
    t_host = time.perf_counter()
    b = ps.Batch(runs, cfg=cfg)
    create_s = time.perf_counter() - t_host
    info = b.info
    for _ in range(args.warmup):
        b.launch()
    b.wait()

    clocks = ClockSampler(local)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.launch()
    ev1.record(stream)
    g64 = b.wait()
    clock_info = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    rot_per_launch = info["rotations"]
    t_max, tot_rot, _ = aggregate_ranks(dist, dev, ms, args.steps * rot_per_launch, args.steps)
    value = tot_rot / (t_max / 1e3)
    amp_updates = world * args.steps * info["amplitude_rotations"] / (t_max / 1e3)
    pass_bytes = 2.0 * 8.0 * info["amplitude_passes"]
    achieved = pass_bytes / (ms / args.steps / 1e3) / 1e9
    peak, peak_kind = hbm_peak()

    # one run at a time through the public single-run API (plans prebuilt,
    # like the batch's windows): copy psi0, apply, overlap
    seq = None
    if not args.no_sequential:
        plans = [ps.Plan(r["n"], ps.PS_C64, r["x"], r["z"], r["phi"]) for r in runs]
        svs = {}
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        for rep in range(2):  # the first pass warms up
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for r, pl in zip(runs, plans):
                n = r["n"]
                if n not in svs:
                    svs[n] = (ps.StateVector(n, tensor=torch.empty(1 << n, dtype=torch.complex64, device=dev)),
                              ps.StateVector(n, tensor=torch.empty(1 << n, dtype=torch.complex64, device=dev)))
                st, p0 = svs[n]
                p0.tensor.copy_(r["psi0"])  # p0 never evolves: its stored scale stays 1
                st.copy_from(p0)
                st.apply_plan(pl)
                st.overlap(p0)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        seq_ms = e0.elapsed_time(e1)
        seq = {"ms": seq_ms, "value": rot_per_launch / (seq_ms / 1e3), "unit": UNIT,
               "how": f"{len(runs)} x (copy psi0, ps_plan_apply of the run's prebuilt plan, ps_overlap), default tuning",
               "speedup_batch_vs_sequential": seq_ms / (ms / args.steps)}
        del plans, svs

    # complex64 vs complex128 (the batch engine in FP64 on the same runs)
    c128 = None
    if world == 1 and not args.no_c128:
        runs128 = [dict(r, psi0=psi0_for(r, torch.complex128), state=None) for r in runs]
        for r in runs:
            r.pop("psi0", None)
        b.close()
        torch.cuda.empty_cache()
        cfg128 = dict(cfg, tile_bits=min(cfg["tile_bits"], 12)) if cfg else None
        b128 = ps.Batch(runs128, dtype=torch.complex128, cfg=cfg128)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        b128.launch()
        b128.wait()
        e0.record(stream)
        b128.launch()
        e1.record(stream)
        g128 = b128.wait()
        ms128 = e0.elapsed_time(e1)
        d = np.abs(g64 - g128)
        c128 = {"value": rot_per_launch / (ms128 / 1e3), "unit": UNIT, "ms": ms128,
                "overlap_max_abs_diff_c64_vs_c128": float(d.max()), "overlap_median_abs_diff": float(np.median(d))}
        b128.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    ns = [r["n"] for r in runs]
    line = {
        "metric": "batched independent runs: rotations/s (qDRIFT and partially randomised, n 14..22, "
                  "one persistent launch per step)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{len(runs)} runs, n {f'= {args.batch_n}' if args.batch_n else 'uniform 14..22'} "
                               f"(mean state {np.mean([8 << n for n in ns]) / 2**20:.1f} MiB), 200-2000 JW-like terms, "
                               f"{args.batch_rotations or '2000-20000'} rotations, half qDRIFT half partial "
                               "(L_D 10%, r 4), 8-determinant psi0 per run",
                   "runs": len(runs), "rotations_per_step": rot_per_launch,
                   "l2": f"{sum(8 << n for n in ns) / 2**30:.2f} GiB of states per step (> 129 MB L2), no flush",
                   "batch": {k: info[k] for k in ("grid", "ctas_per_sm", "lanes", "lane_size", "tile_bits",
                                                    "lane_runs", "single_runs", "resident_runs", "windows", "graph",
                                                    "smem_bytes", "body_bytes")},
                   "parallelism": f"replicas x{world}"},
        "amplitude_updates_per_s": amp_updates,
        "roofline": {"bound": "hbm", "kernel": "k_batch<float,3,2>", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "note": "algorithmic bytes = one read + one write of every run's state per window "
                             "(resident runs stay on chip, lane runs partly in L2)",
                     "peak_source": peak_kind},
        "sequential": seq, "c128": c128, "autotune": tune,
        "host": {"workload_generation_s": host_gen_s, "batch_create_s": create_s},
        "gpu_launches": args.steps, "clocks": clock_info,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------- learned

def run_learned(args):
    """Learned step choice: train the network on Trotter errors the batched
    engine measures (complex128, n 14..18, 200-2000 terms, 8 times, r = 1..64
    plus the Richardson reference runs), then choose r for error 1e-3 on a
    1000-term Hamiltonian at n = 32 (complex64, 32 GiB state) and judge the
    choice with the doubling sweep."""
    import torch
    import paper_2504_17881_gb300 as ps
    from paper_2504_17881_gb300 import learned

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    eps = 1e-3
    P = args.train_problems
    t0 = time.perf_counter()
    probs = learned.synthetic_problems(P, seed=1000, n_range=(14, args.train_nmax), L_range=(200, 2000),
                                       lam_range=(1.0, 10.0), far_every=2)
    times = learned.TIMES16 if args.train_times == 16 else learned.TIMES16[::2]
    torch.cuda.synchronize()
    tg = time.perf_counter()
    X, y, info = learned.training_rows(probs, times=times)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - tg
    gen_rot = sum(probs[pi].L * r for pi in range(P) for _ in times for r in (1, 2, 4, 8, 16, 32, 64, 128))
    hold = max(16, P // 10)  # Hamiltonians held out for the pick margin
    cut = (P - hold) * len(times) * len(learned.R_VALUES)
    m = learned.StepEnsemble(count=4, seed=2)
    tt = time.perf_counter()
    losses = m.fit(X[:cut], y[:cut], epochs=150, batch=256, lr=2e-3, seed=3)[0]
    train_s = time.perf_counter() - tt
    pv = m.predict(X[cut:])
    val_rms = float(np.sqrt(np.mean((pv - y[cut:]) ** 2)))
    margin = m.calibrate_margin(X[cut:], y[cut:], 0.8)
    del X, y, info, probs
    torch.cuda.empty_cache()

    # use: n = use_qubits, 1000 terms, complex64
    n = args.use_qubits
    from paper_2504_17881_gb300 import inputs
    x, z, h = inputs.jw_hamiltonian(n, 1000, seed=1500, lam=8.0)
    prob = learned.Problem(n, x, z, h, psi_seed=1500)
    queries = []
    for t in LEARNED_TIMES:
        tq = time.perf_counter()
        r_ml, _ = m.pick_r(prob, t, eps)
        pick_s = time.perf_counter() - tq
        ts = time.perf_counter()
        r_sw, rot_sw, g_sw = learned.sweep(prob, t, eps, r_max=256)
        torch.cuda.synchronize()
        sweep_s = time.perf_counter() - ts
        # judge: the learned pick's run against the sweep's last (finest) run, 2 r_sw
        tl = time.perf_counter()
        psi0 = ps.StateVector(n, tensor=prob.state(torch.complex64))
        work = ps.StateVector(n, dtype=torch.complex64)
        work.copy_from(psi0)
        work.evolve_trotter(prob.ham, t, r_ml)
        g_ml = work.overlap(psi0)
        torch.cuda.synchronize()
        learned_s = time.perf_counter() - tl
        work.copy_from(psi0)
        work.evolve_trotter(prob.ham, t, 2 * r_sw)
        g_fine = work.overlap(psi0)
        del work, psi0
        torch.cuda.empty_cache()
        queries.append({"t": t, "r_sweep": r_sw, "rotations_sweep": rot_sw, "sweep_s": sweep_s,
                        "r_learned": r_ml, "rotations_learned": r_ml * prob.L, "learned_run_s": learned_s,
                        "pick_s": pick_s, "r_bound": learned.bound_r(prob, t, eps),
                        "err_learned_vs_2r_sweep": abs(g_ml - g_fine),
                        "err_sweep_estimate": 2 * abs(g_sw - g_fine),
                        "rotation_ratio_sweep_over_learned": rot_sw / max(1, r_ml * prob.L)})
    tot_sw = sum(q["rotations_sweep"] for q in queries)
    tot_ml = sum(q["rotations_learned"] for q in queries)
    line = {
        "metric": "learned Trotter step choice: rotations spent by the doubling sweep / by the learned pick "
                  f"(n={n} complex64, eps=1e-3)",
        "value": tot_sw / max(1, tot_ml), "unit": "x", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
        "dtype": "f32 network, c128 training data, c64 use",
        "config": {"workload": f"train: {P} JW-like H (n 14..{args.train_nmax}, 200-2000 terms, one-norm 1..10; every 2nd "
                               f"guiding state with determinants >= 10 flips apart), {len(times)} times "
                               f"{times[0]:.1f}..{times[-1]:.1f}, r 1..64; use: n={n}, 1000 terms, one-norm 8, "
                               f"8-determinant state, {len(LEARNED_TIMES)} times",
                   "training_rows": int(cut), "held_out_rows": int(len(pv)),
                   "network": "4 x (12 -> 128 -> 128 -> 128 -> 1, tanh, FP32, Adam), mean of log errors"},
        "training": {"data_generation_s": gen_s, "data_rotations": gen_rot, "train_s": train_s,
                     "loss_first": float(losses[0]), "loss_last": float(losses[-1]), "val_rms_log_eps": val_rms,
                     "margin": margin, "total_s": time.perf_counter() - t0},
        "queries": queries, "rotations_sweep": tot_sw, "rotations_learned": tot_ml,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------- single-kernel timings

def run_kernels(args):
    """The pair-streaming kernel and the overlap reduction at n = 30 on their
    own (CUDA events per launch, inputs far larger than L2): 64 single-rotation
    windows with an X bit at the top qubit (so the tile kernel cannot take
    them), then 8 overlaps, in complex64 and complex128.  Bytes: one read and
    one write of every amplitude per pair launch, one read of both states per
    overlap."""
    import torch
    import paper_2504_17881_gb300 as ps
    from paper_2504_17881_gb300 import inputs
    torch.cuda.set_device(0)
    n = N_QUBITS
    peak, peak_kind = hbm_peak()
    rng = np.random.default_rng(77)
    count = 64
    x = (rng.integers(0, 1 << (n - 1), size=count, dtype=np.uint64) | np.uint64(1 << (n - 1))).astype(np.uint64)
    z = rng.integers(0, 1 << n, size=count, dtype=np.uint64).astype(np.uint64)
    phi = rng.uniform(-1e-3, 1e-3, size=count)
    out = {}
    for name, tdt, dt in (("c64", torch.complex64, ps.PS_C64), ("c128", torch.complex128, ps.PS_C128)):
        S = 8 if name == "c64" else 16
        a = ps.StateVector(n, dtype=tdt)
        b = ps.StateVector(n, dtype=tdt)
        a.tensor.fill_(1.0 / (1 << (n // 2)))
        b.tensor.fill_(1.0 / (1 << (n // 2)))
        a.set_tuning(kernel_timing=1, max_window=1)
        plan = ps.Plan(n, dt, x, z, phi, tuning={"max_window": 1})
        assert plan.info["pair_windows"] == count
        a.apply_plan(plan)
        a.overlap(b)
        ps.ps_reset_stats(a.handle)
        a.apply_plan(plan)
        for _ in range(8):
            a.overlap(b)
        st = a.stats()
        pair_ms = st["kernel_ms"]["pair"] / st["launches"]["pair"]
        red_ms = st["kernel_ms"]["reduce"] / (st["launches"]["reduce"] / 2)
        out[name] = {
            "pair": {"launches": st["launches"]["pair"], "avg_launch_ms": pair_ms,
                     "gbs": 2.0 * S * (1 << n) / (pair_ms / 1e3) / 1e9,
                     "frac_of_copy": 2.0 * S * (1 << n) / (pair_ms / 1e3) / 1e9 / peak},
            "overlap": {"calls": st["launches"]["reduce"] // 2, "avg_ms": red_ms,
                        "gbs": 2.0 * S * (1 << n) / (red_ms / 1e3) / 1e9,
                        "frac_of_copy": 2.0 * S * (1 << n) / (red_ms / 1e3) / 1e9 / peak}}
        del a, b, plan
        torch.cuda.empty_cache()
    out["fma_tflops"] = {"fp32": ps.ps_measure_fma_rate(ps.PS_C64), "fp64": ps.ps_measure_fma_rate(ps.PS_C128)}
    print(json.dumps({"metric": f"single kernels at n={n}: GB/s per launch", "peak_gbs": peak,
                      "peak_source": peak_kind, "kernels": out}), flush=True)


# ------------------------------------------------------------- Trotter n=26

T26_N = 26
T26_TERMS = 2000
T26_HAM_SEED = 2
T26_PSI0_SEED = 21
T26_TIMES = [0.1 * 2.0 ** (j / 3.0) for j in range(16)]
T26_STEPS = [1, 2, 4, 8, 16, 32, 64]


def run_trotter26(args):
    """The n = 26 first-order Trotter sweep: a 2000-term JW-like Hamiltonian
    (one-norm 3.5), 16 times 0.1 * 2^(j/3) (0.1 .. 3.2), r in {1, 2, ..., 64};
    every (t, r) evolved from the 8-determinant state and closed with the FP64
    overlap, once in complex64 and once in complex128.  Reported: each pair's
    overlaps and their difference, the Trotter error against r = 64 (complex128),
    rotations/s of both dtypes (whole sweep, host scheduling included) and the
    tile kernel's roofline."""
    import torch
    import paper_2504_17881_gb300 as ps
    from paper_2504_17881_gb300 import inputs
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    n = T26_N
    x, z, h = inputs.jw_hamiltonian(n, T26_TERMS, seed=T26_HAM_SEED)
    H = ps.Hamiltonian(n, x, z, h)
    idx, amp = inputs.determinant_state(n, seed=T26_PSI0_SEED)
    peak, peak_kind = hbm_peak()
    out = {}
    per_dtype = {}
    for name, tdt, dt in (("c64", torch.complex64, ps.PS_C64), ("c128", torch.complex128, ps.PS_C128)):
        st0 = ps.StateVector(n, dtype=tdt, device=dev)
        st0.tensor.zero_()
        st0.tensor[torch.as_tensor(idx.astype(np.int64), device=dev)] = torch.as_tensor(amp, device=dev).to(tdt)
        work = ps.StateVector(n, dtype=tdt, device=dev)
        work.set_tuning(kernel_timing=1)
        work.copy_from(st0)
        work.evolve_trotter(H, T26_TIMES[0], 1)  # warm-up
        work.overlap(st0)
        torch.cuda.synchronize(dev)
        ps.ps_reset_stats(work.handle)
        clocks = ClockSampler(0) if name == "c64" else None
        if clocks:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rot = 0
        for t in T26_TIMES:
            for r in T26_STEPS:
                work.copy_from(st0)
                work.evolve_trotter(H, t, r)
                out.setdefault((t, r), {})[name] = work.overlap(st0)
                rot += r * T26_TERMS
        e1.record(stream)
        torch.cuda.synchronize(dev)
        clk = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        stats = work.stats()
        tile_ms = stats["kernel_ms"]["tile"] / max(stats["launches"]["tile"], 1)
        S = 8 if name == "c64" else 16
        per_dtype[name] = {"value": rot / (ms / 1e3), "unit": UNIT, "rotations": rot, "seconds": ms / 1e3,
                           "passes": stats["passes"], "rot_per_pass": rot / max(stats["passes"], 1),
                           "tile_avg_launch_ms": tile_ms,
                           "tile_achieved_gbs": 2.0 * S * (1 << n) / (tile_ms / 1e3) / 1e9 if tile_ms > 0 else None,
                           "gpu_launches": sum(stats["launches"].values()), "clocks": clk}
        del work, st0
        torch.cuda.empty_cache()
    rows = []
    for t in T26_TIMES:
        ref = out[(t, T26_STEPS[-1])]["c128"]
        for r in T26_STEPS:
            g32, g64 = out[(t, r)]["c64"], out[(t, r)]["c128"]
            rows.append({"t": t, "r": r, "g_c64": [g32.real, g32.imag], "g_c128": [g64.real, g64.imag],
                         "c64_vs_c128_abs": abs(g32 - g64), "trotter_err_vs_r64_c128": abs(g64 - ref)})
    c64 = per_dtype["c64"]
    ach = c64["tile_achieved_gbs"]
    line = {
        "metric": f"first-order Trotter sweep at n={n}: rotations/s, complex64 vs FP64", "value": c64["value"],
        "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"trotter n={n}: JW-like H with {T26_TERMS} terms (lambda 3.5, seed {T26_HAM_SEED}), "
                               f"16 times 0.1*2^(j/3), r in {T26_STEPS}, 8-determinant initial state; every (t, r) "
                               f"from psi0 with an FP64 overlap", "pairs": len(rows),
                   "l2": f"inputs larger than L2 ({8 << n >> 20} MiB c64 state), no flush"},
        "roofline": {"bound": "hbm", "kernel": "k_tile<float,3,4>", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak if ach else None, "traffic": None,
                     "peak_source": f"{peak_kind} copy bandwidth"},
        "c64": c64, "c128": per_dtype["c128"],
        "max_c64_vs_c128_abs": max(rw["c64_vs_c128_abs"] for rw in rows), "rows": rows,
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- reference

def run_reference(args):
    """The oracle as it stands, on the host cores: each step applies the next
    REF_ROTATIONS_PER_STEP rotations of the same n = 30 qDRIFT stream on every
    host core and reads the FP64 overlap <psi0|psi>, so the metric and unit
    are the GPU arm's.  A single-threaded figure on the first rotations is
    reported beside it.  Under torchrun only rank 0 runs."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    cores = host_cores()
    threads = cores if oracle.has_openmp() else 1
    total = (args.warmup + args.steps) * REF_ROTATIONS_PER_STEP
    run = OracleRun(total)
    dt1 = run.apply(0, CPU_ROTATIONS_1T, 1)
    run.reset()
    pos = 0
    for _ in range(args.warmup):
        run.apply(pos, REF_ROTATIONS_PER_STEP, cores)
        run.overlap(cores)
        pos += REF_ROTATIONS_PER_STEP
    t0 = time.perf_counter()
    g = 0j
    for _ in range(args.steps):
        run.apply(pos, REF_ROTATIONS_PER_STEP, cores)
        g = run.overlap(cores)
        pos += REF_ROTATIONS_PER_STEP
    dt = time.perf_counter() - t0
    value = args.steps * REF_ROTATIONS_PER_STEP / dt
    sample = (f"{REF_ROTATIONS_PER_STEP} rotations of the same qDRIFT stream at n={N_QUBITS} + the FP64 overlap per "
              f"step (complex128 scatter-form oracle, OpenMP over {threads} threads); {args.steps} timed steps "
              f"after {args.warmup} warm-up")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(), "n": N_QUBITS, "terms": N_TERMS, "samples": N_SAMPLES,
                   "rotations_per_step": REF_ROTATIONS_PER_STEP},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": CPU_ROTATIONS_1T / dt1, "unit": UNIT, "cores": 1,
                                           "sample": f"first {CPU_ROTATIONS_1T} rotations, 1 thread"},
                         "host_cores_available": cores},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "overlap_last": [g.real, g.imag],
    }), flush=True)


def main():
    global N_QUBITS
    args = parse()
    N_QUBITS = args.qubits
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "learned":
        run_learned(args)
    elif args.workload == "trotter26":
        run_trotter26(args)
    elif args.workload == "kernels":
        run_kernels(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
