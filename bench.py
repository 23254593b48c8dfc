#!/usr/bin/env python
"""Benchmark of the lattice-kinetic Kohn-Sham solver on GB300.

The metric is orbital-site updates per second (GLUPS): relaxation steps x
orbitals x grid sites / wall time, through the C ABI.  Default workload: the
8-water cluster, 256^3 grid at h = 0.2 bohr, 40 doubly occupied orbitals,
FP32 populations and collide with FP64 overlaps, Cholesky, energies and
Poisson (about 110 GB on the device); one bench step = one self-consistent
cycle (100 relaxation steps, density, Hartree, LDA, orthonormalisation,
energies), continuing from the previous one.  Workloads that fit a full
solve per step (--workload ch4_128, h2o_96, he_24) run one complete solve
per step to the stop rule of include/lbks.h.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lbks|reference]

--impl reference times the FP64 numpy oracle (the method as the paper states
it, plain CPU code) on the host cores, one relaxation step of the same
workload per bench step (the cluster: the same molecule on a 64^3 grid of
the same box), one oracle process per core as far as host memory allows.

Multi-GPU (torchrun): every rank solves its own replica (independent
systems, no collective on the data path); value = all ranks' updates / the
slowest rank's time.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "GLUPS (orbital-site updates/s)"
UNIT = "GLUPS"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2
KERNEL_SRC = os.path.join(ROOT, "paper_1507_07666_gb300", "csrc", "lbks_relax.cuh")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "stream_collide_ch4_128_fp32.json")
KERNEL_END_MARK = b"// u_(j-1)(r) = -omega sum_{k<j} Lambda_jk psi_k(r)"
# more than eight orbitals: the relaxation step is the wide stream-collide
# kernel plus the tensor-core overlap; their DRAM bytes per orbital-site from
# one ncu capture, valid while both kernels' sources are unchanged
WIDE_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_wide_h2o8_fp32.json")
WIDE_SOURCES = (os.path.join(ROOT, "paper_1507_07666_gb300", "csrc", "lbks_wide.cuh"),
                os.path.join(ROOT, "paper_1507_07666_gb300", "csrc", "lbks_gram_tc.cu"))
# the same step with the two-site stream-collide kernel (tuned variant index 1)
WIDE_PAIR_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "step_wide_pair_h2o8_fp32.json")
WIDE_PAIR_SOURCES = (os.path.join(ROOT, "paper_1507_07666_gb300", "csrc", "lbks_pair.cuh"),
                     os.path.join(ROOT, "paper_1507_07666_gb300", "csrc", "lbks_gram_tc.cu"))

WORKLOADS = {
    "ch4_128": W.ch4_128,
    "he_24": W.he_24,
    "h2o_96": W.water_96,
}
# workloads too large for a full solve per bench step: one step = one SCF cycle
# (n_inner relaxation steps, density, Hartree, LDA, orthonormalisation, energies)
# continuing from the previous cycle
CYCLES = {"h2o8_256": W.cluster_256}
# the oracle cannot hold the cluster's 256^3 populations in host memory: its
# CPU baseline is the same molecule on a coarser grid of the same box
# (batched and served workloads: one water geometry at 96^3)
ORACLE_SAMPLE_OF = {"h2o8_256": W.cluster_sample, "water_scan_64": W.water_96, "serving_mix": W.water_96,
                    "h2o_relax_96": W.water_96}
SERVING = {"serving_mix": 200}  # requests of the mixed stream (Poisson arrivals, mean 200/s, seed 0)
BATCHES = {
    # 64 seeded water geometries (O-H ~ U[1.6, 2.0] bohr, HOH ~ U[95, 115] deg), 96^3 grid, h = 0.2
    "water_scan_64": (64, 0),
}
# Born-Oppenheimer geometry relaxation: one bench step = one relaxation from the
# start geometry (warm-started SCF per move) to max |F| < fmax
# (the O nucleus is held: with the softening a = h the energy depends on where
# a nucleus sits between grid points by tenths of a hartree, and a free
# relaxation slides the O onto a grid point instead of relaxing the bonds)
RELAXATIONS = {"h2o_relax_96": (W.water_96, 2.0, 95.0, 2e-3, [1, 0, 0])}
# concurrent dynamics (Eq. KSLBCD): from the ground state at a stretched
# geometry, one bench step = CD_BLOCKS blocks of CD_NPOT real-time steps, each
# block ending with the potential rebuilt and the nuclei moved
DYNAMICS = {"ch4_cd_128": W.ch4_cd_128}
CD_BLOCKS, CD_NPOT = 10, 10


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["lbks", "reference"], default="lbks")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + sorted(CYCLES) + sorted(BATCHES) + sorted(SERVING)
                    + sorted(RELAXATIONS) + sorted(DYNAMICS), default="h2o8_256")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrent solve slots")
    ap.add_argument("--requests", type=int, default=0, help="serving: requests of the stream (0: the default)")
    ap.add_argument("--precision", choices=["fp32", "fp64", "bf16"], default="fp32")
    ap.add_argument("--storage", choices=["populations", "psi"], default="populations",
                    help="what a relaxation step keeps: the 19 populations per orbital-site (any omega), or, at "
                         "omega = 1, the orbital alone (the same step as a 19-point stencil)")
    ap.add_argument("--poisson-adapt", type=float, default=0.0,
                    help="lbks_params.poisson_adapt: each cycle's Hartree solve stops at max(rtol, min(1e-4, "
                         "value x the previous density change)); 0: the fixed tolerance")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the fused stream-collide kernel (for profiling)")
    ap.add_argument("--kernel-n", type=int, default=0, help="cubic grid edge for --kernel-only (0: workload's)")
    ap.add_argument("--launches", type=int, default=20)
    ap.add_argument("--kernel", choices=["stream_collide", "overlap_tc", "overlap_exact"], default="stream_collide",
                    help="--kernel-only: which step to launch alone")
    ap.add_argument("--relax-variant", type=int, choices=[0, 1, 2, 3, 4], default=0,
                    help="stream-collide variant: 0 tuned per shape, 1 one site per thread, 2 site pairs, "
                         "3 one site with the next orbital prefetched, 4 populations copied by the tensor memory "
                         "accelerator (omega = 1)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------- oracle leg
ORACLE_SAMPLE = r"""
import json, os, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import lattice, lb, scf
w = W.{wl}()
n, h, no = w.n, w.h, w.n_orb
xyz, Z = w.molecule.xyz, w.molecule.Z
dt = lattice.time_step(w.theta, w.omega, h)
psi = lb.orthonormalize(scf.initial_orbitals(n, h, xyz, Z, no), h)
f = lb.equilibrium(psi, w.theta)
sigma = np.ones(no)
V = scf.external_potential(n, h, xyz, Z, h)
times = []
t_end = time.perf_counter() + {seconds}
while len(times) < {min_steps} or (time.perf_counter() < t_end and len(times) < {max_steps}):
    t0 = time.perf_counter()
    r = lb.step(f, sigma, V, w.omega, w.theta, dt, h)
    f, sigma = r["fstar"], r["sigma"]
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times, "updates_per_step": no * n[0] * n[1] * n[2]}}))
"""


def oracle_workload(workload: str):
    fn = WORKLOADS[workload] if workload in WORKLOADS else ORACLE_SAMPLE_OF[workload]
    return fn


def oracle_processes(workload: str) -> int:
    """Concurrent single-thread oracle processes: one per host core, as far as
    half of the available host memory holds them (about six population
    arrays of the sampled workload each, plus 1 GB)."""
    w = oracle_workload(workload)()
    per = 6 * 19 * 8 * w.n_orb * w.sites + (1 << 30)
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    if avail is None:
        avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    return max(1, min(os.cpu_count() or 1, int(0.5 * avail // per)))


def run_oracle_samples(workload: str, seconds: float, min_steps: int, max_steps: int, procs: int = 1):
    """Runs `procs` oracle processes at once (one thread each); returns their
    step timings."""
    code = ORACLE_SAMPLE.format(root=ROOT, wl=oracle_workload(workload).__name__, seconds=seconds,
                                min_steps=min_steps, max_steps=max_steps)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for _ in range(procs)]
    out = []
    for p in ps:
        so, se = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("oracle sample failed:\n" + se[-2000:])
        out.append(json.loads(so.strip().splitlines()[-1]))
    return out


def oracle_rate(samples, skip=0):
    """Whole-host rate of concurrent samples: all processes' timed updates
    over the slowest process's timed seconds."""
    steps = sum(len(s["times"]) - skip for s in samples)
    t = max(sum(s["times"][skip:]) for s in samples)
    return steps * samples[0]["updates_per_step"] / t / 1e9, steps, t


def cpu_baseline(workload: str, seconds: float):
    name = oracle_workload(workload)().name
    one = run_oracle_samples(workload, seconds, 2, 1000)
    v1, n1, t1 = oracle_rate(one)
    procs = oracle_processes(workload)
    many = run_oracle_samples(workload, seconds, 2, 1000, procs)
    v, n, t = oracle_rate(many)
    return {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{n} relaxation steps (Eq. KSLB, all orbitals) of the {name} workload from its Gaussian "
                      f"start in {procs} concurrent FP64 numpy processes of one thread each, {t:.1f} s",
            "one_core": {"value": v1, "cores": 1, "sample": f"{n1} steps, one process, {t1:.1f} s"}}


def main_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = oracle_workload(args.workload)()
    procs = oracle_processes(args.workload)
    samples = run_oracle_samples(args.workload, 0.0, args.warmup + args.steps, args.warmup + args.steps, procs)
    value, steps, t = oracle_rate(samples, skip=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "grid": list(w.n), "h": w.h, "n_orb": w.n_orb,
                   "step": f"one oracle relaxation step of all orbitals in each of {procs} concurrent processes"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{steps} timed relaxation steps of {w.name} in {procs} concurrent FP64 numpy "
                                   "processes of one thread each"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU leg
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags) if f == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def job_totals(dist, device, updates, seconds):
    """Replicas (one independent solve per rank, no collective on the data
    path): the whole job's orbital-site updates and the slowest rank's time.
    dist: torch.distributed or None."""
    if dist is None:
        return float(updates), float(seconds)
    import torch
    u = torch.tensor([float(updates)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_sha():
    """sha256 of lbks_relax.cuh up to the end of the stream-collide kernel (its
    helpers and itself; the launchers below it do not change its traffic)."""
    text = open(KERNEL_SRC, "rb").read()
    end = text.find(KERNEL_END_MARK)
    return hashlib.sha256(text[:end] if end > 0 else text).hexdigest()


def recorded_traffic():
    """dram bytes per launch of the stream-collide kernel from the committed
    ncu summary, if it was taken on the current kernel source."""
    try:
        rec = json.load(open(TRAFFIC_FILE))
        sha = kernel_source_sha()
        if rec.get("kernel_src_sha256") == sha:
            return float(rec["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


WIDE_SEGMENTS = (
    # the wide stream-collide kernel, up to the next kernel of its header
    (b"__global__ void __launch_bounds__(kThreads, 4) k_stream_collide_wide", b"// S = h^3 Psi Psi^T over the packed"),
    # the tensor-core overlap kernel and its device helpers, up to its launcher
    (b"", b"template <bool LAM, bool BULK, int MAXO, int TH = kTcThreads, int TPB = 1>\nstatic cudaError_t gram_tc_launch"),
)


WIDE_PAIR_SEGMENTS = (
    # in the row-kernel header: the two-site helpers (pair types, the two-phase
    # gather) and, from its comment to the end, the wide two-site kernel
    ((b"template <typename TS>\nstruct Pack2;", b"// W consecutive elements of one array"),
     (b"// More than kMaxOrb orbitals: the same two-site update", b"")),
    WIDE_SEGMENTS[1],
)


def wide_sources_sha(variant=0):
    """sha256 over the source text of the wide relaxation step's two kernels
    (each file's segment from its start mark to its end mark); variant 0:
    one site per thread, 1: two sites per thread."""
    h = hashlib.sha256()
    sources, segments = (WIDE_SOURCES, WIDE_SEGMENTS) if variant == 0 else (WIDE_PAIR_SOURCES, WIDE_PAIR_SEGMENTS)
    for path, spans in zip(sources, segments):
        text = open(path, "rb").read()
        for start, end in (spans if isinstance(spans[0], tuple) else (spans,)):
            i = text.find(start) if start else 0
            k = text.find(end, max(i, 0)) if end else len(text)
            h.update(text[i:k] if i >= 0 and k > i else text)
    return h.hexdigest()


def recorded_wide_traffic(units, variant=0):
    """DRAM bytes of one wide relaxation step (stream-collide + overlap) over
    `units` orbital-sites, scaled from the committed ncu capture of a smaller
    grid (traffic grows in proportion to the orbital-sites), if it was taken
    on the current sources of the variant's kernels."""
    path = {0: WIDE_TRAFFIC_FILE, 1: WIDE_PAIR_TRAFFIC_FILE}.get(variant)
    try:
        rec = json.load(open(path))
        if rec.get("sources_sha256") == wide_sources_sha(variant):
            return float(rec["dram_bytes_per_orbital_site"]) * units
    except (OSError, KeyError, ValueError, TypeError):
        pass
    return None


def psi_step_kernels(w, pe, index):
    """Kernels of one orbital-storage step for kernel index (0 tiled, 1 direct,
    2 TMA, 3 z-marching) and its algorithmic HBM bytes per site: psi in and
    out and the collision potential once; more than eight orbitals add the
    overlap kernel's read of psi' and, without the TMA kernel, the W-field
    kernel's read of psi, its write of u and the step's read of u."""
    no, wide = w.n_orb, w.n_orb > 8
    name = ("k_relax_psi_tile", "k_relax_psi", "k_relax_psi_tma", "k_relax_psi_zm")[index]
    if wide and index != 2:
        name = "k_w_field_wide + " + name.replace("k_relax_psi", "k_relax_psi_wide")
    words = 2 * no + ((no if index == 2 else 4 * no - 2) if wide else 0)
    if wide:
        name += " + " + ("k_gram_wide" if pe == 8 else "k_gram_tc") + " (one relaxation step)"
    return name, pe * words + 8


def psi_kernel_index(w, pe, mode):
    """The kernel lbks_relax_step_psi runs under lbks_set_relax_variant(mode)."""
    tma_ok = w.n[0] % (16 // pe) == 0
    k = mode - 1 if mode > 0 else (2 if tma_ok else 0)
    return 0 if (k == 3 and w.n_orb > 8) or (k == 2 and not tma_ok) else k


def time_relax_psi(torch, lbks, w, prec, stream, launches=20, mode=None, shape=None):
    """Average duration of the orbital-storage step (omega = 1) in the
    solver's launch configuration, CUDA events on the launching stream;
    mode: the lbks_set_relax_variant mode to time under, shape: the staged
    stencil's tile shape (lbks_set_psi_tile; None: as set)."""
    if shape is not None:
        prev_shape = lbks.lbks_set_psi_tile(shape)
        try:
            return time_relax_psi(torch, lbks, w, prec, stream, launches, mode)
        finally:
            lbks.lbks_set_psi_tile(prev_shape)
    if mode is not None:
        prev = lbks.lbks_set_relax_variant(mode)
        try:
            return time_relax_psi(torch, lbks, w, prec, stream, launches)
        finally:
            lbks.lbks_set_relax_variant(prev)
    P = torch.float64 if prec == lbks.FP64 else torch.float32
    nx, ny, nz = w.n
    N = nx * ny * nz
    no = w.n_orb
    with torch.cuda.stream(stream):
        pa = torch.rand((no, nz, ny, nx), dtype=P, device="cuda")
        pb = torch.empty_like(pa)
        V = -torch.rand((nz, ny, nx), dtype=torch.float64, device="cuda")
        sig = torch.full((no,), 1e-3, dtype=torch.float64, device="cuda")
        S = torch.empty((no, no), dtype=torch.float64, device="cuda")
        lam_in = torch.tril(torch.rand((no, no), dtype=torch.float64, device="cuda"), -1) * 0.01
        lam = torch.empty_like(S)
        sig2 = torch.empty_like(sig)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    dt = w.theta * w.h * w.h
    bufs = [pa, pb]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * launches)]
    for i in range(3 + launches):
        src, dst = bufs[i % 2], bufs[(i + 1) % 2]
        if i >= 3:
            with torch.cuda.stream(stream):
                flush.fill_(float(i))  # the working set can fit in L2: evict it before every timed launch
            evs[2 * (i - 3)].record(stream)
        lbks.lbks_relax_step_psi(prec, nx, ny, nz, no, w.h, w.theta, dt, src, lam_in, V, sig, dst, S, lam, sig2,
                                 stream=stream)
        if i >= 3:
            evs[2 * (i - 3) + 1].record(stream)
    stream.synchronize()
    ms = [evs[2 * k].elapsed_time(evs[2 * k + 1]) for k in range(launches)]
    del pa, pb, V, flush
    return statistics.mean(ms), N * no


def time_stream_collide(torch, lbks, w, prec, stream, launches=20):
    """Average duration of the fused stream-collide kernel in the solver's own
    launch configuration, CUDA events on the launching stream."""
    T = {lbks.FP32: torch.float32, lbks.FP64: torch.float64, lbks.BF16: torch.bfloat16}[prec]
    P = torch.float64 if prec == lbks.FP64 else torch.float32
    nx, ny, nz = w.n
    N = nx * ny * nz
    no = w.n_orb
    with torch.cuda.stream(stream):
        fa = torch.rand((no, 19, nz, ny, nx), dtype=T, device="cuda")
        fb = torch.empty_like(fa)
        u = torch.rand((max(no - 1, 1), nz, ny, nx), dtype=P, device="cuda") * 0.1
        psi = torch.empty((no, nz, ny, nx), dtype=P, device="cuda")
        V = -torch.rand((nz, ny, nx), dtype=torch.float64, device="cuda")
        sig = torch.full((no,), 1e-3, dtype=torch.float64, device="cuda")
        S = torch.empty((no, no), dtype=torch.float64, device="cuda")
        lam = torch.empty_like(S)
        sig2 = torch.empty_like(sig)
    dt = w.theta * w.h * w.h * (2 - w.omega) / w.omega
    bufs = [fa, fb]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * launches)]
    for i in range(3 + launches):
        src, dst = bufs[i % 2], bufs[(i + 1) % 2]
        if i >= 3:
            evs[2 * (i - 3)].record(stream)
        lbks.lbks_relax_step(prec, nx, ny, nz, no, w.h, w.omega, w.theta, dt, src, u if no > 1 else None, V, sig,
                             dst, psi, S, lam, sig2, stream=stream)
        if i >= 3:
            evs[2 * (i - 3) + 1].record(stream)
    stream.synchronize()
    ms = [evs[2 * k].elapsed_time(evs[2 * k + 1]) for k in range(launches)]
    del fa, fb, u, psi, V
    return statistics.mean(ms), N * no


def time_overlap(torch, lbks, w, prec, stream, tensor_cores, launches=20):
    """Average duration of the overlap (Gram) step S = h^3 Psi Psi^T alone."""
    nx, ny, nz = w.n
    N = nx * ny * nz
    P = torch.float64 if prec == lbks.FP64 else torch.float32
    with torch.cuda.stream(stream):
        psi = torch.randn((w.n_orb, N), dtype=P, device="cuda")
        S = torch.empty((w.n_orb, w.n_orb), dtype=torch.float64, device="cuda")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for i in range(3 + launches):
        if i == 3:
            evs[0].record(stream)
        lbks.lbks_overlap(prec, N, w.n_orb, w.h, psi, S, tensor_cores=tensor_cores, stream=stream)
    evs[1].record(stream)
    stream.synchronize()
    return evs[0].elapsed_time(evs[1]) / launches, N * w.n_orb, psi.element_size()


def main_kernel_only(args):
    """One step launched alone (3 untimed + --launches timed), for ncu: the
    stream-collide, or the overlap on the tensor cores / with exact sums."""
    import torch
    from paper_1507_07666_gb300 import build as build_mod
    build_mod.build()
    from paper_1507_07666_gb300 import lbks
    w = (WORKLOADS.get(args.workload) or CYCLES[args.workload])()
    if args.kernel_n:
        w.n = (args.kernel_n,) * 3
    prec = {"fp32": lbks.FP32, "fp64": lbks.FP64, "bf16": lbks.BF16}[args.precision]
    lbks.lbks_set_relax_variant(args.relax_variant)
    stream = torch.cuda.Stream()
    if args.kernel != "stream_collide":
        ms, units, esz = time_overlap(torch, lbks, w, prec, stream, args.kernel == "overlap_tc", args.launches)
        print(json.dumps({"kernel": "k_gram_tc" if args.kernel == "overlap_tc" and prec != lbks.FP64 else "k_gram",
                          "grid": list(w.n), "n_orb": w.n_orb, "dtype": args.precision, "ms_per_launch": ms,
                          "algorithmic_GBps": units * esz / (ms / 1e3) / 1e9, "launches": args.launches}),
              flush=True)
        return 0
    if args.storage == "psi":
        ms, units = time_relax_psi(torch, lbks, w, prec, stream, launches=args.launches)
        pe = 8 if prec == lbks.FP64 else 4
        N = units // w.n_orb
        kname, per_site = psi_step_kernels(w, pe, psi_kernel_index(w, pe, args.relax_variant))
        nbytes = per_site * N
        print(json.dumps({"kernel": kname, "grid": list(w.n),
                          "n_orb": w.n_orb, "dtype": args.precision, "ms_per_launch": ms,
                          "algorithmic_GBps": nbytes / (ms / 1e3) / 1e9,
                          "orbital_site_updates_per_s": units / (ms / 1e3), "launches": args.launches}), flush=True)
        return 0
    ms, units = time_stream_collide(torch, lbks, w, prec, stream, launches=args.launches)
    elem = {lbks.FP32: 4, lbks.FP64: 8, lbks.BF16: 2}[prec]
    gbs = 38 * elem * units / (ms / 1e3) / 1e9
    print(json.dumps({"kernel": {2: "k_stream_collide_pair", 4: "k_stream_collide_bulk"}.get(args.relax_variant,
                                                                                           "k_stream_collide"),
                      "variant": ("sites (untuned)", "sites", "pairs", "prefetch", "bulk")[args.relax_variant],
                      "grid": list(w.n), "n_orb": w.n_orb, "dtype": args.precision,
                      "ms_per_launch": ms, "algorithmic_GBps": gbs, "launches": args.launches}), flush=True)
    return 0


def main_batch(args):
    """Batched water scan: all geometries relax in the same launches; one
    bench step = one batched solve of every geometry to |dE| < 1e-6 Ha."""
    import torch
    from paper_1507_07666_gb300 import build as build_mod
    build_mod.build()
    from paper_1507_07666_gb300 import lbks
    count, seed = BATCHES[args.workload]
    mols = W.water_scan(count, seed)
    w = W.water_96(mols[0])
    prec = {"fp32": lbks.FP32, "fp64": lbks.FP64, "bf16": lbks.BF16}[args.precision]
    b = lbks.Batch(w.n, w.h, w.n_orb, count, precision=prec, n_inner=w.n_inner, e_tol=w.e_tol, theta=w.theta,
                   omega=w.omega, mix=w.mix, max_cycles=w.max_cycles,
                   storage=lbks.STORE_PSI if args.storage == "psi" else lbks.STORE_POPULATIONS)
    stream = torch.cuda.Stream()
    geoms = [(m.xyz, m.Z) for m in mols]

    def solve():
        b.set_geometries(geoms)
        return b.scf(stream)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = lbks.lbks_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [solve() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = lbks.lbks_kernel_launches() - l0
    elapsed_ms = ev0.elapsed_time(ev1)
    tuned = lbks.lbks_get_relax_variant(b.handle)
    if args.storage == "psi":  # orbital storage names its kernels differently
        tuned = {"variant": ("tiled", "direct", "tma", "zmarch")[tuned["index"]], "ms_tiled": tuned["ms_sites"],
                 "ms_direct": tuned["ms_pairs"], "ms_tma": tuned["ms_prefetch"], "ms_zmarch": tuned["ms_bulk"]}
    updates = sum(r["steps"] for res in results for r in res) * w.n_orb * w.sites
    last = results[-1]
    elem = {lbks.FP32: 4, lbks.FP64: 8, lbks.BF16: 2}[prec]
    line = {
        "metric": METRIC, "value": updates / (elapsed_ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {lbks.FP32: "f32", lbks.FP64: "f64", lbks.BF16: "bf16-storage/f32"}[prec], "data": "synthetic",
        "config": {"workload": f"batched water scan: {count} geometries (seed {seed}), 96^3, h=0.2, one launch "
                               "per relaxation step for all geometries",
                   "grid": list(w.n), "n_orb": w.n_orb, "systems": count, "n_inner": w.n_inner,
                   "storage": args.storage,
                   "l2": "inputs larger than L2 (%s %.1f GB)" % (
                       ("psi pair", 2 * (8 if prec == lbks.FP64 else 4) * w.n_orb * w.sites * count / 1e9)
                       if args.storage == "psi" else
                       ("populations", 2 * 19 * elem * w.n_orb * w.sites * count / 1e9))},
        "solves_per_s": count * args.steps / (elapsed_ms / 1e3),
        "batch": {"converged": sum(r["converged"] for r in last), "cycles_max": max(r["cycles"] for r in last),
                  "cycles_min": min(r["cycles"] for r in last),
                  "E_total_range": [min(r["E_total"] for r in last), max(r["E_total"] for r in last)]},
        "gpu_launches": int(launches), "clocks": clk, "stream_collide_variant": tuned,
    }
    print(json.dumps(line), flush=True)
    b.close()
    return 0


def _serve_arm(lbks, reqs, precision, slots, warm, storage=0):
    """Replays the arrival stream against a server; returns per-request
    latencies (s), the makespan and the results."""
    # the stop rule of include/lbks.h; water's two close occupied levels need up to a few hundred cycles
    srv = lbks.lbks_server_create(lbks.lbks_params_default(precision=precision, storage=storage, max_cycles=600), 0,
                                  slots)
    try:
        for _, w in warm:  # first use of each shape: allocation and graph capture
            rid = lbks.lbks_submit(srv, w.n, w.h, w.molecule.xyz, w.molecule.Z, n_inner=w.n_inner)
            lbks.lbks_server_wait(srv, rid, 600.0)
            lbks.lbks_poll(srv, rid)
        t0 = time.perf_counter()
        ids = []
        for t_arr, w in reqs:
            delay = t0 + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(lbks.lbks_submit(srv, w.n, w.h, w.molecule.xyz, w.molecule.Z, n_inner=w.n_inner))
        out = {}
        while len(out) < len(ids):
            for rid in ids:
                if rid not in out:
                    r = lbks.lbks_poll(srv, rid)
                    if r is not None:
                        out[rid] = r
            time.sleep(0.001)
        makespan = time.perf_counter() - t0
    finally:
        lbks.lbks_server_destroy(srv)
    lat = sorted(out[rid][1]["latency_s"] for rid in ids)
    run = sorted(out[rid][1]["run_s"] for rid in ids)
    return lat, run, makespan, [out[rid][0] for rid in ids]


def percentile(sorted_values, q):
    """Nearest-rank percentile: the smallest value with at least a fraction q
    of the sample at or below it."""
    n = len(sorted_values)
    return sorted_values[min(n - 1, max(0, math.ceil(q * n) - 1))]


def latency_summary(values):
    return {"p50": percentile(values, 0.5), "p90": percentile(values, 0.9), "p99": percentile(values, 0.99),
            "max": values[-1], "n": len(values)}


def main_serving(args):
    """Continuous-batching request loop on a mixed stream of solves against
    the plain single-solve FP64 path (one slot, FP64) on the same stream."""
    import torch
    from paper_1507_07666_gb300 import build as build_mod
    build_mod.build()
    from paper_1507_07666_gb300 import lbks
    reqs = W.serving_stream(args.requests or SERVING[args.workload], 200.0, 0)
    kinds = {}
    for t, w in reqs:
        kinds.setdefault(w.name, (t, w))
    warm = list(kinds.values())
    psi = args.storage == "psi"  # orbital storage: FP32 (it has no bfloat16 form)
    lat, run, span, res = _serve_arm(lbks, reqs, lbks.FP32 if psi else lbks.BF16, args.slots, warm,
                                     lbks.STORE_PSI if psi else lbks.STORE_POPULATIONS)
    lat64, run64, span64, res64 = _serve_arm(lbks, reqs, lbks.FP64, 1, warm)
    de = max(abs(a["E_total"] - b["E_total"]) for a, b in zip(res, res64))
    odd = [{"request": i, "kind": w.name, "h": round(w.h, 4), "converged": a["converged"], "status": a["status"],
            "cycles": a["cycles"], "E_total": a["E_total"], "E_total_fp64": b["E_total"],
            "fp64_converged": b["converged"]}
           for i, ((_, w), a, b) in enumerate(zip(reqs, res, res64))
           if not a["converged"] or not b["converged"] or abs(a["E_total"] - b["E_total"]) > 1e-5]
    line = {
        "metric": "solves/s (served mixed stream)", "value": len(reqs) / span, "unit": "solves/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if psi else "bf16-storage/f32", "data": "synthetic",
        "config": {"workload": f"served stream: {len(reqs)} requests, Poisson arrivals 200/s (seed 0), uniform over "
                               "H2 48^3, He 48^3, LiH 64^3, H2O 96^3, CH4 128^3, h ~ U[0.2, 0.25], jitter 0.05 bohr",
                   "slots": args.slots,
                   "precision": "FP32, orbital storage (omega = 1)" if psi else "BF16 populations + FP32 polish"},
        "latency_s": latency_summary(lat),
        "run_s": latency_summary(run),
        "latency_note": "latency = submit to result (queueing included: the whole stream arrives within about "
                        f"{reqs[-1][0]:.2f} s); run_s = slot start to result",
        "plain_fp64_single_slot": {"solves_per_s": len(reqs) / span64, "latency_s": latency_summary(lat64),
                                   "run_s": latency_summary(run64)},
        "max_abs_dE_vs_fp64_Ha": de,
        "converged": sum(r["converged"] for r in res),
        "fp64_converged": sum(r["converged"] for r in res64),
        "outliers": odd[:12],
    }
    print(json.dumps(line), flush=True)
    return 0


def main_relax(args):
    """Geometry relaxation of a distorted water on the 96^3 grid: every step
    relaxes from the same start (lbks_set_geometry, then lbks_relax_geometry:
    SCF, Hellmann-Feynman forces, steepest-descent moves with warm-started
    SCFs).  value: orbital-site updates of all SCFs of the relaxation per
    second of the whole relaxation (forces, moves and host steps included)."""
    import torch
    from paper_1507_07666_gb300 import build as build_mod
    build_mod.build()
    from paper_1507_07666_gb300 import lbks
    make, r_oh, angle, fmax, fixed = RELAXATIONS[args.workload]
    w = make()
    mol = W.water(r_oh, angle)
    prec = {"fp32": lbks.FP32, "fp64": lbks.FP64, "bf16": lbks.BF16}[args.precision]
    sysm = lbks.System(w.n, w.h, w.n_orb, precision=prec, n_inner=w.n_inner, e_tol=w.e_tol, theta=w.theta,
                       omega=w.omega, mix=w.mix, max_cycles=w.max_cycles,
                       storage=lbks.STORE_PSI if args.storage == "psi" else lbks.STORE_POPULATIONS)
    stream = torch.cuda.Stream()

    def relax():
        sysm.set_geometry(mol.xyz, mol.Z)
        return sysm.relax_geometry(max_steps=60, fmax=fmax, step=0.5, stream=stream, allow_notconv=True,
                                   fixed=fixed)

    for _ in range(args.warmup):
        relax()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = lbks.lbks_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = [relax() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = lbks.lbks_kernel_launches() - l0
    elapsed_ms = ev0.elapsed_time(ev1)
    updates = sum(r["steps"] for r in results) * w.n_orb * w.sites
    last = results[-1]
    # forces call alone (device reduction + host nuclear term + readback)
    t0 = time.perf_counter()
    for _ in range(10):
        sysm.forces()
    forces_ms = (time.perf_counter() - t0) * 100.0
    R = last["xyz"]
    b1, b2 = [R[k] - R[0] for k in (1, 2)]
    d1, d2 = math.sqrt(sum(v * v for v in b1)), math.sqrt(sum(v * v for v in b2))
    ang = math.degrees(math.acos(sum(p * q for p, q in zip(b1, b2)) / (d1 * d2)))
    sysm.close()
    ms, units = time_stream_collide(torch, lbks, w, prec, stream)
    elem = {lbks.FP32: 4, lbks.FP64: 8, lbks.BF16: 2}[prec]
    peak, peak_kind = measured_hbm_peak()
    achieved = 38 * elem * units / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": updates / (elapsed_ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {lbks.FP32: "f32", lbks.FP64: "f64", lbks.BF16: "bf16-storage/f32"}[prec], "data": "synthetic",
        "config": {"workload": f"H2O geometry relaxation from r_OH {r_oh} bohr, HOH {angle} deg to max|F| < {fmax} "
                               "Ha/bohr with the O held, 96^3, h=0.2 (warm-started SCF per move)",
                   "grid": list(w.n), "n_orb": w.n_orb, "storage": args.storage,
                   "l2": "inputs larger than L2 (populations %.2f GB)" % (2 * 19 * elem * units / 1e9)},
        "relaxation": {"relaxed": last["relaxed"], "moves": last["moves"], "scf_cycles": last["cycles"],
                       "E_total": last["E_total"], "r_OH": [float(d1), float(d2)], "HOH_deg": ang,
                       "forces_ms": forces_ms},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_stream_collide", "bytes_per_launch": 38 * elem * units,
                     "ms_per_launch": ms, "peak_source": f"hbm_gbs of {peak_kind}"},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    return 0


ORACLE_CD_SAMPLE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import workloads as W
from oracle import cd, lattice, lb, scf
w = W.{wl}()
n, h, no = w.n, w.h, w.n_orb
dt = lattice.time_step(w.theta, 1.0, h)
psi = lb.orthonormalize(scf.initial_orbitals(n, h, w.molecule.xyz, w.molecule.Z, no), h).astype(complex)
V = scf.external_potential(n, h, w.molecule.xyz, w.molecule.Z, h)
prev, cur = psi, psi
times = []
t_end = time.perf_counter() + {seconds}
while len(times) < 2 or time.perf_counter() < t_end:
    t0 = time.perf_counter()
    prev, cur = cur, cd.cd_step(prev, cur, V, w.theta, dt, h, 0.5 * dt)
    times.append(time.perf_counter() - t0)
print(json.dumps({{"times": times, "updates_per_step": no * n[0] * n[1] * n[2]}}))
"""


def time_cd_step(torch, lbks, w, prec, launches=20):
    """Average duration of one concurrent-dynamics step (k_cd_step, the launch
    configuration of the run) on random levels of the workload's shape, CUDA
    events on the launching stream, L2 flushed before every launch."""
    P = torch.float64 if prec == lbks.FP64 else torch.float32
    nx, ny, nz = w.n
    no = w.n_orb
    dt = w.theta * w.h * w.h
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = torch.rand((no, 2, nz, ny, nx), dtype=P, device="cuda")
        b = torch.rand_like(a)
        c = torch.empty_like(a)
        V = torch.rand((nz, ny, nx), dtype=torch.float64, device="cuda")
        S = torch.zeros((no, no, 2), dtype=torch.float64, device="cuda")
        L = torch.zeros_like(S)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        lbks.lbks_cd_overlap(prec, nx * ny * nz, no, w.h, b, S, L, stream=stream)
        total = 0.0
        for it in range(3 + launches):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lbks.lbks_cd_step(prec, nx, ny, nz, no, w.h, w.theta, 0.5 * dt, a, b, V, L, None, c, S, L, stream=stream)
            e1.record(stream)
            stream.synchronize()
            if it >= 3:
                total += e0.elapsed_time(e1)
    return total / launches, no * nx * ny * nz


def main_dynamics(args):
    """Concurrent dynamics of methane from a stretched geometry: the SCF
    ground state there (untimed), then bench steps of CD_BLOCKS x CD_NPOT
    real-time steps with the potential rebuilt and the nuclei moved after
    every CD_NPOT steps.  value: orbital-site updates of the real-time steps
    per second of the whole run (rebuilds, forces and moves included)."""
    import torch
    from paper_1507_07666_gb300 import build as build_mod
    build_mod.build()
    from paper_1507_07666_gb300 import lbks
    w = DYNAMICS[args.workload]()
    prec = {"fp32": lbks.FP32, "fp64": lbks.FP64, "bf16": lbks.FP32}[args.precision]
    sysm = lbks.System(w.n, w.h, w.n_orb, precision=prec, n_inner=w.n_inner, e_tol=w.e_tol, theta=w.theta,
                       storage=lbks.STORE_PSI)
    sysm.set_geometry(w.molecule.xyz, w.molecule.Z)
    gs = sysm.scf()
    M = W.masses(w.molecule)
    e_start, n_el = sysm.cd_start(n_pot=CD_NPOT)
    vel = np.zeros((len(M), 3))
    energies = []
    for _ in range(args.warmup):
        vel, e, _ = sysm.cd_run(CD_BLOCKS, masses=M, velocities=vel)
        energies.append(e)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    l0 = lbks.lbks_kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vel, e, traj = sysm.cd_run(CD_BLOCKS, masses=M, velocities=vel)
        energies.append(e)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    clk = clocks.stop()
    launches = lbks.lbks_kernel_launches() - l0
    st = sysm.cd_state()
    e_all = np.concatenate(energies)
    total = e_all[:, 0] + e_all[:, 1]
    R = traj[-1]
    r_ch = float(np.mean(np.linalg.norm(R[1:] - R[0], axis=1)))
    sysm.close()
    updates = args.steps * CD_BLOCKS * CD_NPOT * w.n_orb * w.sites
    ms, units = time_cd_step(torch, lbks, w, prec)
    pe = 8 if prec == lbks.FP64 else 4
    per_site = 6 * pe + 8.0 / w.n_orb  # prev and cur read, next written (complex), V once per site
    peak, peak_kind = measured_hbm_peak()
    achieved = per_site * units / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": updates / elapsed / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == lbks.FP64 else "f32", "data": "synthetic",
        "config": {"workload": f"concurrent dynamics (Eq. KSLBCD, Ehrenfest nuclei) of {w.name} from its ground "
                               f"state, {CD_BLOCKS} blocks x {CD_NPOT} steps per bench step, tau = theta h^2 / 2",
                   "grid": list(w.n), "n_orb": w.n_orb,
                   "l2": "levels larger than L2 (3 complex levels %.2f GB)" % (3 * 2 * pe * w.n_orb * w.sites / 1e9),
                   "timing": "wall clock around synchronous lbks_cd_run calls (device synchronised on both sides)"},
        "dynamics": {"ground_state_E": gs["E_total"], "ground_state_cycles": gs["cycles"], "E_start": e_start,
                     "n_electrons": n_el, "time_au": st["time"], "steps": st["steps"],
                     "max_abs_drift_E_total_plus_E_kin_Ha": float(np.abs(total - total[0]).max()),
                     "E_kin_nuclei_end": float(e_all[-1, 1]), "mean_r_CH_end": r_ch},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_cd_step", "bytes_per_launch": per_site * units,
                     "ms_per_launch": ms, "peak_source": f"hbm_gbs of {peak_kind}"},
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        code = ORACLE_CD_SAMPLE.format(root=ROOT, wl=DYNAMICS[args.workload].__name__, seconds=args.cpu_seconds)
        env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
        if r.returncode == 0:
            smp = json.loads(r.stdout.strip().splitlines()[-1])
            v, nsteps, t = oracle_rate([smp])
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"{nsteps} oracle steps (oracle.cd.cd_step) of {w.name}, one FP64 "
                                              f"numpy process, {t:.1f} s"}
    print(json.dumps(line), flush=True)
    return 0


def main_lbks(args):
    import torch
    rank, world, local_rank = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1507_07666_gb300 import build as build_mod
    if rank == 0:
        build_mod.build()
    if dist:
        dist.barrier()
    from paper_1507_07666_gb300 import lbks

    per_cycle = args.workload in CYCLES
    w = (CYCLES if per_cycle else WORKLOADS)[args.workload]()
    prec = {"fp32": lbks.FP32, "fp64": lbks.FP64, "bf16": lbks.BF16}[args.precision]
    psi_mode = args.storage == "psi"
    sysm = lbks.System(w.n, w.h, w.n_orb, precision=prec, n_inner=w.n_inner, e_tol=w.e_tol, theta=w.theta,
                       omega=w.omega, mix=w.mix, max_cycles=w.max_cycles,
                       storage=lbks.STORE_PSI if psi_mode else lbks.STORE_POPULATIONS,
                       poisson_adapt=args.poisson_adapt)
    xyz, Z = w.molecule.xyz, w.molecule.Z
    N = w.sites
    stream = torch.cuda.Stream()

    def solve():
        if per_cycle:
            return sysm.scf_cycles(1, stream)
        sysm.set_geometry(xyz, Z)
        return sysm.scf(stream)

    if per_cycle:
        sysm.set_geometry(xyz, Z)
    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = lbks.lbks_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    results = [solve() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = lbks.lbks_kernel_launches() - l0
    updates, elapsed_s = job_totals(dist, "cuda", sum(r["steps"] for r in results) * w.n_orb * N,
                                    ev0.elapsed_time(ev1) / 1e3)
    elapsed_ms = 1e3 * elapsed_s
    value = updates / elapsed_s / 1e9

    # end to end: host geometry in, energies + density back to the host
    e2e_updates, t_e2e = 0, 0.0
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        sysm.set_geometry(xyz, Z)
        r = sysm.scf_cycles(1, stream) if per_cycle else sysm.scf(stream)
        rho = sysm.density()
        t_e2e += time.perf_counter() - t0
        e2e_updates += r["steps"] * w.n_orb * N
    e2e_updates, t_e2e = job_totals(dist, "cuda", e2e_updates, t_e2e)
    e2e = {"value": e2e_updates / t_e2e / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(xyz.nbytes + Z.nbytes),
           "d2h_bytes_per_step": int(rho.nbytes + 8 * (8 + 2 * w.n_orb + 8))}

    tuned = lbks.lbks_get_relax_variant(sysm.handle)
    tuned_index = tuned["index"]
    psi_shape = None
    if psi_mode:  # orbital storage names its kernels differently
        tuned = {"variant": ("tiled", "direct", "tma", "zmarch")[tuned["index"]], "ms_tiled": tuned["ms_sites"],
                 "ms_direct": tuned["ms_pairs"], "ms_tma": tuned["ms_prefetch"], "ms_zmarch": tuned["ms_bulk"]}
        if tuned_index == 0 and w.n_orb <= 8:  # the staged stencil: its tuned tile shape
            psi_tile = lbks.lbks_get_psi_tile(sysm.handle)
            psi_shape = psi_tile["shape"]
            tuned["tile"] = {"shape": psi_shape, "sites": list(lbks.PSI_TILES[psi_shape]),
                             "sites_per_thread": lbks.PSI_TILE_SITES_PER_THREAD[psi_shape],
                             "plane_sums": lbks.PSI_TILE_PLANE_SUMS[psi_shape]}
    sysm.close()  # the kernel timing below allocates its own population pair

    # dominant kernel alone, same launch configuration
    elem = {lbks.FP32: 4, lbks.FP64: 8, lbks.BF16: 2}[prec]
    wide = w.n_orb > 8
    psi_elem = 8 if prec == lbks.FP64 else 4
    gram_name = "k_gram_wide" if prec == lbks.FP64 else "k_gram_tc"
    if psi_mode:
        # orbital storage: the step the solver runs (its tuned kernel), timed
        # through lbks_relax_step_psi with that kernel forced
        ms, units = time_relax_psi(torch, lbks, w, prec, stream, mode=1 + tuned_index, shape=psi_shape)
        N = units // w.n_orb
        kname, per_site = psi_step_kernels(w, psi_elem, tuned_index)
        bytes_per_launch = per_site * N
    else:
        ms, units = time_stream_collide(torch, lbks, w, prec, stream)
        # more than eight orbitals: the timed step is two kernels, stream-collide
        # and the overlap (Gram) kernel that reads the orbitals it wrote back
        bytes_per_launch = (38 * elem + (2 * psi_elem if wide else 0)) * units
        sc_name = {1: "k_stream_collide_pair", 3: "k_stream_collide_bulk"}.get(tuned_index, "k_stream_collide")
        if wide:
            sc_name = {1: "k_stream_collide_wide_pair", 3: "k_stream_collide_bulk"}.get(tuned_index,
                                                                                        "k_stream_collide_wide")
        kname = ("%s + %s (one relaxation step)" % (sc_name, gram_name)) if wide else sc_name
    peak, peak_kind = measured_hbm_peak()
    achieved = bytes_per_launch / (ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if psi_mode else
                (recorded_wide_traffic(units, tuned_index) if wide and prec == lbks.FP32 else
                 None if wide or tuned_index != 0 else recorded_traffic()),
                "kernel": kname,
                "bytes_per_launch": bytes_per_launch, "ms_per_launch": ms,
                "peak_source": f"hbm_gbs of {peak_kind}"}

    if rank != 0:
        return 0
    last = results[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {lbks.FP32: "f32", lbks.FP64: "f64", lbks.BF16: "bf16-storage/f32"}[prec],
        "data": "synthetic",
        "config": {"workload": w.name + (" SCF cycles (one per step, from the superposition start)" if per_cycle
                                          else " single solve"), "grid": list(w.n), "h": w.h, "n_orb": w.n_orb,
                   "precision": {lbks.FP32: "FP32 populations and collide, FP64 overlaps/energies/Poisson",
                                 lbks.FP64: "FP64 throughout",
                                 lbks.BF16: "BF16 populations, FP32 collide, FP32 polish below |dE| 1e-4, "
                                            "FP64 overlaps/energies/Poisson"}[prec],
                   "n_inner": w.n_inner, "e_tol": w.e_tol, "storage": args.storage,
                   "poisson_adapt": args.poisson_adapt,
                   "l2": ("orbital storage: a solve's working set (psi pair, W field, potentials, Poisson vectors) "
                          "exceeds L2; the kernel timing writes 256 MB before every timed launch") if psi_mode else
                         "inputs larger than L2 (populations %.2f GB)" % (2 * 19 * elem * units / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "solves_per_s": world * args.steps / (elapsed_ms / 1e3),
        "solve": {"E_total": last["E_total"], "eigenvalues": [float(x) for x in last["eigenvalues"]],
                  "cycles": last["cycles"], "steps": last["steps"], "converged": last["converged"],
                  "poisson_iters": last["poisson_iters"], "poisson_s": last["poisson_s"],
                  "poisson_share": last["poisson_s"] / last["wall_s"] if last["wall_s"] > 0 else None},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "roofline": roofline,
        "stream_collide_variant": tuned,
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return main_reference(args)
    if args.kernel_only:
        return main_kernel_only(args)
    if args.relax_variant:
        from paper_1507_07666_gb300 import build as build_mod
        build_mod.build()
        from paper_1507_07666_gb300 import lbks
        lbks.lbks_set_relax_variant(args.relax_variant)
    if args.workload in BATCHES:
        return main_batch(args)
    if args.workload in SERVING:
        return main_serving(args)
    if args.workload in RELAXATIONS:
        return main_relax(args)
    if args.workload in DYNAMICS:
        return main_dynamics(args)
    return main_lbks(args)


if __name__ == "__main__":
    sys.exit(main())
