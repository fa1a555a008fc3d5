"""Benchmark of the coupled LB + Q-tensor step (MLUPS and HBM roofline fraction).

Default workload: 256^3 periodic lattice, BPII unit cells of pitch 32
(q0 = 2 pi / 32), A0 = 0.01, gamma = 3.1, K = 0.01, Gamma = 0.3, xi = 0.7,
tau_f = 2, flow on, Jacobi coupling, FP32 state (FP64 only in diagnostics).
A step is one coupled update of every site.  The state (4.5 GB) is far larger
than L2 (129 MB), so no L2 flush is needed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(a deliberately slow, plain implementation) on the host cores instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 256
Q0 = 2 * np.pi / 32
PARAMS = dict(A0=0.01, gamma=3.1, K=0.01, q0=Q0, Gamma=0.3, xi=0.7, tau_f=2.0)
SEED = 20090119
# algorithmic FP32 bytes per site of each kernel: each value the kernel must
# read or write once (inputs + outputs)
KERNEL_BYTES = {
    # fast path (z-marching, TMA-staged planes)
    "qside": (5 + 4 + 16) * 4,                                 # Q, rho u -> scratch (P, Q*, rho - 1)
    "lbq": (15 + 16 + 4 + 5 + 15 + 4 + 5) * 4,                 # f, scratch, rho u, Q -> f, rho u, Q
    # generic path
    "field": (5 + 5 + 5 + 3) * 4,                              # Q -> H, sigma, tau
    "force_predict": (5 + 5 + 3 + 4 + 3 + 5) * 4,              # Q, H, tau, rho u -> b, Q*
    "lb_correct": (15 + 4 + 5 + 3 + 5 + 5 + 15 + 4 + 5) * 4,   # f, rho u, sigma, b, Q*, Q -> f, rho u, Q
}
KERNELS_FAST = ["qside", "lbq"]
KERNELS_GENERIC = ["field", "force_predict", "lb_correct"]
STATE_BYTES = (15 + 5) * 2 * 4  # read + write of f and Q once per site-step (FP32)
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth (the measured copy peak is the roofline)
# DRAM bytes per site of one launch of each fast kernel (dram__bytes_read.sum +
# dram__bytes_write.sum), from an ncu capture of 160^3 FP32 with its own
# tuning (planes per CTA: k_lbq 9, k_qside 54; one site per thread);
# summary and command in profiles/step_256cube_fast_path.md.  Traffic per
# launch scales with the sites.  Valid only for the kernel sources it was
# taken on (hash below); otherwise null.
MEASURED_TRAFFIC = {
    "sources": ["paper_0901_3293_gb300/csrc/zmarch.cu", "paper_0901_3293_gb300/csrc/common.cuh",
                "paper_0901_3293_gb300/csrc/tma.cuh", "paper_0901_3293_gb300/csrc/kernels.h"],
    "sha256_16": "83a89e0b63237421",
    # one launch of each kernel in the capture (ncu --set full)
    "bytes_per_site": {"qside": (181522432 + 211604224) / 160 ** 3,
                       "lbq": (772152320 + 364112384) / 160 ** 3},
    # smsp__inst_executed.sum (warp instructions) x 32 of the same launches
    "thread_instr_per_site": {"qside": 101004852 * 32 / 160 ** 3, "lbq": 118693712 * 32 / 160 ** 3},
}
ORACLE_SAMPLE = 32  # side of the periodic cube the oracle steps (two BPII unit cells)
WALL_Q = (0.2, 0.0, 0.0, -0.1, 0.0)  # planar anchoring S (x x - I/3), S = 0.3, on the ghost planes


def measured_traffic_per_site(kernel: str):
    """ncu DRAM bytes per site of `kernel`, or None if its sources changed since the capture."""
    import hashlib
    h = hashlib.sha256()
    for f in MEASURED_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != MEASURED_TRAFFIC["sha256_16"]:
        return None
    return MEASURED_TRAFFIC["bytes_per_site"].get(kernel)


def measured_instr_per_site(kernel: str):
    """ncu thread instructions per site of `kernel`, or None if its sources changed since the capture."""
    if measured_traffic_per_site(kernel) is None:
        return None
    return MEASURED_TRAFFIC["thread_instr_per_site"].get(kernel)


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Ranks:
    """The ranks of one run: a barrier and the max over ranks of a timing.
    device "cuda" (NCCL, the bench) or "cpu" (gloo); world 1 needs no process group."""

    def __init__(self, world: int, device: str = "cuda"):
        self.world, self.device = world, device

    def barrier(self) -> None:
        import torch
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
        if self.device == "cuda":
            torch.cuda.synchronize()

    def allmax(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], device=self.device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_mlups(sites_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Replicas: every rank steps its own lattice, so the job advances world x
    sites_per_rank sites per step in the slowest rank's time."""
    return sites_per_rank * steps * world / (ms_max * 1e-3) / 1e6


# multiply-accumulates per site of one surrogate call: conv 15->32, eight 32->32, 32->5 (3^3 taps)
SURROGATE_MAC_PER_SITE = 27 * (15 * 32 + 8 * 32 * 32 + 32 * 5)


def measured_bf16_peak():
    """Dense BF16 TFLOP/s: the measured burst figure (a call is short), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["bf16_tflops"]), "measured burst (MEASURED_PEAKS.json bf16_tflops)"
    return 1900.0, "fallback"


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample_mlups(steps: int, warmup: int = 1, start_at: float = 0.0):
    """FP64 oracle on a periodic 32^3 cube of the same BPII state (two unit
    cells per side), timed on one host core.  The timed loop starts no earlier
    than the wall-clock time start_at, so that concurrent copies overlap.
    Returns (MLUPS, seconds)."""
    from oracle import initial, lbq
    p = lbq.Params(**PARAMS)
    shape = (ORACLE_SAMPLE,) * 3
    Q = initial.init_q9(shape, initial.BPII, p.q0, 0.3, 1e-4, SEED)
    f = lbq.init_f_equilibrium(Q, p)
    for _ in range(warmup):
        f, Q = lbq.step(f, Q, p)
    while time.time() < start_at:
        time.sleep(0.01)
    t0 = time.perf_counter()
    for _ in range(steps):
        f, Q = lbq.step(f, Q, p)
    dt = time.perf_counter() - t0
    return ORACLE_SAMPLE ** 3 * steps / dt / 1e6, dt


def oracle_in_subprocess(steps: int, warmup: int = 1, copies: int = 1):
    """The oracle timed in child processes whose math libraries use one thread
    each: `copies` independent samples stepped at the same time, one per core.
    Returns (MLUPS of all copies together, seconds of the slowest copy)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    start_at = time.time() + (0.0 if copies == 1 else 5.0 + 0.05 * copies)
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "m, dt = bench.oracle_sample_mlups(%d, %d, %r); print(json.dumps([m, dt]))"
            % (ROOT, steps, warmup, start_at))
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                              text=True) for _ in range(copies)]
    dts = []
    for pr in procs:
        out, err = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError(f"oracle sample failed: {err.strip()[-400:]}")
        dts.append(json.loads(out.strip().splitlines()[-1])[1])
    dt = max(dts)
    return copies * ORACLE_SAMPLE ** 3 * steps / dt / 1e6, dt


def host_cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline_entry(steps: int):
    m, dt = oracle_in_subprocess(steps)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    entry = {"value": m, "unit": "MLUPS", "cores": 1, "kind": "oracle",
             "sample": f"{steps} FP64 oracle steps of a periodic {ORACLE_SAMPLE}^3 cube of the same BPII "
                       f"(pitch 32) state, {dt:.1f} s on one host core (numpy, threads pinned to 1)",
             "host": f"{host_cpu_model()}, {cores} cores"}
    if cores > 1:
        ma, dta = oracle_in_subprocess(steps, copies=cores)
        entry["all_cores"] = {"value": ma, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                              "sample": f"{cores} independent copies of the same sample stepped at once, one per "
                                        f"core; the slowest took {dta:.1f} s"}
    return entry


def workload_config(world: int) -> dict:
    """The timed workload, shared by both arms' JSON lines."""
    return {"workload": f"{N_SIDE}^3 periodic BPII (pitch 32), coupled D3Q15 LB + Beris-Edwards, FP32 state",
            "sites_per_gpu": N_SIDE ** 3, "A0": PARAMS["A0"], "gamma": PARAMS["gamma"], "K": PARAMS["K"],
            "q0": PARAMS["q0"], "tau_f": PARAMS["tau_f"], "l2": "state 4.5 GB >> 129 MB L2, no flush",
            "parallelism": f"{world} independent replicas" if world > 1 else "single lattice"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    mlups, dt = oracle_in_subprocess(args.steps, args.warmup)
    line = {
        "impl": "reference", "metric": "coupled LB+Q MLUPS", "value": mlups, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(world),
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"each step is one FP64 oracle step of a periodic {ORACLE_SAMPLE}^3 cube of "
                                   f"the same BPII (pitch 32) state (numpy, one thread); MLUPS scale with sites"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_0901_3293_gb300 import build, lcbp
    if not os.path.exists(lcbp.LIB_PATH):
        build.build()
    dev = torch.cuda.current_device()
    ranks = Ranks(world, "cuda")
    barrier, allmax = ranks.barrier, ranks.allmax

    # every rank holds its own independent 256^3 lattice (replicas: no data exchange)
    n = N_SIDE
    lat = lcbp.Lattice(n, n, n, dtype="f32")
    lat.set_ldg(PARAMS["A0"], PARAMS["gamma"], PARAMS["K"], PARAMS["q0"])
    lat.set_flow(PARAMS["tau_f"], PARAMS["xi"], PARAMS["Gamma"], True, lcbp.JACOBI)
    lat.init_q(lcbp.BPII, 0.3, noise=1e-4, seed=SEED + rank)
    lat.init_f_equilibrium(1.0)
    stream = lat._stream
    lat.step(args.warmup)
    lat.synchronize()

    # ---- timed region: K steps (CUDA-graph replay) on the lattice's stream
    clocks = ClockSampler(dev)
    time.sleep(0.3)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = allmax(e0.elapsed_time(e1))
    sites = n ** 3
    mlups = whole_job_mlups(sites, args.steps, world, ms)
    F = lat.free_energy()  # FP64 diagnostics also check the state is finite
    # the diagnostics pass (row a7): F_h with the defect and non-finite counts,
    # then mass and momentum (f read too), host-timed per call
    t0 = time.perf_counter()
    for _ in range(5):
        lat.free_energy()
    t_F = (time.perf_counter() - t0) / 5
    t0 = time.perf_counter()
    for _ in range(5):
        lat.totals()
    t_tot = (time.perf_counter() - t0) / 5
    diag_line = {"free_energy_ms": 1e3 * t_F, "totals_ms": 1e3 * t_tot,
                 "note": "host-timed lcbp_free_energy / lcbp_totals calls (one pass each, FP64 sums, "
                         "result copy and synchronisation included)"}

    # ---- per-kernel device times, kernel by kernel with events (same kernels)
    kms = lat.profile_steps(max(3, min(args.steps, 10)))
    fast, zc, spt = lat.path()
    zc_lbq, spt_lbq, spt_qside, zc_qside = lat.tuning()
    peak, peak_kind = measured_peaks()
    per_kernel = {}
    # instruction-issue peak: one warp instruction per scheduler per cycle, 4 schedulers per
    # SM, at the SM clock median measured under load (else the maximum)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_hz = 1e6 * (clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0)
    issue_peak = sms * 4 * sm_hz * 32  # thread instructions per second
    for name, t in zip(KERNELS_FAST if fast else KERNELS_GENERIC, kms):
        gbs = KERNEL_BYTES[name] * sites / (t * 1e-3) / 1e9
        per_kernel[name] = {"ms": t, "algorithmic_bytes_per_site": KERNEL_BYTES[name], "GBps": gbs,
                            "frac_of_" + peak_kind: gbs / peak}
        ips = measured_instr_per_site(name) if fast else None
        if ips:
            per_kernel[name]["thread_instr_per_site"] = ips
            per_kernel[name]["frac_of_issue_peak"] = ips * sites / (t * 1e-3) / issue_peak
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    tps = measured_traffic_per_site(dom) if fast else None
    roof = {"bound": "hbm", "achieved": per_kernel[dom]["GBps"], "peak": peak, "unit": "GB/s",
            "frac": per_kernel[dom]["GBps"] / peak, "traffic": tps * sites if tps else None,
            "traffic_note": "ncu DRAM bytes per launch, captured on 160^3 and scaled by sites" if tps else
            "no capture for these kernel sources", "kernel": dom,
            "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs, burst copy)",
            "step_algorithmic_frac": STATE_BYTES * sites * args.steps / (ms * 1e-3) / 1e9 / peak,
            "frac_of_nominal": per_kernel[dom]["GBps"] / HBM_NOMINAL_GBS, "nominal_peak": HBM_NOMINAL_GBS,
            "note": "step_algorithmic_frac counts only the 160 B/site of reading and writing f and Q once; "
                    "frac_of_nominal is against the 7.9 TB/s HBM3e data-sheet figure"}

    # ---- end to end through the C ABI with pinned host buffers: upload f and Q,
    # one step, read back Q and u, every step
    k_e2e = max(2, min(args.steps, 8))
    f_h = torch.empty((15, n, n, n), dtype=torch.float32, pin_memory=True)
    q_h = torch.empty((5, n, n, n), dtype=torch.float32, pin_memory=True)
    u_h = torch.empty((3, n, n, n), dtype=torch.float32, pin_memory=True)
    lat.read_f(out=f_h)
    lat.read_q(out=q_h)

    def e2e_step():
        lat.set_f(f_h)
        lat.set_q(q_h)
        lat.step(1)
        lat.read_q(out=q_h)
        lat.read_u(out=u_h)

    for _ in range(4):  # untimed: the first copies through freshly pinned buffers run slow
        e2e_step()
    # three timed windows of k_e2e steps each; the host link is shared, so the
    # median window is reported and all three are listed
    windows = []
    for _ in range(3):
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            e2e_step()
        barrier()
        windows.append(sites * k_e2e * world / allmax(time.perf_counter() - t0) / 1e6)
    e2e = {"value": sorted(windows)[1], "unit": "MLUPS",
           "h2d_bytes_per_step": (15 + 5) * 4 * sites, "d2h_bytes_per_step": (5 + 3) * 4 * sites,
           "steps": k_e2e, "warmup": 4, "windows": windows,
           "note": "median of three windows of `steps` steps, each step lcbp_set_f + lcbp_set_q from pinned host "
                   "memory, lcbp_step(1), lcbp_read_q + lcbp_read_u to pinned host memory"}
    launches = (2 if fast else 3) * args.steps

    # ---- the same lattice between walls in z (half-way bounce-back, Q anchored
    # to a planar q_wall on the ghost planes): the walled build of the kernels
    lat.set_walls(True, WALL_Q)
    lat.step(max(3, args.warmup))  # tunes the walled build
    lat.synchronize()
    w0 = torch.cuda.Event(enable_timing=True)
    w1 = torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    lat.step(args.steps)
    w1.record(stream)
    w1.synchronize()
    walls_ms = w0.elapsed_time(w1)
    wfast, wzc, wspt = lat.path()
    wkms = lat.profile_steps(max(3, min(args.steps, 10)))
    walls_line = {"ms_per_step": walls_ms / args.steps, "MLUPS": sites * args.steps / (walls_ms * 1e-3) / 1e6,
                  "fast_path": wfast, "planes_per_cta": wzc, "sites_per_thread": wspt,
                  "per_kernel": {name: {"ms": t, "GBps": KERNEL_BYTES[name] * sites / (t * 1e-3) / 1e9,
                                        "frac_of_" + peak_kind: KERNEL_BYTES[name] * sites / (t * 1e-3) / 1e9 / peak}
                                 for name, t in zip(KERNELS_FAST if wfast else KERNELS_GENERIC, wkms)},
                  "q_wall": list(WALL_Q)}

    # ---- the same periodic lattice on the generic kernels (one thread per
    # site, neighbours through L1/L2), which serve the modes the fast path
    # does not (Gauss-Seidel coupling, flow off, L2 != K, nx % 4 != 0)
    lat.set_walls(False)
    lat.set_path(lcbp.PATH_GENERIC)
    lat.step(3)
    lat.synchronize()
    gkms = lat.profile_steps(max(3, min(args.steps, 10)))
    generic_line = {"ms_per_step": sum(gkms), "MLUPS": sites / (sum(gkms) * 1e-3) / 1e6,
                    "per_kernel": {name: {"ms": t, "algorithmic_bytes_per_site": KERNEL_BYTES[name],
                                          "GBps": KERNEL_BYTES[name] * sites / (t * 1e-3) / 1e9,
                                          "frac_of_" + peak_kind: KERNEL_BYTES[name] * sites / (t * 1e-3) / 1e9 / peak}
                                   for name, t in zip(KERNELS_GENERIC, gkms)},
                    "note": "per-kernel event times of lcbp_profile_steps; eager launches"}
    lat.close()

    # ---- the 64x64x256 thin slab (BPII seed for z < 32 inside an x-helix)
    slab = lcbp.Lattice(64, 64, 256, dtype="f32")
    slab.set_ldg_kappa_tau(0.01, 2 * np.pi / 16, 1.0, -0.5)
    slab.set_flow(2.0, 0.7, 0.3, True, lcbp.JACOBI)
    slab.init_q(lcbp.SLAB_BPII_IN_CHOL, 0.3, noise=1e-4, seed=SEED, z0=32)
    slab.init_f_equilibrium(1.0)
    slab.step(max(3, args.warmup))
    slab.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(slab._stream)
    slab.step(args.steps)
    s1.record(slab._stream)
    s1.synchronize()
    slab_ms = s0.elapsed_time(s1)
    slab_line = {"sites": 64 * 64 * 256, "ms_per_step": slab_ms / args.steps,
                 "MLUPS": 64 * 64 * 256 * args.steps / (slab_ms * 1e-3) / 1e6,
                 "note": "state (168 MB) partly L2-resident; not the headline"}
    slab.close()

    # ---- the learned surrogate on the same slab: one call (k = 50 steps' worth
    # of Q change: input packing, ten tensor-core convolutions, Q update)
    # against 50 plain steps, then time to solution of the judged run with the
    # shipped weights against the plain solver (20000 steps, F and the defect
    # fraction logged every 100 steps by both, kappa = 1)
    from paper_0901_3293_gb300 import surrogate_train as st
    k_sur = 50
    t_call, t_plain_k = st.time_call(reps=max(10, min(args.steps, 50)), k=k_sur)
    sur_flop = 2.0 * SURROGATE_MAC_PER_SITE * 64 * 64 * 256
    bf16_peak = measured_bf16_peak()
    weights = os.path.join(ROOT, "paper_0901_3293_gb300", "weights", "slab_k50.lcbpsur")
    run_steps = 20000
    rows, t_plain_run = st.plain_log(1.0, run_steps)
    F_plain = {t: F for t, F, _ in rows}
    jrows, jst, t_judged = st.judged_log(None, 1.0, run_steps, k_sur, 24, 3e-4, weights=weights, warmup=1000)
    f_err = max(abs(F - F_plain[t]) / abs(F_plain[t]) for t, F, _ in jrows)
    sur_line = {"ms_per_call": t_call, "steps_per_call": k_sur, "plain_steps_ms": t_plain_k,
                "speedup_per_call": t_plain_k / t_call,
                "network_tflops": sur_flop / (t_call * 1e-3) / 1e12,
                "frac_of_bf16_peak": sur_flop / (t_call * 1e-3) / 1e12 / bf16_peak[0],
                "bf16_peak": {"tflops": bf16_peak[0], "source": bf16_peak[1]},
                "time_to_solution": {"steps": run_steps, "kappa": 1.0, "plain_s": t_plain_run,
                                     "judged_s": t_judged, "speedup": t_plain_run / t_judged,
                                     "max_rel_F_error_every_100_steps": f_err,
                                     "surrogate_share_of_steps": jst["surrogate_calls"] * k_sur / run_steps,
                                     "segments": jst["segments"], "fallbacks": jst["fallbacks"],
                                     "judge": "24 calls per segment, tol_F 3e-4, 1000 plain warm-up steps",
                                     "weights": "paper_0901_3293_gb300/weights/slab_k50.lcbpsur"},
                "note": "call host-timed over repeated calls (untrained parameters: the arithmetic is the "
                        "same); network FLOPs use the true channel counts (238464 MAC/site); conv kernels are "
                        "the window kernel; both runs are host-timed end to end"}

    # ---- the polarised-light texture of the slab (Sec. 2.3): one image of the
    # current Q (64 x 64 columns of 256 planes, three wavelengths)
    tex_lat = st.slab_lattice(1.0)
    tex_lat.step(20)
    tex_lat.texture()
    tex_lat.synchronize()
    t0 = time.perf_counter()
    for _ in range(20):
        tex_lat.texture()
    tex_ms = 1e3 * (time.perf_counter() - t0) / 20
    tex_line = {"ms_per_image": tex_ms, "sites": 64 * 64 * 256,
                "GBps_of_Q": 64 * 64 * 256 * 5 * 4 / (tex_ms * 1e-3) / 1e9,
                "note": "host-timed lcbp_texture (the column-product kernel, split over z into 3 ranges for "
                        "this 64 x 64 image, the combine kernel and the 16 KB image copy); reads Q (20 B/site) once"}
    tex_lat.close()

    # ---- the 48-replica sweep (32^3 / 48^3, per-replica kappa and tau) in one batch
    from paper_0901_3293_gb300 import workloads
    batch = workloads.replica_sweep_batch(48, SEED, "f32")
    batch.step(max(4, args.warmup))
    batch.synchronize()
    bsites = batch.info()["sites"]
    t0 = time.perf_counter()
    batch.step(args.steps)
    batch.synchronize()
    b_s = time.perf_counter() - t0
    binfo = batch.info()
    bfast, bzc = batch.path()
    # algorithmic bytes of one step per site: the two fast kernels, or the three generic ones
    b_bytes = (KERNEL_BYTES["qside"] + KERNEL_BYTES["lbq"]) if bfast else sum(
        KERNEL_BYTES[k] for k in KERNELS_GENERIC)
    b_gbps = b_bytes * bsites * args.steps / b_s / 1e9
    batch_line = {"replicas": 48, "sites": bsites, "ms_per_step": 1e3 * b_s / args.steps,
                  "MLUPS": bsites * args.steps / b_s / 1e6,
                  "algorithmic_bytes_per_site": b_bytes, "GBps": b_gbps, "frac_of_" + peak_kind: b_gbps / peak,
                  "kernels": "fast (z-marching TMA kernels, 5-D maps per class)" if bfast else "generic",
                  "planes_per_cta": bzc if bfast else None,
                  "tile": None if bfast else binfo["tile"],
                  "persistent_ctas": None if bfast else binfo["persistent_ctas"],
                  "note": "kernel set chosen by timing both on the batch; one launch per kernel over all "
                          "replicas, graph replay; host-timed around lcbp_batch_step + synchronize"}
    batch.close()

    if rank != 0:
        return
    cpu = cpu_baseline_entry(int(os.environ.get("LCBP_ORACLE_STEPS", "40")))
    line = {
        "metric": "coupled LB+Q MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {**workload_config(world),
                   "kernels": "fast (z-marching, TMA-staged planes)" if fast else "generic",
                   "planes_per_cta": {"lbq": zc_lbq, "qside": zc_qside},
                   "sites_per_thread": {"lbq": spt_lbq, "qside": spt_qside}},
        "roofline": roof, "per_kernel": per_kernel, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk, "free_energy_after": F,
        "diagnostics_256cube": diag_line, "walls_256cube": walls_line, "generic_kernels_256cube": generic_line, "slab_64x64x256": slab_line, "surrogate_slab_64x64x256": sur_line, "texture_slab_64x64x256": tex_line,
        "batched_48_replicas": batch_line,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
