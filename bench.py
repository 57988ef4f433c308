#!/usr/bin/env python
"""Throughput of the stabilised DQMC Green's-function path on GB300.

Workload (default, ``n256_beta20``): 16x16 periodic square lattice (N=256),
t=1, U=4, dtau=0.1, beta=20 (M=200), k=10, a batch of 128 Hirsch +-1 field
configurations per GPU; one step = one dqmc_greens call over the batch:
exp(-dtau K), 200 slice products, 20 pivoted-QR re-factorisations, the Loh
inversion and the log det of every instance.  Metric: Green's functions per
second (whole job, all ranks).

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
For N > 1 launch under torch.distributed.run: every rank runs its own batch
(independent instances, no collective on the data path) and the slowest rank's
time sets the job time (weak scaling).

``--impl reference`` times the CPU oracle (NumPy/SciPy FP64, the paper's LAPACK
routines) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import dqmc_inputs as di  # noqa: E402

# FP64 rate of GB300 from its unit counts: 152 SMs x 2 DFMA per clock per SM
# (4 flop) x the 2070 MHz maximum SM clock.  Reported beside the measured
# figure (dqmc_selftest_fp64_rate), which is the roofline denominator.
FP64_DERIVED_TFLOPS = 152 * 4 * 2.070e9 / 1e12


def bf16_peak_tflops():
    """Dense bf16 rate of this machine's GB300 as measured by the pool's driver
    (sustained figure: the tensor-core product runs inside a long step), else
    an earlier sustained measurement of 1.7 PFLOP/s on a GB300."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]), "measured (bf16_tflops_sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


WORKLOADS = {
    # equal-time G + log det (the headline workload)
    "n256_beta20": dict(L=16, U=4.0, dtau=0.1, beta=20.0, k=10, batch=128, config=4),
    # G(tau_j, tau_j) and G(tau_j, 0) on the k-grid
    "tdisplaced_n64": dict(L=8, U=4.0, dtau=0.1, beta=40.0, k=10, batch=256, config=2),
    # log det + gradient for all N*M field entries (continuous field)
    "grad_n144": dict(L=12, g=1.5, dtau=0.1, beta=20.0, k=10, batch=64, config=5),
    # 1024 instances of uneven N and M in one call, k autotuned per N; recorded
    # once as a CUDA graph and replayed
    "ragged_1024": dict(batch=1024, config=3, graphs=True),
    # one small configuration: launch bound, so recorded once as a CUDA graph and replayed
    "n16_beta8": dict(L=4, U=4.0, dtau=0.1, beta=8.0, k=10, batch=1, config=1, graphs=True),
}


# metric and unit of each workload, the same in the GPU arm and the oracle arm
METRICS = {
    "n256_beta20": ("greens_functions_per_second", "G/s"),
    "tdisplaced_n64": ("tdisplaced_sets_per_second", "sets/s"),
    "grad_n144": ("logdet_gradients_per_second", "grads/s"),
    "ragged_1024": ("greens_functions_per_second", "G/s"),
    "n16_beta8": ("greens_functions_per_second", "G/s"),
}


FOLDS = {"sequential": 0, "tree": 1, "auto": 2}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="n256_beta20", choices=sorted(WORKLOADS))
    p.add_argument("--batch", type=int, default=None, help="override instances per GPU")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=8.0,
                   help="oracle seconds per CPU mode for the headline's cpu_baseline")
    p.add_argument("--workload-cpu-seconds", type=float, default=3.0,
                   help="oracle seconds per CPU mode for each entry of 'workloads'")
    p.add_argument("--cpu-mode", default="best", choices=["best", "pool", "threads"],
                   help="--impl reference: process pool (BLAS 1 thread each), one process with "
                        "threaded BLAS, or the faster of the two")
    p.add_argument("--no-workloads", action="store_true",
                   help="headline run only: skip the other BASELINE configurations")
    p.add_argument("--oracle-samples", type=int, default=2,
                   help="instances of the mixed-precision run checked against the CPU oracle")
    p.add_argument("--precision", default="fp64", choices=["fp64"] + [f"bf16x{i}" for i in range(3, 9)],
                   help="chain-product precision of the timed steps (QR and inversions stay FP64)")
    p.add_argument("--no-unshared", action="store_true",
                   help="skip the extra un-pipelined step that times the dominant kernel alone")
    p.add_argument("--graphs", default="auto", choices=["auto", "on", "off"],
                   help="CUDA-graph mode of the handle (auto: on for the launch-bound workloads)")
    p.add_argument("--fold", default="auto", choices=["auto", "tree", "sequential"],
                   help="equal-time chain fold of the handle (auto: tree for small batches)")
    p.add_argument("--gemm-tile", type=int, default=0, choices=[0, 32, 48, 64],
                   help="FP64 product tile edge (0: chosen by size)")
    p.add_argument("--mixed-slices", type=int, default=8,
                   help="also time the mixed chain with this many BF16 slices (0: skip)")
    return p.parse_args()


def make_inputs(wl: dict, rank: int, batch: int):
    """K and the (batch, M, N) fields of this rank's instances (disjoint seeds per rank)."""
    insts = [di.hubbard_instance(wl["L"], wl["U"], wl["dtau"], wl["beta"], wl["k"], sd)
             for sd in rank_seeds(wl, rank, batch)]
    return insts[0].K, np.stack([x.V for x in insts]), insts


def rank_seeds(wl: dict, rank: int, batch: int) -> list[int]:
    """Seeds of this rank's instances: rank r owns instances [r*batch, (r+1)*batch)."""
    return [di.instance_seed(wl["config"], rank * batch + i) for i in range(batch)]


def reduce_max(x: float, device=None) -> float:
    """Max over ranks of a local time (identity outside torch.distributed)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_value(batch: int, world: int, steps: int, max_ms: float) -> float:
    """Whole-job Green's functions per second: all ranks' instances / slowest rank's time."""
    return batch * world * steps / (max_ms / 1e3)


def flops_per_tdisplaced(N: int, M: int, k: int) -> float:
    """Two stacks + per grid point: 2 products for the middle matrix, LU with
    2N right-hand sides, 2 products for G(tau,tau) and G(tau,0)."""
    nc = -(-M // k)
    return (2 * (2.0 * M + nc * (8.0 / 3.0 + 1.0)) + (nc + 1) * (4 + 2.0 / 3.0 + 4 + 4)) * N ** 3


def flops_per_grad(N: int, M: int, k: int) -> float:
    """Two stacks + checkpoint G (2 products, LU, 1 product) + k-1 wraps (2 products
    each) per grid point + the log det."""
    nc = -(-M // k)
    return (2 * (2.0 * M + nc * (8.0 / 3.0 + 1.0)) + (nc + 1) * (4 + 2.0 / 3.0 + 2 + 2)
            + (nc + 1) * (k - 1) * 4 + 2 * (2.0 / 3.0) + 2.0) * N ** 3


def flops_tensor_chain(N: int, M: int, k: int, stacks: int = 1) -> float:
    """Of the counts above, the part the mixed-precision chain moves to the tensor
    cores: per stack, M slice products (2N^3) and ceil(M/k) X updates (N^3)."""
    return stacks * (2.0 * M + -(-M // k)) * N ** 3


def flops_per_greens(N: int, M: int, k: int) -> float:
    """Algorithmic FP64 flops of one G: 2MN^3 chain + ceil(M/k)(8/3 + 1)N^3 QR/update + Loh."""
    nc = -(-M // k)
    loh = 2 * (2.0 / 3.0 + 2.0)   # two LU solves with N right-hand sides
    return (2.0 * M + nc * (8.0 / 3.0 + 1.0) + loh) * N ** 3


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def kernel_source_hash(src: str = "gemm_f64.cu") -> str:
    h = hashlib.sha256()
    with open(os.path.join(ROOT, "paper_2003_05286_gb300", "csrc", src), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, record: str = "chain_gemm_traffic.json",
                     src: str = "gemm_f64.cu"):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary
    (profiles/<record>), or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", record)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get(workload)
    if not e or e.get("kernel_source_sha256_16") != kernel_source_hash(src):
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
def cpu_model() -> str:
    """Host CPU model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def oracle_sampler(name: str, n_inst: int = 4):
    """The oracle routine that matches a workload's metric, as one bounded CPU sample.

    Returns (run, what): ``run(i)`` computes sample i on the host
    cores and returns how many metric units it completed (a fraction for the
    gradient, whose slices the oracle computes one by one from scratch)."""
    from oracle import dqmc as od
    wl = WORKLOADS[name]
    if name == "ragged_1024":
        # the first RAGGED_SAMPLE instances of the workload itself, so that the
        # sample has the workload's mix of N and M (built on first use)
        insts = {}

        def run(i):
            j = i % RAGGED_SAMPLE
            if j not in insts:
                insts[j] = di.ragged_instance(j, 10)
            x = insts[j]
            od.greens(x.K, x.dtau, x.V, x.k)
            return 1.0
        return run, (f"equal-time G of instances i mod {RAGGED_SAMPLE} of the uneven-size "
                     f"workload (its own mix of N and M, k = 10)")
    if name == "grad_n144":
        insts = [di.gaussian_instance(wl["L"], wl["g"], wl["dtau"], wl["beta"], wl["k"], sd)
                 for sd in rank_seeds(wl, 0, n_inst)]
        M = insts[0].M
        per = 2                                   # slices l of dV per sample

        def run(i):
            x = insts[i % len(insts)]
            first = 1 + (per * i) % M
            od.logdet_grad(x.K, x.dtau, x.V, x.k,
                           slices=[(first - 1 + j) % M + 1 for j in range(per)])
            return per / M
        return run, f"{per} of the {M} slices of dV per sample, each G_l from scratch; " \
            f"a gradient counts as {M} slices"
    insts = [di.hubbard_instance(wl["L"], wl["U"], wl["dtau"], wl["beta"], wl["k"], sd)
             for sd in rank_seeds(wl, 0, n_inst)]
    if name == "tdisplaced_n64":
        def run(i):
            x = insts[i % len(insts)]
            od.greens_tdisplaced(x.K, x.dtau, x.V, x.k)
            return 1.0
        return run, "G(tau_j, tau_j) and G(tau_j, 0) on the k-grid of one instance per sample"

    def run(i):
        x = insts[i % len(insts)]
        od.greens(x.K, x.dtau, x.V, x.k)
        return 1.0
    return run, "equal-time G and log det of one instance per sample"


def cpu_rate_threads(name: str, seconds: float):
    """Mode B: samples one after another in this process, BLAS on all cores."""
    run, what = oracle_sampler(name)
    run(0)                                        # warm-up (imports, first-call costs)
    t0 = time.perf_counter()
    n, units = 0, 0.0
    while True:
        units += run(1 + n)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return units / dt, n, dt, what


_POOL_SAMPLERS = {}
RAGGED_SAMPLE = 64      # instances of the ragged workload in its CPU sample


def _pool_run(name: str):
    if name not in _POOL_SAMPLERS:
        _POOL_SAMPLERS[name] = oracle_sampler(name)[0]
    return _POOL_SAMPLERS[name]


def _pool_init():
    # first-call costs (imports, LAPACK set-up) on a tiny problem, outside any timing
    from oracle import dqmc as od
    inst = di.hubbard_instance(2, 4.0, 0.1, 0.5, 5, 1)
    od.greens(inst.K, inst.dtau, inst.V, inst.k)


def _pool_sample(job) -> float:
    name, i = job
    return _pool_run(name)(i)


def _pool_timed(job):
    """One worker of mode A: samples until `seconds` pass; (units, seconds, samples)."""
    name, first, stride, seconds = job
    run = _pool_run(name)
    t0 = time.perf_counter()
    n, units = 0, 0.0
    while True:
        units += run(first + n * stride)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return units, time.perf_counter() - t0, n


class OraclePool:
    """Mode A: one process per host core, each with single-threaded BLAS.

    Started with 'spawn' (a forked child of a process that has touched the GPU
    can hang); BLAS thread counts are set through the environment the children
    inherit, before their NumPy loads."""
    ENV = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")

    def __init__(self, cores: int):
        import multiprocessing as mp
        self.cores = cores
        old = {k: os.environ.get(k) for k in self.ENV}
        for k in self.ENV:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(cores, initializer=_pool_init)
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def round(self, name: str, first: int) -> float:
        """One sample per worker (samples first .. first + cores - 1); units done."""
        return sum(self.pool.map(_pool_sample, [(name, i) for i in range(first, first + self.cores)],
                                 chunksize=1))

    def timed(self, name: str, seconds: float):
        if name == "ragged_1024":
            # every instance of the sample once (their costs differ by ~100x,
            # so a time budget per process would bias the mix)
            t0 = time.perf_counter()
            units = sum(self.pool.map(_pool_sample, [(name, i) for i in range(RAGGED_SAMPLE)],
                                      chunksize=1))
            wall = time.perf_counter() - t0
            return units / wall, RAGGED_SAMPLE, wall
        res = self.pool.map(_pool_timed, [(name, w, self.cores, seconds)
                                          for w in range(self.cores)], chunksize=1)
        units = sum(r[0] for r in res)
        wall = max(r[1] for r in res)
        return units / wall, sum(r[2] for r in res), wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline_line(name: str, seconds: float, pool: "OraclePool | None" = None) -> dict:
    """The oracle on the host cores for about ``seconds`` in each of two modes
    (A: a process per core, BLAS threads = 1; B: one process, BLAS threads =
    all cores); the better mode is the baseline and both are reported."""
    unit = METRICS[name][1]
    cores = os.cpu_count() or 1
    rb, nb, dtb, what = cpu_rate_threads(name, seconds)
    own = pool is None
    if own:
        pool = OraclePool(cores)
    try:
        ra, na, dta = pool.timed(name, seconds)
    finally:
        if own:
            pool.close()
    best = "A" if ra >= rb else "B"
    return {"value": max(ra, rb), "unit": unit, "cores": cores, "kind": "oracle",
            "mode": "A: process pool, BLAS threads = 1" if best == "A"
            else "B: one process, BLAS threads = all cores",
            "cpu_model": cpu_model(),
            "sample": f"{what}; mode A: {cores} processes x BLAS 1 thread, {na} sample(s) in "
                      f"{dta:.1f} s -> {ra:.4g} {unit}; mode B: 1 process x BLAS {cores} threads, "
                      f"{nb} sample(s) in {dtb:.1f} s -> {rb:.4g} {unit} "
                      f"(NumPy/SciPy FP64, the better mode reported)",
            "mode_a": ra, "mode_b": rb}


def run_reference(args, wl, rank, world):
    """The oracle as it stands, on the host cores, on the same workload and metric.

    ``--cpu-mode``: pool (mode A: one step = one sample per core, a process per
    core with single-threaded BLAS), threads (mode B: one step = one sample in
    this process with BLAS on all cores), or best (default: one calibration
    step of each after a warm-up, then the faster one for the timed steps)."""
    if rank != 0:
        return
    name = args.workload
    metric, unit = METRICS[name]
    cores = os.cpu_count() or 1
    run, what = oracle_sampler(name)
    pool = None
    mode = args.cpu_mode
    try:
        if mode in ("pool", "best"):
            pool = OraclePool(cores)
        nxt = [0]

        def step_pool():
            u = pool.round(name, nxt[0])
            nxt[0] += cores
            return u

        def step_threads():
            u = run(nxt[0])
            nxt[0] += 1
            return u

        if mode == "best":
            run(0)                                # first-call costs of this process
            rates = {}
            for m, fn in (("pool", step_pool), ("threads", step_threads)):
                t0 = time.perf_counter()
                u = fn()
                rates[m] = u / (time.perf_counter() - t0)
            mode = max(rates, key=rates.get)
        step = step_pool if mode == "pool" else step_threads
        for _ in range(args.warmup):
            step()
        times, units = [], 0.0
        for _ in range(args.steps):
            t0 = time.perf_counter()
            units += step()
            times.append(time.perf_counter() - t0)
    finally:
        if pool is not None:
            pool.close()
    tot = sum(times)
    value = units / tot
    mdesc = (f"mode A: {cores} processes x BLAS 1 thread, one sample per process per step"
             if mode == "pool" else f"mode B: 1 process x BLAS {cores} threads, one sample per step")
    cfg = {"workload": name, "instances_per_step": units / args.steps, "l2": "n/a (CPU)",
           "cpu_mode": mode}
    cfg.update({key: wl[key] for key in ("L", "U", "g", "dtau", "beta", "k") if key in wl})
    line = {
        "metric": metric, "value": value, "unit": unit,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(),
                         "sample": f"{what}; {args.steps} timed step(s), {mdesc} "
                                   f"(NumPy/SciPy FP64)"},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_fp64_peak(dev_index: int) -> dict:
    """FP64 rate of this GPU from the library's loop kernels (DFMA, and the two
    FP64 mma.sync shapes), with the SM clock sampled during the measurement."""
    import paper_2003_05286_gb300 as dq
    clocks = ClockSampler(dev_index)
    clocks.start()
    out = {}
    for kind, iters in (("dfma", 15000), ("dmma_m8n8k4", 15000), ("dmma_m16n8k8", 3750)):
        tf, ms = dq.selftest_fp64_rate(kind, iters)
        out[kind] = {"tflops": tf, "ms": ms}
    clk = clocks.stop()
    out["clocks"] = clk
    out["derived_tflops"] = FP64_DERIVED_TFLOPS
    return out


def use_graphs(args, wl):
    return args.graphs == "on" or (args.graphs == "auto" and bool(wl.get("graphs")))


def run_gpu(args, wl, rank, world):
    import torch
    import paper_2003_05286_gb300 as dq

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    batch = args.batch or wl["batch"]
    N = wl["L"] ** 2
    M = int(round(wl["beta"] / wl["dtau"]))
    k = wl["k"]
    K_np, V_np, insts = make_inputs(wl, rank, batch)
    K = torch.tensor(K_np, device=dev)
    V = torch.tensor(V_np, device=dev)
    prec = 0 if args.precision == "fp64" else int(args.precision[-1])
    graphs = use_graphs(args, wl)

    # FP64 rate of this GPU (roofline denominator), measured before the timed region
    peak = measure_fp64_peak(dev.index)
    fp64_peak = peak["dfma"]["tflops"]

    h = dq.Handle(chain_precision=prec, graphs=graphs, fold=FOLDS[args.fold])
    h.bind_stream()

    def step():
        return dq.greens(K, wl["dtau"], V, k, handle=h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = h.last_launch_count
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    h.profile(True)
    h.profile_reset()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(float(s))                 # evict L2 between timed steps (not timed)
        ev[s][0].record()
        G, ld, sg, st = step()
        ev[s][1].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall0
    if dist:
        tdist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    tot_ms = reduce_max(tot_ms, dev)
    chain_ms, chain_n, chain_flops = h.profile_read(h.PROF_CHAIN)
    qr_ms, qr_n, qr_flops = h.profile_read(h.PROF_QRP)
    h.profile(False)
    bad = int((st != 0).sum().item())

    value = job_value(batch, world, args.steps, tot_ms)
    fl = flops_per_greens(N, M, k)

    # ---- the dominant kernel once more, not sharing SMs: one extra step with the
    # sub-batch pipeline off (after the timed region; reported beside the roofline)
    unshared = None
    if not args.no_unshared:
        prev = os.environ.get("DQMC_PIPELINE")
        os.environ["DQMC_PIPELINE"] = "0"
        h.set_graph_mode(False)
        h.profile(True)
        h.profile_reset()
        step()
        torch.cuda.synchronize()
        c_ms, c_n, c_fl = h.profile_read(h.PROF_QRP if prec else h.PROF_CHAIN)
        h.profile(False)
        h.set_graph_mode(graphs)
        if prev is None:
            del os.environ["DQMC_PIPELINE"]
        else:
            os.environ["DQMC_PIPELINE"] = prev
        if c_ms > 0:
            u_ach = c_fl / (c_ms / 1e3) / 1e12
            unshared = {"achieved": u_ach, "frac": u_ach / fp64_peak, "launches": c_n,
                        "avg_launch_ms": c_ms / max(c_n, 1),
                        "note": "same kernel in one extra step with the sub-batch pipeline off "
                                "(full batch per launch, no concurrent kernels); not timed"}

    # ---- the same step with the chain products on the tensor cores -----------
    mixed = None
    if args.mixed_slices and prec == 0:
        G64, ld64 = G.clone(), ld.clone()
        hm = dq.Handle(chain_precision=args.mixed_slices)
        hm.bind_stream()
        for _ in range(args.warmup):
            dq.greens(K, wl["dtau"], V, k, handle=hm)
        evm = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        if dist:
            tdist.barrier()
        torch.cuda.synchronize()
        for s_ in range(args.steps):
            flush.fill_(float(s_))
            evm[s_][0].record()
            Gm, ldm, sgm, stm = dq.greens(K, wl["dtau"], V, k, handle=hm)
            evm[s_][1].record()
        torch.cuda.synchronize()
        mms = reduce_max(sum(a.elapsed_time(b) for a, b in evm), dev)
        m_bad = int((stm != 0).sum().item())
        mixed = {"value": job_value(batch, world, args.steps, mms), "unit": "G/s",
                 "ms_per_step": mms / args.steps, "chain_precision": f"bf16x{args.mixed_slices}",
                 "speedup_vs_fp64": tot_ms / mms,
                 "status_nonzero": m_bad,
                 "max_abs_dG_vs_fp64_path": float((Gm - G64).abs().max().item()),
                 "max_rel_dlogdet_vs_fp64_path": float(((ldm - ld64).abs() / ld64.abs()).max().item()),
                 "sign_mismatches": int((sgm != sg).sum().item())}
        # error against the CPU oracle on sampled instances (outside the timed region)
        if args.oracle_samples > 0:
            from oracle import dqmc as od
            n_pick = max(2, args.oracle_samples)
            picks = sorted({round(i * (batch - 1) / (n_pick - 1)) for i in range(n_pick)})
            eg, el, e64 = [], [], []
            for b in picks:
                Go, ldo, so = od.greens(insts[b].K, insts[b].dtau, insts[b].V, insts[b].k)
                scale = max(1.0, float(np.abs(Go).max()))
                eg.append(float(np.abs(Gm[b].cpu().numpy() - Go).max()) / scale)
                e64.append(float(np.abs(G64[b].cpu().numpy() - Go).max()) / scale)
                el.append(abs(float(ldm[b]) - ldo) / abs(ldo))
            mixed["vs_oracle"] = {
                "instances": picks,
                "max_dG_over_max1_maxG": max(eg), "max_rel_dlogdet": max(el),
                "fp64_path_max_dG_over_max1_maxG": max(e64),
                "target": "max|dG| / max(1, max|G|) <= 1e-8 (mixed), <= 1e-10 (FP64)",
                "meets_1e-8": max(eg) <= 1e-8}
        mixed["status_ok"] = m_bad == 0
        hm.close()

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = None
    if not args.no_e2e:
        import ctypes as C
        he = dq.Handle(chain_precision=prec, fold=FOLDS[args.fold])
        he.bind_stream()
        he.set_pointer_mode(True)
        Kh = torch.tensor(K_np).pin_memory()
        Vh = torch.tensor(V_np).pin_memory()
        Gh = torch.empty((batch, N, N), dtype=torch.float64).pin_memory()
        ldh = torch.empty(batch, dtype=torch.float64).pin_memory()
        sgh = torch.empty(batch, dtype=torch.int32).pin_memory()
        sth = torch.empty(batch, dtype=torch.int32).pin_memory()
        p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731

        def e2e_step():
            rc = he._lib.dqmc_greens(he.h, batch, N, M, p(Kh), wl["dtau"], p(Vh), k, p(Gh), p(ldh),
                                     p(sgh), p(sth))
            if rc != 0:
                raise RuntimeError(f"dqmc_greens (host mode) rc={rc}")

        e2e_step()
        if dist:
            tdist.barrier()
        ts = []
        for s in range(max(1, min(args.steps, 3))):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()                      # returns after the outputs are in host memory
            ts.append(time.perf_counter() - t0)
        e2e_s = sum(ts) / len(ts)
        e2e_s = reduce_max(e2e_s, dev)
        e2e = {"value": batch * world / e2e_s, "unit": "G/s",
               "h2d_bytes_per_step": int(Kh.numel() * 8 + Vh.numel() * 8),
               "d2h_bytes_per_step": int(Gh.numel() * 8 + batch * (8 + 4 + 4)),
               "api": "dqmc_greens, DQMC_PTR_HOST (pinned host buffers)"}
        he.close()

    if prec == 0:
        # dominant kernel: the FP64 slice product
        dom_ms, dom_n, dom_flops = chain_ms, chain_n, chain_flops
        dom_kernel = "gemm_f64_kernel (slice-chain product, 2N^3 x batch flops per launch)"
        traffic = measured_traffic(args.workload)
    else:
        # products on the tensor cores: the FP64 pivoted QR dominates the step
        dom_ms, dom_n, dom_flops = qr_ms, qr_n, qr_flops
        dom_kernel = "qrp_fused_kernel (pivoted QR incl. forming Q, 8N^3/3 x batch flops per launch)"
        traffic = measured_traffic(f"{args.workload}_bf16x{prec}", "qrp_fused_traffic.json",
                                   "qrp_f64.cu")
    achieved = (dom_flops / (dom_ms / 1e3)) / 1e12 if dom_ms > 0 else None
    roof_tensor = None
    if prec > 0 and chain_ms > 0:
        pairs = prec * (prec + 1) // 2          # digit pairs p + q <= s + 1
        t_ach = chain_flops * pairs / (chain_ms / 1e3) / 1e12
        t_peak, t_src = bf16_peak_tflops()
        roof_tensor = {"bound": "tensor", "achieved": t_ach, "peak": t_peak, "unit": "TFLOP/s",
                       "frac": t_ach / t_peak, "traffic": None,
                       "kernel": f"ozaki_gemm_kernel ({pairs} BF16 digit-pair products of 2N^3 per "
                                 "slice product and instance)",
                       "launches": chain_n, "avg_launch_ms": chain_ms / max(chain_n, 1),
                       "peak_source": t_src}
    peak_src = (f"measured: DFMA loop kernel (dqmc_selftest_fp64_rate) on this GPU before the "
                f"timed region, median SM clock {peak['clocks']['sm_mhz'] if peak['clocks'] else 'n/a'} MHz"
                f" (derived 152 SM x 4 flop/clk x 2070 MHz = {FP64_DERIVED_TFLOPS:.3f} TFLOP/s)")
    line = {
        "metric": "greens_functions_per_second", "value": value, "unit": "G/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == 0 else f"bf16x{prec}+f64", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "M": M, "k": k, "beta": wl["beta"],
                   "U": wl["U"], "dtau": wl["dtau"], "instances_per_gpu": batch,
                   "chain_precision": args.precision, "cuda_graphs": graphs, "fold": args.fold,
                   "l2": "flushed between timed steps (256 MB write)"},
        "fp64_tflops": fl * batch * world * args.steps / (tot_ms / 1e3) / 1e12,
        "fp64_frac_of_peak": fl * batch * args.steps / (tot_ms / 1e3) / 1e12 / fp64_peak,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": (achieved / fp64_peak) if achieved else None,
                     "traffic": traffic,
                     "kernel": dom_kernel,
                     "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1),
                     "stream_time_share": dom_ms / tot_ms if tot_ms > 0 else None,
                     "unshared": unshared,
                     "peak_source": peak_src,
                     "peak_derived": FP64_DERIVED_TFLOPS,
                     "frac_of_derived": (achieved / FP64_DERIVED_TFLOPS) if achieved else None},
        "fp64_peaks_measured": peak,
        "roofline_tensor": roof_tensor,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "e2e": e2e,
        "mixed": mixed,
        "status_nonzero": bad,
        "wall_s": wall,
    }
    del G, ld, sg, st, V, K, flush
    h.close()
    torch.cuda.empty_cache()
    if rank != 0:
        return
    pool = OraclePool(os.cpu_count() or 1) if world == 1 and not args.no_cpu_baseline else None
    try:
        if world == 1 and not args.no_workloads:
            line["workloads"] = other_workloads(args, peak, pool)
        line["cpu_baseline"] = (cpu_baseline_line(args.workload, args.cpu_seconds, pool)
                                if pool is not None else None)
    finally:
        if pool is not None:
            pool.close()
    print(json.dumps(line), flush=True)


def other_workloads(args, peak, pool=None) -> dict:
    """BASELINE's other configurations, each at few timed steps, for the one JSON line."""
    import torch
    out = {}
    for entry in ("n16_beta8", "tdisplaced_n64", "tdisplaced_n64_bf16x8", "grad_n144",
                  "grad_n144_bf16x8", "ragged_1024", "ragged_1024_bf16x8"):
        name = entry.split("_bf16")[0]
        sub = argparse.Namespace(**vars(args))
        sub.workload = name
        sub.batch = None
        sub.precision = "bf16x8" if entry.endswith("bf16x8") else "fp64"
        # a step of the 4x4 problem is half a millisecond: time more of them
        sub.steps = max(min(args.steps, 3), 20) if name == "n16_beta8" else min(args.steps, 3)
        sub.warmup = 3
        sub.fold = "auto"
        sub.graphs = "auto"
        t0 = time.perf_counter()
        line = measure_other(sub, WORKLOADS[name], 0, 1, peak)
        line["driver_wall_s"] = time.perf_counter() - t0
        line["cpu_baseline"] = (cpu_baseline_line(name, args.workload_cpu_seconds, pool)
                                if pool is not None and entry == name else None)
        out[entry] = line
        torch.cuda.empty_cache()
    return out


def measure_other(args, wl, rank, world, peak=None):
    """The other workloads: same timing rules, whole-step FP64 roofline.  Returns the line."""
    import torch
    import paper_2003_05286_gb300 as dq
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    batch = args.batch or wl["batch"]
    name = args.workload
    prec = 0 if args.precision == "fp64" else int(args.precision[-1])
    graphs = use_graphs(args, wl)
    if peak is None:
        peak = measure_fp64_peak(dev.index)
    fp64_peak = peak["dfma"]["tflops"]
    h = dq.Handle(chain_precision=prec, graphs=graphs, fold=FOLDS[args.fold])
    h.bind_stream()
    if getattr(args, "gemm_tile", 0):
        h.set_gemm_tile(args.gemm_tile)
    extra = {"gemm_tile": getattr(args, "gemm_tile", 0)}
    if name == "ragged_1024":
        from paper_2003_05286_gb300 import tune
        insts0 = [di.ragged_params(rank * batch + i) for i in range(batch)]
        # k per lattice size: tuned on 4 instances at the largest beta of the
        # group, timed with the sequential fold the full ragged batch runs
        kbyL = {}
        for L in sorted({p[0] for p in insts0}):
            idx = [i for i, p in enumerate(insts0) if p[0] == L]
            mx = max(idx, key=lambda i: insts0[i][1])
            sample = [di.ragged_instance(rank * batch + i, 10) for i in idx[:3] + [mx]]
            Mmin = min(x.M for x in sample)
            Ks = torch.tensor(sample[0].K, device=dev)
            Vs = torch.tensor(np.stack([x.V[:Mmin] for x in sample]), device=dev)
            best, _ = tune.tune(Ks, 0.1, Vs, candidates=(5, 10, 15, 20), tiles=(0,), ref_k=2, tol=1e-10,
                                fold=dq._abi.FOLD_SEQUENTIAL)
            kbyL[L] = best["k"]
        insts = [di.ragged_instance(rank * batch + i, kbyL[p[0]]) for i, p in enumerate(insts0)]
        extra["k_by_L"] = kbyL
        Kby = {}   # one hopping matrix per lattice size, shared by its instances
        for x in insts:
            Kby.setdefault(x.N, torch.tensor(x.K, device=dev))
        rb = dq.RaggedBatch([(Kby[x.N], x.dtau, torch.tensor(x.V, device=dev), x.k) for x in insts])
        fl = sum(flops_per_greens(x.N, x.M, x.k) for x in insts)
        fl_tc = sum(flops_tensor_chain(x.N, x.M, x.k) for x in insts)

        def step():
            return rb.run(handle=h)
    else:
        if name == "grad_n144":
            insts = [di.gaussian_instance(wl["L"], wl["g"], wl["dtau"], wl["beta"], wl["k"], sd)
                     for sd in rank_seeds(wl, rank, batch)]
        else:
            insts = [di.hubbard_instance(wl["L"], wl["U"], wl["dtau"], wl["beta"], wl["k"], sd)
                     for sd in rank_seeds(wl, rank, batch)]
        K = torch.tensor(insts[0].K, device=dev)
        V = torch.tensor(np.stack([x.V for x in insts]), device=dev)
        N, M, k = insts[0].N, insts[0].M, wl["k"]
        if name == "tdisplaced_n64":
            fl = batch * flops_per_tdisplaced(N, M, k)
            fl_tc = batch * flops_tensor_chain(N, M, k, 2)

            def step():
                return dq.greens_tdisplaced(K, wl["dtau"], V, k, handle=h)
        elif name == "grad_n144":
            fl = batch * flops_per_grad(N, M, k)
            fl_tc = batch * flops_tensor_chain(N, M, k, 2)

            def step():
                return dq.logdet_grad(K, wl["dtau"], V, k, handle=h)
        else:
            fl = batch * flops_per_greens(N, M, k)
            fl_tc = batch * flops_tensor_chain(N, M, k)

            def step():
                return dq.greens(K, wl["dtau"], V, k, handle=h)
        extra.update(N=N, M=M, k=k)
    metric, unit = METRICS[name]
    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    launches = h.last_launch_count
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(dev.index)
    torch.cuda.synchronize()
    clocks.start()
    for s_ in range(args.steps):
        flush.fill_(float(s_))
        ev[s_][0].record()
        out = step()
        ev[s_][1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    tot = reduce_max(sum(a.elapsed_time(b) for a, b in ev), dev)
    st = out[-1]
    # FP64 roofline of the step: with the tensor-core chain, only the flops that
    # stay on the FP64 pipe (QRs, inversions, wraps) count against its peak
    fl64 = fl if prec == 0 else fl - fl_tc
    ach = fl64 * args.steps / (tot / 1e3) / 1e12
    line = {"metric": metric, "value": job_value(batch, world, args.steps, tot), "unit": unit,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if prec == 0 else f"bf16x{prec}+f64",
            "data": "synthetic",
            "config": dict(workload=name, baseline_config=wl["config"], instances_per_gpu=batch,
                           chain_precision=prec, cuda_graphs=graphs, fold=args.fold,
                           l2="flushed between timed steps (256 MB write)", **extra),
            "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": None,
                         "peak_source": "measured (DFMA loop kernel, dqmc_selftest_fp64_rate)",
                         "frac_of_derived": ach / FP64_DERIVED_TFLOPS,
                         "kernel": "whole step (all kernels), algorithmic FP64 flops"
                                   + ("" if prec == 0 else " of the kernels that stay in FP64 (QRs, "
                                      "inversions, wraps); the chain products and X updates run on "
                                      "the tensor cores and are not counted")},
            "gpu_launches": launches * args.steps, "clocks": clk,
            "status_nonzero": int((st != 0).sum().item()), "e2e": None}
    h.close()
    return line


def run_gpu_other(args, wl, rank, world):
    line = measure_other(args, wl, rank, world)
    if rank != 0:
        return
    line["cpu_baseline"] = (cpu_baseline_line(args.workload, args.cpu_seconds)
                            if world == 1 and not args.no_cpu_baseline else None)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
    try:
        if args.workload == "n256_beta20":
            run_gpu(args, wl, rank, world)
        else:
            run_gpu_other(args, wl, rank, world)
    finally:
        if world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


if __name__ == "__main__":
    main()
