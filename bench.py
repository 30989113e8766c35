#!/usr/bin/env python3
"""Benchmark of the QEM E-step hot path (arXiv 2503.08264) on GB300.

One step = one iteration of Alg. 1 on the device: E-step (sample, local
factors, K x K forward contraction, plate sums, root, adjoint, moments) then
EMA + M-step, on a seeded synthetic workload.  The metric is E-step
log-factor pairs per second, pairs = sum over non-root plate elements of
K_parent * K_child.

  python bench.py [--gpus N --steps K --warmup W] [--workload NAME] [--precision P]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the same workload

Under torchrun (N > 1) every rank runs an independent instance of the
workload (weak scaling, no collective on the data path); rank 0 prints one
JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2503_08264_gb300 import synth as S  # noqa: E402

METRIC = "E-step K^2 x plate-elt log-factor pairs/s"
UNIT = "pairs/s"

# workload name -> (builder(seed), K, default precision)
WORKLOADS = {
    "conjugate_gaussian_M8_N16_K16": (lambda seed: S.conjugate_gaussian(M=8, N=16, seed=seed), 16, "fp32"),
    "hier_logistic_M5000_N10_K1024": (lambda seed: S.hier_logistic(M=5000, N=10, seed=seed), 1024, "bf16x3"),
    "hier_logistic_M300_N5_K128": (lambda seed: S.hier_logistic(M=300, N=5, seed=seed), 128, "fp32"),
    # profiling case: the large workload's shapes with a fifth of its plate (fits an ncu capture)
    "hier_logistic_M1000_N10_K1024": (lambda seed: S.hier_logistic(M=1000, N=10, seed=seed), 1024, "bf16x3"),
    "batched_three_level_256_K256": (lambda seed: S.batched_three_level(n_inst=256, seed=seed), 256, "bf16x3"),
    # the Covid model's chain plate: 92 regions x 109 days of a random walk under a global latent
    "chain_poisson_R92_T109_K128": (lambda seed: S.chain_poisson(R=92, T=109, seed=seed), 128, "fp32"),
}
DEFAULT_WORKLOAD = "hier_logistic_M5000_N10_K1024"
EMA_LAMBDA = 0.5
CONVERGE_ITERS = 100   # Alg. 1 iterations run before the timed region (EM steady state)


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    p.add_argument("--precision", default=None, choices=["fp32", "bf16", "bf16x3", "tf32"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--ref-seconds", type=float, default=150.0,
                   help="reference arm: total oracle time the samples are sized for")
    p.add_argument("--metric", choices=["pairs", "time_to_tol"], default="pairs",
                   help="pairs: E-step throughput (default); time_to_tol: the warm-start study")
    p.add_argument("--root", choices=["grouped", "split"], default="grouped",
                   help="split: the root's mean and log-variance as separate latents (K^2 parent pairs)")
    p.add_argument("--qcond", action="store_true",
                   help="leaf level with the parent-conditioned proposal (permutation copies; two-level, FP32)")
    p.add_argument("--unit-peaks", action="store_true",
                   help="measure the per-SM rates of the exponential unit, the FP32 pipe and tcgen05.mma")
    p.add_argument("--small-case", choices=["estep", "estep_steady", "mlp"], default=None,
                   help="run a small case for a profiler (no JSON line): estep = 12 EM iterations of "
                        "hier_logistic M=1000 N=10 K=1024 bf16x3 on the host loop; estep_steady = 100 "
                        "iterations, then 3 inside the NVTX range small_case; mlp = the warm-start "
                        "network's forward and gradient on 16384 users, twice")
    p.add_argument("--train-instances", type=int, default=2000)
    p.add_argument("--test-instances", type=int, default=16)
    return p.parse_args(argv)


# --------------------------------------------------------------------------- distributed helpers
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def dist_init(ws: int, backend: str):
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(local_ms: float, local_units: float, ws: int, device=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the units)."""
    if ws == 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled every 5 ms during the
    timed region, read through NVML (libnvidia-ml, the library nvidia-smi
    reports from; read-only queries), with `nvidia-smi -lms 50` as the fallback.
    The GPU is found by its PCI address, so the sample follows the CUDA device
    under any CUDA_VISIBLE_DEVICES."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of nvmlDeviceGetCurrentClocksEventReasons
    REASON_BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                   0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}
    PERIOD_S = 0.005

    def __init__(self, cuda_device: int):
        self.dev = cuda_device
        self.proc = None
        self.path = None
        self.thread = None
        self.samples = []
        self.nvml = None
        self.handle = None

    def _nvml_open(self):
        import ctypes as C
        try:
            nv = C.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if nv.nvmlInit_v2() != 0:
            return False
        h = C.c_void_p()
        ok = False
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.dev)
            bus = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0".encode()
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) == 0
        except Exception:
            ok = False
        if not ok:
            ok = nv.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.dev), C.byref(h)) == 0
        if not ok:
            return False
        self.nvml, self.handle = nv, h
        return True

    def _nvml_read(self):
        import ctypes as C
        sm, smax, pw, rs = C.c_uint(), C.c_uint(), C.c_uint(), C.c_ulonglong()
        nv, h = self.nvml, self.handle
        if nv.nvmlDeviceGetClockInfo(h, 1, C.byref(sm)) != 0:          # NVML_CLOCK_SM
            return None
        nv.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(smax))
        nv.nvmlDeviceGetPowerUsage(h, C.byref(pw))
        f = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        f(h, C.byref(rs))
        return float(sm.value), float(smax.value), pw.value / 1000.0, int(rs.value)

    def _loop(self):
        while not self.stop_evt.is_set():
            r = self._nvml_read()
            if r is not None:
                self.samples.append(r)
            self.stop_evt.wait(self.PERIOD_S)

    def start(self):
        import threading
        if self._nvml_open() and self._nvml_read() is not None:
            self.stop_evt = threading.Event()
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 2.0:
                time.sleep(0.001)
            return
        try:
            fd, self.path = tempfile.mkstemp(prefix="qem_clocks_", suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler is producing samples
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.thread is not None:
            self.stop_evt.set()
            self.thread.join(timeout=2.0)
            sm = [x[0] for x in self.samples]
            smax = [x[1] for x in self.samples]
            reasons = sorted({nm for x in self.samples for bit, nm in self.REASON_BITS.items() if x[3] & bit})
            return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                    "reasons": reasons, "samples": len(sm), "source": "NVML, 5 ms period",
                    "power_w_max": max(x[2] for x in self.samples) if self.samples else None}
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 50 ms period"}


# --------------------------------------------------------------------------- roofline
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# Binding-unit model of each contraction path (per log-factor pair of one
# launch): FP32 CUDA-core path = FP32 pipe (128 lanes/clk/SM), tensor-core
# path = MUFU ex2 (1 exponential per pair; 32 per clk per SM on GB300).
SMS = 152
# where the per-SM unit rates come from (probe method, cycle counts, clocks)
PEAK_SOURCE = "profiles/mufu_fp32_peaks.md"


# DRAM bytes per launch of a dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), with the git blob hash of the
# kernel's source file at capture time: reported only while that file is
# unchanged (the summary under profiles/ gives the capture command).
NCU_TRAFFIC = {
    # the element-resident forward (k_fwd_res) and adjoint (k_adj_res),
    # captured at the EM steady state of the 1000-element small case
    # (bench.py --small-case estep_steady) and scaled by elements to the 5000
    # of this workload: their traffic is per element (the element's rows
    # once, its output row written once; the parent's rows stay in L2)
    ("forward", "hier_logistic_M5000_N10_K1024", "bf16x3"): {
        "bytes": 5 * (164162304 + 4952064), "source": "paper_2503_08264_gb300/csrc/qem_tc_res.cu",
        "blob": "43d2408ea249832ce023fd0f37d3de37c1c2b225",
        "profile": "profiles/fwd_res_bf16x3_hier_logistic_M1000_K1024.md"},
    ("adjoint", "hier_logistic_M5000_N10_K1024", "bf16x3"): {
        "bytes": 5 * (167880704 + 5359104), "source": "paper_2503_08264_gb300/csrc/qem_tc_res.cu",
        "blob": "43d2408ea249832ce023fd0f37d3de37c1c2b225",
        "profile": "profiles/adj_res_bf16x3_hier_logistic_M1000_K1024.md"},
}


def git_blob_hash(path: str) -> str:
    import hashlib
    with open(os.path.join(ROOT, path), "rb") as f:
        data = f.read()
    return hashlib.sha1(b"blob %d\0" % len(data) + data).hexdigest()


def ncu_traffic(kind: str, workload: str, precision: str):
    e = NCU_TRAFFIC.get((kind, workload, precision))
    try:
        return e["bytes"] if e and git_blob_hash(e["source"]) == e["blob"] else None
    except OSError:
        return None


def roofline_for(kind: str, precision: str, D: int, pairs: float, ms: float, sm_max_mhz: float):
    clk = (sm_max_mhz or 2070.0) * 1e6
    if precision == "fp32":
        ops_per_pair = 3 * D + 4          # (z-m), ^2, fma per dim; shift, exp, accumulate, max
        peak = SMS * 128 * clk / ops_per_pair
        model = f"FP32 pipe: {ops_per_pair} lane-ops/pair, 128 lanes/clk/SM x {SMS} SMs x {clk / 1e6:.0f} MHz"
    else:
        peak = SMS * 32 * clk
        model = f"MUFU ex2: 1/pair, 32/clk/SM x {SMS} SMs x {clk / 1e6:.0f} MHz"
    achieved = pairs / (ms * 1e-3)
    return {"bound": "alu", "kernel": kind, "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": None, "model": model + " (derived from unit counts and max clock)",
            "peak_source": PEAK_SOURCE}


# --------------------------------------------------------------------------- CPU oracle baseline
def cpu_oracle_sample(workload: str, target_s: float, seed: int = 7, qcond: bool = False, split: bool = False):
    """Time the FP64 oracle E-step on a bounded sample of the workload (all host cores).

    The sample keeps the workload's shapes (K, dimensions, observations per
    element) and takes a prefix of its plate elements (2-level workloads) or a
    smaller batch of instances (batched workloads), sized from a short
    calibration run so that the timed run takes about target_s seconds.
    Chain workloads take whole regions and the chain oracle (numpy, one
    thread for its own loops)."""
    import numpy as np
    from oracle import oracle as O
    O.build()
    builder, K, _ = WORKLOADS[workload]
    full = builder(seed)
    two_level = len(full.levels) == 2
    T = int(getattr(full.levels[1], "chain", 1) or 1) if two_level else 1
    total = full.levels[1].n // T if two_level else full.n_inst

    def sub(count):
        count = int(max(1, min(total, count)))
        if two_level:
            lv = full.levels[1]
            n = count * T
            users = S.Level(n=n, dim=lv.dim, prior=lv.prior, prior_a=lv.prior_a, prior_b=lv.prior_b, lik=lv.lik,
                            lik_var=lv.lik_var, n_obs=lv.n_obs, qfam=lv.qfam,
                            parent=np.zeros(n, np.int64), x=lv.x[:n], y=lv.y[:n], chain=T, qcond=int(qcond))
            what = "regions" if T > 1 else "plate elements"
            return S.Model([full.levels[0], users]), f"{count} of {total} {what}"
        return S.batched_three_level(n_inst=count, seed=seed), f"{count} of {total} instances"

    # grow the sample until one run takes at least 60% of the target (the
    # per-element cost only shows once the fixed per-call cost is amortised)
    count = 4 if two_level else 1
    for _ in range(5):
        model, desc = sub(count)
        t = oracle_estep_seconds(model, K, 1, split)
        if t >= 0.6 * target_s or count >= total:
            break
        count = min(total, count * min(50.0, target_s / max(t, 1e-3)))
    pairs = model.pairs(K) * (K if split else 1)
    cores = 1 if (T > 1 or qcond or split) else O.max_threads()
    noise = "supplied noise" if (T > 1 or qcond or split) else "counter-based noise"
    return {"value": pairs / t, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one FP64 E-step on {desc} of {workload} ({noise}), {t:.1f} s"}, model


def oracle_estep_seconds(model, K: int, it: int, split: bool = False) -> float:
    """Seconds of one FP64 oracle E-step of `model` (the chain oracle for chain plates,
    the conditional-proposal oracle for qcond levels, the split-root oracle with split)."""
    if split:
        from oracle import split_root as R
        eps = S.noise(model, K, seed=it)
        t0 = time.perf_counter()
        R.estep(model, S.initial_q(model), K, eps)
        return time.perf_counter() - t0
    if len(model.levels) == 2 and int(getattr(model.levels[1], "qcond", 0) or 0):
        from oracle import conditional as QC
        eps = S.noise(model, K, seed=it)
        rng = np.random.default_rng(it)
        perm = np.stack([rng.permutation(K) for _ in range(model.levels[1].n)])
        t0 = time.perf_counter()
        QC.estep(model, S.initial_q(model), K, eps, perm)
        return time.perf_counter() - t0
    if len(model.levels) == 2 and int(getattr(model.levels[1], "chain", 1) or 1) > 1:
        from oracle import chain as C
        eps = S.noise(model, K, seed=it)
        t0 = time.perf_counter()
        C.estep(model, S.initial_q(model), K, eps)
        return time.perf_counter() - t0
    from oracle import oracle as O
    t0 = time.perf_counter()
    O.estep(model, S.initial_q(model), K, seed=1, it=it)
    return time.perf_counter() - t0


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    builder, K, _ = WORKLOADS[args.workload]
    # size one step's sample so that warmup + steps fit in about three minutes
    per_step = max(0.2, args.ref_seconds / max(1, args.steps + args.warmup))
    split = args.root == "split"
    base, model = cpu_oracle_sample(args.workload, per_step, qcond=args.qcond, split=split)
    times = []
    for i in range(args.warmup + args.steps):
        t = oracle_estep_seconds(model, K, i + 1, split)
        if i >= args.warmup:
            times.append(t)
    pairs = model.pairs(K) * (K if split else 1)
    value = pairs * len(times) / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "K": K, "sample": base["sample"],
                       "proposal": "parent-conditioned, permutation copies" if args.qcond else "factorised",
                       "root": "split (mean and log-variance as separate latents)" if split else "grouped"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------- time to tolerance
# The second metric: wall time for QEM to bring every test instance to
# convergence, plain FP32 QEM (cold start, one instance per plan) against the
# mixed-precision (split-BF16), batched (all instances in one plan) and
# warm-started (users' q from the trained network) form.
#   iteration  Alg. 1 with the constant new-estimate weight 0.5
#   plateau    per instance and run, the mean of log P_MP over the second
#              half of the run's TOL_T_MAX iterations
#   converged  first iteration t at which the mean of log P_MP over
#              iterations t-4 .. t is within TOL_DELTA nats of the plateau
# log P_MP, the method's estimate of the evidence, is the convergence signal:
# the moments of the 36-dimensional global node are not reproducible across
# noise streams at K = 128 (its importance weights are nearly degenerate, so
# its proposal wanders from one stream to the next), and the plateau itself
# moves by up to a few tens of nats between streams, so each run is measured
# against its own plateau.
TOL_LAMBDA = 0.5
TOL_DELTA = 10.0
TOL_WINDOW = 5
TOL_REF_T = 200
TOL_T_MAX = 100
TOL_K = 128
TOL_M, TOL_N = 300, 5
TRAIN_SEED, TEST_SEED = 10000, 90000


def qem_trajectory(plan, q0, T, seed, callback=None):
    """Plain host loop of Alg. 1 from the proposal q0 (device, flat);
    callback(t, q, log_pmp) sees every iteration; returns the final (m, q)."""
    import torch
    q = q0.clone()
    m = plan.mean_params(q)
    mom = torch.empty(plan.q_len, dtype=torch.float64, device=q.device)
    lp = torch.empty(plan.n_inst, dtype=torch.float64, device=q.device)
    for t in range(1, T + 1):
        plan.estep(q, None, seed=seed, it=t, moments=mom, log_pmp=lp)
        if callback is not None:
            callback(t, q, lp)
        plan.mstep(mom, m, q, TOL_LAMBDA, t=t)
    return m, q


def log_pmp_trace(plan, q0, T, seed):
    """[T, n_inst] log P_MP of every iteration."""
    import torch
    rows = []
    qem_trajectory(plan, q0, T, seed, callback=lambda t, q, lp: rows.append(lp.clone()))
    return torch.stack(rows).cpu().numpy()


def reference_plateau(plan, q0, T=TOL_REF_T, seed=4242):
    """Per instance: mean log P_MP over the second half of a T-iteration run."""
    return log_pmp_trace(plan, q0, T, seed)[T // 2:].mean(0)


def iterations_to_tol(plan, q0, T_max=TOL_T_MAX, seed=777):
    """Per instance: (first iteration at which the windowed log P_MP is within
    TOL_DELTA of the run's plateau, the plateau)."""
    tr = log_pmp_trace(plan, q0, T_max, seed)
    plateau = tr[T_max // 2:].mean(0)
    hit = []
    for j in range(tr.shape[1]):
        h = T_max
        for t in range(TOL_WINDOW, T_max + 1):
            if tr[t - TOL_WINDOW:t, j].mean() >= plateau[j] - TOL_DELTA:
                h = t
                break
        hit.append(h)
    return hit, [float(x) for x in plateau]


def train_warm_start(n_train, seed=TRAIN_SEED, T=60, epochs=8, batch=4096, lr=2e-3, shuffle_seed=5):
    """QEM on n_train seeded instances (split-BF16, batched), then the network
    trained on the users' final proposals.  Returns (network, seconds, losses)."""
    import torch
    from paper_2503_08264_gb300 import qem
    from paper_2503_08264_gb300.warmstart import WarmStart
    t0 = time.perf_counter()
    model = S.hier_logistic_batch(n_train, M=TOL_M, N=TOL_N, seed=seed)
    plan = qem.Plan(model, TOL_K, precision="bf16x3")
    q0 = plan.flat(S.initial_q(model))
    m = plan.mean_params(q0)
    q = q0.clone()
    plan.run(T, TOL_LAMBDA, m, q, seed=seed)
    users = plan.split_q(q)[1]                                  # [n_users, 2, D] on the host
    lv = model.levels[1]
    perm = np.random.default_rng(shuffle_seed).permutation(lv.n)
    net = WarmStart(seed=seed)
    feats = net.features(torch.as_tensor(lv.x[perm]).cuda(), torch.as_tensor(lv.y[perm]).cuda())
    target = torch.as_tensor(np.ascontiguousarray(users[perm])).cuda()
    plan.close()
    losses = net.train(feats, target, epochs=epochs, batch=batch, lr=lr)
    torch.cuda.synchronize()
    return net, time.perf_counter() - t0, losses


def warm_start_fn(plan, net):
    """A function that writes the network's proposal for the users into a
    fresh copy of the cold proposal (features, forward and to_q run on the
    device each call); the instance data and the cold proposal are uploaded
    once, outside it."""
    import torch
    lv = plan.model.levels[1]
    x_d = torch.as_tensor(lv.x).cuda()
    y_d = torch.as_tensor(lv.y).cuda()
    cold = plan.flat(S.initial_q(plan.model))
    off = plan.model.levels[0].n * 2 * plan.model.levels[0].dim

    def fn():
        q = cold.clone()
        qu = net.predict_q(net.features(x_d, y_d))
        q[off:off + qu.numel()].copy_(qu.reshape(-1))
        return q
    return fn


def cold_start_fn(plan):
    cold = plan.flat(S.initial_q(plan.model))
    return lambda: cold.clone()


def timed_qem(plan, q_init, T, seed):
    """CUDA-event seconds of q_init() (the warm start's kernels, or a copy of
    the cold proposal) plus T iterations of Alg. 1 in one qem_run launch,
    on the plan's stream; returns (seconds, final q on the device).  The loop
    graph is built by an untimed 2-iteration run first."""
    import torch
    q = q_init()
    plan.run(2, TOL_LAMBDA, plan.mean_params(q), q, seed=seed + 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    q = q_init()
    plan.run(T, TOL_LAMBDA, plan.mean_params(q), q, seed=seed)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e-3, q


def oracle_reference(n_inst, T, seed, K=TOL_K):
    """Alg. 1 in FP64 with the oracle's E-step on the first n_inst test
    instances, from the cold proposal with the counter-based noise of `seed`
    (the GPU runs' stream for the same instances of the batch).  Returns per
    user [n_users, 2, D] the proposal (loc, scale) averaged over iterations
    T/2+1..T, and per instance the mean log P_MP over those iterations."""
    from oracle import oracle as O
    O.build()
    model = S.hier_logistic_batch(n_inst, M=TOL_M, N=TOL_N, seed=TEST_SEED)
    q = [np.asarray(a, np.float64) for a in S.initial_q(model)]
    m = [np.stack([a[:, 0], a[:, 0] ** 2 + a[:, 1] ** 2], 1) for a in q]
    acc, lp = None, []
    for t in range(1, T + 1):
        r = O.estep(model, q, K, None, seed=seed, it=t)
        m = [O.ema(m[l], r["mom"][l], TOL_LAMBDA) for l in range(2)]
        q = [O.mstep(O.Q_GAUSS, m[l]) for l in range(2)]
        if t > T // 2:
            acc = q[1].copy() if acc is None else acc + q[1]
            lp.append(r["log_pmp"])
    return acc / (T - T // 2), np.mean(lp, 0)


def moment_error(q_users, ref):
    """Per user and dimension: |loc - loc_ref| / scale_ref and
    |scale - scale_ref| / scale_ref; their mean and maximum."""
    q_users = np.asarray(q_users, np.float64)[:ref.shape[0]]
    el = np.abs(q_users[:, 0] - ref[:, 0]) / ref[:, 1]
    es = np.abs(q_users[:, 1] - ref[:, 1]) / ref[:, 1]
    return {"loc_mean": float(el.mean()), "loc_max": float(el.max()), "scale_mean": float(es.mean()),
            "scale_max": float(es.max())}


def iterations_to_target(plan, q0, target, T_max=TOL_T_MAX, seed=777):
    """Per instance: the first iteration at which the mean log P_MP over the
    last TOL_WINDOW iterations reaches target[i] (T_max when never)."""
    tr = log_pmp_trace(plan, q0, T_max, seed)
    hit = []
    for j in range(tr.shape[1]):
        h = T_max
        for t in range(TOL_WINDOW, T_max + 1):
            if tr[t - TOL_WINDOW:t, j].mean() >= target[j]:
                h = t
                break
        hit.append(h)
    return hit


def run_time_to_tol(args):
    import torch
    from paper_2503_08264_gb300 import qem
    torch.cuda.set_device(0)
    seed = 777                                    # the noise stream of every run below
    net, train_s, losses = train_warm_start(args.train_instances)
    n_test = args.test_instances
    t0 = time.perf_counter()
    ref, ref_lp = oracle_reference(n_test, TOL_REF_T, seed)
    oracle_s = time.perf_counter() - t0
    # the same reference from another noise stream on two instances: the
    # chain-to-chain spread of the converged moments (the floor of moment_err)
    ref2, _ = oracle_reference(2, TOL_REF_T, seed + 1)
    spread = moment_error(ref2, ref[:2 * TOL_M])
    target = ref_lp - TOL_DELTA
    # the plain FP32 baseline, one instance per plan, each run for its own iterations
    it_plain, sec_plain, q_plain = [], [], []
    for i in range(n_test):
        mdl = S.hier_logistic(M=TOL_M, N=TOL_N, seed=TEST_SEED + i)
        plan = qem.Plan(mdl, TOL_K, precision="fp32")
        init = cold_start_fn(plan)
        h = iterations_to_target(plan, init(), target[i:i + 1], seed=seed)
        sec, q = timed_qem(plan, init, h[0], seed)
        it_plain += h
        sec_plain.append(sec)
        q_plain.append(plan.split_q(q)[1])
        plan.close()
    batch = S.hier_logistic_batch(n_test, M=TOL_M, N=TOL_N, seed=TEST_SEED)
    out = {}
    for name, prec, warm in (("batched_bf16x3_cold", "bf16x3", False), ("batched_bf16x3_warm", "bf16x3", True),
                             ("batched_fp32_warm", "fp32", True)):
        plan = qem.Plan(batch, TOL_K, precision=prec)
        init = warm_start_fn(plan, net) if warm else cold_start_fn(plan)
        its = iterations_to_target(plan, init(), target, seed=seed)
        sec, q = timed_qem(plan, init, max(its), seed)
        out[name] = {"iterations": its, "seconds": sec, "ms_per_iteration": sec * 1e3 / max(its),
                     "moment_err": moment_error(plan.split_q(q)[1], ref)}
        plan.close()
    plain_s = float(sum(sec_plain))
    fast = out["batched_bf16x3_warm"]
    line = {"metric": "time to tolerance (all test instances)", "value": fast["seconds"], "unit": "s",
            "higher_is_better": False, "n_gpus": 1, "dtype": "bf16x3", "data": "synthetic",
            "vs_plain_fp32": plain_s / fast["seconds"] if fast["seconds"] > 0 else None,
            "plain_fp32": {"seconds": plain_s, "iterations": it_plain,
                           "moment_err": moment_error(np.concatenate(q_plain), ref)},
            "variants": out,
            "oracle_reference": {"instances": n_test, "iterations": TOL_REF_T, "seconds": round(oracle_s, 1),
                                 "plateau_log_pmp": [round(float(x), 2) for x in ref_lp],
                                 "chain_to_chain_moment_spread": spread},
            "config": {"workload": f"hier_logistic_M{TOL_M}_N{TOL_N}_K{TOL_K} x {n_test} test instances",
                       "train": f"{args.train_instances} instances, {len(losses)} epochs, {train_s:.1f} s",
                       "train_loss_last": losses[-1], "lambda": TOL_LAMBDA, "noise_seed": seed,
                       "criterion": f"per instance, the mean log P_MP over {TOL_WINDOW} iterations reaches the "
                                    f"FP64 oracle's plateau less {TOL_DELTA} nats (the same target for every "
                                    "run); plateau: the oracle's Alg. 1 from the cold proposal, mean log P_MP "
                                    f"over its iterations {TOL_REF_T // 2 + 1}-{TOL_REF_T}",
                       "max_iterations": TOL_T_MAX,
                       "time": "CUDA events around each run: the warm start's features, forward and to_q "
                               "(warm variants) and the iterations to tolerance in one qem_run launch; "
                               "plain FP32 sums its per-instance runs",
                       "moment_err": "every user at the iteration of tolerance (the last instance's, for the "
                                     "batched runs) against the oracle's proposal averaged over iterations "
                                     f"{TOL_REF_T // 2 + 1}-{TOL_REF_T}: |loc - loc_ref| / scale_ref and "
                                     "|scale - scale_ref| / scale_ref; chain_to_chain_moment_spread is the same "
                                     "measure between two oracle runs that differ only in their noise stream "
                                     "(two instances): the floor of any run's moment error"}}
    print(json.dumps(line))
    return 0


def run_small_case(kind: str):
    """Small, short workloads for ncu captures (a few GB at most, seconds of GPU time)."""
    import torch
    from paper_2503_08264_gb300 import qem
    if kind in ("estep", "estep_steady"):
        # estep: 12 iterations from q_0 (the adjoint still on the small-set
        # kernel); estep_steady: 100 iterations to the EM steady state, then 3
        # inside the NVTX range "small_case" (both tensor-core contractions
        # element-resident, the adjoint over ~800 kept parent samples)
        model = S.hier_logistic(M=1000, N=10, seed=1000)
        plan = qem.Plan(model, 1024, precision="bf16x3")
        q = plan.flat(S.initial_q(model))
        m = plan.mean_params(q)
        mom = torch.empty(plan.q_len, dtype=torch.float64, device="cuda")
        n_pre, n_in = (12, 0) if kind == "estep" else (100, 3)
        for t in range(1, n_pre + n_in + 1):
            if t == n_pre + 1:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push("small_case")
            plan.estep(q, None, seed=5, it=t, moments=mom)
            plan.mstep(mom, m, q, EMA_LAMBDA, t=t)
        if n_in:
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print("small case", kind, ": log P_MP", plan.log_pmp(), "tensor-core adjoint pairs", plan.adjoint_pairs())
        return 0
    from paper_2503_08264_gb300.warmstart import WarmStart
    n = 16384
    model = S.hier_logistic(M=n, N=5, seed=3)
    rng = np.random.default_rng(1)
    target = torch.as_tensor(np.stack([rng.standard_normal((n, 18)), rng.uniform(0.2, 1.2, (n, 18))],
                                      1).astype(np.float32)).cuda()
    net = WarmStart(seed=1)
    f = net.features(torch.as_tensor(model.levels[1].x).cuda(), torch.as_tensor(model.levels[1].y).cuda())
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        net.forward(f)
        net.loss_grad(f, target, loss)
    torch.cuda.synchronize()
    print("small case mlp: loss", loss.item())
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist_init(ws, "nccl")
    from paper_2503_08264_gb300 import _lib as L
    from paper_2503_08264_gb300 import qem  # fails loudly when libqem.so is missing

    builder, K, default_prec = WORKLOADS[args.workload]
    precision = args.precision or default_prec
    model = builder(1000 + rank)
    if args.qcond:
        if len(model.levels) != 2 or precision != "fp32":
            raise SystemExit("--qcond needs a two-level workload and the fp32 path")
        model.levels[1].qcond = 1
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = qem.Plan(model, K, precision=precision, stream=stream, tile=L.QEM_TILE_AUTO)
        q0 = S.initial_q(model)
        q_d = plan.flat(q0)
        m_d = plan.mean_params(q_d)
        mom_d = torch.empty(plan.q_len, dtype=torch.float64, device="cuda")
        lp_d = torch.empty(plan.n_inst, dtype=torch.float64, device="cuda")
    pairs = float(model.pairs(K))
    seed = 12345 + rank

    def step(t):
        plan.estep(q_d, None, seed=seed, it=t, moments=mom_d, log_pmp=lp_d)
        plan.mstep(mom_d, m_d, q_d, EMA_LAMBDA, t=t)

    with torch.cuda.stream(stream):
        # EM steady state before anything is timed: a fixed number of Alg. 1
        # iterations from q_0 as one graph launch (the first call autotunes the
        # launch shapes), whatever --warmup and --steps are; the adjoint's work
        # grows with the root samples that keep weight as the proposal converges
        plan.run(CONVERGE_ITERS, EMA_LAMBDA, m_d, q_d, moments=mom_d, seed=seed)
    t_iter = CONVERGE_ITERS + 1
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(t_iter)
            t_iter += 1
    stream.synchronize()
    per_iter, per_call = plan.run_kernels()
    plan.log_pmp()  # raises on a non-finite estimate or a device error
    m_g, q_g = m_d.clone(), q_d.clone()  # the single-launch loop (timed below) continues from a copy
    barrier(ws)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        torch.cuda.nvtx.range_push("qem_timed")  # the timed steps, for profilers (ncu --nvtx-include)
        ev0.record(stream)
        for _ in range(args.steps):
            step(t_iter)
            t_iter += 1
        ev1.record(stream)
        torch.cuda.nvtx.range_pop()
    stream.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    clk = clocks.stop()
    local_ms = ev0.elapsed_time(ev1)
    lp_host = plan.log_pmp()
    max_ms, tot_pairs = aggregate(local_ms, pairs * args.steps, ws, device="cuda")
    value = tot_pairs / (max_ms * 1e-3)

    # per-kernel device times from a second pass of as many steps (every kernel
    # bracketed by CUDA events on the plan's stream; not the headline pass)
    plan.profile(True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        pe0.record(stream)
        for _ in range(args.steps):
            step(t_iter)
            t_iter += 1
        pe1.record(stream)
    stream.synchronize()
    prof = plan.profile_read()
    prof_ms = pe0.elapsed_time(pe1)
    plan.profile(False)

    # the same iterations as one graph launch (device-side loop, no host
    # round trip between iterations)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(ws)
    with torch.cuda.stream(stream):
        g0.record(stream)
        plan.run(args.steps, EMA_LAMBDA, m_g, q_g, moments=mom_d, seed=seed)
        g1.record(stream)
    stream.synchronize()
    g_ms, g_pairs = aggregate(g0.elapsed_time(g1), pairs * args.steps, ws, device="cuda")
    graph_loop = {"ms_per_step": g_ms / args.steps, "value": g_pairs / (g_ms * 1e-3),
                  "launches": int(per_iter * args.steps + per_call)}

    # rooflines of the two contraction kernels (CUDA events on the plan's
    # stream); the headline one is the kernel with the larger share of the step.
    # Work per step: the forward evaluates every pair (K_parent x K_child per
    # element); the adjoint only the pairs of kept parent samples (its
    # compaction), counted from the last E-step's kept lists.
    kept_tc, kept_all = plan.adjoint_pairs()
    adj_pairs = kept_all if precision == "fp32" else kept_tc
    gpu_launches = int(per_iter * args.steps)
    sm_max = clk.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    D_child = model.levels[-1].dim
    rooflines = {}
    for kind, work in (("forward", pairs), ("adjoint", adj_pairs)):
        k_ms, k_n = prof.get(kind, (0.0, 0))
        if k_ms <= 0 or work <= 0:
            continue
        r = roofline_for(kind, precision, D_child, work * args.steps, k_ms, sm_max)
        r["pairs_per_step"] = work
        r["launches"] = k_n
        r["ms_per_launch"] = k_ms / k_n
        r["traffic"] = ncu_traffic(kind, args.workload, precision)
        if r["traffic"] is not None:
            r["traffic_unit"] = "bytes per launch (ncu dram read + write)"
        r["share_of_step"] = k_ms / prof_ms if prof_ms else None
        rooflines[kind] = r
    kind = max(rooflines, key=lambda k: rooflines[k]["share_of_step"] or 0.0)
    roof = rooflines[kind]

    # end to end through the C ABI with host buffers: the step's inputs are
    # copied from pinned host memory each step and its results read back
    e2e = None
    if not args.no_e2e:
        host_in = [t.cpu().pin_memory() for t in plan._keep if isinstance(t, torch.Tensor)]
        dev_in = [t for t in plan._keep if isinstance(t, torch.Tensor)]
        m_host = m_d.cpu().pin_memory()
        mom_host = torch.empty_like(mom_d, device="cpu").pin_memory()
        lp_host_t = torch.empty_like(lp_d, device="cpu").pin_memory()
        m_back = torch.empty_like(m_d, device="cpu").pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host_in) + m_host.numel() * 8
        d2h = mom_host.numel() * 8 + lp_host_t.numel() * 8 + m_back.numel() * 8
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                for h, d in zip(host_in, dev_in):
                    d.copy_(h, non_blocking=True)
                m_d.copy_(m_host, non_blocking=True)
                plan.mstep(None, m_d, q_d, EMA_LAMBDA, t=t_iter)
                step(t_iter)
                t_iter += 1
                mom_host.copy_(mom_d, non_blocking=True)
                lp_host_t.copy_(lp_d, non_blocking=True)
                m_back.copy_(m_d, non_blocking=True)
            e1.record(stream)
        stream.synchronize()
        barrier(ws)
        e_ms, e_pairs = aggregate(e0.elapsed_time(e1), pairs * args.steps, ws, device="cuda")
        e2e = {"value": e_pairs / (e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if ws == 1 and rank == 0 and not args.no_cpu_baseline:
        cpu, _ = cpu_oracle_sample(args.workload, args.cpu_seconds, qcond=args.qcond)

    if rank == 0:
        ws_bytes = plan.workspace_bytes
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "bf16": "bf16",
                                                                   "bf16x3": "bf16x3", "tf32": "tf32"}[precision],
                "data": "synthetic",
                "config": {"workload": args.workload, "K": K, "pairs_per_step_per_gpu": pairs,
                           "precision": precision, "noise": "in-kernel Philox4x32-10",
                           "step": "qem_estep + qem_mstep (one Alg. 1 iteration)",
                           "state": f"EM steady state: {CONVERGE_ITERS} iterations from q_0 before the "
                                    f"{args.warmup} warm-up and {args.steps} timed steps",
                           "l2": f"working set {ws_bytes / 1e9:.2f} GB > 129 MB L2 (no flush)",
                           "parallelism": f"replicas x{ws} (independent instances)",
                           "launch_shapes": plan.tuning(),
                           "proposal": "parent-conditioned, permutation copies" if args.qcond else "factorised"},
                "graph_loop": graph_loop,
                "roofline": roof, "rooflines": rooflines, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": gpu_launches,
                "clocks": clk, "kernels_ms": {k: round(v[0], 4) for k, v in prof.items()},
                "log_pmp_last": float(lp_host[0])}
        print(json.dumps(line))
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_split_root(args):
    """E-step + M-step with the split root (qem_estep_split_root): pairs per
    step = users x K^2 parent pairs x K child samples.  One GPU; FP32."""
    import torch

    from paper_2503_08264_gb300 import qem

    builder, K, _ = WORKLOADS[args.workload]
    model = builder(1000)
    if len(model.levels) != 2 or model.levels[1].prior != S.PRIOR_NORMAL_MEAN_LOGVAR:
        raise SystemExit("--root split needs a two-level mean/log-variance model")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        plan = qem.Plan(model, K, precision="fp32", stream=stream)
        q_d = plan.flat(S.initial_q(model))
        m_d = plan.mean_params(q_d)
        mom_d = torch.empty(plan.q_len, dtype=torch.float64, device="cuda")
        lp_d = torch.empty(plan.n_inst, dtype=torch.float64, device="cuda")
        rw_d = torch.empty((plan.n_inst, 2, K), dtype=torch.float32, device="cuda")
    n_users = model.levels[1].n
    pairs = float(n_users) * K ** 3
    seed = 4321

    def step(t):
        plan.estep_split_root(q_d, None, seed=seed, it=t, moments=mom_d, log_pmp=lp_d, root_weights=rw_d)
        plan.mstep(mom_d, m_d, q_d, EMA_LAMBDA, t=t)

    t_iter = 1
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(t_iter)
            t_iter += 1
    stream.synchronize()
    plan.log_pmp()
    clocks = ClockSampler(0)
    clocks.start()
    plan.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            step(t_iter)
            t_iter += 1
        ev1.record(stream)
    stream.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = plan.profile_read()
    plan.profile(False)
    lp_host = plan.log_pmp()
    sm_max = clk.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2070.0)
    f_ms, f_n = prof["forward"]
    roof = roofline_for("forward", "fp32", model.levels[1].dim, pairs * f_n, f_ms, sm_max)
    roof["traffic"] = None
    roof["share_of_step"] = f_ms / ms if ms else None
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import split_root as R
        m_s = max(1, min(n_users, 40))
        sub = S.hier_logistic(M=m_s, N=model.levels[1].n_obs, D=model.levels[1].dim, seed=7)
        q_s = S.initial_q(sub)
        eps_s = S.noise(sub, K, seed=8)
        t0 = time.perf_counter()
        R.estep(sub, q_s, K, eps_s)
        dt = time.perf_counter() - t0
        cpu = {"value": m_s * K ** 3 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one FP64 split-root E-step of {m_s} users (numpy; the oracle's BLAS may use more "
                         f"threads), {dt:.1f} s"}
    line = {"metric": METRIC, "value": pairs * args.steps / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "root": "split (mean and log-variance as separate latents)",
                       "K": K, "pairs_per_step_per_gpu": pairs, "precision": "fp32",
                       "noise": "in-kernel Philox4x32-10",
                       "step": "qem_estep_split_root + qem_mstep (one Alg. 1 iteration)"},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            "kernels_ms": {k: round(v[0], 4) for k, v in prof.items()}, "log_pmp_last": float(lp_host[0])}
    print(json.dumps(line))
    plan.close()
    return 0


def run_unit_peaks():
    """The roofline denominators' per-SM unit rates, measured on this GPU
    (probes/unit_peaks.cu), with the clocks seen while they ran."""
    from paper_2503_08264_gb300 import build as B
    exe = B.build_unit_peaks()
    clocks = ClockSampler(0)
    clocks.start()
    r = subprocess.run([exe], capture_output=True, text=True)
    clk = clocks.stop()
    if r.returncode != 0:
        raise SystemExit(f"unit_peaks failed ({r.returncode}): {r.stderr[-500:]}")
    line = json.loads(r.stdout.strip().splitlines()[-1])
    line["clocks"] = clk
    print(json.dumps(line))
    return 0


def main(argv=None):
    args = parse(argv)
    if args.unit_peaks:
        return run_unit_peaks()
    if args.impl == "reference":
        return run_reference(args)
    if args.small_case:
        return run_small_case(args.small_case)
    if args.metric == "time_to_tol":
        return run_time_to_tol(args)
    if args.root == "split":
        return run_split_root(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
