#!/usr/bin/env python
"""Throughput benchmark of the batched PN inspiral integrator on B300.

One step = one pass of the hot path over one batch: integrate the
1,048,576-binary ensemble (equal mass, chi_i ~ U[0,1], isotropic spins,
M omega 0.01 -> 0.05; Dormand-Prince 5(4) at tolerance 5e-7, h0 = 10, stop on
omega_f) with the inputs resident in HBM.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank integrates its own ensemble (a different seed) of the
same size: independent binaries, no data exchange ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import csv
import ctypes as C
import hashlib
import io
import json
import re
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "inspirals/sec (Mω 0.01→0.05) & % FP64 peak; mixed vs FP64 at ≤1e-6 dot err"
WORKLOAD = ("1,048,576 binaries, m1 = m2 = 0.5, chi_i ~ U[0,1], isotropic spin directions, L-hat = z, "
            "M omega 0.01 -> 0.05, DP5(4) tol 5e-7, h0 = 10, stop on omega_f")

# Algorithmic floating-point operations of one Dormand-Prince attempt, as the
# plain FP64 formulation counts them (each +, -, *, / one operation; no FMA):
# the right-hand side of Eqs. (1)-(4) is 118 operations (+ 1 cbrt + 1 log) and
# is evaluated 6 times per attempt; the stages, the error norm and the step
# control add 633 (+ 1 sqrt + 1 pow).  tests/test_bench_constants.py checks
# these against the oracle's operation counter.
FLOPS_RHS = 118
FLOPS_STEP = 633
FLOPS_ATTEMPT = 6 * FLOPS_RHS + FLOPS_STEP
FP64_DATASHEET_TFLOPS = 1.25  # nominal dense FP64 of one B300

# DRAM traffic of the integration kernel per binary from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, profiles/); valid only while
# the kernel sources hash (kernel_sha) to the recorded value.
PROFILED = {"kernel_sha": "c18364a7dbdf2184", "dram_bytes_per_binary": (55.538e6 + 16.341e6) / 131072}


# Executed floating-point thread instructions per attempt of each integration kernel
# k_integrate_mx<PREC> (PREC 0 FP64, 1 FP32 right-hand side, 2 double-single) at the persistent
# schedule, and of the double-single kernel at the plain schedule (its own register budget), from one
# ncu capture of the 131,072-binary case (profiles/k_integrate_pipes_C1_131072.md): sums of
# smsp__sass_thread_inst_executed_op_{ffma,fadd,fmul,ffma2,fadd2,fmul2,dfma,dadd,dmul}_pred_on over
# the launch divided by its attempts.  Valid only while the kernel sources hash to kernel_sha.
EXECUTED = {"kernel_sha": "c18364a7dbdf2184", "per_attempt": {
    0: {"ffma": 130.84, "fadd": 397.46, "fmul": 93.55, "ffma2": 0.0, "fadd2": 0.0, "fmul2": 0.0,
        "dfma": 505.94, "dadd": 44.96, "dmul": 242.83},
    1: {"ffma": 232.97, "fadd": 29.45, "fmul": 267.58, "ffma2": 190.0, "fadd2": 395.0, "fmul2": 55.0,
        "dfma": 15.97, "dadd": 10.96, "dmul": 10.91},
    2: {"ffma": 1252.84, "fadd": 2745.46, "fmul": 516.83, "ffma2": 495.0, "fadd2": 1090.0, "fmul2": 165.0,
        "dfma": 45.94, "dadd": 60.96, "dmul": 18.83}},
    "per_attempt_plain": {
    2: {"ffma": 1252.84, "fadd": 2745.46, "fmul": 516.83, "ffma2": 495.0, "fadd2": 1090.0, "fmul2": 165.0,
        "dfma": 45.94, "dadd": 60.96, "dmul": 17.89}}}


def executed_flops(prec: int, plain: bool = False):
    """(FP32, FP64) flops one attempt executes (an FMA is 2, a packed pair instruction 2 lanes) in the
    kernel of that precision at the persistent schedule (or at the plain one, where it was captured), or
    None when no capture of the current kernel sources is recorded."""
    table = EXECUTED["per_attempt"]
    if plain and prec in EXECUTED["per_attempt_plain"]:
        table = EXECUTED["per_attempt_plain"]
    if EXECUTED["kernel_sha"] != kernel_sha() or prec not in table:
        return None
    c = table[prec]
    f32 = 2 * c["ffma"] + c["fadd"] + c["fmul"] + 2 * (2 * c.get("ffma2", 0) + c.get("fadd2", 0) + c.get("fmul2", 0))
    f64 = 2 * c["dfma"] + c["dadd"] + c["dmul"]
    return f32, f64


def kernel_sha() -> str:
    """Hash of the integration kernel's sources with comments and blank space removed (so an edit to a
    comment does not count as a kernel change)."""
    h = hashlib.sha256()
    for f in ("pn_device.cuh", "pn_kernels.cu", "pn_internal.h"):
        with open(os.path.join(ROOT, "paper_0908_3889_b300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=1_048_576, help="binaries per rank (default: the full workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape 'plain|persistent:BLOCK[:BPT]' for every precision instead of the "
                         "autotuner (a run under a profiler uses it: the tuner's own timings are distorted there)")
    ap.add_argument("--science", choices=("ks",), default=None,
                    help="instead of the benchmark: Sec. V B's uniformity test at the paper's size (equal mass, "
                         "chi = 0.7, isotropic spins, M omega 0.00395 -> 0.05, 362,799,815 inspirals), sampled "
                         "and integrated on the device in chunks, final S1-hat.S2-hat binned into 2^20 bins, "
                         "one-sample KS test against U[-1, 1]")
    ap.add_argument("--science-n", type=int, default=362_799_815)
    ap.add_argument("--science-precision", type=int, default=0, help="0 FP64, 1 FP32 RHS, 2 double-single")
    ap.add_argument("--profile-case", choices=("integrate", "stops", "adjoint", "adjoint_ds"), default=None,
                    help="no timing, the small cases the ncu section captures run: 'integrate' integrates the "
                         "first --n binaries of the workload once per precision (persistent schedule, 256 "
                         "threads), then in double-single at the plain schedule (128 threads); 'stops' "
                         "integrates them in FP64 once with the landing stop and once with the "
                         "first-crossing stop; 'adjoint' runs one pn_batch_adjoint over the 65,536-binary "
                         "adjoint ensemble, 'adjoint_ds' the same with the double-single reverse sweep")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Each rank integrates its own ensemble of the same shape (independent binaries: weak scaling)."""
    import workloads
    return workloads.SEED_BASE + 1 + 1000 * rank


def aggregate_rate(world: int, n_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job inspirals/s: all ranks' binaries over the slowest rank's time."""
    return world * n_per_rank * steps / (max_ms * 1e-3)


def init_dist(backend: str, device_id=None, timeout_s: float | None = None):
    """Join the process group with a bounded timeout.

    A rank that never joins makes the others' rendezvous fail after timeout_s, and a
    rank that leaves between steps makes the others' next barrier or reduction raise
    (at once when its connection closes, else after timeout_s) instead of waiting
    forever.  Default: PN_DIST_TIMEOUT_S from the environment, else 300 s.
    """
    import datetime

    import torch.distributed as tdist
    if timeout_s is None:
        timeout_s = float(os.environ.get("PN_DIST_TIMEOUT_S", "300"))
    kw = {"timeout": datetime.timedelta(seconds=timeout_s)}
    if device_id is not None:
        kw["device_id"] = device_id
    tdist.init_process_group(backend, **kw)
    return tdist


def reduce_max(x: float, tdist, device) -> float:
    """Max over ranks (a timing reduction only; no data moves between ranks)."""
    if tdist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index: int):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(index), "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                smax.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peak_probe(index: int = 0):
    """FP64 and FP32 FMA throughput (flop/s) measured live, and the clocks sampled while the probe ran."""
    from paper_0908_3889_b300.build import PEAK_LIB
    lib = C.CDLL(PEAK_LIB)
    lib.pn_peak_probe.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
    f64, f32 = C.c_double(), C.c_double()
    clocks = ClockSampler(index)
    time.sleep(0.3)  # the sampler's first reading
    rc = lib.pn_peak_probe(C.byref(f64), C.byref(f32))
    ck = clocks.stop()
    lib.pn_peak_probe_packed.argtypes = [C.POINTER(C.c_double)] * 4
    f2, l32, l2, l64 = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    if lib.pn_peak_probe_packed(C.byref(f2), C.byref(l32), C.byref(l2), C.byref(l64)) == 0:
        ck["packed_f32x2_fma_tflops"] = f2.value / 1e12
        ck["fma_latency_cycles"] = {"f32": l32.value, "f32x2": l2.value, "f64": l64.value}
    if rc != 0:
        return None, None, ck
    return f64.value, f32.value, ck


def cpu_oracle_rate(ens, target_s: float = 10.0, threads: int = 0):
    """Time the CPU oracle on a bounded sample of the ensemble (about target_s seconds)."""
    import oracle
    import workloads
    n_all = ens["m1"].shape[0]
    calib = workloads.take(ens, np.arange(min(2048, n_all)))
    oracle.integrate(calib, threads=threads)  # builds/loads the oracle
    t0 = time.perf_counter()
    r = oracle.integrate(calib, threads=threads)
    dt = time.perf_counter() - t0
    rate = calib["m1"].shape[0] / dt
    m = int(min(n_all, max(2048, rate * target_s)))
    sample = workloads.take(ens, np.arange(m))
    t0 = time.perf_counter()
    r = oracle.integrate(sample, threads=threads)
    dt = time.perf_counter() - t0
    return m / dt, m, int(r["threads_used"]), dt


def science_ks(args, pn, torch, dev):
    """Sec. V B: is the final S1-hat.S2-hat uniform?  Device sampling (pn_batch_sample), integration and a
    2^20-bin histogram per chunk of 2^24 binaries; the counts are summed on the host and tested with
    pn_ks_uniform.  Prints one JSON line."""
    total, chunk, bins = args.science_n, 1 << 24, 1 << 20
    d = pn.dist(q=(1.0, 1.0), q_mode=0, chi=(0.7, 0.7), chi_mode=0, omega0=(0.00395, 0.00395), omega_f=0.05)
    counts = np.zeros(bins, dtype=np.int64)
    status = np.zeros(8, dtype=np.int64)
    attempts = 0
    ms = 0.0
    t0 = time.perf_counter()
    with pn.Batch(min(chunk, total), pn.params(precision=args.science_precision)) as b:
        inp = pn.alloc_inputs(min(chunk, total), dev)
        out = pn.alloc_outputs(min(chunk, total), dev)
        done, c = 0, 0
        while done < total:
            n = min(chunk, total - done)
            pn.pn_batch_sample(b.handle, workloads_seed(c), d, n, inp)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            pn.pn_batch_integrate(b.handle, n, inp, out)
            e1.record()
            counts += pn.pn_batch_histogram(b.handle, n, inp, out, pn.native.PN_Q_FINAL_S1S2, bins)
            ms += e0.elapsed_time(e1)
            st = b.stats(inp, out, n)
            status += np.array(st["count_by_status"], dtype=np.int64)
            attempts += st["acc_total"] + st["rej_total"] + st["land_total"]
            done += n
            c += 1
    wall = time.perf_counter() - t0
    ks = pn.pn_ks_uniform(counts, -1.0, 1.0)
    hist100 = counts.reshape(100, -1).sum(axis=1) if bins % 100 == 0 else np.add.reduceat(
        counts, (np.arange(100) * bins) // 100)
    line = {"science": "Sec. V B uniformity of the final S1-hat.S2-hat (one-sample KS against U[-1, 1])",
            "n": total, "chunks": c, "precision": args.science_precision,
            "workload": "m1 = m2 = 0.5, chi1 = chi2 = 0.7, isotropic spin directions, L-hat = z, "
                        "M omega 0.00395 -> 0.05, DP5(4) tol 5e-7, h0 = 10",
            "integrate_ms": ms, "inspirals_per_s": total / (ms * 1e-3), "wall_s": wall,
            "attempts_per_binary": attempts / total, "count_by_status": status.tolist(),
            "ks": ks, "histogram_100_bins": hist100.tolist(),
            "paper": {"n": 362_799_815, "p_value": 5.17e-5, "hardware": "Tesla S1070 GPUs, FP32"}}
    print(json.dumps(line), flush=True)


def workloads_seed(chunk: int) -> int:
    """Seed of chunk c of the science run (counter-based draws: chunks are independent)."""
    return 0x0908_3889_5B00 + chunk


def bench_config(n: int, world: int) -> dict:
    """The workload both arms measure (the same dict in the GPU line and the oracle's line)."""
    return {"workload": WORKLOAD, "n_binaries_per_gpu": n, "precision": "fp64",
            "l2": "GPU arm: L2 flushed before each step (256 MB write)", "parallelism": f"replicas x{world}"}


def reference_arm(args, rank, world):
    """The oracle, as it stands, on the host cores: the base contract's reference arm for this path."""
    if rank != 0:
        return
    import workloads
    ens = workloads.config("C1", n=args.n)
    _, m, threads, _ = cpu_oracle_rate(ens, target_s=1.0)
    per_step = max(1024, m)
    import oracle
    total, count = 0.0, 0
    for s in range(args.warmup + args.steps):
        idx = (np.arange(per_step) + s * per_step) % ens["m1"].shape[0]
        sample = workloads.take(ens, idx)
        t0 = time.perf_counter()
        oracle.integrate(sample)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            total += dt
            count += per_step
    value = count / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "inspirals/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(ens["m1"].shape[0], world),
            "cpu_baseline": {"value": value, "unit": "inspirals/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} binaries of the 1,048,576-binary ensemble per step"},
            "e2e": {"value": value, "unit": "inspirals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_0908_3889_b300 as pn
    import workloads
    from paper_0908_3889_b300.build import build

    if world > 1:
        torch.cuda.set_device(local)
        tdist = init_dist("nccl", device_id=torch.device("cuda", local))
    else:
        tdist = None
        torch.cuda.set_device(0)
    if rank == 0:
        build()
    if tdist:
        tdist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if tdist:
            tdist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, tdist, dev)

    n = args.n
    ens = workloads.config("C1", n=n, seed=rank_seed(rank))
    inp = pn.to_device(ens, device=dev)
    out = pn.alloc_outputs(n, dev)
    if args.science == "ks":
        science_ks(args, pn, torch, dev)
        return
    if args.profile_case in ("adjoint", "adjoint_ds"):
        c4 = workloads.config("C4")
        n4 = c4["m1"].shape[0]
        inp4 = pn.to_device(c4, device=dev)
        cot = {"dot_s1s2": torch.ones(n4, dtype=torch.float64, device=dev)}
        grads = {f: torch.empty(n4, dtype=torch.float64, device=dev) for f in pn.native.GRAD_FIELDS}
        with pn.Batch(n4, pn.params(precision=2 if args.profile_case == "adjoint_ds" else 0)) as b:
            pn.pn_batch_adjoint(b.handle, n4, inp4, cot, grads)
            torch.cuda.synchronize()
        print(json.dumps({"profile_case": "C4 " + args.profile_case, "n": n4}))
        return
    if args.profile_case == "integrate":
        attempts = {}
        persist, plain = pn.native.PN_SCHED_PERSISTENT, pn.native.PN_SCHED_PLAIN
        runs = [(pn.native.PN_FP64, persist, 256), (pn.native.PN_MIXED, persist, 256),
                (pn.native.PN_MIXED_DS, persist, 256), (pn.native.PN_MIXED_DS, plain, 128)]
        for prec, sched, block in runs:
            with pn.Batch(n, pn.params(precision=prec, schedule=sched, block=block, bpt=1)) as b:
                b.integrate(inp, out)
                torch.cuda.synchronize()
                st = b.stats(inp, out)
                key = str(prec) + ("" if sched == persist else " plain")
                attempts[key] = st["acc_total"] + st["rej_total"] + st["land_total"]
        print(json.dumps({"profile_case": "C1", "n": n, "launches": ["fp64", "fp32 rhs", "double-single",
                                                                     "double-single plain 128"],
                          "attempts": attempts}))
        return
    if args.profile_case == "stops":
        attempts = {}
        for mode in (pn.native.PN_STOP_LAND, pn.native.PN_STOP_FIRST_CROSS):
            with pn.Batch(n, pn.params(precision=pn.native.PN_FP64, schedule=pn.native.PN_SCHED_PERSISTENT,
                                       block=256, stop_mode=mode)) as b:
                b.integrate(inp, out)
                torch.cuda.synchronize()
                st = b.stats(inp, out)
                attempts[mode] = st["acc_total"] + st["rej_total"] + st["land_total"]
        print(json.dumps({"profile_case": "C1 stops", "n": n, "stop_modes": [0, 1], "attempts": attempts}))
        return
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2 (126 MB)

    f64_peak, f32_peak, probe_clocks = peak_probe(torch.cuda.current_device())

    def timed_run(b, steps, warmup):
        for _ in range(warmup):
            b.integrate(inp, out)
        barrier()
        clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
        t_wall0 = time.perf_counter()
        total_ms = 0.0
        kernel_ms = 0.0
        stream = torch.cuda.current_stream()
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.integrate(inp, out)
            e1.record(stream)
            e1.synchronize()
            total_ms += e0.elapsed_time(e1)
            kernel_ms += b.timing()[1]  # the integration kernel alone (events on the batch's stream)
        barrier()
        wall = time.perf_counter() - t_wall0
        ck = clocks.stop() if clocks else None
        timed_run.kernel_ms = kernel_ms
        return total_ms, wall, ck

    fixed = None
    if args.shape:
        parts = args.shape.split(":")
        fixed = {"schedule": {"plain": 1, "persistent": 2}[parts[0]], "block": int(parts[1]),
                 "bpt": int(parts[2]) if len(parts) > 2 else 1}

    def shaped(b, prec_params):
        """Fix the batch's launch shape, or let the autotuner choose it; returns the shape."""
        if fixed is None:
            return b.autotune(inp)
        b.set_params(pn.params(**prec_params, **fixed))
        return dict(fixed)

    nvtx = torch.cuda.nvtx  # phase ranges for profilers
    nvtx.range_push("fp64 headline")
    # FP64 headline.
    prm = pn.params(precision=0)
    with pn.Batch(n, prm) as b:
        tune = shaped(b, {"precision": 0})
        total_ms, wall, clocks = timed_run(b, args.steps, args.warmup)
        kernel_ms_step = timed_run.kernel_ms / args.steps
        st = b.stats(inp, out)
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = aggregate_rate(world, n, args.steps, total_ms)
    attempts = st["acc_total"] + st["rej_total"] + st["land_total"]
    flops_launch = FLOPS_ATTEMPT * attempts
    achieved = flops_launch / (kernel_ms_step * 1e-3)
    fp64_out = {k: out[k].clone() for k in ("dot_s1s2", "dot_ls1", "dot_ls2", "status", "t", "omega", "S1", "S2",
                                            "Lhat")}
    sha = kernel_sha()
    traffic = (PROFILED["dram_bytes_per_binary"] * n
               if PROFILED["kernel_sha"] == sha and PROFILED["dram_bytes_per_binary"] else None)
    roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": (f64_peak or 0) / 1e12, "unit": "TFLOP/s",
            "frac": achieved / f64_peak if f64_peak else None, "traffic": traffic,
            "pipe": "FP64", "peak_source": "FP64 FMA throughput measured live by the peak probe (2 flops per FMA)",
            "datasheet_peak": FP64_DATASHEET_TFLOPS, "frac_of_datasheet": achieved / 1e12 / FP64_DATASHEET_TFLOPS,
            "flops_per_attempt": FLOPS_ATTEMPT, "attempts_per_launch": attempts,
            "kernel": "pn::k_integrate_mx<FP64>", "kernel_ms_per_launch": kernel_ms_step,
            "timing": "CUDA events around the integration kernel alone on the batch's stream (pn_batch_timing), "
                      "averaged over the timed steps"}
    ex64 = executed_flops(0)
    if ex64 is not None and f64_peak:
        roof["fp64_flops_per_attempt_executed"] = ex64[1]
        roof["fp64_pipe_executed_frac"] = ex64[1] * attempts / (kernel_ms_step * 1e-3) / f64_peak

    # Mixed precision on the same ensemble: FP32 right-hand side (PN_MIXED) and
    # double-single right-hand side on the FP32 pipe (PN_MIXED_DS).
    def mixed_run(prec):
        with pn.Batch(n, pn.params(precision=prec)) as b:
            tn = shaped(b, {"precision": prec})
            mix_ms, _, _ = timed_run(b, args.steps, 1)
            mix_kernel_ms = timed_run.kernel_ms / args.steps
            mst = b.stats(inp, out)
        mix_ms = max_over_ranks(mix_ms)
        ok = (fp64_out["status"] == 0) & (out["status"] == 0)
        errs = {}
        for k in ("dot_s1s2", "dot_ls1", "dot_ls2"):
            d = (out[k] - fp64_out[k]).abs()[ok & torch.isfinite(fp64_out[k])]
            errs[k] = {"max": float(d.max()), "p99": float(torch.quantile(d[:1_000_000].float(), 0.99)),
                       "p50": float(d.median())}
        # other outputs: relative error of t and omega; S1, S2, L-hat components scaled by their
        # vector's FP64 magnitude
        for k in ("t", "omega"):
            d = ((out[k] - fp64_out[k]).abs() / fp64_out[k].abs())[ok]
            errs[k] = {"max": float(d.max()), "p50": float(d.median())}
        for k in ("S1", "S2", "Lhat"):
            mag = torch.linalg.vector_norm(fp64_out[k], dim=0)
            keep = ok & (mag > 0)
            d = ((out[k] - fp64_out[k]).abs().amax(dim=0) / torch.where(mag > 0, mag, 1.0))[keep]
            errs[k] = {"max": float(d.max()), "p50": float(d.median())}
        m_attempts = mst["acc_total"] + mst["rej_total"] + mst["land_total"]
        sec = mix_kernel_ms * 1e-3  # the integration kernel alone
        plain = tn["schedule"] == pn.native.PN_SCHED_PLAIN
        ex = executed_flops(prec, plain=plain)
        roof_m = None
        if ex is not None and f32_peak and f64_peak:
            a32, a64 = ex[0] * m_attempts / sec, ex[1] * m_attempts / sec
            roof_m = {"bound": "issue/latency", "pipe": "FP32", "achieved": a32 / 1e12, "peak": f32_peak / 1e12,
                      "unit": "TFLOP/s", "frac": a32 / f32_peak,
                      "peak_source": "FP32 FMA throughput measured live by the peak probe (2 flops per FMA)",
                      "fp32_flops_per_attempt_executed": ex[0],
                      "fp64_pipe": {"achieved": a64 / 1e12, "peak": f64_peak / 1e12, "frac": a64 / f64_peak,
                                    "fp64_flops_per_attempt_executed": ex[1]},
                      "counts": "executed instructions per attempt from ncu (profiles/), scaled by this run's attempts",
                      "kernel": f"pn::k_integrate_mx<{prec}, {'plain' if plain else 'persistent'}>",
                      "kernel_ms_per_launch": mix_kernel_ms}
        return {"value": aggregate_rate(world, n, args.steps, mix_ms), "unit": "inspirals/s",
                "ms_per_step": mix_ms / args.steps, "speedup_vs_fp64": total_ms / mix_ms,
                "dot_err_vs_fp64": {k: errs[k] for k in ("dot_s1s2", "dot_ls1", "dot_ls2")},
                "other_err_vs_fp64": {k: errs[k] for k in ("t", "omega", "S1", "S2", "Lhat")},
                "schedule": {1: "plain", 2: "persistent"}.get(tn["schedule"]), "block": tn["block"],
                "attempts_per_binary": m_attempts / n,
                "algorithmic_tflops": FLOPS_ATTEMPT * m_attempts / sec / 1e12, "roofline": roof_m}

    nvtx.range_pop()
    nvtx.range_push("mixed precision")
    mixed = mixed_ds = None
    if not args.no_mixed:
        mixed = mixed_run(1)
        mixed["rhs"] = "FP32"
        mixed_ds = mixed_run(2)
        mixed_ds["rhs"] = "double-single (pairs of FP32) on the FP32 pipe"

    nvtx.range_pop()
    nvtx.range_push("end to end")
    # End to end through the host-buffer entry point (pinned host memory).
    e2e = None
    if not args.no_e2e:
        hin = pn.to_device(ens, device="cpu", pin_memory=True)
        hout = pn.alloc_outputs(n, pin_memory=True)
        with pn.Batch(n, prm) as b:
            shaped(b, {"precision": 0})
            for _ in range(max(1, args.warmup)):
                pn.pn_batch_integrate_host_async(b.handle, n, hin, hout)
            pn.pn_batch_host_wait(b.handle)
            barrier()
            # Each step copies its inputs in and its results out; consecutive asynchronous calls
            # overlap those copies with the neighbouring steps' integrations.
            t0 = time.perf_counter()
            for _ in range(args.steps):
                pn.pn_batch_integrate_host_async(b.handle, n, hin, hout)
            pn.pn_batch_host_wait(b.handle)
            barrier()
            e2e_s = max_over_ranks(time.perf_counter() - t0)
            # The synchronous call (copy in, integrate, copy out, wait) per step, for comparison.
            t0 = time.perf_counter()
            for _ in range(args.steps):
                pn.pn_batch_integrate_host(b.handle, n, hin, hout)
            barrier()
            sync_s = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": aggregate_rate(world, n, args.steps, e2e_s * 1e3), "unit": "inspirals/s",
               "h2d_bytes_per_step": 15 * 8 * n, "d2h_bytes_per_step": (14 * 8 + 4 * 4) * n,
               "api": "pn_batch_integrate_host_async per step (pinned host buffers), pn_batch_host_wait at the end",
               "synchronous_calls": {"value": aggregate_rate(world, n, args.steps, sync_s * 1e3),
                                     "api": "pn_batch_integrate_host per step"}}

    nvtx.range_pop()
    nvtx.range_push("extras")
    # Extras: the uneven-length ensemble (persistent vs plain schedule) and the adjoint.
    extras = None
    if not args.no_extras:
        extras = {}
        # The headline ensemble at fixed schedules: the plain FP64 kernel against the persistent
        # double-single one (the mixed form at the 1e-6 dot bar, in the persistent schedule).
        c1_shapes = {}
        for key, prec, sched, block in (("fp64_plain", 0, 1, 256), ("mixed_ds_persistent", 2, 2, 128)):
            with pn.Batch(n, pn.params(precision=prec, schedule=sched, block=block)) as b:
                rate_ms, _, _ = timed_run(b, args.steps, 1)
            rate_ms = max_over_ranks(rate_ms)
            c1_shapes[key] = {"value": aggregate_rate(world, n, args.steps, rate_ms), "unit": "inspirals/s",
                              "ms_per_step": rate_ms / args.steps, "block": block,
                              "schedule": {1: "plain", 2: "persistent"}[sched]}
        c1_shapes["mixed_ds_persistent"]["speedup_vs_fp64_plain"] = (
            c1_shapes["mixed_ds_persistent"]["value"] / c1_shapes["fp64_plain"]["value"])
        extras["C1_fixed_schedules"] = c1_shapes
        c2 = workloads.config("C2", seed=workloads.SEED_BASE + 2 + 1000 * rank)
        n2 = c2["m1"].shape[0]
        inp2 = pn.to_device(c2, device=dev)
        out2 = pn.alloc_outputs(n2, dev)
        for name, sched in (("plain", 1), ("persistent", 2)):
            for prec, pname in ((0, "fp64"), (2, "mixed_ds")):
                blk2 = 256 if prec == 0 else 128  # each precision's best block (double-single: 3 blocks per SM)
                with pn.Batch(n2, pn.params(precision=prec, schedule=sched, block=blk2)) as b:
                    b.integrate(inp2, out2)
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    b.integrate(inp2, out2)
                    e1.record()
                    e1.synchronize()
                    ms2 = max_over_ranks(e0.elapsed_time(e1))
                    st2 = b.stats(inp2, out2)
                extras[f"uneven_C2_{pname}_{name}"] = {"value": aggregate_rate(world, n2, 1, ms2),
                                                      "unit": "inspirals/s", "ms": ms2, "block": blk2,
                                                      "accepted_steps_min_max": [st2["acc_min"], st2["acc_max"]],
                                                      "attempts_min_max": [st2["attempts_min"], st2["attempts_max"]]}
        del inp2, out2
        c4 = workloads.config("C4", seed=workloads.SEED_BASE + 4 + 1000 * rank)
        n4 = c4["m1"].shape[0]
        inp4 = pn.to_device(c4, device=dev)
        cot = {"dot_s1s2": torch.ones(n4, dtype=torch.float64, device=dev)}
        grads = {f: torch.empty(n4, dtype=torch.float64, device=dev) for f in pn.native.GRAD_FIELDS}
        def adjoint_ms(precision):
            with pn.Batch(n4, pn.params(precision=precision)) as b:
                pn.pn_batch_adjoint(b.handle, n4, inp4, cot, grads)
                ms_adj = []
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    pn.pn_batch_adjoint(b.handle, n4, inp4, cot, grads)  # recording forward + reverse sweep
                    e1.record()
                    e1.synchronize()
                    ms_adj.append(e0.elapsed_time(e1))
            return max_over_ranks(min(ms_adj))

        ms4 = adjoint_ms(0)
        ms4ds = adjoint_ms(2)
        # Sec. IV's performance workload: one test inspiral, omega 0.004 -> 0.1, replicated (lock-step).
        pp = workloads.config("PAPER_PERF", n=1_048_576, seed=workloads.SEED_BASE + 6 + 1000 * rank)
        inpp = pn.to_device(pp, device=dev)
        outp = pn.alloc_outputs(pp["m1"].shape[0], dev)
        pp_dots = {}
        for prec, key in ((0, "paper_test_inspiral_fp64"), (1, "paper_test_inspiral_mixed_fp32"),
                          (2, "paper_test_inspiral_mixed_ds")):
            with pn.Batch(pp["m1"].shape[0], pn.params(precision=prec)) as b:
                b.integrate(inpp, outp)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                b.integrate(inpp, outp)
                e1.record()
                e1.synchronize()
                msp = max_over_ranks(e0.elapsed_time(e1))
            dots = {k: outp[k].clone() for k in ("dot_s1s2", "dot_ls1", "dot_ls2")}
            if prec == 0:
                pp_dots = dots
            extras[key] = {
                "value": aggregate_rate(world, pp["m1"].shape[0], 1, msp), "unit": "inspirals/s", "ms": msp,
                "workload": "one seeded inspiral, omega 0.004 -> 0.1, 1,048,576 copies (Sec. IV lock-step test)",
                "paper_gpu_2009": {"value": 2700.0, "unit": "inspirals/s",
                                   "hardware": "1 GPU of a Tesla S1070, FP32"}}
            if prec != 0:
                extras[key]["speedup_vs_fp64"] = extras["paper_test_inspiral_fp64"]["ms"] / msp
                extras[key]["max_dot_diff_vs_fp64"] = max(float((dots[k] - pp_dots[k]).abs().max())
                                                          for k in dots)
        del inpp, outp, pp_dots
        # Sec. V B-D's parameter sweeps: ten 100,000-binary ensembles (omega 0.00395 -> 0.05) in one
        # integrate launch, per-ensemble statistics from one segmented reduction.
        sw = workloads.paper_sweeps()
        sizes = [e["m1"].shape[0] for _, _, e in sw]
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        cat = {k: np.concatenate([e[k] for _, _, e in sw], axis=-1) for k in sw[0][2]}
        inps = pn.to_device(cat, device=dev)
        outs = pn.alloc_outputs(int(off[-1]), dev)
        with pn.Batch(int(off[-1]), pn.params(precision=0)) as b:
            b.integrate(inps, outs)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            b.integrate(inps, outs)
            e1.record()
            sst = b.stats_segments(inps, outs, off)
            e2.record()
            e2.synchronize()
            mss = max_over_ranks(e0.elapsed_time(e1))
        extras["paper_sweeps_one_launch"] = {
            "value": aggregate_rate(world, int(off[-1]), 1, mss), "unit": "inspirals/s", "ms": mss,
            "stats_ms": e1.elapsed_time(e2),
            "workload": "Sec. V B-D sweeps: r vs chi (0.1..0.9), the m1 = 0.4 chi = 0.05 ring, r vs m1 (0.5..0.3); "
                        "10 x 100,000 binaries, omega 0.00395 -> 0.05, one pn_batch_integrate + one "
                        "pn_batch_stats_segments",
            "pearson_s1s2": {f"{kind}={val}": s_["pearson_s1s2"] for (kind, val, _), s_ in zip(sw, sst)}}
        del inps, outs
        extras["adjoint_C4"] = {"value": aggregate_rate(world, n4, 1, ms4), "unit": "gradients/s", "ms": ms4,
                                "workload": "65,536 binaries, q ~ U[1,4], chi = 1, omega 0.01 -> 0.05; "
                                            "d(S1-hat.S2-hat final)/d(S1-hat, S2-hat, q), checkpoint every 64"}
        extras["adjoint_C4_ds_sweep"] = {"value": aggregate_rate(world, n4, 1, ms4ds), "unit": "gradients/s",
                                         "ms": ms4ds, "sweep": "double-single recording pass and reverse sweep"}

    nvtx.range_pop()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the host baseline is an N = 1 figure
        rate, m, threads, dt = cpu_oracle_rate(ens, target_s=10.0)
        rate1, m1_, _, _ = cpu_oracle_rate(workloads.take(ens, np.arange(4096)), target_s=2.0, threads=1)
        import oracle
        pp = workloads.config("PAPER_PERF", n=64)
        t0 = time.perf_counter()
        oracle.integrate(pp, threads=1)
        paper_rate = 64 / (time.perf_counter() - t0)
        cpu = {"value": rate, "unit": "inspirals/s", "cores": threads, "kind": "oracle",
               "sample": f"first {m} binaries of the ensemble ({dt:.1f} s on {threads} threads)",
               "single_thread_value": rate1,
               "paper_test_inspiral_single_thread": {"value": paper_rate, "unit": "inspirals/s",
                                                      "workload": "one inspiral omega 0.004 -> 0.1, 64 copies",
                                                      "paper_value_2009_xeon_e5410": 57.0}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "inspirals/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": bench_config(n, world),
                "launch": {"schedule": {1: "plain", 2: "persistent"}.get(tune["schedule"], tune["schedule"]),
                           "block": tune["block"], "binaries_per_thread": tune["bpt"],
                           "attempts_per_binary": attempts / n, "kernel_sha": sha},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                # per step: the lanes' order (k_len_key, k_len_count, k_scan_above, k_len_scatter) when
                # on, k_setup, k_integrate_mx, k_dots (the queue reset and the sort's bins are memset nodes)
                "gpu_launches": (7 if pn.params().order == pn.native.PN_ORDER_LENGTH else 3) * args.steps,
                "clocks": clocks, "mixed": mixed, "mixed_ds": mixed_ds, "extras": extras,
                "fp32_fma_peak_tflops": (f32_peak or 0) / 1e12, "fp64_fma_peak_tflops": (f64_peak or 0) / 1e12,
                "peak_probe_clocks": probe_clocks}
        print(json.dumps(line), flush=True)
    if tdist:
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
