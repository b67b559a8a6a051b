#!/usr/bin/env python
"""Throughput of scaling-and-squaring exp(A) (Bader, Blanes, Casas, arXiv:1710.10989)
through libbbcexpm.so. Prints one JSON line (rank 0).

Default workload (dense4096): one step = exp(A) of twelve 4096 x 4096 matrices:
six Gaussian N(0,1)/sqrt(N) rescaled to 1-norms {0.01, 0.1, 1, 5, 20, 100}
(seeds 1-6) and six non-normal upper-triangular ones (diagonal N(0,1), strict
upper N(0,1)*10, seeds 101-106) at the same norms; (m, s) by the theta rule at
u = 2^-53. The timed form is the split-precision one (products rebuilt from 6
BF16 slices on the tensor cores, exact slice sums, deflated diagonals: the
fewest slices that keep every run of this workload inside its 1e-12 relative
Frobenius tolerance); the plain FP64 form is timed beside it, and every run
checks the tolerance against it (FP64 GPU results sit within 1e-14 of the
oracle on this workload).

Other workloads (--workload): batch (20000 matrices, N in {8..256}, binary32
storage, one persistent graph-captured launch per step), small (one 64 x 64
matrix, latency), large (8192 x 8192, norms 0.5/5/50).
--impl reference times the CPU oracle instead, on the host cores.
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

from paper_1710_10989_gb300 import workloads as W  # noqa: E402

PI = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}
# DRAM traffic per launch of the dominant kernels from one ncu capture each (profiles/),
# keyed to the hash of the sources the captured kernel is compiled from (its .cu file
# and the headers with inline device code), valid only while those are unchanged.
NCU_TRAFFIC = {
    "k_ozaki_pair": (("gemm_ozaki.cu", "internal.h", "slices.h"),
                     "cadb546e09d9627e042990469a781607e0fe320a0562a3492d6f5b3365f89be2", 4096,
                     ((2.930344e9 + 0.159464e9) + (1.159916e9 + 0.097516e9)) / 2),
}


def ncu_traffic(kernel: str, n: int):
    import hashlib
    if kernel not in NCU_TRAFFIC:
        return None
    sources, sha, n_cap, traffic = NCU_TRAFFIC[kernel]
    h = hashlib.sha256()
    try:
        for src in sources:
            h.update(open(os.path.join(ROOT, "paper_1710_10989_gb300", "csrc", src), "rb").read())
    except OSError:
        return None
    return traffic if (h.hexdigest() == sha and n == n_cap) else None


# FP64 pipe: the GB300's nominal 1.25 TFLOP/s FP64 is 2 DFMA per clock per SM:
# 152 SMs x 2 DFMA x 2 flop x 2.07 GHz (maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=("dense4096", "batch", "small", "large", "learned", "compare4096",
                                           "complex2048", "integrator"),
                    default="dense4096")
    ap.add_argument("--precision", choices=("ozaki", "fp64"), default="ozaki")
    ap.add_argument("--slices", type=int, default=6,
                    help="BF16 slices of the split-precision products (6: the fastest that keeps every "
                         "dense-4096 run within the 1e-12 tolerance; the library's own default is 7)")
    ap.add_argument("--n", type=int, default=0, help="override the matrix size of dense workloads")
    ap.add_argument("--count", type=int, default=W.BATCH_COUNT, help="batch size of --workload batch")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--u", choices=("double", "single"), default="double",
                    help="batch workload: backward-error target of the (m, s) selection, 2^-53 or 2^-24 "
                         "(Table 2's single-precision thresholds)")
    ap.add_argument("--selector", choices=("plain", "learned", "alpha"), default="learned",
                    help="(m, s) selection of the batch workload")
    return ap.parse_args()


# ------------------------------------------------------------------ workloads
def dense_workload(n: int):
    mats = [W.dense_case(i, n=n) for i in range(len(W.DENSE_NORMS))]
    mats += [W.dense_case(i, n=n, nonnormal=True) for i in range(len(W.DENSE_NORMS))]
    return mats


def large_workload(n: int):
    return [W.large_case(i, n=n) for i in range(len(W.LARGE_NORMS))]


def products_of(mats, u=2.0 ** -53, select=None) -> list[int]:
    """pi_m + s of each matrix's (m, s) by the theta rule: the library's selection,
    or `select(norm, u)` (the reference arm passes the oracle's)."""
    if select is None:
        from paper_1710_10989_gb300 import api
        select = api.select
    out = []
    for A in mats:
        m, s = select(float(np.abs(A.astype(np.float64)).sum(axis=0).max()), u)
        out.append(PI[m] + s)
    return out


# Order in which the reference arm's steps visit the twelve dense-workload matrices
# (indices into dense_workload: 0-5 Gaussian, 6-11 upper triangular, norms ascending):
# every run of four consecutive steps holds 28 products, the workload's mean of 7 per
# matrix, so any number of steps that is a multiple of four samples the mix exactly.
DENSE_CYCLE = (5, 6, 2, 9, 11, 0, 8, 3, 4, 7, 10, 1)
# The pair the main arm's CPU-baseline leg times (and checks the timed form against):
# the norm-100 Gaussian and the norm-100 upper-triangular matrix (12 products each).
DENSE_CPU_SAMPLE = (5, 11)


def dense_config(args, n: int, mats, prods, world: int) -> dict:
    """The workload description both arms print (inputs and their (m, s) only)."""
    return {"workload": WORKLOAD_DESC[args.workload].format(n=n),
            "n": n, "matrices_per_step": len(mats), "products_per_step": sum(prods),
            "u": "2^-53", "parallelism": "replicas" if world > 1 else "single",
            "l2": f"inputs larger than L2 (each exp(A) streams ~10 N^2 FP64 buffers of "
                  f"{n * n * 8 / 2 ** 20:.0f} MiB)"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.others_before = -1

    def other_compute_apps(self) -> int:
        """Compute processes on this GPU other than this one (GPU sharing check)."""
        try:
            out = subprocess.run(["nvidia-smi", "--query-compute-apps=pid", "--format=csv,noheader",
                                  "-i", str(self.device)], capture_output=True, text=True, timeout=10).stdout
        except (FileNotFoundError, OSError, subprocess.TimeoutExpired):
            return -1
        pids = [p.strip() for p in out.splitlines() if p.strip().isdigit()]
        return sum(1 for p in pids if int(p) != os.getpid())

    def start(self):
        self.others_before = self.other_compute_apps()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons),
                "other_compute_apps": max(self.others_before, self.other_compute_apps())}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


METRICS = {
    "dense4096": "expm/s (dense 4096x4096 exp(A), rel. Frobenius error <= 1e-12 vs FP64)",
    "large": "expm/s (dense 8192x8192 exp(A), rel. Frobenius error <= 1e-10 vs FP64)",
    "batch": "expm/s (batched exp(A), 20000 matrices N in 8..256, binary32 storage)",
    "small": "expm/s (single 64x64 exp(A), FP64, graph-replayed)",
    "learned": "expm/s (4096 held-out matrices N in 16..512, learned certified (m,s) selection)",
    "compare4096": "expm/s (dense 4096x4096 exp(A), new Taylor scheme; Paterson-Stockmeyer and Pade r_26 beside it)",
    "complex2048": "expm/s (dense complex 2048x2048 exp(A) via the 4096x4096 real form, rel. Frobenius error vs "
                   "the complex oracle)",
    "integrator": "system-steps/s (Lie-Euler steps Y <- exp(h Omega) Y, 4096 skew-symmetric systems N in 8..64, "
                  "one persistent launch per step)",
}
WORKLOAD_DESC = {
    "dense4096": "dense{n}: 6 Gaussian N(0,1)/sqrt(N) (seeds 1-6) + 6 non-normal upper-triangular "
                 "(seeds 101-106), 1-norms 0.01,0.1,1,5,20,100",
    "large": "large{n}: Gaussian N(0,1)/sqrt(N), seeds 1-3, 1-norms 0.5,5,50",
    "batch": "batch: N uniform on {{8,...,256}}, 1-norms log-uniform [1e-3, 1e2], half Gaussian, "
             "half V diag(lambda) V^-1 (cond(V)=1e3), seed 7",
    "small": "small64: N(0,1) seed 0, 1-norm 1.0, (m,s) = (18,0)",
    "compare4096": "the six Gaussian matrices of dense4096 (seeds 1-6, 1-norms 0.01,0.1,1,5,20,100)",
    "complex2048": "complex{n}: (N(0,1) + i N(0,1)) entries, seeds 201-203, complex 1-norms 0.5, 5, 50",
    "integrator": "4096 systems, seed 31: N uniform on {8,...,64}, h Omega = skew part of N(0,1) scaled to "
                  "1-norms log-uniform [0.01, 3], Y_0 orthogonal (QR), binary64",
    "learned": "4096 held-out matrices (GPU generator, seed 12): N uniform 16..512, 1-norms log-uniform "
               "[1e-3, 1e2], half Gaussian, half V diag(lambda) V^-1 (cond(V)=1e3)",
}


# ------------------------------------------------------------------ CPU oracle legs
def host_cpu() -> str:
    """Model name of the host CPU that ran the oracle (for the CPU-baseline record)."""
    try:
        with open("/proc/cpuinfo", errors="replace") as f:
            for row in f:
                if row.lower().startswith("model name"):
                    return row.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts list no model name in /proc/cpuinfo; lscpu decodes it
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for row in out.splitlines():
            if row.strip().lower().startswith("model name"):
                return row.split(":", 1)[1].strip()
    except (OSError, ValueError, subprocess.SubprocessError):
        pass
    return os.uname().machine


def cpu_dense_sample(mats, prods, idx=DENSE_CPU_SAMPLE):
    """The oracle, as it stands, on matrices `idx` of the workload (all host cores).
    Its time per product is scaled to the workload's mean products per exp(A)
    (the oracle's products all cost the same 2 N^3 triple loop); the sample's own
    rate is reported beside it. Returns the baseline and the oracle's outputs."""
    from oracle import oracle as O
    O.theta_array("new")  # thresholds are constants: computed (and cached) before timing
    outs, done = {}, 0
    t0 = time.perf_counter()
    for i in idx:
        A = mats[i]
        is_upper = not np.any(np.tril(A, -1))
        outs[i], info = O.expm_upper(A, "new") if is_upper else O.expm(A, "new")
        done += info.products
    dt = time.perf_counter() - t0
    mean_p = sum(prods) / len(prods)
    cpu = {"value": 1.0 / (dt / done * mean_p), "unit": "expm/s", "cores": O.num_threads(), "kind": "oracle",
           "value_of_sample": len(idx) / dt,
           "sample": (f"oracle exp(A) of workload matrices {list(idx)} (N={mats[0].shape[0]}, 1-norms "
                      f"{[round(float(np.abs(mats[i]).sum(0).max()), 3) for i in idx]}, {done} products in all) "
                      f"in {dt:.1f} s on {O.num_threads()} threads; its seconds per product scaled to the "
                      f"workload's mean of {mean_p:.2f} products per exp(A) (oracle selection)")}
    return cpu, outs


def cpu_batch_sample(mats, k=200):
    """The oracle on the first k matrices of the batch (a uniform sample of sizes/norms)."""
    from oracle import oracle as O
    O.theta_array("new")
    t0 = time.perf_counter()
    for A in mats[:k]:
        O.expm(A.astype(np.float64), "new")
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "expm/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"oracle exp(A) of the first {k} of the batch's matrices (binary32 inputs promoted "
                      f"to binary64) in {dt:.1f} s"}


def run_reference(args, rank: int, world: int):
    """The oracle as it stands on the host cores, on this arm's workload and config.
    Dense workloads: each step is the oracle's exp(A) of the next matrix of the
    workload (DENSE_CYCLE), value = matrices / seconds over the timed steps; no
    library code is loaded. The CPU needs no warm-up: --warmup is accepted and not run."""
    if rank != 0:
        return
    from oracle import oracle as O
    metric = METRICS[args.workload]
    O.theta_array("new")
    if args.workload == "batch":
        mats = W.batch_matrices(min(args.count, 400))
        cfg = {"workload": WORKLOAD_DESC["batch"], "count": args.count}
        k, t_all = 0, 0.0
        for st in range(args.steps):
            A = mats[st % len(mats)].astype(np.float64)
            t0 = time.perf_counter()
            O.expm(A, "new")
            t_all += time.perf_counter() - t0
            k += 1
        sample = f"one batch matrix per step (binary32 inputs promoted to binary64), {k} matrices"
    else:
        n = args.n or (W.LARGE_N if args.workload == "large" else 64 if args.workload == "small" else W.DENSE_N)
        mats = (large_workload(n) if args.workload == "large" else [W.small_case()] if args.workload == "small"
                else dense_workload(n))
        prods = products_of(mats, select=lambda v, u: O.select(v, "new", u))
        cfg = dense_config(args, n, mats, prods, world)
        cycle = DENSE_CYCLE if len(mats) == len(DENSE_CYCLE) else tuple(range(len(mats)))
        k, t_all, done = 0, 0.0, []
        for st in range(args.steps):
            i = cycle[st % len(cycle)]
            A = mats[i]
            is_upper = n > 1 and not np.any(np.tril(A, -1))
            t0 = time.perf_counter()
            _, info = O.expm_upper(A, "new") if is_upper else O.expm(A, "new")
            t_all += time.perf_counter() - t0
            done.append(info.products)
            k += 1
        sample = (f"one workload matrix per step, in the order {list(cycle)} (any four consecutive steps hold "
                  f"the workload's mean of {sum(prods) / len(prods):.2f} products per exp(A)); {k} matrices, "
                  f"{sum(done)} products")
    value = k / t_all
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": value, "unit": "expm/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": "expm/s", "cores": O.num_threads(), "kind": "oracle",
                         "cpu_model": host_cpu(), "sample": sample, "seconds": t_all},
        "e2e": {"value": value, "unit": "expm/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
        flush=True)


# ------------------------------------------------------------------ GPU legs
def timed(torch, dist, world, stream, fn, steps):
    """Barrier + sync on both sides, CUDA events on the launching stream; max over ranks."""
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t = torch.tensor([ev0.elapsed_time(ev1)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def flags_for(api, precision, slices):
    return api.SCHEME_NEW | (api.PREC_FP64 if precision == "fp64" else api.PREC_OZAKI | api.ozaki_slices(slices))


def run_dense(args, torch, dist, api, rank, world, local):
    n = args.n or (W.LARGE_N if args.workload == "large" else W.DENSE_N)
    mats = large_workload(n) if args.workload == "large" else dense_workload(n)
    prods = products_of(mats)
    h = api.Handle(local)
    stream = torch.cuda.current_stream()
    flags = flags_for(api, args.precision, args.slices)
    dA = [torch.from_numpy(A).cuda() for A in mats]
    dO = [torch.empty_like(a) for a in dA]

    def step():
        for a, o in zip(dA, dO):
            h.expm(a, o, 0.0, flags, stream)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    h.profile_enable(True)
    clocks.start()
    ms = timed(torch, dist, world, stream, step, args.steps)
    clk = clocks.stop()
    launches, _ = h.profile_read(api.KERNEL_ALL)
    prod_launches, prod_ms = h.profile_read(api.KERNEL_PRODUCT)
    prod_flops = h.profile_flops(api.KERNEL_PRODUCT)   # algorithmic: 2N^3 dense, N(N+1)(N+2)/3 triangular
    split_launches, split_ms = h.profile_read(api.KERNEL_SPLIT)
    _, norm_ms = h.profile_read(api.KERNEL_NORM)
    _, lincomb_ms = h.profile_read(api.KERNEL_LINCOMB)
    h.profile_enable(False)
    value = len(mats) * args.steps * world / (ms / 1e3)

    # plain FP64 form beside it, and how far the two results are apart
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64_compare:
        f64 = flags_for(api, "fp64", 0)
        dF = [torch.empty_like(a) for a in dA]

        def step64():
            for a, o in zip(dA, dF):
                h.expm(a, o, 0.0, f64, stream)
        step64()
        ms64 = timed(torch, dist, world, stream, step64, 1)
        diffs = [float(torch.linalg.norm(o - f) / torch.linalg.norm(f)) for o, f in zip(dO, dF)]
        tol = 1e-12 if args.workload == "dense4096" else 1e-10
        fp64 = {"value": len(mats) * world / (ms64 / 1e3), "unit": "expm/s", "steps": 1, "warmup": 1,
                "max_rel_fro_diff_vs_chosen": max(diffs), "rel_fro_diff_per_matrix": diffs,
                "tolerance": tol, "tolerance_met": max(diffs) <= tol - 1e-14}
        del dF

    e2e = None
    if not args.no_e2e:
        hA = [torch.from_numpy(A).pin_memory() for A in mats]
        hO = [torch.empty_like(a).pin_memory() for a in hA]
        e2e_steps = max(1, min(args.steps, 2))
        # the public host-buffer call: copies of neighbouring matrices overlap the computation
        h.expm_host_many(hA, hO, 0.0, flags, stream)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            h.expm_host_many(hA, hO, 0.0, flags, stream)
        te = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": len(mats) * e2e_steps * world / float(te.item()), "unit": "expm/s",
               "h2d_bytes_per_step": len(mats) * n * n * 8, "d2h_bytes_per_step": len(mats) * n * n * 8,
               "steps": e2e_steps, "api": "bbc_expm_host_many (pinned host buffers, pipelined copies)"}

    pk = peaks()
    avg_ms = prod_ms / max(1, prod_launches)
    flops_per_product = prod_flops / max(1, prod_launches)   # mean over dense and triangular launches
    logical = flops_per_product / (avg_ms / 1e3) / 1e12
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": logical, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": logical / FP64_PEAK_TFLOPS, "traffic": ncu_traffic("k_gemm_f64", n),
                "kernel": "k_gemm_f64<64,64>",
                "peak_source": "FP64 pipe, 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                "flops_per_launch": flops_per_product, "avg_launch_ms": avg_ms, "launches": prod_launches}
    else:
        pairs = args.slices * (args.slices + 1) // 2
        executed = pairs * flops_per_product / (avg_ms / 1e3) / 1e12
        peak = pk.get("bf16_tflops", 1899.1)
        roof = {"bound": "tensor", "achieved": executed, "peak": peak, "unit": "TFLOP/s",
                "frac": executed / peak,
                "traffic": ncu_traffic("k_ozaki_pair", n) if args.slices == 6 else None,
                "traffic_note": "mean of ncu captures of one dense and one triangle product at 6 slices "
                                "(the workload's launch mix is half and half; profiles/k_ozaki_pair_dense4096.md)",
                "kernel": f"k_ozaki_pair ({args.slices} BF16 slices: {pairs} slice products per FP64 product)",
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS)" if "bf16_tflops" in pk
                                else "fallback 1.9 PFLOP/s bf16"),
                "flops_per_launch": pairs * flops_per_product, "avg_launch_ms": avg_ms,
                "launches": prod_launches, "logical_fp64_tflops": logical,
                "split_ms_per_product": split_ms / max(1, split_launches / 3)}
    # the CPU-baseline leg: the oracle timed on a sample of the workload (the whole
    # workload for the 8192 one); its outputs are also the reference the timed form's
    # results (and, at 8192, every precision form's) are checked against (same (m, s))
    cpu, oracle_check, forms = None, None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        idx = DENSE_CPU_SAMPLE if len(mats) == 12 else tuple(range(len(mats)))
        cpu, outs = cpu_dense_sample(mats, prods, idx)
        tol = 1e-12 if args.workload == "dense4096" else 1e-10
        errs = []
        for i in idx:
            got = dO[i].cpu().numpy()
            errs.append(float(np.linalg.norm(got - outs[i]) / np.linalg.norm(outs[i])))
        oracle_check = {"matrices": list(idx), "rel_fro_vs_oracle": errs, "tolerance": tol,
                        "tolerance_met": max(errs) <= tol}
        if args.workload == "large":
            forms = large_forms(torch, api, h, stream, dA, outs, prods)
        del outs
    h.close()
    line = {
        "metric": METRICS[args.workload],
        "value": value, "unit": "expm/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else f"bf16x{args.slices}-slices(exact sums)->f64",
        "data": "synthetic",
        "config": dense_config(args, n, mats, prods, world),
        "form": {"scheme": "new (reduced-product Taylor)", "precision": args.precision,
                 "slices": args.slices if args.precision != "fp64" else None,
                 "structure": "upper triangular inputs (the non-normal six) are detected in the 1-norm pass and "
                              "run on the triangles, with the exact diagonal and superdiagonal put back "
                              "(Section 5); the flop figures count the triangle products' own work"},
        "oracle_check": oracle_check, "precision_forms": forms,
        "tflops_logical": prod_flops * world / (ms / 1e3) / 1e12,
        "time_share": {"product_ms": prod_ms, "split_ms": split_ms, "norm_ms": norm_ms,
                       "lincomb_and_exact_diagonal_ms": lincomb_ms, "timed_ms": ms},
        "roofline": roof, "plain_fp64": fp64, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk,
    }
    return line


def large_forms(torch, api, h, stream, dA, outs, prods):
    """The precision config's forms on the 8192 matrices, one pass each (event-timed,
    after one untimed pass), with every run's relative Frobenius error against the
    oracle's result at the same (m, s): the exact slices, the stated literal splits
    (3 BF16 terms, 2 TF32 terms) with and without the squarings on the FP64 pipe,
    FP32-accurate products (3 TF32 terms), and all-FP64 products."""
    res = {}
    for name, fl in (("exact 6 BF16 slices", api.PREC_OZAKI | api.ozaki_slices(6)),
                     ("exact 7 BF16 slices", api.PREC_OZAKI),
                     ("literal 3 BF16 terms", api.PREC_SPLIT | api.ozaki_slices(3)),
                     ("literal 3 BF16 terms, FP64 squarings", api.PREC_SPLIT | api.ozaki_slices(3)
                      | api.square_fp64_last(15)),
                     ("literal 2 TF32 terms", api.PREC_SPLIT_TF32 | api.ozaki_slices(2)),
                     ("literal 2 TF32 terms, FP64 squarings", api.PREC_SPLIT_TF32 | api.ozaki_slices(2)
                      | api.square_fp64_last(15)),
                     ("FP32 products (3 TF32 terms)", api.PREC_FP32),
                     ("FP64 products", api.PREC_FP64)):
        out = torch.empty_like(dA[0])
        runs = []
        for i, a in enumerate(dA):
            h.expm(a, out, 0.0, api.SCHEME_NEW | fl, stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = h.expm(a, out, 0.0, api.SCHEME_NEW | fl, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            runs.append({"m": info.m, "s": info.s, "ms": e0.elapsed_time(e1),
                         "rel_fro_vs_oracle": float(np.linalg.norm(got - outs[i]) / np.linalg.norm(outs[i]))})
        res[name] = {"expm_per_s": len(dA) / (sum(r["ms"] for r in runs) / 1e3), "runs": runs,
                     "meets_1e-10": all(r["rel_fro_vs_oracle"] <= 1e-10 for r in runs)}
        del out
    return res


def run_batch(args, torch, dist, api, rank, world, local, mats):
    """20000 uneven matrices: the chosen form (4-slice split products + learned
    selection, by default) against plain FP64 products with the paper's rule."""
    from paper_1710_10989_gb300 import selector as SEL
    h = api.Handle(local)
    split = args.precision == "ozaki"
    h.batch_reserve(256, api.PREC_OZAKI if split else 0)
    tuning = None
    if split:  # the autotuner's per-size product family and grid (measured here, or restored from its cache)
        from paper_1710_10989_gb300 import tuner
        t0 = time.perf_counter()
        mask, ctas = tuner.tuned(h, 256)
        tuning = {"split_mask": f"0x{mask:08x}", "ctas": ctas, "seconds": round(time.perf_counter() - t0, 2),
                  "split_buckets_N": [8 * (b + 1) for b in range(32) if (mask >> b) & 1]}
    sel_flag = {"plain": 0, "learned": api.SELECT_LEARNED, "alpha": api.SELECT_ALPHA}[args.selector]
    if args.selector == "learned":
        SEL.install(h)
    flags = (api.PREC_OZAKI if split else 0) | sel_flag
    order = api.batch_order([A.shape[0] for A in mats])
    mats = [mats[i] for i in order]
    # the matrices back to back in one device buffer (inputs) and one more (outputs), so that an
    # end-to-end step moves the whole batch with one copy each way
    sizes = [A.size for A in mats]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    dtype_t = torch.from_numpy(mats[0]).dtype
    din = torch.empty(int(offs[-1]), dtype=dtype_t, device="cuda")
    dout = torch.empty_like(din)
    for A, o in zip(mats, offs[:-1]):
        din[int(o):int(o) + A.size].copy_(torch.from_numpy(A.ravel()))
    ins = [din[int(o):int(o) + A.size].view(A.shape) for A, o in zip(mats, offs[:-1])]
    outs = [dout[int(o):int(o) + A.size].view(A.shape) for A, o in zip(mats, offs[:-1])]
    batch = api.Batch(ins, outs)
    stream = torch.cuda.Stream()

    u_batch = 2.0 ** -24 if args.u == "single" else 0.0

    def capture(fl, tol=u_batch):
        with torch.cuda.stream(stream):
            h.expm_batched(batch, tol=tol, flags=fl, stream=stream)  # warm-up outside the capture
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                h.expm_batched(batch, tol=tol, flags=fl, stream=stream)
        return g

    graph = capture(flags)
    cur = torch.cuda.current_stream()  # replays run on the current stream, so the events go there too
    for _ in range(args.warmup):
        graph.replay()
    clocks = ClockSampler(local)
    h.profile_enable(True)
    clocks.start()
    ms = timed(torch, dist, world, cur, graph.replay, args.steps)
    clk = clocks.stop()
    h.profile_enable(False)
    torch.cuda.synchronize()
    infos = batch.infos()
    bad = sum(1 for i in infos if i["status"] != 0)
    products = sum(i["products"] for i in infos)
    flops = sum(2.0 * A.shape[0] ** 3 * i["products"] for A, i in zip(mats, infos))
    bytes_io = sum(2 * A.size * 4 for A in mats)
    value = len(mats) * args.steps * world / (ms / 1e3)
    logical = flops / (ms / args.steps / 1e3) / 1e12
    sel = np.array([i["selector"] for i in infos])
    chosen_out = [o.cpu().numpy() for o in outs[::200]]

    plain = None
    if flags != 0 and not args.no_fp64_compare:
        g64 = capture(0, 0.0)
        g64.replay()
        ms64 = timed(torch, dist, world, cur, g64.replay, 1)
        inf64 = batch.infos()
        plain = {"value": len(mats) * world / (ms64 / 1e3), "unit": "expm/s", "steps": 1,
                 "mean_products": float(np.mean([i["products"] for i in inf64])), "form": "FP64 products, paper's rule"}
        # the Pade comparator on the same batch (r_10 or r_26 by cost, FP64 products, one-CTA LU solve)
        gp = capture(api.SCHEME_PADE, 0.0)
        gp.replay()
        msp = timed(torch, dist, world, cur, gp.replay, 1)
        infp = batch.infos()
        plain["pade_fp64"] = {"value": len(mats) * world / (msp / 1e3), "unit": "expm/s",
                              "mean_products_plus_solve": float(np.mean([i["products"] for i in infp])),
                              "r10_share": float(np.mean([i["m"] == 10 for i in infp])),
                              "new_over_pade_time": ms64 / msp}
        del gp

    # accuracy of the chosen form against the oracle on every 200th matrix
    from oracle import oracle as O
    errs = []
    for A, E in zip(mats[::200], chosen_out):
        ref, _ = O.expm(A.astype(np.float64))
        errs.append(float(np.linalg.norm(E.astype(np.float64) - ref) / np.linalg.norm(ref)))

    e2e = None
    if not args.no_e2e:
        hin = din.cpu().pin_memory()           # the whole batch, packed, in pinned host memory
        hout = torch.empty_like(hin).pin_memory()
        e2e_steps = max(1, min(args.steps, 2))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            din.copy_(hin, non_blocking=True)   # host -> device, one copy
            graph.replay()
            hout.copy_(dout, non_blocking=True)  # device -> host, one copy
            torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": len(mats) * e2e_steps * world / te, "unit": "expm/s", "h2d_bytes_per_step": bytes_io // 2,
               "d2h_bytes_per_step": bytes_io // 2, "steps": e2e_steps,
               "api": "bbc_expm_batched on the packed batch, one pinned copy each way per step"}
    cpu = cpu_batch_sample(mats[::max(1, len(mats) // 200)]) if (rank == 0 and world == 1
                                                                 and not args.no_cpu_baseline) else None
    h.close()
    pk = peaks()
    if split:
        # executed work: 10 BF16 slice products per product on the warp-level MMAs (padding to 32 excluded),
        # counted for the matrices whose size bucket the autotuner gave split products
        mask_v = int(tuning["split_mask"], 16) if tuning else 0xFFFFFFFF
        flops_split = sum(2.0 * A.shape[0] ** 3 * i["products"] for A, i in zip(mats, infos)
                          if A.shape[0] <= 256 and (mask_v >> ((A.shape[0] - 1) // 8)) & 1)
        executed = 10 * flops_split / (ms / args.steps / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": executed, "peak": 0.32 * pk.get("bf16_tflops", 1899.1),
                "unit": "TFLOP/s", "frac": executed / (0.32 * pk.get("bf16_tflops", 1899.1)), "traffic": None,
                "kernel": "k_batched_expm (4-slice BF16 mma.sync products)",
                "peak_source": "mma.sync m16n8k16 BF16 measured at 604 TFLOP/s on this GB300 (0.32 of the "
                               "MEASURED_PEAKS bf16 figure, which is tcgen05/cuBLAS)",
                "logical_fp64_tflops": logical}
    else:
        roof = {"bound": "alu", "achieved": logical, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": logical / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_batched_expm (FP64 products)",
                "peak_source": "FP64 pipe, 2 DFMA/clk/SM x 152 SMs x 2.07 GHz"}
    return {
        "metric": METRICS["batch"], "value": value,
        "unit": "expm/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("bf16x4-slices(exact group sums)->f64" if split else "f64") + " (binary32 storage)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["batch"].format(),
                   "count": len(mats) * world, "products_per_step": products, "statuses_not_ok": bad,
                   "parallelism": f"{world} ranks, LPT shards of the batch, no collective" if world > 1 else "single",
                   "precision": args.precision, "selector": args.selector,
                   "graph": "one persistent kernel per step, replayed from a CUDA graph",
                   "u": "2^-24" if args.u == "single" else "2^-53",
                   "autotuner": tuning,
                   "l2": "per-CTA binary64 work slots; inputs+outputs 3.7 GB per step (larger than L2)"},
        "tflops_logical": logical,
        "selector_stats": {"fallback_rate": float(np.mean(sel == 4)), "accepted_by_norm": float(np.mean(sel == 2)),
                           "accepted_by_alpha2": float(np.mean(sel == 3))} if args.selector == "learned" else None,
        "max_rel_err_vs_oracle_sample": max(errs), "error_sample": len(errs), "tolerance": 1e-6,
        "plain_fp64": plain, "roofline": roof,
        "hbm_gbs_io": bytes_io / (ms / args.steps / 1e3) / 1e9,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk,
    }


def run_compare(args, torch, dist, api, rank, world, local):
    """The paper's comparison (Section 4, Fig. 1: cost of the new Taylor scheme
    against Paterson-Stockmeyer and Pade r_26 over a range of norms) in wall time on
    this GPU: each method's exp(A) of the six Gaussian 4096 matrices, with split
    products (6 slices) and with FP64 products. The Pade solve is an LU with
    partial pivoting (the paper's 4/3-product step)."""
    mats = [W.dense_case(i) for i in range(len(W.DENSE_NORMS))]
    h = api.Handle(local)
    dA = [torch.from_numpy(A).cuda() for A in mats]
    out = torch.empty_like(dA[0])
    ref = torch.empty_like(dA[0])
    stream = torch.cuda.current_stream()
    split = api.PREC_OZAKI | api.ozaki_slices(6)
    methods = [("new", api.SCHEME_NEW, split), ("ps", api.SCHEME_PS, split), ("pade26", api.SCHEME_PADE26, split),
               ("pade", api.SCHEME_PADE, split), ("new_fp64", api.SCHEME_NEW, api.PREC_FP64),
               ("pade26_fp64", api.SCHEME_PADE26, api.PREC_FP64), ("pade_fp64", api.SCHEME_PADE, api.PREC_FP64)]
    res = {}
    for name, scheme, prec in methods:
        rows = []
        for A, a in zip(mats, dA):
            h.expm(a, out, 0.0, scheme | prec, stream)       # warm-up
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = h.expm(a, out, 0.0, scheme | prec, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            h.expm(a, ref, 0.0, api.SCHEME_NEW | split, stream)
            diff = float(torch.linalg.norm(out - ref) / torch.linalg.norm(ref))
            rows.append({"norm1": round(info.norm1, 4), "m": info.m, "s": info.s, "products": info.products,
                         "ms": e0.elapsed_time(e1), "rel_fro_vs_new": diff})
        res[name] = rows
    ms_new = sum(r["ms"] for r in res["new"])
    h.close()
    return {
        "metric": METRICS["compare4096"], "value": len(mats) / (ms_new / 1e3), "unit": "expm/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": ms_new, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x6-slices(exact sums)->f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["compare4096"], "n": 4096, "u": "2^-53",
                   "pade_solve": "LU with partial pivoting, N right-hand sides (blocked: cluster-factored panels, "
                                 "FP64 rank-32 updates; the library's own kernels)"},
        "comparison": res,
        "wall_time_ratio_new_over_pade": {p: sum(r["ms"] for r in res[a]) / sum(r["ms"] for r in res[b])
                                          for p, a, b in (("split", "new", "pade26"),
                                                          ("fp64", "new_fp64", "pade26_fp64"),
                                                          ("split_r10_r26", "new", "pade"),
                                                          ("fp64_r10_r26", "new_fp64", "pade_fp64"))},
    }


def cpu_small_sample(A):
    """The oracle on the 64 x 64 case (paper's scheme): one thread and all threads,
    repeated for about a second each."""
    from oracle import oracle as O
    O.theta_array("new")
    full = O.num_threads()
    res = {}
    for cores in (1, full):
        O.set_num_threads(cores)
        O.expm(A, "new")
        n, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 1.0:
            O.expm(A, "new")
            n += 1
        res[cores] = n / (time.perf_counter() - t0)
    O.set_num_threads(full)
    return {"value": res[full], "unit": "expm/s", "cores": full, "kind": "oracle",
            "single_core": res[1],
            "sample": f"oracle exp(A) of the 64 x 64 case, repeated for 1 s on {full} threads and on 1"}


def complex_workload(n):
    mats = []
    for seed, norm in ((201, 0.5), (202, 5.0), (203, 50.0)):
        rng = np.random.default_rng(seed)
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        mats.append(A * (norm / np.max(np.sum(np.abs(A), axis=0))))
    return mats


def run_complex(args, torch, dist, api, rank, world, local):
    """Complex A through bbc_expm_complex (the 2N x 2N real form on the real
    path): the chosen product precision and FP64 beside it, errors against the
    complex oracle on the first (cheapest) matrix."""
    n = args.n or 2048
    mats = complex_workload(n)
    h = api.Handle(local)
    stream = torch.cuda.current_stream()
    flags = flags_for(api, args.precision, args.slices)
    dA = [torch.from_numpy(A).cuda() for A in mats]
    dO = [torch.empty_like(a) for a in dA]
    infos = []

    def step():
        infos.clear()
        for a, o in zip(dA, dO):
            infos.append(h.expm_complex(a, o, 0.0, flags, stream))

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    h.profile_enable(True)
    clocks.start()
    ms = timed(torch, dist, world, stream, step, args.steps)
    clk = clocks.stop()
    launches, _ = h.profile_read(api.KERNEL_ALL)
    prod_launches, prod_ms = h.profile_read(api.KERNEL_PRODUCT)
    prod_flops = h.profile_flops(api.KERNEL_PRODUCT)
    h.profile_enable(False)
    value = len(mats) * args.steps * world / (ms / 1e3)
    f64 = flags_for(api, "fp64", 0)
    dF = [torch.empty_like(a) for a in dA]

    def step64():
        for a, o in zip(dA, dF):
            h.expm_complex(a, o, 0.0, f64, stream)
    step64()
    ms64 = timed(torch, dist, world, stream, step64, 1)
    diffs = [float(torch.linalg.norm(o - f) / torch.linalg.norm(f)) for o, f in zip(dO, dF)]
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import complex_oracle as CO
        t0 = time.perf_counter()
        want, _ = CO.expm(mats[0])
        dt = time.perf_counter() - t0
        got = dO[0].cpu().numpy()
        err = {"rel_fro_vs_complex_oracle_first": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
               "oracle_seconds": dt}
    pk = peaks()
    avg_ms = prod_ms / max(1, prod_launches)
    fpl = prod_flops / max(1, prod_launches)
    logical = fpl / (avg_ms / 1e3) / 1e12
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": logical, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": logical / FP64_PEAK_TFLOPS, "traffic": None, "kernel": "k_gemm_f64<64,64> on the real form"}
    else:
        pairs = args.slices * (args.slices + 1) // 2
        peak = pk.get("bf16_tflops", 1899.1)
        ex = pairs * logical
        roof = {"bound": "tensor", "achieved": ex, "peak": peak, "unit": "TFLOP/s", "frac": ex / peak,
                "traffic": None, "kernel": f"k_ozaki_pair ({args.slices} slices) on the real form",
                "logical_fp64_tflops": logical}
    h.close()
    return {
        "metric": METRICS["complex2048"], "value": value, "unit": "expm/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else f"bf16x{args.slices}-slices(exact sums)->f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["complex2048"].format(n=n), "n": n, "real_form_n": 2 * n,
                   "ms": [(i.m, i.s) for i in infos], "precision": args.precision},
        "roofline": roof, "error": err,
        "plain_fp64": {"value": len(mats) * world / (ms64 / 1e3), "unit": "expm/s",
                       "max_rel_fro_diff_vs_chosen": max(diffs)},
        "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk,
    }


def run_integrator(args, torch, dist, api, rank, world, local):
    """Lie-Euler steps of many orthogonal systems at once: Y_i <- exp(h Omega_i) Y_i
    in place through bbc_expm_apply_batched, 10 steps per graph replay."""
    count = 4096
    rng = np.random.default_rng(31)
    ns = rng.integers(1, 9, size=count) * 8
    norms = np.exp(rng.uniform(np.log(0.01), np.log(3.0), size=count))
    gens, ys = [], []
    for n, v in zip(ns, norms):
        G = rng.standard_normal((n, n))
        S = G - G.T
        gens.append(S * (v / np.max(np.sum(np.abs(S), axis=0))))
        ys.append(np.linalg.qr(rng.standard_normal((n, n)))[0])
    order = api.batch_order([int(n) for n in ns])
    h = api.Handle(local)
    h.batch_reserve(64)
    dG = [torch.from_numpy(gens[i]).cuda() for i in order]
    dY = [torch.from_numpy(ys[i].copy()).cuda() for i in order]
    b = api.Batch(dG, dY, rhs=dY)
    stream = torch.cuda.Stream()
    per_replay = 10
    with torch.cuda.stream(stream):
        h.expm_apply_batched(b, stream=stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(per_replay):
                h.expm_apply_batched(b, stream=stream)
    cur = torch.cuda.current_stream()
    for _ in range(args.warmup):
        g.replay()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed(torch, dist, world, cur, g.replay, args.steps)
    clk = clocks.stop()
    infos = b.infos()
    drift = max(float(torch.linalg.norm(y.T @ y - torch.eye(y.shape[0], dtype=y.dtype, device=y.device)))
                for y in dY[::64])
    products = sum(i["products"] for i in infos)
    nsorted = [int(ns[i]) for i in order]
    flops_launch = sum(2.0 * n ** 3 * inf["products"] for n, inf in zip(nsorted, infos))
    achieved = flops_launch * per_replay * args.steps / (ms / 1e3) / 1e12
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        k = 64
        t0 = time.perf_counter()
        for i in range(k):
            O.expm(gens[i], "new")[0] @ ys[i]
        dt = time.perf_counter() - t0
        cpu = {"value": k / dt, "unit": "system-steps/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"oracle exp(h Omega) Y for the first {k} systems in {dt:.2f} s"}
    h.close()
    steps_total = count * per_replay * args.steps * world
    return {
        "metric": METRICS["integrator"], "value": steps_total / (ms / 1e3), "unit": "system-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["integrator"], "count": count, "lie_euler_steps_per_replay": per_replay,
                   "products_per_launch": products},
        "orthogonality_drift_max": drift,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_batched_expm (FP64 products, one CTA per system)",
                     "flops_per_launch": flops_launch},
        "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": 2 * per_replay * args.steps, "clocks": clk,
    }


def run_small(args, torch, dist, api, rank, world, local):
    """One 64 x 64 matrix: graph-replayed exp(A) through the batched kernel (count 1:
    a cluster of CTAs shares the matrix, (m, s) chosen on the device), the three
    methods graph-replayed at their (m, s) through bbc_expm_fixed_async, and the
    plain bbc_expm call (host synchronisations included)."""
    A = W.small_case()
    h = api.Handle(local)
    h.batch_reserve(64)
    csize, _ = h.batch_launch_shape(1)   # one matrix: a cluster of CTAs shares it
    a = torch.from_numpy(A).cuda()
    o = torch.empty_like(a)
    batch = api.Batch([a], [o])
    stream = torch.cuda.Stream()
    reps = 200
    with torch.cuda.stream(stream):
        h.expm_batched(batch, stream=stream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(reps):
                h.expm_batched(batch, stream=stream)
    cur = torch.cuda.current_stream()
    for _ in range(args.warmup):
        graph.replay()
    clocks = ClockSampler(local)
    clocks.start()
    ms = timed(torch, dist, world, cur, graph.replay, args.steps)
    clk = clocks.stop()
    us_graph = ms * 1e3 / (args.steps * reps)
    # single calls of bbc_expm (two host synchronisations each), and the same method
    # at its (m, s) graph-replayed through bbc_expm_fixed_async: the paper's scheme,
    # Paterson-Stockmeyer and the Pade r_26 comparator on the same matrix
    us_call, us_async = {}, {}
    status = torch.zeros(1, dtype=torch.int32, device=a.device)
    for name, fl in (("new", api.SCHEME_NEW), ("ps", api.SCHEME_PS), ("pade26", api.SCHEME_PADE26),
                     ("pade", api.SCHEME_PADE)):
        for _ in range(5):
            h.expm(a, o, 0.0, fl, cur)
        t0 = time.perf_counter()
        for _ in range(50):
            info = h.expm(a, o, 0.0, fl, cur)
        us_call[name] = {"us": (time.perf_counter() - t0) / 50 * 1e6, "m": info.m, "s": info.s,
                         "products": info.products}
        with torch.cuda.stream(stream):
            h.expm_fixed_async(a, o, info.m, info.s, fl | api.DENSE, stream=stream, status=status)
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                for _ in range(reps):
                    h.expm_fixed_async(a, o, info.m, info.s, fl | api.DENSE, stream=stream, status=status)
        for _ in range(args.warmup):
            g.replay()
        ms_a = timed(torch, dist, world, cur, g.replay, args.steps)
        if int(status.item()) != 0:
            raise RuntimeError(f"{name}: status {int(status.item())}")
        us_async[name] = {"us": ms_a * 1e3 / (args.steps * reps), "m": info.m, "s": info.s,
                          "expm_per_s": args.steps * reps / (ms_a / 1e3)}
    h.close()
    cpu = cpu_small_sample(A) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    flops = 2.0 * 64 ** 3 * 5
    return {
        "metric": METRICS["small"], "value": 1e6 / us_graph, "unit": "expm/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["small"], "exp_per_step": reps, "ctas_per_matrix": csize},
        "us_per_expm_graph": us_graph, "graph_fixed": us_async, "single_call": us_call,
        "roofline": {"bound": "latency", "achieved": flops / (us_graph * 1e-6) / 1e12, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": flops / (us_graph * 1e-6) / 1e12 / FP64_PEAK_TFLOPS,
                     "traffic": None},
        "cpu_baseline": cpu, "e2e": None, "gpu_launches": 2 * reps * args.steps, "clocks": clk,
    }


def run_learned(args, torch, dist, api, rank, world, local):
    """The learned selector against the paper's rule and the closed-form alpha rule
    on the same held-out matrices (one persistent launch per step each)."""
    from paper_1710_10989_gb300 import selector as SEL
    h = api.Handle(local)
    h.batch_reserve(512)
    _, meta = SEL.install(h)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    rng = np.random.default_rng(12)
    mats = []
    while len(mats) < 4096:
        n = int(rng.integers(16, 513))
        mats += list(SEL.gpu_matrices(torch, n, min(64, 4096 - len(mats)), gen).unbind(0))
    order = api.batch_order([A.shape[0] for A in mats])
    mats = [mats[i].contiguous() for i in order]
    cur = torch.cuda.current_stream()
    res = {}
    for name, flags in (("plain", 0), ("alpha", api.SELECT_ALPHA), ("learned", api.SELECT_LEARNED)):
        outs = [torch.empty_like(a) for a in mats]
        b = api.Batch(mats, outs)
        for _ in range(args.warmup):
            h.expm_batched(b, flags=flags, stream=cur)
        clocks = ClockSampler(local)
        clocks.start()
        ms = timed(torch, dist, world, cur, lambda: h.expm_batched(b, flags=flags, stream=cur), args.steps)
        clk = clocks.stop()
        inf = b.infos()
        sel = np.array([i["selector"] for i in inf])
        flops = sum(2.0 * A.shape[0] ** 3 * i["products"] for A, i in zip(mats, inf))
        res[name] = {"value": len(mats) * args.steps * world / (ms / 1e3), "ms_per_step": ms / args.steps,
                     "mean_products": float(np.mean([i["products"] for i in inf])),
                     "statuses_not_ok": int(sum(i["status"] != 0 for i in inf)),
                     "tflops": flops / (ms / args.steps / 1e3) / 1e12, "clocks": clk,
                     "fallback_rate": float(np.mean(sel == 4)) if name == "learned" else None,
                     "accepted_by_norm": float(np.mean(sel == 2)) if name == "learned" else None,
                     "accepted_by_alpha2": float(np.mean(sel == 3)) if name == "learned" else None}
        res[name]["outs"] = outs
    from oracle import oracle as O
    idx = np.linspace(0, len(mats) - 1, 16).astype(int)
    for name in res:
        errs = []
        for i in idx:
            A = mats[i].cpu().numpy()
            ref, _ = O.expm(A)
            errs.append(float(np.linalg.norm(res[name]["outs"][i].cpu().numpy() - ref) / np.linalg.norm(ref)))
        res[name]["max_rel_err_vs_oracle_sample16"] = max(errs)
        del res[name]["outs"]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = [mats[i].cpu().numpy() for i in idx]
        O.theta_array("new")
        t0 = time.perf_counter()
        for A in sample:
            O.expm(A)
        dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "expm/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": f"oracle exp(A) of 16 of the held-out matrices spread over sizes, in {dt:.1f} s"}
    h.close()
    learned = res["learned"]
    return {
        "metric": METRICS["learned"], "value": learned["value"], "unit": "expm/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": learned["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC["learned"], "count": len(mats),
                   "network": f"5-{meta['hidden']}-{meta['hidden']}-{6 * meta['S']} MLP trained on "
                              f"{meta['count']} matrices (train accuracy {meta['train_accuracy']:.3f})",
                   "selector": "MLP proposal, certified by ||A||_1 or alpha_2 bound, else theta rule"},
        "learned": learned, "plain": res["plain"], "alpha_rule": res["alpha"],
        "roofline": {"bound": "alu", "achieved": learned["tflops"], "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": learned["tflops"] / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_batched_expm (FP64 products, learned selection)"},
        "cpu_baseline": cpu, "e2e": None, "gpu_launches": 2 * 3 * (args.steps + args.warmup),
        "clocks": learned["clocks"],
    }


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    # the batch is generated by spawned workers (safe before or after CUDA starts); with
    # several ranks the global batch is world x count matrices and each rank builds its
    # longest-processing-time shard of it on the cost N^3 (pi_m + s), (m, s) by the
    # library's theta rule on each matrix's 1-norm (weak scaling, no data-path collective)
    mats = None
    if args.workload == "batch" and world == 1:
        mats = W.batch_matrices(args.count)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        from paper_1710_10989_gb300 import build as B
        B.build()
    if world > 1:
        dist.barrier()
    from paper_1710_10989_gb300 import api
    if args.workload == "batch" and world > 1:
        from paper_1710_10989_gb300 import sharding
        ns, norms = W.batch_spec(count=args.count * world)
        u = api.U_SINGLE if args.u == "single" else api.U_DOUBLE
        prods = [PI[m] + s for m, s in (api.select(float(v), u) for v in norms)]
        mats = W.batch_matrices_subset(sharding.shard_indices(ns, rank, world, prods), count=args.count * world)
    if args.workload == "batch":
        line = run_batch(args, torch, dist, api, rank, world, local, mats)
    elif args.workload == "small":
        line = run_small(args, torch, dist, api, rank, world, local)
    elif args.workload == "learned":
        line = run_learned(args, torch, dist, api, rank, world, local)
    elif args.workload == "integrator":
        line = run_integrator(args, torch, dist, api, rank, world, local)
    elif args.workload == "complex2048":
        line = run_complex(args, torch, dist, api, rank, world, local)
    elif args.workload == "compare4096":
        line = run_compare(args, torch, dist, api, rank, world, local)
    else:
        line = run_dense(args, torch, dist, api, rank, world, local)
    if rank == 0:
        if isinstance(line.get("cpu_baseline"), dict):
            line["cpu_baseline"].setdefault("cpu_model", host_cpu())
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
