#!/usr/bin/env python
"""Throughput of scaling-and-squaring exp(A) (Bader, Blanes, Casas, arXiv:1710.10989)
on the dense 4096 x 4096 FP64 workload, through libbbcexpm.so.

One step = exp(A) of every matrix of the workload: six Gaussian N(0,1)/sqrt(N)
matrices rescaled to 1-norms {0.01, 0.1, 1, 5, 20, 100} (seeds 1-6) and six
non-normal upper-triangular ones (diagonal N(0,1), strict upper N(0,1)*10,
seeds 101-106) at the same norms; (m, s) chosen by the theta rule at u = 2^-53.

Prints one JSON line (rank 0). --impl reference times the CPU oracle instead.
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

L2_BYTES = 129 * 2 ** 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp64", "ozaki"), default="fp64")
    ap.add_argument("--slices", type=int, default=0, help="BF16 slices for --precision ozaki (0 = 7)")
    ap.add_argument("--n", type=int, default=W.DENSE_N, help="matrix size (default: the 4096 workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(n: int):
    mats, names = [], []
    for i, nrm in enumerate(W.DENSE_NORMS):
        mats.append(W.dense_case(i, n=n))
        names.append(f"gauss_{nrm:g}")
    for i, nrm in enumerate(W.DENSE_NORMS):
        mats.append(W.dense_case(i, n=n, nonnormal=True))
        names.append(f"upper_{nrm:g}")
    return mats, names


def products_per_matrix(mats) -> list[int]:
    """(m, s) by the theta rule from each matrix's 1-norm; products = pi_m + s."""
    from paper_1710_10989_gb300 import api
    pi = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}
    out = []
    for A in mats:
        m, s = api.select(float(np.abs(A).sum(axis=0).max()))
        out.append(pi[m] + s)
    return out


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


# FP64 pipe: the GB300's nominal 1.25 TFLOP/s FP64 is 2 DFMA per clock per SM:
# 152 SMs x 2 DFMA x 2 flop x 2.07 GHz (maximum SM clock).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def cpu_oracle_sample(mats, prods):
    """The oracle on matrix 0 of the workload (its cheapest), scaled to expm/s of
    the whole workload by products: value = 1 / (t_per_product * mean products)."""
    from oracle import oracle as O
    A = mats[0]
    O.theta_array("new")  # thresholds are constants: computed (and cached) before timing
    t0 = time.perf_counter()
    _, info = O.expm(A, "new")
    dt = time.perf_counter() - t0
    per_product = dt / max(1, info.products)
    mean_p = sum(prods) / len(prods)
    return {"value": 1.0 / (per_product * mean_p), "unit": "expm/s", "cores": O.num_threads(),
            "kind": "oracle",
            "sample": (f"oracle exp(A) of the workload's first matrix (N={A.shape[0]}, 1-norm 0.01, "
                       f"{info.products} products) in {dt:.1f} s; scaled by products to the workload's "
                       f"mean of {mean_p:.2f} products per exp(A)")}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    mats, _ = workload(args.n)
    prods = products_per_matrix(mats)
    vals = []  # the CPU needs no warm-up steps; --warmup is accepted and not run
    for _ in range(args.steps):
        r = cpu_oracle_sample(mats, prods)
        vals.append(r["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": "expm/s (dense 4096x4096 exp(A), FP64)", "value": value,
            "unit": "expm/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "dense4096: 6 Gaussian + 6 non-normal upper-triangular, norms 0.01-100",
                       "n": args.n, "matrices_per_step": len(mats)},
            "cpu_baseline": {"value": value, "unit": "expm/s", "cores": r["cores"], "kind": "oracle",
                             "sample": "per step: " + r["sample"]},
            "e2e": {"value": value, "unit": "expm/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

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

    flags = api.SCHEME_NEW | (api.PREC_FP64 if args.precision == "fp64"
                              else api.PREC_OZAKI | api.ozaki_slices(args.slices))
    mats, names = workload(args.n)
    n = args.n
    prods = products_per_matrix(mats)
    h = api.Handle(local)
    dA = [torch.from_numpy(A).cuda() for A in mats]
    dO = [torch.empty_like(a) for a in dA]
    stream = torch.cuda.current_stream()

    def step():
        infos = []
        for a, o in zip(dA, dO):
            infos.append(h.expm(a, o, 0.0, flags, stream))
        return infos

    for _ in range(args.warmup):
        infos = step()
    assert [i.products for i in infos] == prods, ([i.products for i in infos], prods)

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    h.profile_enable(True)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches, _ = h.profile_read(api.KERNEL_ALL)
    prod_launches, prod_ms = h.profile_read(api.KERNEL_PRODUCT)
    split_launches, split_ms = h.profile_read(api.KERNEL_SPLIT)
    norm_launches, norm_ms = h.profile_read(api.KERNEL_NORM)
    h.profile_enable(False)
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    total = len(mats) * args.steps * world
    value = total / (ms_max / 1e3)

    # end to end through the C-ABI host entry point: H2D of A and D2H of exp(A) every call
    e2e = None
    if not args.no_e2e:
        hA = [torch.from_numpy(A).pin_memory() for A in mats]
        hO = [torch.empty_like(a).pin_memory() for a in hA]
        e2e_steps = max(1, min(args.steps, 2))
        for a, o in zip(hA, hO):
            h.expm_host(a, o, 0.0, flags, stream)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            for a, o in zip(hA, hO):
                h.expm_host(a, o, 0.0, flags, stream)
        te = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": len(mats) * e2e_steps * world / float(te.item()), "unit": "expm/s",
               "h2d_bytes_per_step": len(mats) * n * n * 8, "d2h_bytes_per_step": len(mats) * n * n * 8,
               "steps": e2e_steps}

    pk = peaks()
    flops_per_product = 2.0 * n ** 3
    avg_ms = prod_ms / max(1, prod_launches)
    achieved = flops_per_product / (avg_ms / 1e3) / 1e12
    if args.precision == "fp64":
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_gemm_f64<64,64> (dense product + fused epilogue)",
                "peak_source": "FP64 pipe, 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)",
                "avg_launch_ms": avg_ms, "launches": prod_launches}
    else:
        # the tcgen05 kernel executes k(k+1)/2 BF16 slice products per FP64 product
        slices = args.slices or 7
        pairs = slices * (slices + 1) // 2
        executed = pairs * flops_per_product / (avg_ms / 1e3) / 1e12
        peak = pk.get("bf16_tflops", 1899.1)
        roof = {"bound": "tensor", "achieved": executed, "peak": peak, "unit": "TFLOP/s",
                "frac": executed / peak, "traffic": None,
                "kernel": f"k_ozaki_gemm ({slices} BF16 slices, {pairs} slice products per FP64 product)",
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst, cuBLAS)" if "bf16_tflops" in pk
                               else "fallback 1.9 PFLOP/s bf16",
                "flops_per_launch": pairs * flops_per_product, "avg_launch_ms": avg_ms,
                "launches": prod_launches, "logical_fp64_tflops": achieved,
                "split_kernels_ms_per_product": split_ms / max(1, split_launches / 3)}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_oracle_sample(mats, prods)
        line = {
            "metric": "expm/s (dense 4096x4096 exp(A), FP64)", "value": value, "unit": "expm/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "bf16-slices(exact f32 sums)->f64",
            "data": "synthetic",
            "config": {"workload": "dense4096: 6 Gaussian N(0,1)/sqrt(N) (seeds 1-6) + 6 non-normal "
                                   "upper-triangular (seeds 101-106), 1-norms 0.01,0.1,1,5,20,100",
                       "n": n, "matrices_per_step": len(mats), "products_per_step": sum(prods),
                       "scheme": "new (reduced-product Taylor)", "precision": args.precision,
                       "u": "2^-53", "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (each exp(A) streams ~10 N^2 FP64 buffers of "
                             f"{n * n * 8 / 2 ** 20:.0f} MiB)"},
            "tflops_logical": sum(prods) * flops_per_product * args.steps * world / (ms_max / 1e3) / 1e12,
            "time_share": {"product_ms": prod_ms, "split_ms": split_ms, "norm_ms": norm_ms,
                           "timed_ms": ms},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
