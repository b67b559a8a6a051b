"""Run one kernel class of libbbcexpm.so on a synthetic case, for profilers.

    python -m paper_1710_10989_gb300.profile_case --kernel gemm --n 4096 --reps 2
    python -m paper_1710_10989_gb300.profile_case --kernel expm --n 1024 --norm 5
    python -m paper_1710_10989_gb300.profile_case --kernel gemm --n 4096 --precision tf32
    python -m paper_1710_10989_gb300.profile_case --kernel solve --n 4096

Inputs are seeded Gaussians; nothing is checked (the test suite does that).
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=("gemm", "expm", "norm", "batched", "solve"), default="gemm")
    ap.add_argument("--count", type=int, default=512, help="matrices of --kernel batched")
    ap.add_argument("--selector", choices=("plain", "learned"), default="learned")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--norm", type=float, default=1.0)
    ap.add_argument("--precision", choices=("fp64", "ozaki", "bf16x3", "tf32"), default="fp64",
                    help="FP64 products, exact BF16 slices, or the literal 3-term BF16 / 2-term TF32 splits")
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--upper", action="store_true", help="upper triangular operands (triangle products)")
    ap.add_argument("--small", action="store_true",
                    help="--kernel batched on --count copies of the 64 x 64 single-matrix case (binary64)")
    a = ap.parse_args()

    import torch

    from paper_1710_10989_gb300 import api
    from paper_1710_10989_gb300 import workloads as W

    flags = {"fp64": api.PREC_FP64, "ozaki": api.PREC_OZAKI | api.ozaki_slices(a.slices),
             "bf16x3": api.PREC_SPLIT | api.ozaki_slices(3), "tf32": api.PREC_SPLIT_TF32 | api.ozaki_slices(2)}[a.precision]
    if a.kernel == "batched":  # the batched workload's distribution, binary32 storage
        mats = [W.small_case()] * a.count if a.small else W.batch_matrices(a.count)
        h = api.Handle(0)
        bflags = 0 if a.precision == "fp64" else api.PREC_OZAKI
        h.batch_reserve(256, bflags)
        if a.selector == "learned":
            from paper_1710_10989_gb300 import selector as SEL
            SEL.install(h)
            bflags |= api.SELECT_LEARNED
        order = api.batch_order([m.shape[0] for m in mats])
        ins = [torch.from_numpy(mats[i]).cuda() for i in order]
        outs = [torch.empty_like(x) for x in ins]
        b = api.Batch(ins, outs)
        for _ in range(a.reps):
            h.expm_batched(b, flags=bflags)
        torch.cuda.synchronize()
        h.close()
        print("done", a)
        return
    h = api.Handle(0)
    if a.upper:
        A = torch.from_numpy(W.nonnormal_upper(a.n, 1, a.norm)).cuda()
        B = torch.from_numpy(W.nonnormal_upper(a.n, 2, a.norm)).cuda()
        flags |= api.UPPER
    else:
        A = torch.from_numpy(W.gaussian(a.n, 1, a.norm)).cuda()
        B = torch.from_numpy(W.gaussian(a.n, 2, a.norm)).cuda()
    C = torch.empty_like(A)
    if a.kernel == "solve":  # the Pade comparator's solve on a Gaussian system (row interchanges throughout)
        for _ in range(a.reps):
            M, X = A.clone(), B.clone()
            h.solve(M, X)
        torch.cuda.synchronize()
        h.close()
        print("done", a)
        return
    for _ in range(a.reps):
        if a.kernel == "gemm":
            h.gemm(A, B, C, flags)
        elif a.kernel == "norm":
            h.norm1(A)
        else:
            h.expm(A, C, 0.0, api.SCHEME_NEW | flags)
    torch.cuda.synchronize()
    h.close()
    print("done", a)


if __name__ == "__main__":
    main()
