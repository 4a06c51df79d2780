"""Time the tensor-core split-product GEMM alone (CUDA events, after warm-up).

    python -m paper_1312_1549_gb300.gemm_bench --m 1024 --n 13312 --k 6656 [--npass 3] [--reps 5]

C (m x n) = A (m x k) B (n x k)^T through omm_kernel_gemm_tc; the default shape is the
operator-on-direction product of the Si512 workload ([H~ D; S D], n = 1024, 2m = 13312,
m = 6656). Prints the kernel time including the operand splits and the flop rate.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import build as _build


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=1024)
    ap.add_argument("--n", type=int, default=13312)
    ap.add_argument("--k", type=int, default=6656)
    ap.add_argument("--npass", type=int, default=3)
    ap.add_argument("--reps", type=int, default=5)
    args = ap.parse_args()
    _build.build()
    from . import solver as S
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(args.m, args.k, dtype=torch.float64, device="cuda", generator=g)
    B = torch.randn(args.n, args.k, dtype=torch.float64, device="cuda", generator=g)
    C = torch.empty(args.m, args.n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        S.gemm_tc(A, B, C, npass=args.npass)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        S.gemm_tc(A, B, C, npass=args.npass)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    ref = A[:64].double() @ B[:64].double().T
    err = float(((C[:64, :64] - ref[:, :64]).abs() / (A[:64].abs() @ B[:64].abs().T)).max())
    flop = 2.0 * args.m * args.n * args.k * args.npass
    print(json.dumps({"m": args.m, "n": args.n, "k": args.k, "npass": args.npass,
                      "ms_with_splits": ms, "tflops_issued_with_splits": flop / ms / 1e9,
                      "max_rel_err": err}))


if __name__ == "__main__":
    main()
