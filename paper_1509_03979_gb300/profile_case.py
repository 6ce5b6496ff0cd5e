"""Run one small, fixed case of the CUDA path for profiling (e.g. under ncu).

    python -m paper_1509_03979_gb300.profile_case --case apply --N 262144 --batch 16 --reps 2
    python -m paper_1509_03979_gb300.profile_case --case sp --N 262144 --batch 1
    python -m paper_1509_03979_gb300.profile_case --case apply --impl streamed --batch 64

Cases: apply / apply_t (batched A or A^T over `batch` random vectors, through the batched
implementation `impl`: auto, cluster or streamed), sp / omp / ompr (batched recovery of `batch`
synthetic signals with M = N/4, K = M/10).
"""
import argparse

import numpy as np
import torch

from paper_1509_03979_gb300 import binding, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="apply", choices=["apply", "apply_t", "sp", "omp", "ompr"])
    ap.add_argument("--N", type=int, default=1 << 18)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--impl", default="auto", choices=["auto", "cluster", "streamed"])
    a = ap.parse_args()
    N, M = a.N, a.N // 4
    op = binding.Operator(N, M, 0x0C5002)
    op.set_batched_impl(a.impl)
    dev = torch.device("cuda")
    g = torch.Generator(device=dev).manual_seed(0)
    if a.case in ("apply", "apply_t"):
        X = torch.randn((a.batch, N), device=dev, generator=g)
        U = torch.randn((a.batch, M), device=dev, generator=g)
        for _ in range(a.reps):
            if a.case == "apply":
                op.apply_batched(X)
            else:
                op.apply_t_batched(U)
    else:
        K = max(1, M // 10)
        S = np.stack([synth.sparse_gaussian(N, K, 100 + b) for b in range(a.batch)]).astype(np.float32)
        Y = op.apply_batched(torch.from_numpy(S).to(dev))
        for _ in range(a.reps):
            binding.recover_batched([op] * a.batch, [Y[b] for b in range(a.batch)], [K] * a.batch,
                                    [a.case] * a.batch, 1e-6, 100)
    torch.cuda.synchronize()
    print("ok", a.case, N, a.batch)


if __name__ == "__main__":
    main()
