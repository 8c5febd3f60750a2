"""Autotune the sampler's launch configuration on this GPU and write the
tuning table that the library (and bench.py) load.

  python -m paper_1905_00165_gb300.tune [--n 16384] [--precision 3xtf32]
      [--form hermitian|lu|complex|aztec|batched] [--draws 12] [--out tune_gb300.json]

The kernel timed is the benchmark's workload of that form: K = Q diag(lam) Q^H
with Q Haar and lam ~ Beta(1/2, 1/2) (Hermitian, real or complex),
K = D^{-1} S D (general), the Aztec-diamond tiling kernel whose 4 d^2 edges
come closest to --n (general complex), or, for the batched sampler, 4096
L-ensemble marginal kernels of order U{64..--n} (the CTA size is tuned). Entries already in the output file are kept unless
this run replaces their key.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
DEFAULT_OUT = os.path.join(HERE, "tune_gb300.json")


def main(argv=None) -> int:
    p = argparse.ArgumentParser()
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--precision", default="3xtf32", choices=["fp64", "3xtf32", "bf16x6"])
    p.add_argument("--form", default="hermitian",
                   choices=["hermitian", "lu", "complex", "aztec", "batched"])
    p.add_argument("--draws", type=int, default=12)
    p.add_argument("--max-streams", type=int, default=8)
    p.add_argument("--out", default=DEFAULT_OUT)
    args = p.parse_args(argv)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import paper_1905_00165_gb300 as dpp
    from paper_1905_00165_gb300 import _lib, build
    import workloads as W
    build.build()
    dev = "cuda"
    if args.form == "batched":
        if os.path.exists(args.out):
            _lib.tune_load(args.out)
        Ks = W.lensemble_batch_torch(4096, seed=0, nmin=64, nmax=args.n, device=dev)
        best = dpp.BatchedSampler(Ks).autotune(draws=max(2, args.draws // 4))
        _lib.tune_save(args.out)
        print(json.dumps({"form": args.form, "n_max": args.n, "best": best}))
        return 0
    if args.form == "lu":
        K, _ = W.lu_similarity_kernel(args.n, seed=0, device=dev)
        Kd = torch.from_numpy(np.ascontiguousarray(K.T)).to(dev).t()
    elif args.form == "aztec":
        d = max(1, int(round((args.n / 4) ** 0.5)))
        Kd, _, _ = W.aztec_kernel(d, device=dev, return_torch=True)
    else:
        Kd = W.hermitian_kernel(args.n, seed=0, kind="beta", complex_=args.form == "complex",
                                device=dev, return_torch=True)
        Kd = Kd.t().contiguous().t()
    if os.path.exists(args.out):
        _lib.tune_load(args.out)
    best = dpp.autotune(Kd, hermitian=args.form in ("hermitian", "complex"), precision=args.precision,
                        max_streams=args.max_streams, draws=args.draws)
    _lib.tune_save(args.out)
    print(json.dumps({"form": args.form, "n": args.n, "precision": args.precision, "best": best}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
