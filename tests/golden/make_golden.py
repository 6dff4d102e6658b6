"""Writes the stored expected values under tests/golden/ from the FP64 CPU
oracle alone (nothing here touches the CUDA library).

    python tests/golden/make_golden.py lowest_8x8x8x16 [--workers 8]

lowest_8x8x8x16: the 24 eigenvalues of Q of smallest |lambda| on the 8^3 x 16
field of the workload "check_8x8x8x16" in workloads.json, by the oracle's
Chebyshev-filtered subspace iteration on Q^2 (oracle/chefsi.py), with their
eigen-residuals.  It is the completeness reference of the GPU eigensolver (the
paper warns after Algorithm 1 that the Rayleigh quotient iteration can miss a
wanted mode).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def lowest(case: str, workers: int, k: int, nb: int, degree: int):
    import numpy as np

    import synth
    from oracle import chefsi, dirac

    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)[case]
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    op = dirac.WilsonClover(U, cfg["m0"], cfg["csw"], tuple(cfg["bc"]))
    qb = chefsi.q_norm_bound(op)
    start = synth.gaussian_vectors(dims, nb, cfg["seed"] + 7)
    fmap = chefsi.ParallelFilter(op, workers) if workers > 1 else None
    t0 = time.time()
    try:
        lam, V, res, info = chefsi.lowest_abs_eigenpairs(op.Q, start, k, qb, degree=degree, tol=1e-11,
                                                         filter_map=fmap, log=lambda m: print(m, flush=True))
    finally:
        if fmap is not None:
            fmap.close()
    # an independent re-check of each pair with the oracle stencil
    resid = [dirac.norm(op.Q(V[i]) - lam[i] * V[i]) for i in range(k)]
    out = dict(
        doc="eigenvalues of Q of smallest |lambda| (ordered by |lambda|, then lambda) by Chebyshev-filtered "
            "subspace iteration on Q^2 (oracle/chefsi.py); written by tests/golden/make_golden.py",
        workload=case, dims=list(dims), eps=cfg["eps"], seed=cfg["seed"], m0=cfg["m0"], csw=cfg["csw"],
        bc=cfg["bc"], block=nb, degree=degree, q_bound=qb, iterations=info["iters"], seconds=time.time() - t0,
        eigenvalues=[float(x) for x in lam], residuals=[float(r) for r in resid],
        block_sqrt_mu=info["block_sqrt_mu"],
    )
    assert info["converged"] and max(resid) <= 1e-10, (info, resid)
    path = os.path.join(HERE, f"lowest_Q_{case.split('_', 1)[1]}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, f"{time.time() - t0:.0f} s")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["lowest_8x8x8x16"])
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    if args.what == "lowest_8x8x8x16":
        lowest("check_8x8x8x16", args.workers, k=24, nb=48, degree=80)


if __name__ == "__main__":
    main()
