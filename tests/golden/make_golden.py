"""Writes the stored expected values under tests/golden/ from the FP64 CPU
oracle alone (nothing here touches the CUDA library).

    python tests/golden/make_golden.py lowest_8x8x8x16 [--workers 8]
    python tests/golden/make_golden.py oracle_work_8x8x8x16

lowest_8x8x8x16: the 24 eigenvalues of Q of smallest |lambda| on the 8^3 x 16
field of the workload "check_8x8x8x16" in workloads.json, by the oracle's
Chebyshev-filtered subspace iteration on Q^2 (oracle/chefsi.py), with their
eigen-residuals.  It is the completeness reference of the GPU eigensolver (the
paper warns after Algorithm 1 that the Rayleigh quotient iteration can miss a
wanted mode).

oracle_work_8x8x8x16: one complete oracle eigensolve (setup and Algorithm 1,
20 pairs to 1e-10) on the same field, its wall time on the host that ran it and
the number of each oracle operation it performed; the CPU baseline of bench.py
prices these operation counts with live oracle timings.
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


def oracle_work(case: str):
    """A complete oracle eigensolve (setup + Algorithm 1 with the default
    additions) of the workload's n_eig pairs, with its wall time and the count of
    every oracle operation it performed.  The counters wrap the oracle's own
    functions in this process only; the arithmetic is untouched."""
    import numpy as np

    import synth
    from oracle import dirac, krylov, mg, rqi

    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)[case]
    dims = tuple(cfg["dims"])
    counts = dict(fine_D_vectors=0, sap_cycles=0, coarse_builds=0, interp_builds=0, restricts=0, prolongs=0,
                  coarse_applies=0, krylov_steps_fine=0, krylov_steps_coarse=0, fine_vdots=0)
    nfine = int(np.prod(dims)) * 12

    def wrap(obj, name, key, weight=lambda *a, **k: 1):
        fn = getattr(obj, name)

        def counted(*a, **k):
            counts[key] += weight(*a, **k)
            return fn(*a, **k)
        setattr(obj, name, counted)

    wrap(dirac.WilsonClover, "D", "fine_D_vectors",
         lambda self, psi: int(np.prod(psi.shape[:-6])) if psi.ndim > 6 else 1)
    wrap(mg.SAP, "smooth", "sap_cycles", lambda self, b, x, sigma, cycles, mr: cycles)
    wrap(mg, "coarse_operator", "coarse_builds")
    wrap(mg.Interpolation, "__init__", "interp_builds")
    wrap(mg.Interpolation, "restrict", "restricts")
    wrap(mg.Interpolation, "prolong", "prolongs")
    wrap(mg.CoarseOperator, "apply", "coarse_applies")
    # Arnoldi steps of GMRES / FGMRES, split by the vector length (fine or coarse)
    arn = krylov._arnoldi_cycle

    def arnoldi_counted(apply_A, precond, r0, beta, m, tol_abs, flexible):
        out = arn(apply_A, precond, r0, beta, m, tol_abs, flexible)
        counts["krylov_steps_fine" if r0.size == nfine else "krylov_steps_coarse"] += out[2]
        return out
    krylov._arnoldi_cycle = arnoldi_counted
    vdot = np.vdot

    def vdot_counted(a, b):
        if np.size(a) == nfine:
            counts["fine_vdots"] += 1
        return vdot(a, b)
    np.vdot = vdot_counted
    try:
        U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
        t0 = time.time()
        op = dirac.WilsonClover(U, cfg["m0"], cfg["csw"], tuple(cfg["bc"]))
        params = dict(mg.DEFAULT_PARAMS, agg=tuple(cfg["agg"]), ntv=cfg["n_tv"], sap_block=tuple(cfg["sap_block"]))
        W0 = synth.uniform_vectors(dims, cfg["n_tv"], cfg["seed"])
        lam, V, res, st = rqi.eigensolve(op, W0, cfg["n_eig"], cfg["tol"], params, seed=cfg["seed"],
                                         log=lambda m: print(m, flush=True))
        wall = time.time() - t0
    finally:
        np.vdot = vdot
        krylov._arnoldi_cycle = arn
    out = dict(doc="work of one complete oracle eigensolve (setup + Algorithm 1) and its wall time; written by "
                   "tests/golden/make_golden.py", workload=case, dims=list(dims), n_eig=cfg["n_eig"],
               tol=cfg["tol"], wall_s=wall, host_cores_used=1, counts=counts, rqi_stats=st,
               eigenvalues=[float(x) for x in lam], residuals=[float(r) for r in res])
    path = os.path.join(HERE, f"oracle_work_{case.split('_', 1)[1]}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, f"{wall:.0f} s", counts)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["lowest_8x8x8x16", "oracle_work_8x8x8x16"])
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    args = ap.parse_args()
    if args.what == "lowest_8x8x8x16":
        lowest("check_8x8x8x16", args.workers, k=24, nb=48, degree=80)
    elif args.what == "oracle_work_8x8x8x16":
        oracle_work("check_8x8x8x16")


if __name__ == "__main__":
    main()
