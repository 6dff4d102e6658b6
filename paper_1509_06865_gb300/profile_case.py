"""Small, self-terminating GPU cases for kernel profiling (ncu).

    python -m paper_1509_06865_gb300.profile_case --case eig16

eig16: the 16^3 x 32 benchmark field (eps = 0.2, c_sw = 1.9, m0 of the tuned
workload), multigrid setup with one refinement pass, then one sweep of
Algorithm 1 on 3 vectors without guards to eigen-residual 1e-3.  It launches
every kernel of the hot path (stencils, SAP, restriction, prolongation, the
coarse-operator build and the persistent coarse GMRES) a few hundred times at
the benchmark's lattice size, in a few seconds and a few GB of device memory.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="eig16", choices=["eig16"])
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import synth
    from paper_1509_06865_gb300 import MIXED, Context

    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)["bench_16x16x16x32"]
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    ctx = Context(dims)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], n_tv=cfg["n_tv"], precision=MIXED, setup_iters=1,
                   max_sweeps=1, n_guard=0)
    ctx.load_gauge(U)
    ctx.setup(cfg["seed"])
    _, _, _, st = ctx.eigensolve(3, 1e-3, want_vectors=False)
    ctx.close()
    print("profile case", args.case, st)


if __name__ == "__main__":
    main()
