"""Small, self-terminating GPU cases for kernel profiling (ncu).

    python -m paper_1509_06865_gb300.profile_case --case eig16
    python -m paper_1509_06865_gb300.profile_case --case stencil32

stencil32: five FP32 applications of Q - sigma on a 32^3 x 64 lattice with unit
links (the stencil's memory traffic does not depend on the link values), about
4 GB of device memory.

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
    ap.add_argument("--case", default="eig16", choices=["eig16", "stencil32"])
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import synth
    from paper_1509_06865_gb300 import MIXED, OP_Q, PREC_F32, Context

    if args.case == "stencil32":
        dims = (32, 32, 32, 64)
        ctx = Context(dims)
        ctx.set_params(m0=-0.05, csw=1.9, n_tv=20, precision=MIXED)
        ctx.load_gauge(synth.unit_gauge(dims))
        nbytes = 32 * 32 * 32 * 64 * 12 * 8
        x, y = ctx.alloc_dev(nbytes), ctx.alloc_dev(nbytes)
        ctx.pack_spinors(synth.gaussian_vectors(dims, 1, 77)[0], x, PREC_F32)
        for _ in range(5):
            ctx.apply_dev(x, y, 1e-3, OP_Q, PREC_F32)
        ctx.close()
        print("profile case", args.case, "ok")
        return

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
