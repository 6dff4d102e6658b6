#!/usr/bin/env python
"""Benchmark: seconds per 20 lowest eigenpairs of Q = gamma5 D at eigen-residual
1e-10 on a 16^3 x 32 lattice (the multigrid Rayleigh quotient iteration of
arXiv:1509.06865, Algorithm 1), mixed precision against the all-FP64 GPU path.

One step = the whole hot path on one synthetic gauge field already in device
memory: gauge packing and the clover term, the multigrid setup (test vectors,
P, coarse operator) and Algorithm 1 for the 20 lowest pairs.  `value` is the
device time per step (lower is better); `e2e` repeats the step through the
public C ABI from pinned host memory, copying the eigenvectors back.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle instead (see cpu_baseline()).
N > 1 runs N independent replicas, one per rank (the path does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s per 20 lowest Q eigenpairs at resid 1e-10, mixed vs FP64; stencil HBM GB/s"
WORKLOAD = dict(
    workload="16^3x32 Wilson-clover, SU(3) links exp(i 0.2 H), c_sw=1.9, m0 near-critical; "
             "20 lowest eigenpairs of Q to resid 1e-10; 2-level MG (4^4 aggregates, 20 test vectors, SAP 4^4)",
    dims=[16, 16, 16, 32], eps=0.2, seed=1002, csw=1.9, n_eig=20, tol=1e-10,
)
COUNTS_FILE = os.path.join(ROOT, "bench_counts.json")
# library timer classes that are one kernel each (the BLAS classes are several)
SINGLE_KERNEL_CLASSES = ("coarse_gmres", "stencil_f64", "stencil_f32", "sap_f32", "sap_f64", "restrict", "prolong",
                         "coarse_apply", "coarse_build", "interp_build")
# DRAM bytes (read + write) per launch from an ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum); None where none was taken
DRAM_BYTES_PER_LAUNCH = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:coarse_gmres -s 20 -c 3 on
    # `python -m paper_1509_06865_gb300.profile_case --case eig16` (same 16^3x32 coarse grid): 66.0 MB read +
    # 0.17 MB written per launch, whatever the number of GMRES steps (the coarse operator is read from DRAM once per
    # solve and then served by L2)
    "coarse_gmres": 66.17e6,
}


def load_m0() -> float:
    with open(os.path.join(ROOT, "workloads.json")) as f:
        m0 = json.load(f)["bench_16x16x16x32"]["m0"]
    if m0 is None:
        raise RuntimeError("workloads.json: m0 of the 16^3x32 workload not tuned yet")
    return float(m0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return dict(hbm=float(p["hbm_gbs"]), bf16=float(p["bf16_tflops"]), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, src="fallback")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0, None
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    dist.init_process_group("nccl" if os.environ.get("MGEIG_BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return rank, ws, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x: float, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# GPU arm


def stencil_microbench(ctx, dims, flush, peak_hbm, n=40):
    """Q - sigma on device buffers, one launch per timed interval, L2 flushed
    before each launch; CUDA events on the context's own stream."""
    import numpy as np
    import torch

    import synth
    from paper_1509_06865_gb300 import OP_Q, PREC_F32, PREC_F64

    V = int(np.prod(dims))
    s = torch.cuda.ExternalStream(ctx.stream())
    x_host = synth.gaussian_vectors(tuple(dims), 1, 77)
    out = {}
    # algorithmic bytes per site: x, y (12 complex each), 4 links (two rows in
    # FP32, full in FP64), clover (72 reals)
    for prec, name, per_site in ((PREC_F32, "f32", 96 + 96 + 192 + 288), (PREC_F64, "f64", 192 + 192 + 576 + 576)):
        nbytes = V * 12 * (8 if prec == PREC_F32 else 16)
        x = ctx.alloc_dev(nbytes)
        y = ctx.alloc_dev(nbytes)
        ctx.pack_spinors(x_host, x, prec)
        for _ in range(3):
            ctx.apply_dev(x, y, 1e-3, OP_Q, prec)
        times = []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            ctx.apply_dev(x, y, 1e-3, OP_Q, prec)
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        gbs = per_site * V / (ms * 1e-3) / 1e9
        out[name] = dict(ms=ms, gbs=gbs, frac_hbm=gbs / peak_hbm, bytes_per_site=per_site,
                         gflops=1872.0 * V / (ms * 1e-3) / 1e9)
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import synth
    from paper_1509_06865_gb300 import FP64, MIXED, Context

    rank, ws, local, dist = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    dims = tuple(w["dims"])
    m0 = load_m0()
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    U_pinned = torch.from_numpy(U.view(np.float64).reshape(-1)).pin_memory()
    U_dev = U_pinned.to(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)    # > 129 MB L2

    def make_ctx(precision):
        ctx = Context(dims, device=local)
        ctx.set_params(m0=m0, csw=w["csw"], n_tv=20, precision=precision)
        return ctx

    def step(ctx, seed):
        flush.fill_(rank & 0xFF)
        torch.cuda.synchronize()
        ctx.load_gauge_dev(U_dev.data_ptr())
        ctx.setup(seed)
        lam, _, res, st = ctx.eigensolve(w["n_eig"], w["tol"], want_vectors=False)
        return lam, res, st

    def timed(ctx, steps, seed):
        barrier(dist)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")     # lets a profiler select the timed steps
        e0.record()
        out = [step(ctx, seed) for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        barrier(dist)
        return e0.elapsed_time(e1) / 1e3, out

    ctx = make_ctx(MIXED)
    ctx.load_gauge_dev(U_dev.data_ptr())
    sten = stencil_microbench(ctx, dims, flush, peaks()["hbm"])
    # the same stencil on the 32^3 x 64 lattice of the larger workloads (unit links:
    # the stencil's memory traffic does not depend on the link values)
    big = (32, 32, 32, 64)
    ctxb = Context(big, device=local)
    ctxb.set_params(m0=m0, csw=w["csw"], n_tv=20, precision=MIXED)
    ctxb.load_gauge(synth.unit_gauge(big))
    sten_big = stencil_microbench(ctxb, big, flush, peaks()["hbm"], n=20)
    ctxb.close()
    # the last warm-up step records every kernel class (the per-class breakdown);
    # the timed steps record events for the dominant single kernel only
    for i in range(args.warmup):
        if i == args.warmup - 1:
            ctx.set_timing(True)
        step(ctx, w["seed"])
    kt = ctx.kernel_times()
    top = max((k for k in SINGLE_KERNEL_CLASSES if k in kt), key=lambda k: kt[k]["ms"])
    ctx.set_timing_classes([top])
    n_launch0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        t_mixed, outs = timed(ctx, args.steps, w["seed"])
    launches = ctx.launch_count() - n_launch0
    kt_top = ctx.kernel_times()[top]
    ctx.set_timing(False)
    lam, res, st = outs[-1]
    t_mixed = max_over_ranks(dist, t_mixed, dev)

    # e2e through the public API with host buffers: gauge from pinned host
    # memory in, eigenvalues and eigenvectors out
    barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        ctx.load_gauge(U_pinned.numpy().view(np.complex128))
        ctx.setup(w["seed"])
        lam_e, V_e, res_e, _ = ctx.eigensolve(w["n_eig"], w["tol"], want_vectors=True)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(dist, time.perf_counter() - t0, dev) / e2e_steps
    ctx.close()

    # the all-FP64 GPU path at the same accuracy (--fp64-steps 0 skips it)
    fp64 = None
    if args.fp64_steps > 0:
        ctx64 = make_ctx(FP64)
        step(ctx64, w["seed"])
        t_fp64, outs64 = timed(ctx64, args.fp64_steps, w["seed"])
        lam64, res64, st64 = outs64[-1]
        ctx64.close()
        t_fp64 = max_over_ranks(dist, t_fp64, dev) / args.fp64_steps
        fp64 = dict(value=t_fp64, unit="s", steps=args.fp64_steps, max_resid=float(max(res64)),
                    sweeps=st64["sweeps"], outer_iters=st64["outer_iters"],
                    max_abs_diff_vs_mixed=float(np.max(np.abs(np.asarray(lam) - np.asarray(lam64)))))

    if rank != 0:
        return
    pk = peaks()
    # the dominant single kernel, its algorithmic bytes over its event-timed
    # duration inside the timed region
    achieved = kt_top["bytes"] / (kt_top["ms"] / 1e3) / 1e9 if kt_top["ms"] > 0 else None
    with open(COUNTS_FILE + ".new", "w") as f:
        json.dump(dict(workload=w["workload"], steps=1, kernels=kt, stats=st), f, indent=1)
    value = t_mixed / (args.steps * ws)
    line = dict(
        metric=METRIC, value=value, unit="s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=1e3 * t_mixed / args.steps, higher_is_better=False, scaling="weak", vs_baseline=None,
        dtype="f64 outer / f32 preconditioner", data="synthetic",
        config=dict(workload=w["workload"], dims=w["dims"], m0=load_m0(), n_eig=w["n_eig"], tol=w["tol"],
                    parallelism=f"replicas{ws}", l2="flushed (256 MB write) before every step"),
        fp64_path=fp64,
        mixed_over_fp64_speedup=(fp64["value"] / value) if fp64 else None,
        result=dict(lambda_min=float(lam[0]), lambda_max=float(lam[-1]), max_resid=float(max(res)),
                    sweeps=st["sweeps"], solves=st["solves"], outer_iters=st["outer_iters"],
                    mg_cycles=st["mg_cycles"], coarse_iters=st["coarse_iters"]),
        stencil=dict(sten, l2="flushed before every launch", lattice=w["dims"],
                     lattice_32x32x32x64=sten_big),
        roofline=dict(bound="hbm", kernel=top, achieved=achieved, peak=pk["hbm"], unit="GB/s",
                      frac=(achieved / pk["hbm"]) if achieved else None,
                      traffic=DRAM_BYTES_PER_LAUNCH.get(top),
                      launches=kt_top["launches"], ms=kt_top["ms"],
                      bytes_per_launch=kt_top["bytes"] / max(1, kt_top["launches"]),
                      peak_src=f"{pk['src']} hbm_gbs (burst copy)"),
        e2e=dict(value=t_e2e, unit="s", h2d_bytes_per_step=int(U.nbytes),
                 d2h_bytes_per_step=int(V_e.nbytes + lam_e.nbytes + res_e.nbytes)),
        gpu_launches=int(launches),
        clocks=clk.summary(),
        kernels={k: dict(launches=v["launches"], ms=round(v["ms"], 3), gbs=(v["bytes"] / v["ms"] / 1e6) if v["ms"] else None)
                 for k, v in kt.items() if v["launches"]},
        kernels_note="per-class device time of one step (the last warm-up step, every class timed)",
    )
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(kt_counts=kt, stats=st, steps=1)   # kt covers one step
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# CPU oracle (baseline and --impl reference)


def cpu_baseline_subprocess(kt_counts=None, stats=None, steps=1):
    """Run the oracle sample in a fresh single-threaded process."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    payload = json.dumps(dict(kernels=kt_counts, stats=stats, steps=steps))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"], input=payload,
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return dict(kind="oracle", error=r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_sample(counts: dict | None):
    """Per-operation oracle times at 16^3x32, combined with the method's operation
    counts per step (kernel launches by class of one GPU step; they are work
    units of the algorithm on this workload, not results)."""
    import numpy as np

    import synth
    from oracle import dirac, krylov, mg

    w = WORKLOAD
    dims = tuple(w["dims"])
    t_all = time.perf_counter()
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    t = time.perf_counter()
    op = dirac.WilsonClover(U, load_m0(), w["csw"])
    t_clover = time.perf_counter() - t
    x = synth.gaussian_vectors(dims, 1, 1)[0]
    t = time.perf_counter()
    y = op.Q_sigma(x, 1e-3)
    t_stencil = time.perf_counter() - t
    Wt = synth.uniform_vectors(dims, 20, 5)
    t = time.perf_counter()
    P = mg.Interpolation(Wt, (4, 4, 4, 4))
    t_interp = time.perf_counter() - t
    t = time.perf_counter()
    rc = P.restrict(x)
    t_restrict = time.perf_counter() - t
    t = time.perf_counter()
    P.prolong(rc)
    t_prolong = time.perf_counter() - t
    # coarse operator: two of its 40 columns, scaled
    t = time.perf_counter()
    for c, j in ((0, 0), (1, 0)):
        wv = P.column(c, j)
        part = dirac.apply_local(op.A, op.m0, wv)
        for mu in range(4):
            part = part + dirac.hop_forward(op.U, wv, mu, op.bc) + dirac.hop_backward(op.U, wv, mu, op.bc)
            P.restrict(part)
            P.restrict(part)
        P.restrict(part)
    t_coarse_build = (time.perf_counter() - t) * 20
    Dc = np.zeros((9, P.nagg, 40, 40), dtype=np.complex128)
    C = mg.CoarseOperator(Dc, P.cdims, 20)
    t = time.perf_counter()
    C.apply(rc, 1e-3)
    t_capply = time.perf_counter() - t
    sap = mg.SAP(op, (4, 4, 4, 4))
    t = time.perf_counter()
    r = x - op.D_sigma(x, 1e-3)
    sap.block_mr(r, 0, 1e-3, 4)
    t_sap = time.perf_counter() - t          # one colour = one sweep
    t = time.perf_counter()
    for _ in range(4):
        np.vdot(x, y)
        y = y + 0.5 * x
    t_blas = (time.perf_counter() - t) / 8
    per_op = dict(stencil_f64=t_stencil, stencil_f32=t_stencil, sap_f64=t_sap, sap_f32=t_sap,
                  restrict=t_restrict, prolong=t_prolong, coarse_apply=t_capply, coarse_build=t_coarse_build,
                  interp_build=t_interp, blas_f64=t_blas * 3, blas_low=t_blas * 3 * 40 / V_ratio(),
                  other=t_clover)
    if counts and counts.get("kernels"):
        kt = counts["kernels"]
        steps = max(1, int(counts.get("steps", 1)))
        est = sum(per_op.get(k, 0.0) * v["launches"] / steps for k, v in kt.items())
        how = "per-op oracle times x the method's per-step launch counts"
    else:
        est = None
        how = "per-op oracle times only (no launch counts)"
    return dict(value=est, unit="s", cores=1, kind="oracle",
                sample=f"oracle FP64 at 16^3x32: 1 stencil, 1 SAP sweep, P build, restrict, prolong, "
                       f"2 of 40 coarse-operator columns (x20), 1 coarse apply, BLAS-1, clover; {how}",
                sample_seconds=time.perf_counter() - t_all, per_op_s=per_op)


def V_ratio():
    # BLAS-1 on coarse vectors (512 x 40 complex) vs fine vectors (131072 x 12)
    return 131072 * 12 / (512 * 40)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    counts = None
    if os.path.exists(COUNTS_FILE):
        with open(COUNTS_FILE) as f:
            counts = json.load(f)
    vals = []
    for _ in range(args.warmup):
        pass
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        r = cpu_baseline_subprocess_from(counts)
        vals.append(r.get("value"))
    elapsed = time.perf_counter() - t0
    v = statistics.median([x for x in vals if x is not None]) if any(x is not None for x in vals) else None
    line = dict(impl="reference", metric=METRIC, value=v, unit="s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", config=dict(workload=WORKLOAD["workload"], dims=WORKLOAD["dims"]),
                cpu_baseline=dict(r, value=v),
                e2e=dict(value=v, unit="s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                wall_s=elapsed)
    print(json.dumps(line), flush=True)


def cpu_baseline_subprocess_from(counts):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample"],
                       input=json.dumps(counts or {}), capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return dict(kind="oracle", error=r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        payload = sys.stdin.read()
        counts = json.loads(payload) if payload.strip() else None
        print(json.dumps(oracle_sample(counts)))
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
