#!/usr/bin/env python
"""Benchmark: seconds per 20 lowest eigenpairs of Q = gamma5 D at eigen-residual
1e-10 on a 16^3 x 32 lattice (the multigrid Rayleigh quotient iteration of
arXiv:1509.06865, Algorithm 1), mixed precision against the all-FP64 GPU path.

One step = the whole hot path on one synthetic gauge field already in device
memory: gauge packing and the clover term, the multigrid setup (test vectors,
P, coarse operator) and Algorithm 1 for the 20 lowest pairs.  `value` is the
device time per step (lower is better); `e2e` repeats the step through the
public C ABI from pinned host memory, copying the eigenvectors back.  The line
also carries the 20 lowest pairs of the 32^3 x 64 field (one step, after the
timed region), the stencil microbenchmark and the FP64 / FP32 FMA roofs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --profile-case eig16|stencil32      (small cases for ncu)

--impl reference times the FP64 CPU oracle instead (see oracle_baseline()).
N > 1 runs N independent replicas, one per rank (the path does not shard).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
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
# library timer classes that are one kernel each (the BLAS classes are several)
SINGLE_KERNEL_CLASSES = ("coarse_gmres", "stencil_f64", "stencil_f32", "sap_f32", "sap_f64", "restrict", "prolong",
                         "coarse_apply", "coarse_build", "interp_build")
# DRAM bytes (read + write) per launch from an ncu capture of the current kernel
# (dram__bytes_read.sum + dram__bytes_write.sum); None where none was taken
DRAM_BYTES_PER_LAUNCH = {
    # ncu --set full -k regex:coarse_gmres -s 20 -c 2 on `python bench.py --profile-case eig16` (the same
    # 16^3x32 coarse grid and the current kernel): 66.0 MB read + 0.46 MB written per launch, whatever the number
    # of GMRES steps (the coarse operator is read from DRAM once per solve and then served by L2)
    "coarse_gmres": 66.47e6,
}


def workload(name: str) -> dict:
    with open(os.path.join(ROOT, "workloads.json")) as f:
        return json.load(f)[name]


def load_m0() -> float:
    m0 = workload("bench_16x16x16x32")["m0"]
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


def stencil_microbench(ctx, dims, flush, peak_hbm, n=40, nrhs=0):
    """Q - sigma on device buffers, one launch per timed interval, L2 flushed
    before each launch; CUDA events on the context's own stream.  With nrhs > 0
    also the FP32 stencil on nrhs fields in one launch (links and clover read
    once for all of them)."""
    import numpy as np
    import torch

    import synth
    from paper_1509_06865_gb300 import OP_Q, PREC_F32, PREC_F32_F64_DS, PREC_F64, PREC_F64_DS

    V = int(np.prod(dims))
    s = torch.cuda.ExternalStream(ctx.stream())
    x_host = synth.gaussian_vectors(tuple(dims), 1, 77)

    def timeit(launch):
        for _ in range(3):
            launch()
        times = []
        for _ in range(n):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            launch()
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.median(times)

    out = {}
    # algorithmic bytes per site: x, y (12 complex each), 4 links (two rows in
    # FP32, full in FP64), clover (72 reals)
    for prec, name, per_site in ((PREC_F32, "f32", 96 + 96 + 192 + 288), (PREC_F64, "f64", 192 + 192 + 576 + 576)):
        nbytes = V * 12 * (8 if prec == PREC_F32 else 16)
        x = ctx.alloc_dev(nbytes)
        y = ctx.alloc_dev(nbytes)
        ctx.pack_spinors(x_host, x, prec)
        ms = timeit(lambda: ctx.apply_dev(x, y, 1e-3, OP_Q, prec))
        gbs = per_site * V / (ms * 1e-3) / 1e9
        out[name] = dict(ms=ms, gbs=gbs, frac_hbm=gbs / peak_hbm, bytes_per_site=per_site,
                         gflops=1872.0 * V / (ms * 1e-3) / 1e9)
        if prec == PREC_F64:
            # the mixed solver's FP64-output stencil in double-float arithmetic:
            # FP64 in (x 192 B), and FP32 in (x 96 B, the outer FGMRES matvec);
            # links and clover as float pairs (the FP64 byte counts)
            x32 = ctx.alloc_dev(V * 12 * 8)
            ctx.pack_spinors(x_host, x32, PREC_F32)
            for dprec, dname, xin in ((PREC_F64_DS, "f64_ds", x), (PREC_F32_F64_DS, "f32in_f64_ds", x32)):
                ms = timeit(lambda: ctx.apply_dev(xin, y, 1e-3, OP_Q, dprec))
                ps = per_site - (96 if dprec == PREC_F32_F64_DS else 0)
                gbs = ps * V / (ms * 1e-3) / 1e9
                out[dname] = dict(ms=ms, gbs=gbs, frac_hbm=gbs / peak_hbm, bytes_per_site=ps,
                                  flop_per_site=1872, speedup_vs_f64=out["f64"]["ms"] / ms)
    if nrhs > 0:
        nbytes = V * 12 * 8
        x = ctx.alloc_dev(nbytes * nrhs)
        y = ctx.alloc_dev(nbytes * nrhs)
        ctx.pack_spinors(np.repeat(x_host, nrhs, axis=0), x, PREC_F32)
        ms = timeit(lambda: ctx.apply_dev_nrhs(x, y, nrhs, 1e-3, OP_Q, PREC_F32))
        per_site = nrhs * (96 + 96) + 192 + 288
        gbs = per_site * V / (ms * 1e-3) / 1e9
        out[f"f32_nrhs{nrhs}"] = dict(ms=ms, ms_per_rhs=ms / nrhs, gbs=gbs, frac_hbm=gbs / peak_hbm,
                                      bytes_per_site=per_site)
    return out


def coarse_tc_microbench(flush, device, peak_hbm, nrhs=12, n=10):
    """The coarse operator of the 32^3 x 64 lattice (4^4 aggregates, 20 test
    vectors: 8192 coarse sites, 40 x 40 blocks; 943 MB in FP32, 472 MB in BF16,
    out of L2) applied to nrhs coarse vectors: BF16 links with per-link FP32
    scale on the tensor cores in one launch, against the FP32-link CUDA-core apply
    one right-hand side after another.  CUDA events on the context's stream, L2
    flushed before each timed call."""
    import torch

    import synth
    from paper_1509_06865_gb300 import LINKS_BF16, LINKS_LEVEL, MIXED, Context

    cfg = workload("large_32x32x32x64")
    dims = tuple(cfg["dims"])
    out = {}
    for links, name in ((LINKS_BF16, "bf16_tensor_cores"), (LINKS_LEVEL, "f32_cuda_cores")):
        ctx = Context(dims, device=device)
        ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], agg=cfg["agg"], n_tv=cfg["n_tv"], sap_block=cfg["sap_block"],
                       precision=MIXED, coarse_links=links, setup_iters=0)
        ctx.load_gauge(synth.unit_gauge(dims))
        ctx.setup(cfg["seed"])
        n2 = 2 * cfg["n_tv"]
        nc = ctx.coarse_sites * n2
        X = torch.randn(nrhs * nc, dtype=torch.complex64, device=torch.device("cuda", device))
        Y = torch.empty_like(X)
        s = torch.cuda.ExternalStream(ctx.stream())
        torch.cuda.synchronize()

        def timeit(k):
            for _ in range(3):
                ctx.coarse_apply_dev_nrhs(X.data_ptr(), Y.data_ptr(), k, 0.01)
            times = []
            for _ in range(n):
                flush.fill_(2)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                ctx.coarse_apply_dev_nrhs(X.data_ptr(), Y.data_ptr(), k, 0.01)
                e1.record(s)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            return statistics.median(times)

        link_b = 9 * ctx.coarse_sites * n2 * n2 * (4 if links == LINKS_BF16 else 8)
        ms_n = timeit(nrhs)
        ms_1 = timeit(1)
        byt = link_b + nrhs * 2 * nc * 8
        out[name] = dict(nrhs=nrhs, ms=ms_n, ms_per_rhs=ms_n / nrhs, ms_one_rhs=ms_1, link_mb=link_b / 1e6,
                         gbs=byt / (ms_n * 1e-3) / 1e9, frac_hbm=byt / (ms_n * 1e-3) / 1e9 / peak_hbm)
        ctx.close()
        del X, Y
    out["speedup_per_rhs"] = out["f32_cuda_cores"]["ms_per_rhs"] / out["bf16_tensor_cores"]["ms_per_rhs"]
    return out


def run_gpu(args):
    import numpy as np
    import torch

    import synth
    from paper_1509_06865_gb300 import FP64, MIXED, PREC_F32, PREC_F64, Context

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
    alu = dict(fp64_tflops=ctx.fma_peak(PREC_F64) / 1e12, fp32_tflops=ctx.fma_peak(PREC_F32) / 1e12,
               how="own kernel: 8 independent FMA chains per thread on every SM, best of 5 launches, CUDA events")
    sten = stencil_microbench(ctx, dims, flush, peaks()["hbm"])
    # the same stencil on the 32^3 x 64 lattice of the larger workloads (unit links:
    # the stencil's memory traffic does not depend on the link values)
    big = (32, 32, 32, 64)
    ctxb = Context(big, device=local)
    ctxb.set_params(m0=m0, csw=w["csw"], n_tv=20, precision=MIXED)
    ctxb.load_gauge(synth.unit_gauge(big))
    sten_big = stencil_microbench(ctxb, big, flush, peaks()["hbm"], n=20, nrhs=12)
    ctxb.close()
    coarse_tc = coarse_tc_microbench(flush, local, peaks()["hbm"])
    for k in ("f32", "f64"):
        for sd in (sten, sten_big):
            sd[k]["frac_fp64_fma_peak" if k == "f64" else "frac_fp32_fma_peak"] = \
                sd[k]["gflops"] / 1e3 / (alu["fp64_tflops"] if k == "f64" else alu["fp32_tflops"])
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

    # the 20 lowest pairs of the 32^3 x 64 field (one step each, after the timed region)
    large = None if args.no_large else large_field(args, flush, local)
    # like for like: the GPU eigensolve of the 4^4 field on which the CPU baseline
    # times the oracle's complete eigensolve
    small, small_pairs = small_field(flush, local)

    if rank != 0:
        return
    pk = peaks()
    # the dominant single kernel, its algorithmic bytes over its event-timed
    # duration inside the timed region
    achieved = kt_top["bytes"] / (kt_top["ms"] / 1e3) / 1e9 if kt_top["ms"] > 0 else None
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
        eigensolve_32x32x32x64=large,
        like_for_like_4x4x4x4=small,
        alu_peaks=alu,
        stencil=dict(sten, l2="flushed before every launch", lattice=w["dims"],
                     lattice_32x32x32x64=sten_big),
        coarse_apply_12rhs_32x32x32x64=coarse_tc,
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
        vec_path = os.path.join(tempfile.mkdtemp(prefix="mgeig_oracle_"), "V.npy")
        line["cpu_baseline"] = oracle_baseline_subprocess(vec_path)
        cs = line["cpu_baseline"].get("complete_4x4x4x4")
        if cs:
            small["oracle_s"] = cs["wall_s"]
            small["oracle_over_gpu"] = cs["wall_s"] / small["gpu_s"]
        if cs and small_pairs is not None:
            # the error of the GPU's result against the FP64 oracle's
            try:
                small["vs_oracle"] = pairs_vs_oracle(small_pairs[0], small_pairs[1], cs["lam"], np.load(vec_path))
            except Exception as e:  # the line is printed whatever this comparison meets
                small["vs_oracle"] = dict(error=repr(e)[:300])
    print(json.dumps(line), flush=True)


def large_field(args, flush, device):
    """The 20 lowest pairs of Q on the 32^3 x 64 field to 1e-10 (mixed, and FP64
    with --large-fp64), one step each, CUDA events around the step."""
    import numpy as np
    import torch

    import synth
    from paper_1509_06865_gb300 import FP64, MIXED, Context

    cfg = workload("large_32x32x32x64")
    if cfg["m0"] is None:
        return dict(skipped="m0 of the 32^3x64 workload not tuned")
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    U_dev = torch.from_numpy(U.view(np.float64).reshape(-1)).to(torch.device("cuda", device))
    out = dict(workload=f"32^3x64 Wilson-clover, links exp(i {cfg['eps']} H), c_sw={cfg['csw']}, m0={cfg['m0']}; "
                        f"{cfg['n_eig']} lowest eigenpairs of Q to resid {cfg['tol']}",
               dims=cfg["dims"], m0=cfg["m0"], n_eig=cfg["n_eig"], tol=cfg["tol"])
    for prec, name in ((MIXED, "mixed"), (FP64, "fp64")):
        if prec == FP64 and not args.large_fp64:
            continue
        ctx = Context(dims, device=device)
        ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                       sap_block=cfg["sap_block"], precision=prec)
        flush.fill_(3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.load_gauge_dev(U_dev.data_ptr())
        st0 = ctx.setup(cfg["seed"])
        lam, _, res, st = ctx.eigensolve(cfg["n_eig"], cfg["tol"], want_vectors=False)
        e1.record()
        torch.cuda.synchronize()
        ctx.close()
        out[name] = dict(value=e0.elapsed_time(e1) / 1e3, unit="s", setup_s=st0["seconds"], eig_s=st["seconds"],
                         converged=st["converged"], max_resid=float(max(res)), lambda_min=float(lam[0]),
                         lambda_max=float(lam[-1]), sweeps=st["sweeps"], solves=st["solves"],
                         outer_iters=st["outer_iters"], coarse_iters=st["coarse_iters"])
    del U_dev
    return out


def learned_study(device=0, steps=2500, batch=4, sigma=0.0, name="bench_16x16x16x32"):
    """The learned smoother on a workload's field (default the 16^3 x 32 benchmark field): trained on the GPU
    on steps x batch (residual, SAP correction) pairs the method generates
    (10^4 by default, the training-set size of the learned-smoother workload),
    then one shifted solve (Q - sigma) x = b (b Z2 noise) to 1e-10 by the FP64
    FGMRES with the two-grid preconditioner whose post-smoother is SAP, the
    network, or nothing; the true residual is re-computed with the FP64 stencil."""
    import numpy as np

    import synth
    from paper_1509_06865_gb300 import LEARNED, MIXED, OP_Q, PREC_F64, SAP, Context

    w = workload(name)
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    kw = dict(m0=w["m0"], csw=w["csw"], n_tv=w["n_tv"], agg=w["agg"], sap_block=w["sap_block"], precision=MIXED,
              outer_maxiter=400)
    ctx = Context(dims, device=device)
    ctx.set_params(**kw)
    ctx.load_gauge(U)
    ctx.setup(w["seed"])
    ctx.net_init(1)
    t0 = time.perf_counter()
    losses = ctx.net_train(steps, batch, 2e-3, 99)
    t_train = time.perf_counter() - t0
    b = synth.z2_noise(dims, 1, 21)[0]
    out = dict(dims=list(dims), pairs=steps * batch, train_s=t_train, loss_first=float(np.mean(losses[:10])),
               loss_last=float(np.mean(losses[-10:])), sigma=sigma, tol=1e-10)
    for name, extra in (("sap", dict(smoother=SAP)), ("learned", dict(smoother=LEARNED)),
                        ("none", dict(smoother=SAP, sap_cycles=0))):
        ctx.set_params(**kw, **extra)
        ctx.setup(w["seed"])
        try:
            x, st = ctx.solve(b, sigma, 1e-10)
        except Exception as e:   # a capped solve without smoother reports ENOCONV
            out[name] = dict(error=str(e))
            continue
        r = ctx.apply(x[None], sigma, OP_Q, PREC_F64)[0] - b
        out[name] = dict(outer_iters=st["outer_iters"], s=st["seconds"], converged=st["converged"],
                         true_resid=float(np.linalg.norm(r) / np.linalg.norm(b)))
    ctx.close()
    print(json.dumps(out), flush=True)
    return out


def config3_study(device=0, n_eig=50, setup_iters=30):
    """The larger 32^3 x 64 workload: approximate modes straight from a setup of
    `setup_iters` iterations (their Rayleigh quotients and eigen-residuals,
    Sec. 3.3: about 1e-3 there), then the `n_eig` lowest pairs to 1e-10 by
    Algorithm 1 (mixed precision, BF16 coarse links with per-link FP32 scale)."""
    import numpy as np

    import synth
    from paper_1509_06865_gb300 import LINKS_BF16, MIXED, Context

    cfg = workload("large_32x32x32x64")
    dims = tuple(cfg["dims"])
    ctx = Context(dims, device=device)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                   sap_block=cfg["sap_block"], precision=MIXED, coarse_links=LINKS_BF16, setup_iters=setup_iters)
    ctx.load_gauge(synth.gauge_field(dims, cfg["eps"], cfg["seed"]))
    t0 = time.perf_counter()
    st0 = ctx.setup(cfg["seed"])
    t_setup = time.perf_counter() - t0
    appr = ctx.lma_prepare(cfg["n_tv"], None, 0.75)
    order = np.argsort(np.abs(appr["lam"]))
    t0 = time.perf_counter()
    lam, _, res, st = ctx.eigensolve(n_eig, cfg["tol"], want_vectors=False)
    t_eig = time.perf_counter() - t0
    ctx.close()
    out = dict(dims=list(dims), coarse_links="bf16", setup_iters=setup_iters, setup_s=t_setup,
               approx_modes=dict(n=cfg["n_tv"], lam=[float(appr["lam"][i]) for i in order],
                                 eps=[float(appr["eps"][i]) for i in order],
                                 eps_median=float(np.median(appr["eps"])), n_kept_cutoff_0_75=int(appr["n_kept"])),
               n_eig=n_eig, eig_s=t_eig, converged=st["converged"], max_resid=float(max(res)),
               lambda_min=float(lam[0]), lambda_max=float(lam[-1]), sweeps=st["sweeps"], solves=st["solves"],
               outer_iters=st["outer_iters"], coarse_iters=st["coarse_iters"])
    print(json.dumps(out), flush=True)
    return out


def small_field(flush, device):
    """The 4 lowest pairs of the 4^4 workload (mixed, to 1e-10), the field of the
    oracle's complete eigensolve in the CPU baseline: the like-for-like ratio of
    two complete runs."""
    import torch

    import synth
    from paper_1509_06865_gb300 import MIXED, Context

    cfg = workload("dense_4x4x4x4")
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    times = []
    for _ in range(3):
        ctx = Context(dims, device=device)
        ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                       sap_block=cfg["sap_block"], precision=MIXED)
        flush.fill_(5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.load_gauge(U)
        ctx.setup(cfg["seed"])
        lam, _, res, st = ctx.eigensolve(cfg["n_eig"], cfg["tol"], want_vectors=False)
        e1.record()
        torch.cuda.synchronize()
        ctx.close()
        times.append(e0.elapsed_time(e1) / 1e3)
    # the same eigensolve once more, untimed, for the eigenvectors that are set
    # beside the oracle's
    out = dict(gpu_s=statistics.median(times), max_resid=float(max(res)), converged=st["converged"],
               n_eig=cfg["n_eig"], outer_iters=st["outer_iters"], solves=st["solves"])
    try:
        ctx = Context(dims, device=device)
        ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                       sap_block=cfg["sap_block"], precision=MIXED)
        ctx.load_gauge(U)
        ctx.setup(cfg["seed"])
        lam_v, V, _, _ = ctx.eigensolve(cfg["n_eig"], cfg["tol"], want_vectors=True)
        ctx.close()
        return out, (lam_v, V)
    except Exception as e:  # the timed numbers above stand without the comparison
        out["vs_oracle"] = dict(error=repr(e)[:300])
        return out, None


def pairs_vs_oracle(lam, V, lam_o, V_o):
    """How far the GPU's eigenpairs lie from the oracle's on the same field: the
    largest eigenvalue difference relative to the largest |lambda| (both lists
    sorted by value), and the smallest norm of a GPU eigenvector's projection on
    the span of the oracle's eigenvectors (1 when the sets agree; basis-free, so
    degenerate pairs compare too)."""
    import numpy as np

    lam, lam_o = np.sort(np.asarray(lam, float)), np.sort(np.asarray(lam_o, float))
    if lam.shape != lam_o.shape:
        return dict(error=f"{lam.size} GPU pairs against {lam_o.size} oracle pairs")
    G = np.asarray(V).reshape(len(V), -1)
    O = np.asarray(V_o).reshape(len(V_o), -1)
    Qo, _ = np.linalg.qr(O.T)                 # orthonormal basis of the oracle's span
    proj = np.linalg.norm(Qo.conj().T @ G.T, axis=0) / np.linalg.norm(G, axis=1)
    return dict(max_rel_dlambda=float(np.max(np.abs(lam - lam_o)) / np.max(np.abs(lam_o))),
                min_span_overlap=float(np.min(proj)), lambda_gpu=lam.tolist(), lambda_oracle=lam_o.tolist())


# ---------------------------------------------------------------------------
# CPU oracle (baseline and --impl reference)


def oracle_outer_iteration_s(name: str, iters: int):
    """Seconds per outer FGMRES iteration of the oracle on a workload's field: one
    two-grid cycle (the coarse GMRES at its iteration cap, the SAP cycles), one
    FP64 application of Q - sigma and the Arnoldi Gram-Schmidt step, timed over
    `iters` iterations of one shifted solve (sigma = 0, P from the workload's
    number of Philox-uniform test vectors; building P and the coarse operator is
    not timed)."""
    import numpy as np

    import synth
    from oracle import dirac, krylov, mg

    cfg = workload(name)
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    m0 = cfg["m0"] if cfg.get("m0") is not None else load_m0()
    op = dirac.WilsonClover(U, m0, cfg["csw"], tuple(cfg.get("bc", (1, 1, 1, 1))))
    params = dict(mg.DEFAULT_PARAMS, agg=tuple(cfg["agg"]), ntv=cfg["n_tv"], sap_block=tuple(cfg["sap_block"]),
                  coarse_tol=0.0)
    # the two-grid preconditioner with a seeded random coarse operator of the
    # right shape: at a fixed coarse iteration count its cost does not depend on
    # the operator's values, and the oracle's Galerkin build (minutes at 16^3 x 32)
    # is not part of an outer iteration
    W = synth.uniform_vectors(dims, cfg["n_tv"], cfg["seed"])
    B = object.__new__(mg.TwoGrid)
    B.op, B.p, B.W, B._defl = op, params, np.array(W), None
    B.P = mg.Interpolation(B.W, params["agg"])
    n2 = 2 * cfg["n_tv"]
    rng = np.random.default_rng(cfg["seed"])
    B.Dc = rng.standard_normal((9, B.P.nagg, n2, n2)) + 1j * rng.standard_normal((9, B.P.nagg, n2, n2))
    B.coarse = mg.CoarseOperator(B.Dc, B.P.cdims, B.P.ntv)
    B.sap = mg.SAP(op, params["sap_block"])
    b = synth.gaussian_vectors(dims, 1, 3)[0]
    B(b, 0.0)   # the coarse deflation data, outside the timed region
    t0 = time.perf_counter()
    krylov.fgmres(lambda v: op.Q_sigma(v, 0.0), lambda v: B(v, 0.0), b, tol=0.0, restart=iters, maxiter=iters)
    return (time.perf_counter() - t0) / iters


def oracle_complete_small(vectors_path=None):
    """One complete oracle eigensolve (setup and Algorithm 1 with the library's
    default additions) of the 4^4 workload's 4 lowest pairs to 1e-10: its wall
    time, work and eigenvalues; the eigenvectors go to `vectors_path` (.npy)
    when one is given."""
    import numpy as np

    import synth
    from oracle import dirac, mg, rqi

    cfg = workload("dense_4x4x4x4")
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    t0 = time.perf_counter()
    op = dirac.WilsonClover(U, cfg["m0"], cfg["csw"])
    params = dict(mg.DEFAULT_PARAMS, agg=tuple(cfg["agg"]), ntv=cfg["n_tv"], sap_block=tuple(cfg["sap_block"]))
    lam, V, res, st = rqi.eigensolve(op, synth.uniform_vectors(dims, cfg["n_tv"], cfg["seed"]), cfg["n_eig"],
                                     cfg["tol"], params)
    wall = time.perf_counter() - t0
    assert float(np.max(res)) <= cfg["tol"], res
    if vectors_path:
        np.save(vectors_path, np.asarray(V))
    return dict(wall_s=wall, n_eig=cfg["n_eig"], sweeps=st["sweeps"], solves=st["solves"],
                outer_iters=st["outer_iters"], max_res=float(np.max(res)), lam=np.asarray(lam).tolist())


def oracle_baseline(c_big=None, vectors_path=None):
    """The FP64 CPU oracle, measured: a complete oracle eigensolve of the 4^4
    workload (4 pairs to 1e-10, about 40 s), scaled to the 20 pairs of the 16^3 x
    32 benchmark field by the oracle's own measured cost of one outer FGMRES
    iteration on both fields (about 20 s on the large one) and the pair count:
        value = T(4^4, complete) * C(16^3x32) / C(4^4) * 20 / 4.
    The premise is the method's: outer iterations per eigenpair hardly depend on
    the volume (the paper's Fig. 1), the cost of each grows with it.  `cores` is
    the CPU time of the sample over its wall time (numpy's element-wise kernels
    use one core, its LAPACK calls more)."""
    c0 = time.process_time()
    t0 = time.perf_counter()
    small = oracle_complete_small(vectors_path)
    c_small = oracle_outer_iteration_s("dense_4x4x4x4", 6)
    if c_big is None:
        c_big = oracle_outer_iteration_s("bench_16x16x16x32", 1)
    wall = time.perf_counter() - t0
    cores = (time.process_time() - c0) / wall
    big_pairs = WORKLOAD["n_eig"]
    value = small["wall_s"] * (c_big / c_small) * (big_pairs / small["n_eig"])
    return dict(value=value, unit="s", cores=round(cores, 2), nproc=os.cpu_count(), kind="oracle",
                sample="a complete FP64 oracle eigensolve of the 4^4 workload (4 pairs to 1e-10, wall time measured) "
                       "scaled to 20 pairs on the 16^3x32 field by the oracle's measured seconds per outer FGMRES "
                       "iteration on both fields (two-grid cycle + FP64 stencil + Gram-Schmidt) and the pair ratio",
                sample_seconds=wall, complete_4x4x4x4=small, outer_iteration_s=dict(small=c_small, bench=c_big))


def oracle_baseline_subprocess(vectors_path=None):
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample"]
    if vectors_path:
        cmd += ["--oracle-vectors", vectors_path]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        return dict(kind="oracle", error=r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args):
    """The oracle arm: every warm-up and timed step is a complete oracle_baseline()
    measurement on this host; value = their median."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # the oracle's cost of one outer iteration on the 16^3 x 32 field (about a
    # minute with its operator build) is measured once; every warm-up and timed
    # step runs the complete 4^4 eigensolve and the 4^4 outer-iteration sample
    c_big = oracle_outer_iteration_s("bench_16x16x16x32", 1)
    for _ in range(args.warmup):
        oracle_baseline(c_big)
    t0 = time.perf_counter()
    runs = [oracle_baseline(c_big) for _ in range(max(1, args.steps))]
    elapsed = time.perf_counter() - t0
    v = statistics.median(r["value"] for r in runs)
    last = runs[-1]
    line = dict(impl="reference", metric=METRIC, value=v, unit="s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * elapsed / max(1, args.steps), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD["workload"], dims=WORKLOAD["dims"], m0=load_m0(),
                            n_eig=WORKLOAD["n_eig"], tol=WORKLOAD["tol"]),
                cpu_baseline=dict(last, value=v, values=[r["value"] for r in runs]),
                e2e=dict(value=v, unit="s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
                wall_s=elapsed)
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the cost of Algorithm 1 against the number of wanted pairs, and with P built
# from a subset of the modes (the trend of Fig. 2 and the remark after it, Sec. 2.2)


def neig_study(device=0):
    import torch

    import synth
    from paper_1509_06865_gb300 import MIXED, Context

    w = WORKLOAD
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    rows = []
    cases = [(n, -1) for n in (4, 8, 12, 16, 20, 24, 32)] + [(20, 12), (20, 6)]
    for n_eig, p_modes in cases:
        ctx = Context(dims, device=device)
        ctx.set_params(m0=load_m0(), csw=w["csw"], n_tv=20, precision=MIXED, p_modes=p_modes)
        ctx.load_gauge(U)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ctx.setup(w["seed"])
        lam, _, res, st = ctx.eigensolve(n_eig, w["tol"], want_vectors=False)
        e1.record()
        torch.cuda.synchronize()
        ctx.close()
        rows.append(dict(n_eig=n_eig, p_modes=p_modes if p_modes > 0 else 20, s=e0.elapsed_time(e1) / 1e3,
                         converged=st["converged"], max_resid=float(res.max()), sweeps=st["sweeps"],
                         solves=st["solves"], outer_iters=st["outer_iters"], coarse_iters=st["coarse_iters"]))
        print(json.dumps(rows[-1]), flush=True)
    return rows


# ---------------------------------------------------------------------------
# batched shifted solves of several fields (the batched workload: 16 shifts in
# [0, 0.05] x 12 Z2 + iZ2 right-hand sides per field; fields of three sizes)


def batch_study(device=0, nrhs=12, nsig=16):
    import torch

    import synth
    from paper_1509_06865_gb300 import MIXED, Context, solve_batch

    # the six fields of uneven size (two each of 8^4, 12^3 x 24, 16^3 x 32); the
    # 12^3 x 24 lattice takes SAP blocks of 3^4 (an even number of blocks per direction)
    fields = [((8, 8, 8, 8), 1101), ((8, 8, 8, 8), 1102), ((12, 12, 12, 24), 1105), ((12, 12, 12, 24), 1106),
              ((16, 16, 16, 32), 1103), ((16, 16, 16, 32), 1104)]
    ctxs, rhs = [], []
    for dims, seed in fields:
        ctx = Context(dims, device=device)
        sap = (3, 3, 3, 3) if dims[0] == 12 else (4, 4, 4, 4)
        # m0 above the critical value of the 16^3x32 workload: min |lambda| > max sigma (no singular system)
        ctx.set_params(m0=load_m0() + 0.06, csw=1.9, n_tv=20, precision=MIXED, sap_block=sap)
        ctx.load_gauge(synth.gauge_field(dims, 0.2, seed))
        ctx.setup(seed)
        ctxs.append(ctx)
        rhs.append(synth.z2_noise(dims, nrhs, seed))
    sigmas = [0.05 * k / (nsig - 1) for k in range(nsig)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xs, st = solve_batch(ctxs, sigmas, rhs, 1e-10)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nsys = len(fields) * nsig * nrhs
    out = dict(fields=[list(d) for d, _ in fields], shifts=nsig, rhs_per_field=nrhs, systems=nsys, s=dt,
               systems_per_s=nsys / dt, converged=st["converged"], outer_iters=st["outer_iters"],
               mean_outer_per_system=st["outer_iters"] / nsys, note="host buffers in and out, tol 1e-10")
    for ctx in ctxs:
        ctx.close()
    print(json.dumps(out), flush=True)
    return out


# ---------------------------------------------------------------------------
# small self-terminating cases for ncu (one GPU, a few GB)


def profile_case(case: str):
    """stencil32: five FP32 applications of Q - sigma on a 32^3 x 64 lattice with
    unit links (the stencil's memory traffic does not depend on the link values),
    about 4 GB of device memory.

    eig16: the 16^3 x 32 benchmark field, multigrid setup with one refinement
    pass, then one sweep of Algorithm 1 on 3 vectors without guards to
    eigen-residual 1e-3: every kernel of the hot path a few hundred times at the
    benchmark's lattice size, in a few seconds and a few GB of device memory.

    learned16: four training steps of the learned smoother (batch 4) on the
    16^3 x 32 field: the BF16 tensor-core convolutions forward, data and weight
    gradients, about 3 GB of device memory.

    coarse32: three BF16 tensor-core coarse applies on 12 right-hand sides on
    the coarse grid of the 32^3 x 64 lattice (unit links, setup without
    iterations), about 6 GB of device memory."""
    import synth
    from paper_1509_06865_gb300 import MIXED, OP_Q, PREC_F32, Context

    if case == "learned16":
        # the learned smoother's training and inference kernels on the 16^3 x 32 field
        w = workload("bench_16x16x16x32")
        dims = tuple(w["dims"])
        ctx = Context(dims)
        ctx.set_params(m0=w["m0"], csw=w["csw"], n_tv=w["n_tv"], agg=w["agg"], sap_block=w["sap_block"],
                       precision=MIXED, setup_iters=1)
        ctx.load_gauge(synth.gauge_field(dims, w["eps"], w["seed"]))
        ctx.setup(w["seed"])
        ctx.net_init(1)
        ctx.net_train(4, 4, 2e-3, 99)
        ctx.close()
        print("profile case", case, "ok")
        return
    if case == "coarse32":
        # the BF16 tensor-core coarse apply on 12 right-hand sides, 32^3 x 64 coarse grid
        import torch
        from paper_1509_06865_gb300 import LINKS_BF16
        cfg = workload("large_32x32x32x64")
        dims = tuple(cfg["dims"])
        ctx = Context(dims)
        ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], agg=cfg["agg"], n_tv=cfg["n_tv"], sap_block=cfg["sap_block"],
                       precision=MIXED, coarse_links=LINKS_BF16, setup_iters=0)
        ctx.load_gauge(synth.unit_gauge(dims))
        ctx.setup(cfg["seed"])
        nc = ctx.coarse_sites * 2 * cfg["n_tv"]
        X = torch.randn(12 * nc, dtype=torch.complex64, device="cuda:0")
        Y = torch.empty_like(X)
        torch.cuda.synchronize()
        for _ in range(3):
            ctx.coarse_apply_dev_nrhs(X.data_ptr(), Y.data_ptr(), 12, 0.01)
        torch.cuda.synchronize()
        ctx.close()
        print("profile case", case, "ok")
        return
    if case == "stencil32":
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
        print("profile case", case, "ok")
        return
    cfg = workload("bench_16x16x16x32")
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    ctx = Context(dims)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], n_tv=cfg["n_tv"], precision=MIXED, setup_iters=1,
                   max_sweeps=1, n_guard=0)
    ctx.load_gauge(U)
    ctx.setup(cfg["seed"])
    _, _, _, st = ctx.eigensolve(3, 1e-3, want_vectors=False)
    ctx.close()
    print("profile case", case, st)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 32^3x64 eigensolve")
    ap.add_argument("--large-fp64", action="store_true", help="also the all-FP64 32^3x64 eigensolve")
    ap.add_argument("--profile-case", choices=["eig16", "stencil32", "coarse32", "learned16"])
    ap.add_argument("--neig-study", action="store_true",
                    help="time Algorithm 1 on the 16^3x32 field for 4..32 wanted pairs and with P from 12 / 6 modes")
    ap.add_argument("--learned-study", action="store_true",
                    help="16^3x32: train the learned smoother on 10^4 pairs, then SAP vs net vs none at 1e-10")
    ap.add_argument("--config3-study", action="store_true",
                    help="32^3x64: approximate modes after a 30-iteration setup, then the 50 lowest pairs")
    ap.add_argument("--batch-study", action="store_true",
                    help="16 shifts x 12 Z2 right-hand sides on six fields (8^4, 12^3x24, 16^3x32) with mgeig_solve_batch")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-vectors", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_sample:
        print(json.dumps(oracle_baseline(vectors_path=args.oracle_vectors)))
        return
    if args.profile_case:
        profile_case(args.profile_case)
        return
    if args.neig_study:
        neig_study()
        return
    if args.batch_study:
        batch_study()
        return
    if args.config3_study:
        config3_study()
        return
    if args.learned_study:
        learned_study()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
