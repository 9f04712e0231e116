#!/usr/bin/env python
"""Benchmark of the GB300 FlashEigen hot path (arXiv 1602.01421).

Workload (default): R-MAT scale 22 (4.19M vertices, edge factor 16, a/b/c/d 0.57/0.19/0.19/
0.05, seed 1, symmetrised, self-loops/duplicates removed, 0/1 int32 CSR).  One step = one
plain FP64 Block Krylov-Schur solve for the 8 largest-magnitude eigenpairs, block 4, 8 blocks
(subspace 32), tol 1e-8, counter-RNG start: SpMM, block Gram/update re-orthogonalisation (the
restart product and the second Gram-Schmidt pass on the tensor cores), CholQR2, Rayleigh-Ritz,
restarts and the explicit residual check, all on the GPU.
Beside it (one results line): the SpMM sweep b in {1,2,4,8,16} x {FP32, FP64} in GB/s of
compulsory bytes, the roofline of the step's dominant kernel and of the tensor-core kernels,
the same solve with all-FP64 orthogonalisation arithmetic, the full solve at R-MAT scale 14,
the mixed-precision and learned-start solves, 32 and 64 eigenpairs with 128- and 256-vector
subspaces, R-MAT scale 24 (mixed vs FP64 at subspace 64; learned vs random starts), the SVD of
a directed R-MAT graph, the semi-external SpMM, the end-to-end time through host buffers, and
the CPU oracle on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--scale S]
    python bench.py --config mixed24|learned24|semiext27     (single configurations; semiext27
                                                              is not in the default run: its
                                                              graph generation alone takes ~2 min)
    python bench.py --only solve [--solve-mode mixed]        (timed solves only)
    python bench.py --only spmm1|gram1|ugram1|tcrestart|tcupdate|tcgram
                                                             (launches of one kernel, for
                                                              profiler captures)

Under torchrun (N > 1) every rank solves its own copy of the workload (replicas: one solve
runs on one GPU and is not split across GPUs); value = all ranks' solves / the slowest rank's
time.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMM GB/s & % HBM peak; time to 8 eigenpairs @1e-8, plain vs mixed/learned"
NEV, BLOCK, NBLOCKS, TOL = 8, 4, 8, 1e-8
# the scale-22 solve needs about 500 restarts (a tight cluster at -221); the cap only bounds
# a run that does not converge
MAX_RESTARTS = 5000
NOMINAL_HBM = 8000.0
# FP64 on GB300: 2 FP64 operations per clock per SM x 152 SMs x 2.07 GHz = 629 G/s (1.26
# TFLOP/s counting an FMA as two); the FP64 SpMM is bound by its adds, not by HBM.
FP64_ADD_PEAK_G = 2 * 152 * 2.07
# dram__bytes_read.sum + dram__bytes_write.sum of one spmm_main_kernel<double,4> launch on
# R-MAT scale 22 (ncu, the one-launch capture of `bench.py --only spmm1 --prec f64 --b 4`)
SPMM_F64_B4_DRAM_BYTES = 1455201024 + 109192192


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def spmm_bytes(n, nnz, b, s):
    """Compulsory bytes of one SpMM: colidx + rowptr + X read once + Y written."""
    return 4 * nnz + 4 * (n + 1) + 2 * n * b * s


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev_index, path):
        self.path = path
        self.proc = None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(dev_index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_aggregate(ms_local, steps, dist=None, device="cpu"):
    """Replicas: every rank runs `steps` solves; the job time is the slowest rank's, and the
    whole-job throughput counts all ranks' solves.  Returns (value, max_ms, world_size)."""
    ws = 1
    ms = float(ms_local)
    if dist is not None and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ws * steps / (ms / 1000.0), ms, ws


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_full_solves():
    """Full oracle solves of the benchmark graphs (block SpMM counts, restarts, time), written by
    tests/golden/make_oracle_solves.py, which calls only the oracle."""
    p = os.path.join(ROOT, "tests", "golden", "oracle_solves.json")
    return json.load(open(p)) if os.path.exists(p) else {}


def run_reference(args):
    """The oracle (plain CPU FP64 Block Krylov-Schur) timed on the host cores.

    Each timed step is one bounded sample of the workload: the oracle's solve stopped after
    --ref-cycles Krylov-Schur cycles (the first cycle builds all 8 blocks, every later one 3),
    so steps x ms_per_step is time actually spent.  `value` extrapolates the sample's time per
    block SpMM step to the block count of the oracle's OWN full solve of the same graph
    (tests/golden/oracle_solves.json).  The first cycles orthogonalise against fewer blocks
    than the average cycle, so the extrapolation errs on the fast side for the oracle."""
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    import graphgen
    from oracle import bks
    g = graphgen.rmat(args.scale, seed=1)
    cores = os.cpu_count()
    full = oracle_full_solves().get(f"rmat{args.scale}")
    for _ in range(args.warmup):
        bks.block_krylov_schur(g.rowptr, g.colidx, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                               max_restarts=0)
    times, blocks = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = bks.block_krylov_schur(g.rowptr, g.colidx, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                                   max_restarts=args.ref_cycles - 1)
        times.append(time.perf_counter() - t0)
        blocks.append(r.spmm_blocks)
    per_block = sum(times) / sum(blocks)
    if full is not None:
        full_blocks, basis = full["spmm_blocks"], (f"the oracle's own full solve of this graph "
                                                   f"({full['spmm_blocks']} block SpMMs, "
                                                   f"{full['restarts']} restarts)")
    else:
        full_blocks, basis = blocks[0], "no full oracle solve recorded for this scale: the sample itself"
    t_solve = per_block * full_blocks
    sample = (f"{args.ref_cycles} Krylov-Schur cycle(s) of the oracle on R-MAT scale {args.scale} "
              f"({blocks[0]} block SpMMs, {statistics.median(times):.2f} s median) per step; "
              f"time per block SpMM x {full_blocks} block SpMMs of {basis}")
    # config 1 (scale 14): the oracle's full solve fits in seconds -- timed once, in full
    t14 = None
    if args.scale != 14 and not args.no_config1:
        g14 = graphgen.rmat(14, seed=1)
        t0 = time.perf_counter()
        r14 = bks.block_krylov_schur(g14.rowptr, g14.colidx, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                                     max_restarts=5000)
        t14 = {"workload": "rmat14-ef16 FP64 Block Krylov-Schur nev8 b4 m32 tol1e-8 (full solve)",
               "s": round(time.perf_counter() - t0, 3), "restarts": int(r14.restarts),
               "spmm_blocks": int(r14.spmm_blocks), "converged": bool(r14.converged)}
    value = 1.0 / t_solve
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}-ef16 FP64 Block Krylov-Schur nev8 b4 m32 tol1e-8",
                       "n": g.n, "nnz": g.nnz},
            "sample": {"ms_per_step": 1000.0 * statistics.mean(times), "block_spmms_per_step": blocks[0],
                       "s_per_block_spmm": per_block},
            "extrapolation": {"full_solve_block_spmms": full_blocks, "basis": basis,
                              "s_per_solve": t_solve},
            "full_solve_config1": t14,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_cuda(fn, reps, torch):
    s = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    torch.cuda.synchronize()
    for a, b in evs:
        a.record(s)
        fn()
        b.record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


UGRAM_NV = 7


def ugram_inputs(fe, torch, n):
    """Inputs of the roofline launch: V = 7 FP64 blocks of n x 4 (the second classical
    Gram-Schmidt pass against 7 blocks), C (28 x 4, small), W (n x 4)."""
    Vg = fe.random_normal(UGRAM_NV * n, 4, dtype=torch.float64, seed=5).view(UGRAM_NV, n, 4)
    Wg = fe.random_normal(n, 4, dtype=torch.float64, seed=6)
    Cg = 1e-3 * torch.randn(UGRAM_NV * 4, 4, dtype=torch.float64, device=Wg.device,
                            generator=torch.Generator(device=Wg.device).manual_seed(7))
    return Vg, Cg, Wg


def cpu_baseline(g, scale, cycles=2):
    """The oracle on a bounded sample (its first `cycles` Krylov-Schur cycles), time per block
    SpMM scaled to the block count of the oracle's own full solve of the graph."""
    from oracle import bks
    t0 = time.perf_counter()
    r = bks.block_krylov_schur(g.rowptr, g.colidx, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                               max_restarts=cycles - 1)
    t = time.perf_counter() - t0
    full = oracle_full_solves().get(f"rmat{scale}")
    blocks = full["spmm_blocks"] if full else r.spmm_blocks
    t_solve = t / r.spmm_blocks * blocks
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{cycles} Krylov-Schur cycles ({r.spmm_blocks} block SpMMs, {t:.1f} s) of the "
                      f"oracle on the same graph; time per block SpMM x {blocks} block SpMMs "
                      + ("of the oracle's own full solve" if full else "(no full solve recorded)")}


def run_ours(args):
    import numpy as np
    import torch
    import graphgen
    import paper_1602_01421_gb300 as fe

    ws, rank, local = dist_setup()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    lib = fe.load()
    lib.fe_kernel_launches.restype = ctypes.c_int64
    hbm_peak, peak_kind = peaks()

    t_gen = time.perf_counter()
    g = graphgen.rmat(args.scale, seed=1)
    t_gen = time.perf_counter() - t_gen
    n, nnz = g.n, g.nnz
    t0 = time.perf_counter()
    # --index-format applies to the profiler mode spmm1; the step uses the default plan
    h = fe.Csr.from_graph(g, index_format=args.index_format if args.only == "spmm1" else "auto")
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    info = h.info()

    if args.only == "gram1":
        # one Gram launch at the FP64 solve's mean shape (7 blocks of n x 4 against n x 4)
        Vg = fe.random_normal(7 * n, 4, dtype=torch.float64, seed=5).view(7, n, 4)
        Wg = fe.random_normal(n, 4, dtype=torch.float64, seed=6)
        for _ in range(args.warmup + args.steps):
            fe.block_gram(Vg, Wg)
        torch.cuda.synchronize()
        print(json.dumps({"only": "gram1", "n": n, "nv": 7, "b": 4}))
        return
    if args.only in ("tcrestart", "tcupdate", "tcgram"):
        # the tensor-core kernels at the FP64 solve's shapes: the restart product (8 blocks of
        # n x 4 into 5), the second pass's update W - V G1 (8 blocks into 1), its Gram (9 blocks
        # against n x 4)
        gen = torch.Generator(device="cuda").manual_seed(7)
        Vt = fe.random_normal((9 if args.only == "tcgram" else 8) * n, 4, dtype=torch.float64,
                              seed=5).view(-1, n, 4)
        Wt = fe.random_normal(n, 4, dtype=torch.float64, seed=6)
        Yt = torch.randn(32, 20, dtype=torch.float64, device="cuda", generator=gen)
        Ot = torch.empty((5, n, 4), dtype=torch.float64, device="cuda")
        Ct = (torch.randn(32, 4, dtype=torch.float64, device="cuda", generator=gen) * 1e-3)
        for _ in range(args.warmup + args.steps):
            if args.only == "tcrestart":
                fe.block_combine(Vt, Yt, 5, Ot, engine="tc")
            elif args.only == "tcupdate":
                fe.block_update(Vt, Ct, Wt, -1.0, 1.0, engine="tc")
            else:
                fe.block_gram(Vt, Wt, engine="tc")
        torch.cuda.synchronize()
        print(json.dumps({"only": args.only, "n": n}))
        return
    if args.only == "ugram1":
        # one fused update + Gram launch at the FP64 solve's shape (7 blocks of n x 4)
        Vg, Cg, Wg = ugram_inputs(fe, torch, n)
        for _ in range(args.warmup + args.steps):
            fe.block_update_gram(Vg, Cg, Wg, alpha=-1.0, beta=1.0)
        torch.cuda.synchronize()
        print(json.dumps({"only": "ugram1", "n": n, "nv": UGRAM_NV, "b": 4}))
        return
    if args.only == "spmm1":
        # one SpMM launch (for a single-kernel profiler capture)
        tdt = torch.float32 if args.prec == "f32" else torch.float64
        Xs = fe.random_normal(n, args.b, dtype=tdt, seed=3)
        Ys = torch.empty_like(Xs)
        for _ in range(args.warmup):
            fe.spmm(h, Xs, Ys)
        for _ in range(args.steps):
            fe.spmm(h, Xs, Ys)
        torch.cuda.synchronize()
        print(json.dumps({"only": "spmm1", "n": n, "nnz": nnz, "b": args.b, "prec": args.prec}))
        return

    def solve(mode="fp64"):
        return fe.eigs(h, NEV, BLOCK, NBLOCKS, TOL, "LM", mode=mode, seed=1, max_restarts=MAX_RESTARTS)

    for _ in range(args.warmup):
        ev, X, st = solve(args.solve_mode if args.only == "solve" else "fp64")
        assert st["converged"], "warm-up solve did not converge"
    if args.only == "solve":
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(args.steps):
            ev, X, st = solve(args.solve_mode)
        s1.record()
        torch.cuda.synchronize()
        print(json.dumps({"only": "solve", "mode": args.solve_mode, "n": n, "nnz": nnz,
                          "s_per_solve": s0.elapsed_time(s1) / 1e3 / max(args.steps, 1),
                          "restarts": st["restarts"], "spmm_blocks": st["spmm_blocks"],
                          "evals": [float(x) for x in ev]}))
        return

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    clk = Clocks(dev, os.path.join(args.outdir, f"clocks_rank{rank}.csv"))
    time.sleep(0.3)
    barrier()
    l0 = lib.fe_kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        ev, X, st = solve()
        stats.append(st)
    e1.record(stream)
    barrier()
    launches = lib.fe_kernel_launches() - l0
    clocks = clk.stop()
    value, ms, _ = replica_aggregate(e0.elapsed_time(e1), args.steps, dist, device="cuda")
    ms_per_step = ms / args.steps
    blocks = stats[-1]["spmm_blocks"]

    # ---- SpMM sweep (compulsory-byte GB/s), b in {1,2,4,8,16} x {f32, f64}
    sweep = {}
    for prec, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        for b in (1, 2, 4, 8, 16):
            Xs = fe.random_normal(n, b, dtype=tdt, seed=3)
            Ys = torch.empty_like(Xs)
            for _ in range(3):
                fe.spmm(h, Xs, Ys)
            t = time_cuda(lambda: fe.spmm(h, Xs, Ys), args.sweep_reps, torch)
            med = statistics.median(t)
            gb = spmm_bytes(n, nnz, b, es) / (med / 1000.0) / 1e9
            # secondary: gather-inclusive bytes (every nonzero's X row counted, as an SpMM with
            # no X reuse in any cache would move them)
            gather_b = spmm_bytes(n, nnz, b, es) - n * b * es + nnz * b * es
            sweep[f"{prec}_b{b}"] = {"ms": round(med, 4), "GBps": round(gb, 1),
                                     "frac_measured": round(gb / hbm_peak, 4),
                                     "frac_nominal": round(gb / NOMINAL_HBM, 4),
                                     "gather_GBps": round(gather_b / (med / 1000.0) / 1e9, 1)}
            del Xs, Ys
    # SpMM roofline (the metric's kernel), FP32 b = 4 and the solve's FP64 b = 4
    spmm_roofline = {}
    for key, es in (("f32_b4", 4), ("f64_b4", 8)):
        achieved = sweep[key]["GBps"]
        spmm_roofline[key] = {"kernel": "spmm_main_kernel + hub_reduce_kernel", "bound": "hbm",
                              "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                              "frac": round(achieved / hbm_peak, 4), "peak_kind": peak_kind,
                              "bytes_per_launch": spmm_bytes(n, nnz, 4, es)}
    # dominant kernel of the FP64 solve (launch list: 25.6% of the kernel time), the SpMM with an
    # FP64 block of 4 columns; bound by FP64 adds (one per non-zero and column), reported against
    # the nominal FP64 add rate
    t64 = sweep["f64_b4"]["ms"]
    adds = float(nnz) * 4
    gadds = adds / (t64 / 1000.0) / 1e9
    roofline = {"kernel": "spmm_main_kernel<double,4> + hub_reduce_kernel (FP64 SpMM, b = 4)",
                "bound": "alu", "achieved": round(gadds, 1), "peak": FP64_ADD_PEAK_G,
                "unit": "G FP64 adds/s", "frac": round(gadds / FP64_ADD_PEAK_G, 4),
                "peak_kind": "nominal FP64 add rate (2 per clock per SM x 152 SMs x 2.07 GHz)",
                "traffic": SPMM_F64_B4_DRAM_BYTES if args.scale == 22 else None,
                "adds_per_launch": adds, "bytes_per_launch": spmm_bytes(n, nnz, 4, 8),
                "ms_per_launch": t64, "stream": "torch current stream",
                "hbm_frac": round(spmm_bytes(n, nnz, 4, 8) / (t64 / 1000.0) / 1e9 / hbm_peak, 4)}
    # the tensor-core split-product kernels at the solve's shapes, against HBM: the restart
    # product V Y (8 blocks of n x 4 into 5) and the second-pass Gram [V_0..V_7 W]^T W
    roofline_tc = {}
    try:
        Vt = fe.random_normal(8 * n, 4, dtype=torch.float64, seed=5).view(8, n, 4)
        Yt = torch.randn(32, 20, dtype=torch.float64, device=Vt.device,
                         generator=torch.Generator(device=Vt.device).manual_seed(7))
        Ot = fe.block_combine(Vt, Yt, 5, engine="tc")
        tcm = statistics.median(time_cuda(lambda: fe.block_combine(Vt, Yt, 5, Out=Ot, engine="tc"), 10, torch))
        bc = 8.0 * n * (32 + 20)
        roofline_tc["tc_combine_pipe_kernel<4,32> (restart V Y, 8 -> 5 blocks)"] = {
            "bound": "hbm", "achieved": round(bc / (tcm / 1000.0) / 1e9, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(bc / (tcm / 1000.0) / 1e9 / hbm_peak, 4),
            "bytes_per_launch": bc, "ms_per_launch": round(tcm, 4),
            "fma_engine_ms": round(statistics.median(time_cuda(
                lambda: fe.block_combine(Vt, Yt, 5, Out=Ot, engine="fma"), 5, torch)), 4)}
        del Ot
        # the second pass's update W <- W - V G1 at its largest shape (8 blocks into 1)
        Wt = fe.random_normal(n, 4, dtype=torch.float64, seed=6)
        Ct = Yt[:, :4].contiguous() * 1e-3
        tum = statistics.median(time_cuda(lambda: fe.block_update(Vt, Ct, Wt, -1.0, 1.0, engine="tc"), 10, torch))
        bu = 8.0 * n * (32 + 4 + 4)
        roofline_tc["tc_combine_pipe_kernel<4,16> (update W - V G1, 8 blocks)"] = {
            "bound": "hbm", "achieved": round(bu / (tum / 1000.0) / 1e9, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(bu / (tum / 1000.0) / 1e9 / hbm_peak, 4),
            "bytes_per_launch": bu, "ms_per_launch": round(tum, 4),
            "fma_engine_ms": round(statistics.median(time_cuda(
                lambda: fe.block_update(Vt, Ct, Wt, -1.0, 1.0, engine="fma"), 5, torch)), 4)}
        del Ct, Yt
        Vx = torch.cat([Vt, Wt.view(1, n, 4)], 0)
        Gt = fe.block_gram(Vx, Wt, engine="tc")
        tgm = statistics.median(time_cuda(lambda: fe.block_gram(Vx, Wt, G=Gt, engine="tc"), 10, torch))
        bg = 8.0 * n * (36 + 4)
        roofline_tc["tc_gram_pipe_kernel<4> ([V_0..V_7 W]^T W)"] = {
            "bound": "hbm", "achieved": round(bg / (tgm / 1000.0) / 1e9, 1), "peak": hbm_peak,
            "unit": "GB/s", "frac": round(bg / (tgm / 1000.0) / 1e9 / hbm_peak, 4),
            "bytes_per_launch": bg, "ms_per_launch": round(tgm, 4),
            "fma_engine_ms": round(statistics.median(time_cuda(
                lambda: fe.block_gram(Vx, Wt, G=Gt, engine="fma"), 5, torch)), 4)}
        del Vt, Wt, Vx, Gt
    except Exception as e:
        roofline_tc = {"error": str(e)}

    # ---- the same FP64 solve with every orthogonalisation product in FP64 arithmetic
    # (orth_pass1 = fp64: no FP32-arithmetic first Gram-Schmidt pass or small corrections)
    fp64_all = None
    if not args.no_fp64_all:
        try:
            out = {}
            def run_all64():
                out["r"] = fe.eigs(h, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1, orth_pass1="fp64",
                                   max_restarts=MAX_RESTARTS)
            run_all64()
            ta = time_cuda(run_all64, 1, torch)[0]
            eva, Xa, sta = out["r"]
            fp64_all = {"s": ta / 1000.0, "restarts": sta["restarts"], "spmm_blocks": sta["spmm_blocks"],
                        "converged": sta["converged"], "max_resid": sta["max_resid"],
                        "max_rel_eval_diff_vs_step": float(np.max(np.abs(eva - ev) / np.abs(ev))),
                        "time_vs_step": ta / ms_per_step}
        except Exception as e:
            fp64_all = {"error": str(e)}

    # ---- config 1: R-MAT scale 14, the full plain FP64 solve (the oracle arm times its own
    # full solve of the same graph)
    config1 = None
    if not args.no_config1 and args.scale != 14:
        try:
            g14 = graphgen.rmat(14, seed=1)
            with fe.Csr.from_graph(g14) as h14:
                out = {}
                def run14():
                    out["r"] = fe.eigs(h14, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1,
                                       max_restarts=MAX_RESTARTS)
                for _ in range(3):
                    run14()
                t14 = statistics.median(time_cuda(run14, 5, torch))
                ev14, _, st14 = out["r"]
            full14 = oracle_full_solves().get("rmat14")
            config1 = {"workload": "rmat14-ef16 FP64 Block Krylov-Schur nev8 b4 m32 tol1e-8 (full solve)",
                       "s": t14 / 1000.0, "restarts": st14["restarts"], "spmm_blocks": st14["spmm_blocks"],
                       "converged": st14["converged"],
                       "max_rel_eval_diff_vs_oracle": (float(np.max(np.abs(ev14 - np.array(full14["evals"]))
                                                                    / np.abs(np.array(full14["evals"]))))
                                                       if full14 else None)}
        except Exception as e:
            config1 = {"error": str(e)}

    # ---- mixed-precision solve on the same graph (time to 8 eigenpairs)
    t_mixed = None
    if not args.no_mixed:
        try:
            out = {}
            def run_mixed():
                out["r"] = solve("mixed")
            run_mixed()
            tm = time_cuda(run_mixed, 1, torch)[0]
            ev2, X2, st2 = out["r"]
            t_mixed = {"s": tm / 1000.0, "spmm_blocks": st2["spmm_blocks"],
                       "spmm_blocks_fp32": st2["spmm_blocks_fp32"], "restarts": st2["restarts"],
                       "restarts_fp32": st2["restarts_fp32"], "seconds_fp32": st2["seconds_fp32"],
                       "max_rel_eval_diff_vs_fp64": float(np.max(np.abs(ev2 - ev) / np.abs(ev))),
                       "converged": st2["converged"], "speedup_vs_fp64": ms_per_step / tm}
        except Exception as e:  # reported, not hidden
            t_mixed = {"error": str(e)}

    # ---- learned start: MLP trained on small R-MAT graphs, time to 8 pairs on this graph
    learned_res = None
    learned_params = None
    if not args.no_learned:
        try:
            from paper_1602_01421_gb300 import learned as L
            t0 = time.perf_counter()
            # span loss against the nev wanted Ritz vectors of each training graph
            ex = [L.make_subspace_example(graphgen.rmat(sc, seed=100 + i))
                  for i, sc in enumerate([12, 13, 14, 15, 16, 17] * 3)]
            params, losses = L.train(ex, hidden=64, b=BLOCK, steps=1500, lr=2e-3, loss="span")
            learned_params = params
            t_train = time.perf_counter() - t0
            out = {}
            def run_learned():
                out["r"] = fe.eigs(h, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1, mlp_weights=params,
                                   mlp_hidden=64, max_restarts=MAX_RESTARTS)
            run_learned()
            tl = time_cuda(run_learned, 1, torch)[0]
            ev4, X4, st4 = out["r"]
            learned_res = {"s": tl / 1000.0, "spmm_blocks": st4["spmm_blocks"],
                           "spmm_start_calls": st4["spmm_start"], "restarts": st4["restarts"],
                           "speedup_vs_fp64_random": ms_per_step / tl,
                           "max_rel_eval_diff_vs_fp64": float(np.max(np.abs(ev4 - ev) / np.abs(ev))),
                           "train": {"graphs": len(ex), "scales": "12-17", "steps": 1500,
                                     "loss": "span vs the 8 wanted Ritz vectors",
                                     "final_loss": float(np.mean(losses[-50:])),
                                     "s": round(t_train, 2)}}
            # the learned start with the mixed-precision iteration
            def run_learned_mixed():
                out["rm"] = fe.eigs(h, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1, mlp_weights=params,
                                    mlp_hidden=64, mode="mixed", max_restarts=MAX_RESTARTS)
            run_learned_mixed()
            tlm = time_cuda(run_learned_mixed, 1, torch)[0]
            ev5, X5, st5 = out["rm"]
            learned_res["mixed"] = {
                "s": tlm / 1000.0, "spmm_blocks": st5["spmm_blocks"], "restarts": st5["restarts"],
                "speedup_vs_fp64_random": ms_per_step / tlm,
                "max_rel_eval_diff_vs_fp64": float(np.max(np.abs(ev5 - ev) / np.abs(ev)))}
        except Exception as e:
            learned_res = {"error": str(e)}

    # ---- many eigenvalues: nev 32 with the paper's setting for larger sets (block 4 and as
    # many blocks as eigenvalues: m = 128), FP64 and mixed
    many = None
    if not args.no_many:
        try:
            many = {"nev": 32, "block": 4, "nblocks": 32}
            out = {}
            ev32 = None
            for mode in ("fp64", "mixed"):
                def run_many():
                    out["r"] = fe.eigs(h, 32, 4, 32, TOL, "LM", seed=1, mode=mode,
                                       max_restarts=MAX_RESTARTS)
                run_many()
                tmn = time_cuda(run_many, 1, torch)[0]
                evm, Xm, stm = out["r"]
                many[mode] = {"s": tmn / 1000.0, "restarts": stm["restarts"],
                              "spmm_blocks": stm["spmm_blocks"], "converged": stm["converged"],
                              "max_resid": stm["max_resid"]}
                if ev32 is None:
                    ev32 = evm
                else:
                    many[mode]["max_rel_eval_diff_vs_fp64"] = float(np.max(np.abs(evm - ev32) / np.abs(ev32)))
            many["evals_8_vs_nev8_solve"] = float(np.max(np.abs(ev32[:NEV] - ev) / np.abs(ev)))
        except Exception as e:
            many = {"error": str(e)}

    # ---- many eigenvalues with a 256-vector subspace (nev 64, block 4, 64 blocks), mixed mode
    if many is not None and "error" not in many and not args.no_many:
        try:
            out = {}
            def run_many256():
                out["r"] = fe.eigs(h, 64, 4, 64, TOL, "LM", seed=1, mode="mixed",
                                   max_restarts=MAX_RESTARTS)
            run_many256()
            t256 = time_cuda(run_many256, 1, torch)[0]
            ev256, _, st256 = out["r"]
            many["nev64_m256_mixed"] = {"s": t256 / 1000.0, "restarts": st256["restarts"],
                                        "spmm_blocks": st256["spmm_blocks"],
                                        "converged": st256["converged"], "max_resid": st256["max_resid"],
                                        "evals_32_vs_nev32_solve": float(np.max(np.abs(ev256[:32] - ev32) / np.abs(ev32)))}
        except Exception as e:
            many["nev64_m256_mixed"] = {"error": str(e)}

    # ---- SVD of a directed graph (the paper's page-graph method): directed R-MAT of the same
    # scale, 8 singular values through A^T A, block 2 and 2 x 8 blocks (the paper's setting)
    svd_res = None
    if not args.no_svd:
        try:
            out = {}
            gd = graphgen.rmat(args.scale, seed=1, directed=True)
            svd_res = {"graph": f"directed rmat{args.scale}-ef16", "n": gd.n, "nnz": gd.nnz,
                       "nsv": 8, "block": 2, "nblocks": 16}
            with fe.Csr.from_graph(gd) as hd:
                for key, fn in (("spmm", fe.spmm), ("spmm_t", fe.spmm_t)):
                    Xs = fe.random_normal(gd.n, 2, dtype=torch.float32, seed=3)
                    Ys = torch.empty_like(Xs)
                    fn(hd, Xs, Ys)
                    ts = statistics.median(time_cuda(lambda: fn(hd, Xs, Ys), 10, torch))
                    svd_res[f"{key}_f32_b2"] = {
                        "ms": round(ts, 4),
                        "GBps": round(spmm_bytes(gd.n, gd.nnz, 2, 4) / (ts / 1000.0) / 1e9, 1)}
                sv0 = None
                for mode in ("fp64", "mixed"):
                    def run_svd():
                        out["s"] = fe.svds(hd, 8, 2, 16, TOL, seed=1, mode=mode,
                                           max_restarts=MAX_RESTARTS)
                    run_svd()
                    tsv = time_cuda(run_svd, 1, torch)[0]
                    sv, Vr, Ul, sts = out["s"]
                    svd_res[mode] = {"s": tsv / 1000.0, "restarts": sts["restarts"],
                                     "ata_applications": sts["spmm_blocks"],
                                     "converged": sts["converged"]}
                    if sv0 is None:
                        sv0 = sv
                        svd_res["svals_head"] = [float(x) for x in sv[:3]]
                    else:
                        svd_res[mode]["max_rel_sval_diff_vs_fp64"] = float(np.max(np.abs(sv - sv0) / sv0))
            del gd
        except Exception as e:
            svd_res = {"error": str(e)}

    # ---- semi-external: the same SpMM with the CSR streamed from pinned host memory
    semi = None
    if not args.no_semi:
        try:
            cap = 256 << 20
            semi = {"cap_bytes": cap}
            # staged copies or direct reads of the pinned panels; packed (default) or plain
            # column indices
            for mode, direct, fmt in (("staged", False, "auto"), ("staged_plain", False, "plain"),
                                      ("direct", True, "auto")):
                with fe.Csr.from_graph(g, device_mem_cap_bytes=cap, semi_direct=direct,
                                       index_format=fmt) as hs:
                    si = hs.info()
                    Xs = fe.random_normal(n, 4, dtype=torch.float32, seed=3)
                    Ys = torch.empty_like(Xs)
                    fe.spmm(hs, Xs, Ys)
                    ts = statistics.median(time_cuda(lambda: fe.spmm(hs, Xs, Ys), 5, torch))
                semi[mode] = {"panels": si["panels"], "device_bytes": si["device_bytes"],
                              "index_format": "packed" if si["index_format"] == 2 else "plain",
                              "index_bytes": si["index_bytes"], "f32_b4_ms": round(ts, 3),
                              "GBps": round(spmm_bytes(n, nnz, 4, 4) / (ts / 1000.0) / 1e9, 1),
                              "index_read_GBps": round(si["index_bytes"] / (ts / 1000.0) / 1e9, 1)}
        except Exception as e:
            semi = {"error": str(e)}

    # ---- R-MAT scale 24: the mixed-precision solve against the plain FP64 one (block 8,
    # subspace 64), and the learned start against random starts (block 4, subspace 32, mixed),
    # each result with its explicit residual from the oracle's SpMM
    scale24 = None
    if not args.no_scale24 and args.scale == 22:
        try:
            scale24 = config24(args, fe, graphgen, torch, learned_params)
        except Exception as e:
            scale24 = {"error": str(e)}

    # ---- end to end through host buffers: CSR create (H2D) + solve + evecs D2H
    e2e_times = []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with fe.Csr.from_graph(g) as h2:
            ev3, X3, st3 = fe.eigs(h2, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1, max_restarts=MAX_RESTARTS)
            host = X3.cpu().numpy()
        torch.cuda.synchronize()
        if i > 0:
            e2e_times.append(time.perf_counter() - t0)
    e2e = {"value": 1.0 / statistics.mean(e2e_times), "unit": "solves/s",
           # the SpMM plan fe_csr_create uploads (the handle's device bytes minus the hub
           # partial-sum buffer, 16 doubles per hub chunk, which is allocated, not copied)
           "h2d_bytes_per_step": int(info["device_bytes"] - 128 * info["hub_chunks"]),
           "d2h_bytes_per_step": int(host.nbytes) + 8 * NEV}

    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"rmat{args.scale}-ef16 FP64 Block Krylov-Schur nev8 b4 m32 tol1e-8",
                       "n": n, "nnz": nnz, "rmat": "a/b/c/d=0.57/0.19/0.19/0.05 seed1 permuted",
                       "l2": "inputs larger than L2 (CSR %.0f MB)" % ((4 * nnz + 8 * n) / 1e6),
                       "parallelism": f"replicas{ws}"},
            "time_to_8_eigenpairs_s": ms_per_step / 1000.0,
            "eigs": {"restarts": stats[-1]["restarts"], "spmm_blocks": blocks,
                     "evals_head": [float(x) for x in ev[:3]], "max_resid": stats[-1]["max_resid"]},
            "fp64_all_orth": fp64_all, "config1": config1, "scale24": scale24, "mixed": t_mixed,
            "learned": learned_res, "many_eigs": many, "svd": svd_res, "semi_external": semi,
            "spmm_sweep": sweep, "spmm_roofline": spmm_roofline, "roofline": roofline,
            "roofline_tc": roofline_tc,
            "clocks": clocks, "e2e": e2e,
            "gpu_launches": int(launches),
            "setup": {"graph_gen_s": round(t_gen, 2), "csr_create_s": round(t_create, 3),
                      "device_bytes": info["device_bytes"]}}
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(g, args.scale)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def config24(args, fe, graphgen, torch, learned_params):
    """R-MAT scale 24 (16.8M vertices, edge factor 16): plain FP64 vs mixed precision (nev 8,
    block 8, 8 blocks: subspace 64, tol 1e-8), and learned vs random starts (nev 8, block 4,
    8 blocks, mixed, tol 1e-8; the network trained on small graphs, this graph unseen)."""
    import numpy as np
    from oracle import core
    t0 = time.perf_counter()
    g = graphgen.rmat(24, seed=1)
    res = {"workload": "rmat24-ef16", "n": g.n, "nnz": g.nnz, "gen_s": round(time.perf_counter() - t0, 1)}

    def resid(ev, X):
        Xh = X.cpu().numpy()
        R = core.spmm(g.rowptr, g.colidx, Xh) - Xh * ev
        return float((np.linalg.norm(R, axis=0) / np.abs(ev)).max())

    with fe.Csr.from_graph(g) as h:
        def timed(**kw):
            out = {}
            def run():
                out["r"] = fe.eigs(h, max_restarts=MAX_RESTARTS, **kw)
            t = time_cuda(run, 1, torch)[0] / 1000.0
            return out["r"] + (t,)

        ev64, X64, st64, t64 = timed(nev=8, block=8, nblocks=8, tol=TOL, which="LM", seed=1)
        res["fp64_b8_m64"] = {"s": t64, "restarts": st64["restarts"], "spmm_blocks": st64["spmm_blocks"],
                              "converged": st64["converged"], "max_rel_resid_oracle_spmm": resid(ev64, X64)}
        del X64
        evm, Xm, stm, tm = timed(nev=8, block=8, nblocks=8, tol=TOL, which="LM", seed=1, mode="mixed")
        res["mixed_b8_m64"] = {"s": tm, "restarts": stm["restarts"], "restarts_fp32": stm["restarts_fp32"],
                               "spmm_blocks": stm["spmm_blocks"], "converged": stm["converged"],
                               "max_rel_resid_oracle_spmm": resid(evm, Xm),
                               "max_rel_eval_diff_vs_fp64": float(np.max(np.abs(evm - ev64) / np.abs(ev64))),
                               "speedup_vs_fp64": t64 / tm}
        del Xm
        if learned_params is not None:
            rnd = []
            for sd in (1, 2, 3):
                ev, X, st, t = timed(nev=8, block=BLOCK, nblocks=NBLOCKS, tol=TOL, which="LM", seed=sd,
                                     mode="mixed", return_vectors=False)
                rnd.append({"seed": sd, "s": t, "spmm_blocks": st["spmm_blocks"]})
            evl, Xl, stl, tl = timed(nev=8, block=BLOCK, nblocks=NBLOCKS, tol=TOL, which="LM", seed=1,
                                     mode="mixed", mlp_weights=learned_params, mlp_hidden=64)
            res["learned_start_mixed"] = {
                "train": "span loss, 18 R-MAT graphs at scales 12-17, 1500 Adam steps (the learned leg's network)",
                "random": rnd, "learned": {"s": tl, "spmm_blocks": stl["spmm_blocks"],
                                           "spmm_start_calls": stl["spmm_start"],
                                           "max_rel_resid_oracle_spmm": resid(evl, Xl)},
                "spmm_ratio_vs_random_median": stl["spmm_blocks"] / float(np.median([x["spmm_blocks"] for x in rnd]))}
    return res


def run_config(args):
    """The other measurement configurations (one results line each, not the step metric)."""
    import numpy as np
    import torch
    import graphgen
    import paper_1602_01421_gb300 as fe
    from oracle import core
    torch.cuda.set_device(0)
    out = {"config": args.config}
    if args.config in ("mixed24", "learned24"):
        t0 = time.perf_counter()
        g = graphgen.rmat(24, seed=1 if args.config == "mixed24" else 24)
        out.update(n=g.n, nnz=g.nnz, gen_s=round(time.perf_counter() - t0, 1))
        h = fe.Csr.from_graph(g)

        def timed(**kw):
            torch.cuda.synchronize()
            t = time.perf_counter()
            ev, X, st = fe.eigs(h, max_restarts=MAX_RESTARTS, **kw)
            torch.cuda.synchronize()
            return ev, X, st, time.perf_counter() - t

        def cpu_resid(ev, X):
            """explicit residuals with the CPU oracle's SpMM (FP64) on the returned vectors"""
            Xh = X.cpu().numpy()
            R = core.spmm(g.rowptr, g.colidx, Xh) - Xh * ev
            return (np.linalg.norm(R, axis=0) / np.abs(ev)).max()

        if args.config == "mixed24":
            b, nb = 8, 8
            ev64, X64, st64, t64 = timed(nev=8, block=b, nblocks=nb, tol=1e-8, which="LM", seed=1)
            evm, Xm, stm, tm = timed(nev=8, block=b, nblocks=nb, tol=1e-8, which="LM", seed=1, mode="mixed")
            out.update(workload="rmat24-ef16 nev8 b8 m64 tol1e-8",
                       fp64={"s": t64, "restarts": st64["restarts"], "spmm_blocks": st64["spmm_blocks"],
                             "max_rel_resid_cpu": cpu_resid(ev64, X64)},
                       mixed={"s": tm, "restarts": stm["restarts"], "restarts_fp32": stm["restarts_fp32"],
                              "spmm_blocks": stm["spmm_blocks"], "spmm_blocks_fp32": stm["spmm_blocks_fp32"],
                              "s_fp32": stm["seconds_fp32"], "max_rel_resid_cpu": cpu_resid(evm, Xm),
                              "max_rel_eval_diff_vs_fp64": float(np.max(np.abs(evm - ev64) / np.abs(ev64)))},
                       speedup=t64 / tm, evals=[float(x) for x in ev64])
        else:
            from paper_1602_01421_gb300 import learned as L
            ex = [L.make_subspace_example(graphgen.rmat(sc, seed=100 + i))
                  for i, sc in enumerate([14, 15, 16, 17, 18, 19, 20] * args.learned_graphs)]
            params, losses = L.train(ex, hidden=64, b=BLOCK, steps=args.learned_steps, lr=2e-3,
                                     loss="span")
            res = []
            for sd in (1, 2, 3):
                ev, X, st, t = timed(nev=8, block=BLOCK, nblocks=NBLOCKS, tol=1e-8, which="LM", seed=sd,
                                     mode="mixed", return_vectors=False)
                res.append({"seed": sd, "s": t, "spmm_blocks": st["spmm_blocks"]})
            ev, X, st, t = timed(nev=8, block=BLOCK, nblocks=NBLOCKS, tol=1e-8, which="LM", seed=1,
                                 mode="mixed", mlp_weights=params, mlp_hidden=64)
            out.update(workload="rmat24-ef16 (fresh seed) nev8 b4 m32 tol1e-8 mixed",
                       train={"graphs": len(ex), "scales": "14-20", "steps": args.learned_steps,
                              "loss": "span vs the 8 wanted Ritz vectors",
                              "final_loss": float(np.mean(losses[-50:]))},
                       random=res, learned={"s": t, "spmm_blocks": st["spmm_blocks"],
                                            "spmm_start_calls": st["spmm_start"],
                                            "max_rel_resid_cpu": cpu_resid(ev, X)})
        h.close()
    elif args.config == "semiext27":
        t0 = time.perf_counter()
        g = graphgen.rmat(27, seed=1)
        out.update(n=g.n, nnz=g.nnz, gen_s=round(time.perf_counter() - t0, 1))
        cap = 6 << 30
        t0 = time.perf_counter()
        h = fe.Csr.from_graph(g, device_mem_cap_bytes=cap, semi_direct=args.semi_direct,
                              index_format=args.index_format)
        info = h.info()
        out.update(create_s=round(time.perf_counter() - t0, 1), cap_bytes=cap, panels=info["panels"],
                   device_bytes=info["device_bytes"], index_bytes=info["index_bytes"],
                   index_format="packed" if info["index_format"] == 2 else "plain")
        for prec, tdt, es in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
            X = fe.random_normal(g.n, 4, dtype=tdt, seed=3)
            Y = torch.empty_like(X)
            fe.spmm(h, X, Y)
            tt = statistics.median(time_cuda(lambda: fe.spmm(h, X, Y), 3, torch))
            rows = np.random.default_rng(0).integers(0, g.n, 20000)
            ref = core.spmm_rows(g.rowptr, g.colidx, X.cpu().numpy(), rows)
            err = float(np.max(np.abs(Y.cpu().numpy()[rows] - ref) /
                               (core.spmm_rows(g.rowptr, g.colidx, np.abs(X.cpu().numpy()), rows) + 1e-300)))
            out[f"spmm_{prec}_b4"] = {"ms": round(tt, 2), "GBps": round(spmm_bytes(g.n, g.nnz, 4, es) / tt / 1e6, 1),
                                      "index_read_GBps": round(info["index_bytes"] / tt / 1e6, 1),
                                      "max_rel_err_sampled_rows": err}
            del X, Y
        # the configuration's solve: 8 eigenpairs at tol 1e-8, block 4, 8 blocks, FP64 subspace in
        # HBM while the CSR streams; explicit residuals checked with the oracle's SpMM
        for mode in args.semi_modes.split(","):
            if not mode:
                continue
            torch.cuda.synchronize()
            t = time.perf_counter()
            ev, X, st = fe.eigs(h, NEV, BLOCK, NBLOCKS, TOL, "LM", seed=1, mode=mode,
                                max_restarts=MAX_RESTARTS, raise_on_noconverge=False)
            torch.cuda.synchronize()
            ts = time.perf_counter() - t
            Xh = X.cpu().numpy()
            R = core.spmm(g.rowptr, g.colidx, Xh) - Xh * ev
            out[f"solve_{mode}"] = {"s": round(ts, 2), "converged": st["converged"],
                                    "restarts": st["restarts"], "spmm_blocks": st["spmm_blocks"],
                                    "max_rel_resid_cpu": float((np.linalg.norm(R, axis=0) / np.abs(ev)).max()),
                                    "orth": float(np.abs(Xh.T @ Xh - np.eye(NEV)).max()),
                                    "evals": [float(x) for x in ev]}
            del X, Xh, R
            print(json.dumps({"progress": f"solve_{mode}", **out[f"solve_{mode}"]}), flush=True)
        h.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--sweep-reps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-scale24", action="store_true",
                    help="skip the R-MAT scale-24 legs (mixed vs FP64 at subspace 64, learned start)")
    ap.add_argument("--no-fp64-all", action="store_true",
                    help="skip the FP64 solve with all-FP64 orthogonalisation arithmetic")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-many", action="store_true", help="skip the nev 32 (m = 128) leg")
    ap.add_argument("--no-svd", action="store_true", help="skip the directed-graph SVD leg")
    ap.add_argument("--no-semi", action="store_true")
    ap.add_argument("--index-format", default="auto", choices=["auto", "plain", "packed"],
                    help="semiext27 and --only spmm1: column-index format of the CSR")
    ap.add_argument("--semi-modes", default="mixed,fp64",
                    help="semiext27: solve modes to time on the semi-external handle ('' = none)")

    ap.add_argument("--ref-cycles", type=int, default=2,
                    help="reference arm: Krylov-Schur cycles of the oracle per timed sample")
    ap.add_argument("--no-config1", action="store_true",
                    help="skip the full scale-14 solves (both arms)")
    ap.add_argument("--outdir", default=os.path.join(ROOT, "bench_out"),
                    help="where the clock samples are written")
    ap.add_argument("--only", default="all",
                    choices=["all", "solve", "spmm1", "gram1", "ugram1", "tcrestart", "tcupdate", "tcgram"],
                    help="solve: warm-up + timed solves only; spmm1 / gram1 / ugram1 / tcrestart / "
                         "tcupdate / tcgram: launches of one kernel only (profiler captures)")
    ap.add_argument("--b", type=int, default=4)
    ap.add_argument("--solve-mode", default="fp64", choices=["fp64", "mixed"],
                    help="--only solve: which solve to run")
    ap.add_argument("--config", default="rmat22", choices=["rmat22", "mixed24", "learned24", "semiext27"],
                    help="rmat22: the step metric (default); others print their own results line")
    ap.add_argument("--learned-graphs", type=int, default=2)
    ap.add_argument("--semi-direct", action="store_true",
                    help="semiext27: kernels read the pinned panels directly (no staging copies)")
    ap.add_argument("--learned-steps", type=int, default=1500)
    ap.add_argument("--prec", default="f64", choices=["f32", "f64"])
    args = ap.parse_args()
    os.makedirs(args.outdir, exist_ok=True)
    if args.impl == "reference":
        run_reference(args)
    elif args.config != "rmat22":
        run_config(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
