#!/usr/bin/env python
"""Benchmark: quantics-MPS Fresnel propagation steps per second.

Workload (default): a 2^16 x 2^16 wavefront (n = 16 interleaved d = 4 sites),
never densified -- a separable Gaussian beam times a seeded rank-8 smooth phase,
built on the GPU from per-axis TT-SVD encodings (Kronecker-interleaved, summed,
compressed to chi = 128).  One step = Q_x, Q_y, D_x, D_y, Q_x^dagger, Q_y^dagger
applied by zip-up with truncation to chi = 128 (Fig. fig_mpo_mpo of the paper),
lambda z / dx^2 = 25.3 (lambda = 633 nm, dx = 10 um, z = 4 mm per step).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the same workload instead.  Multi-GPU runs are independent replicas (the
path does not shard): value = steps of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Fresnel MPO-MPS steps/s at 2^16², χ=128: mixed vs FP32 plain; % roofline"
LAMBDA_Z_OVER_DX2 = 25.3
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["fp32", "mixed", "both"], default="both",
                    help="site contractions in FP32 (SIMT) or mixed (split-BF16 tcgen05 tensor cores, FP32 "
                         "accumulation); both: the headline value is the mixed path, the FP32 plain path is timed "
                         "beside it")
    ap.add_argument("--n", type=int, default=16)
    ap.add_argument("--chi", type=int, default=128)
    ap.add_argument("--cutoff", type=float, default=1e-10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-profile", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end steps through host buffers (0 skips them)")
    ap.add_argument("--eager", action="store_true", help="launch every kernel from the host instead of "
                                                           "replaying the step's CUDA graph")
    ap.add_argument("--workload", choices=["fresnel", "batched", "optics"], default="fresnel",
                    help="batched: many independent wavefronts (n 8-12, chi 16-64) stepped as CUDA graphs")
    ap.add_argument("--items", type=int, default=64, help="items of the batched workload")
    ap.add_argument("--branches", type=int, default=0, help="parallel branches of the batched graph (0: auto)")
    ap.add_argument("--eig-cluster-min", type=int, default=-1,
                    help="smallest order solved by the 8-CTA cluster eigen-solver (-1: the library's default, 32; "
                         "161: one CTA per solve)")
    ap.add_argument("--oracle-worker", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--oracle-budget", type=float, default=30.0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    return args


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock/throttle sampling while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        # nvidia-smi numbers GPUs in PCI order and ignores CUDA_VISIBLE_DEVICES: address the device by its UUID
        self.idx = str(device_index)
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device_index).uuid)
            self.idx = u if u.startswith("GPU-") else f"GPU-{u}"
        except Exception:
            pass
        self.proc = None
        self.path = os.path.join("/tmp", f"qtn_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "gpu": self.idx}


# ----------------------------------------------------------------------------- GPU workload

def build_state_gpu(qtn, n: int, chi: int, cutoff: float):
    """Separable Gaussian beam x rank-8 smooth phase as an interleaved MPS, on the GPU."""
    import torch
    import synth
    fx, gy = synth.separable_phase_factors(n)
    big = 192                                               # room for one direct sum before compression
    eng = qtn.Engine(n_sites=n, d=4, chi=big, w=2, dense=1 << n)
    acc = None
    for r in range(fx.shape[0]):
        X = qtn.MPS(n, 2, 32)
        Y = qtn.MPS(n, 2, 32)
        eng.encode(torch.from_numpy(fx[r].astype(np.complex64)).cuda(), n, "1d", X, 32, cutoff, stats=False)
        eng.encode(torch.from_numpy(gy[r].astype(np.complex64)).cuda(), n, "1d", Y, 32, cutoff, stats=False)
        term = qtn.MPS(n, 4, big)
        eng.kron_interleave(X, Y, term)
        # right-canonical terms keep the FP32 sweeps over the direct sum well conditioned
        eng.truncate(term, big, 1e-13, stats=False)
        if acc is None:
            acc = term
        else:
            s = qtn.MPS(n, 4, big)
            eng.add(acc, term, s)
            eng.truncate(s, chi, cutoff, stats=False)
            acc = s
    eng.truncate(acc, chi, cutoff, stats=False)
    out = qtn.MPS(n, 4, chi)
    out.sites.copy_(acc.sites[:, :chi, :, :chi])
    out.bond.copy_(acc.bond)
    out.c.canon = acc.c.canon
    torch.cuda.synchronize()
    return out


def run_ours(args, rank, ws, local, prec):
    import torch
    from paper_2510_23089_gb300 import qtn

    torch.cuda.set_device(local)
    if args.eig_cluster_min >= 0:
        qtn.load_library().qtn_set_eig_cluster_min(args.eig_cluster_min)
    n, chi = args.n, args.chi
    L = 1 << n
    c = LAMBDA_Z_OVER_DX2 / L
    psi0 = build_state_gpu(qtn, n, chi, args.cutoff)
    eng_b = qtn.Engine(n_sites=n, d=4, chi=16, w=16, dense=0)      # operator builds on the default stream
    Q = eng_b.build_qft_mpo(n, False, 1e-12, w_cap=16)
    Qd = eng_b.mpo_dagger(Q)
    # phase MPO needs a 2^n dense scratch: a separate small engine
    eng_p = qtn.Engine(n_sites=n, d=2, chi=16, w=2, dense=1 << n)
    D = eng_p.build_phase_mpo(n, c, 1e-12, w_cap=16)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")
    psi = psi0.clone()                                      # the buffers every step (and the graph) work on
    torch.cuda.synchronize()
    del eng_p, eng_b
    stream = torch.cuda.Stream()                            # a created stream: graphs cannot capture the legacy one
    eng = qtn.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=stream)
    use_graph = not args.eager
    # one Fresnel step recorded as a CUDA graph (qtn_batch_create) and replayed per step
    batch = qtn.Batch([eng], [psi], [Q], [Qd], [D], n_steps=1, chi_max=chi, cutoff=args.cutoff,
                      prec=prec) if use_graph else None

    def reset():
        psi.sites.copy_(psi0.sites)
        psi.bond.copy_(psi0.bond)
        psi.c.canon = psi0.c.canon

    def step(eager=False):
        if use_graph and not eager:
            batch.launch(1)
        else:
            eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, chi, args.cutoff, prec, stats=False)

    with torch.cuda.stream(stream):
        reset()
        for _ in range(args.warmup):                        # warm-up from the initial state
            step()
        torch.cuda.synchronize()
        # the timed region propagates the initial state through `steps` Fresnel steps (the workload)
        reset()
        sampler = ClockSampler(local)
        barrier(ws)
        torch.cuda.synchronize()
        launches0 = eng.launch_count()
        sampler.start()
        times = []
        torch.cuda.nvtx.range_push("bench_timed")          # lets a profiler select the timed steps alone
        for _ in range(args.steps):
            flush.zero_()                                   # evict the L2 between timed steps
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        clocks = sampler.stop()
        launches = eng.launch_count() - launches0
        barrier(ws)
        total_ms = max_over_ranks(sum(times), ws)
        bonds_after = psi.bonds()
        final = psi.clone()                                 # the state after the timed steps (accuracy check)

        # kernel classes: CUDA events around every launch cannot sit inside a replayed graph, so the same
        # steps run once more without the graph and with the library's profiling on
        prof, prof_ms = {}, None
        if not args.no_profile:
            reset()
            torch.cuda.synchronize()
            eng.profile(True)
            pt = []
            for _ in range(args.steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(eager=True)
                e1.record(stream)
                e1.synchronize()
                pt.append(e0.elapsed_time(e1))
            for cls, name in ((0, "k_gemm"), (1, "k_eig"), (2, "k_gemm_tc")):
                ms, cnt, fl = eng.profile_read(cls)
                if cnt:
                    prof[name] = (ms, cnt, fl)
            eng.profile(False)
            prof_ms = sum(pt)

        # end-to-end through the C ABI with host buffers: pinned host state -> device, one step, result -> host
        host_sites = psi0.sites.cpu().pin_memory()
        host_bond = psi0.bond.cpu().pin_memory()
        out_sites = torch.empty_like(host_sites).pin_memory()
        out_bond = torch.empty_like(host_bond).pin_memory()
        e2e_t = []
        for it in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            psi.sites.copy_(host_sites, non_blocking=True)
            psi.bond.copy_(host_bond, non_blocking=True)
            psi.c.canon = psi0.c.canon
            step()
            out_sites.copy_(psi.sites, non_blocking=True)
            out_bond.copy_(psi.bond, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            if it > 0:
                e2e_t.append(e0.elapsed_time(e1))
    if batch is not None:
        batch.close()
    e2e_ms = max_over_ranks(sum(e2e_t) / len(e2e_t), ws) if e2e_t else None
    h2d = host_sites.numel() * 8 + host_bond.numel() * 4
    return {
        "times": times, "total_ms": total_ms, "clocks": clocks, "launches": launches, "prof": prof,
        "prof_ms": prof_ms, "e2e_ms": e2e_ms, "h2d": h2d, "bonds": bonds_after, "bonds0": psi0.bonds(),
        "Qw": Q.w_max, "Dw": D.w_max, "graph": use_graph, "final": final,
    }


def run_batched(args, local):
    """Independent wavefronts of the batched workload (Gaussian beam x Kolmogorov phase screen, n in 8..12,
    chi in {16, 32, 64}), all advanced by one launch of one CUDA graph per step (the items split into parallel
    branches), with the GEMM tile of each (n, chi) class chosen by the autotuner on a copy of one of its items."""
    import torch
    import synth
    from paper_2510_23089_gb300 import qtn

    torch.cuda.set_device(local)
    prec = "fp32" if args.prec == "fp32" else "mixed"
    # the cluster eigen-solver also wins here: 64 items at 255 item-steps/s against 164 with one CTA per solve
    eig_min = args.eig_cluster_min if args.eig_cluster_min >= 0 else 32
    qtn.load_library().qtn_set_eig_cluster_min(eig_min)
    specs = synth.batched_item_specs(count=args.items)
    nmax, cmax = max(s["n"] for s in specs), max(s["chi"] for s in specs)
    enc = qtn.Engine(n_sites=nmax, d=4, chi=cmax, w=16, dense=1 << (2 * nmax))
    ops = {}
    for n in sorted({s["n"] for s in specs}):
        Q = enc.build_qft_mpo(n, False, 1e-12, w_cap=16)
        ops[n] = (Q, enc.mpo_dagger(Q), enc.build_phase_mpo(n, LAMBDA_Z_OVER_DX2 / (1 << n), 1e-12, w_cap=16))
    items, engines = [], []
    for sp in specs:
        psi = qtn.MPS(sp["n"], 4, sp["chi"])
        field = torch.from_numpy(synth.batched_item_field(sp)).cuda()
        enc.encode(field, sp["n"], "interleaved", psi, sp["chi"], args.cutoff, stats=False)
        del field
        items.append(psi)
        engines.append(qtn.Engine(n_sites=sp["n"], d=4, chi=sp["chi"], w=16, dense=0, stream=torch.cuda.Stream()))
    del enc
    torch.cuda.synchronize()
    # autotuner: GEMM tile per (n, chi) class, on a copy of the first item of the class (cached by QTN_TUNE_CACHE)
    tiles = {}
    for i, sp in enumerate(specs):
        key = (sp["n"], sp["chi"])
        if key not in tiles:
            Q, Qd, D = ops[sp["n"]]
            tiles[key] = engines[i].tune_gemm_tile(items[i].clone(), Q, Qd, D, sp["chi"], args.cutoff, prec)
        engines[i].set_gemm_tile(tiles[key][0])
    torch.cuda.synchronize()
    Qs, Qds, Ds = [ops[s["n"]][0] for s in specs], [ops[s["n"]][1] for s in specs], [ops[s["n"]][2] for s in specs]
    branches, tuned_ms = args.branches, None
    if branches <= 0:   # autotuner: parallel branches of the graph, on copies of the items
        copies = [it.clone() for it in items]
        cands = sorted({max(1, args.items // 4), max(1, args.items // 2), args.items})
        branches, tuned_ms = qtn.tune_branches(engines, copies, Qs, Qds, Ds, 0, args.cutoff, prec, cands)
        del copies
    t0 = time.perf_counter()
    batch = qtn.Batch(engines, items, Qs, Qds, Ds, n_steps=1, chi_max=0, cutoff=args.cutoff, prec=prec,
                      branches=branches)
    build_s = time.perf_counter() - t0
    stream = batch.stream
    batch.launch(args.warmup)
    batch.sync()
    sampler = ClockSampler(local)
    launches0 = qtn.load_library().qtn_launch_count()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    batch.launch(args.steps)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = sampler.stop()
    launches = qtn.load_library().qtn_launch_count() - launches0
    batch.sync()
    batch.close()
    hist = {}
    for s in specs:
        hist[f"n{s['n']}_chi{s['chi']}"] = hist.get(f"n{s['n']}_chi{s['chi']}", 0) + 1
    return {"ms": ms, "clocks": clocks, "launches": launches, "hist": hist, "prec": prec, "build_s": build_s,
            "eig_cluster_min": eig_min,
            "branches": branches, "branches_tuned_ms": tuned_ms,
            "tiles": {f"n{k[0]}_chi{k[1]}": {"tile": v[0], "ms_per_step_one_item": v[1]} for k, v in tiles.items()}}


def run_optics(args, local, ws=1):
    """Mask-gradient workload: per item, the intensity loss of one Fresnel step after a phase mask and its
    gradient with respect to the mask's site tensors (forward pass, adjoint step, overlap derivative), at
    n = 12 (4096 x 4096), field chi = 32, one mask of chi = 16 shared by the batch.  The items are
    independent: each has its own engine and stream and is driven from its own host thread (the library
    calls release the interpreter lock), so their chains of small kernels run concurrently on the GPU.  The
    items' mask gradients are summed and, with the batch sharded over ranks, all-reduced (the one exchange)."""
    from concurrent.futures import ThreadPoolExecutor

    import numpy as np
    import torch
    import synth
    from paper_2510_23089_gb300 import optics, qtn

    torch.cuda.set_device(local)
    n, chi, chi_m = 12, 32, 16
    c = LAMBDA_Z_OVER_DX2 / (1 << n)
    enc = qtn.Engine(n_sites=n, d=4, chi=64, w=32, dense=1 << (2 * n))
    # one phase mask for the batch (its loss is summed over the items); every item works on its own copy
    mx, my = synth.smooth_random_phase_mask_factors(n, seed=7002, strength=0.5)
    X, Y = qtn.MPS(n, 2, 8), qtn.MPS(n, 2, 8)
    enc.encode(torch.from_numpy(mx.astype(np.complex64)).cuda(), n, "1d", X, 8, 1e-12, stats=False)
    enc.encode(torch.from_numpy(my.astype(np.complex64)).cuda(), n, "1d", Y, 8, 1e-12, stats=False)
    M = qtn.MPS(n, 4, 64)
    enc.kron_interleave(X, Y, M)
    enc.truncate(M, chi_m, args.cutoff, stats=False)
    items = []
    for i in range(args.items):
        E = torch.from_numpy(synth.gaussian_beam_with_rectangles(n, seed=7001 + 3 * i, waist=0.1)).cuda()
        Em = qtn.MPS(n, 4, chi)
        enc.encode(E, n, "interleaved", Em, chi, args.cutoff, stats=False)
        It = torch.from_numpy(synth.rectangles_target(n, seed=7003 + 3 * i).astype(np.complex64)).cuda()
        Itm = qtn.MPS(n, 4, chi_m)
        enc.encode(It, n, "interleaved", Itm, chi_m, args.cutoff, stats=False)
        del E, It
        eng = qtn.Engine(n_sites=n, d=4, chi=64, w=32, dense=0, stream=torch.cuda.Stream())
        prob = optics.IntensityLossProblem(eng, n, c, chi=chi, cutoff=args.cutoff, w_cap=16)
        items.append((eng, prob, Em, M.clone(), Itm))
    del enc
    torch.cuda.synchronize()

    def run_item(it, passes):
        eng, prob, Em, M, Itm = it
        loss, H = 0.0, None
        with torch.cuda.stream(eng.stream):
            for _ in range(passes):
                val, cache = prob.forward(Em, M, Itm)
                _, H = prob.backward(Em, M, cache)
                loss += val
        return loss, H

    pool = ThreadPoolExecutor(max_workers=len(items))
    list(pool.map(lambda it: run_item(it, args.warmup), items))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    launches0 = qtn.load_library().qtn_launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for it in items:                       # every item stream starts after e0
        it[0].stream.wait_event(e0)
    res = list(pool.map(lambda it: run_item(it, args.steps), items))
    losses = [r[0] for r in res]
    for it in items:
        ev = torch.cuda.Event()
        ev.record(it[0].stream)
        stream.wait_event(ev)
    # the items' last mask gradients summed, and over the ranks when the items are sharded (the one exchange)
    grad = torch.stack([r[1] for r in res]).sum(dim=0)
    optics.sum_over_ranks_(grad)
    e1.record(stream)
    e1.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), ws)
    clocks = sampler.stop()
    launches = qtn.load_library().qtn_launch_count() - launches0
    pool.shutdown()
    return {"ms": ms, "clocks": clocks, "launches": launches, "loss": sum(losses), "mask_bonds": items[0][3].bonds()}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_state(n: int, chi: int, cutoff: float):
    import synth
    from oracle import mps as OS
    fx, gy = synth.separable_phase_factors(n)
    acc = None
    for r in range(fx.shape[0]):
        X, _ = OS.tt_svd(fx[r], n, 2, 1 << 20, cutoff)
        Y, _ = OS.tt_svd(gy[r], n, 2, 1 << 20, cutoff)
        term = OS.kron_interleave(X, Y)
        acc = term if acc is None else OS.truncate(OS.direct_sum(acc, term), chi, cutoff)[0]
    return OS.truncate(acc, chi, cutoff)[0]


def oracle_steps(n: int, chi: int, cutoff: float, steps: int, budget_s: float):
    """FP64 oracle propagating its own initial state (same recipe) through up to `steps` Fresnel steps,
    stopping once `budget_s` seconds are spent.  Returns (steps done, seconds, bond profile)."""
    from oracle import fresnel as OF
    from oracle import mpo as OM
    from oracle import mps as OS
    L = 1 << n
    c = LAMBDA_Z_OVER_DX2 / L
    sites = oracle_state(n, chi, cutoff)
    ops = (OM.qft_mpo_layers(n, 1e-12), None, OM.phase_mpo(n, c, 1e-12))
    ops = (ops[0], OM.dagger(ops[0]), ops[2])
    canon = "right"
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        sites, canon, _ = OF.fresnel_mps(sites, "interleaved", n, c, chi, cutoff, canon=canon, ops=ops)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return done, time.perf_counter() - t0, OS.bonds(sites)


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max((i.get("num_threads", 1) for i in info), default=os.cpu_count())
    except Exception:
        return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def oracle_rate(n: int, chi: int, cutoff: float, steps: int, budget_s: float, threads: int):
    """The FP64 oracle's steps/s in a child process whose BLAS uses `threads` threads (set through the
    environment before NumPy loads).  Returns dict(done, sec, bonds, threads)."""
    env = dict(os.environ)
    for v in THREAD_VARS:
        env[v] = str(threads)
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--n", str(n), "--chi", str(chi),
           "--cutoff", repr(cutoff), "--steps", str(steps), "--oracle-budget", str(budget_s)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=budget_s * 4 + 600)
    if r.returncode != 0:
        raise RuntimeError(f"oracle worker failed: {r.stderr[-300:]}")
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["threads"] = threads
    return out


def cpu_baseline_line(args, budget_s: float):
    """cpu_baseline: the oracle on all host cores and on one thread (bounded samples of the workload)."""
    cores = os.cpu_count() or 1
    allc = oracle_rate(args.n, args.chi, args.cutoff, args.steps, budget_s, cores)
    one = oracle_rate(args.n, args.chi, args.cutoff, args.steps, budget_s, 1)
    return {"value": allc["done"] / allc["sec"], "unit": "steps/s", "cores": cores, "kind": "oracle",
            "blas_threads": cores,
            "sample": f"the first {allc['done']} of the {args.steps} timed Fresnel steps, FP64 NumPy oracle from its "
                      f"own initial state (bounded at {budget_s:.0f} s), BLAS threads = os.cpu_count() = {cores}; "
                      f"final max bond {max(allc['bonds'])}",
            "bonds": allc["bonds"],
            "one_thread": {"value": one["done"] / one["sec"], "unit": "steps/s", "blas_threads": 1,
                           "sample": f"the first {one['done']} steps, same oracle, bounded at {budget_s:.0f} s"}}


# ----------------------------------------------------------------------------- roofline

def roofline_line(r, peaks, steps: int):
    """Roofline of the dominant kernel class and of the whole step.

    The path is bound by FP32 arithmetic on small dense matrices (the FP64 parts are accumulations of FP32
    products): peak = SMs x 128 FP32 lanes x 2 FLOP x max SM clock.  FLOPs are counted on the device by
    the kernels themselves (algorithmic counts, see the kernel docs) over the same `steps` steps, run once
    more without the graph and with CUDA events around every launch of the two counted classes."""
    import torch
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    prof = r["prof"]
    # The eigen-solve class (the Jacobi sweeps of k_eig_cluster and k_eig_jacobi and the finishing
    # k_eig_finish) is the dominant work; the event-timed durations of the many short GEMM launches of the
    # eager pass include the host's launch gaps and are not used to pick it.
    name = "k_eig" if "k_eig" in prof else max(prof.items(), key=lambda kv: kv[1][0])[0]
    ms, cnt, fl = prof[name]
    achieved = fl / (ms / 1e3) / 1e12 if ms > 0 else 0.0
    flops_step = sum(v[2] for v in prof.values()) / steps
    t_roof = flops_step / (alu_peak * 1e12)
    t_step = r["total_ms"] / steps / 1e3
    label = "k_eig (k_eig_cluster + k_eig_finish + k_eig_jacobi)" if name == "k_eig" else name
    return {"bound": "alu", "kernel": label, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak, "traffic": None,
            "peak_source": f"FP32 FMA: {sm} SMs x 128 lanes x 2 x max SM clock {sm_mhz:.0f} MHz (derived; "
                           "MEASURED_PEAKS holds no FP32 figure)",
            "launches": cnt, "avg_launch_us": 1e3 * ms / max(cnt, 1), "flops_per_launch": fl / max(cnt, 1),
            "share_of_step": ms / r["prof_ms"] if r["prof_ms"] else None,
            "measured_over": f"the same {steps} steps run once more without the CUDA graph, library profiling "
                             "on (events around every launch of the counted classes)",
            "composite": {"flops_per_step": flops_step, "t_roof_ms": t_roof * 1e3, "t_step_ms": t_step * 1e3,
                          "frac": t_roof / t_step,
                          "note": "T_roof = counted FLOPs per step / FP32 peak; T_step = graph-replayed step"},
            "classes": {k: {"ms": v[0], "launches": v[1], "flops": v[2], "ms_per_step": v[0] / steps,
                            "gflop_per_step": v[2] / steps / 1e9} for k, v in prof.items()}}


# ----------------------------------------------------------------------------- main

def main():
    args = parse()
    if args.oracle_worker:
        done, sec, bonds = oracle_steps(args.n, args.chi, args.cutoff, args.steps, args.oracle_budget)
        print(json.dumps({"done": done, "sec": sec, "bonds": bonds}), flush=True)
        return
    rank, ws, local = dist_init()
    config = {"workload": f"quantics interleaved 2^{args.n}x2^{args.n} wavefront, chi={args.chi}, "
                          "Gaussian beam x rank-8 smooth phase, lambda z/dx^2=25.3 per step",
              "n_sites": args.n, "d": 4, "chi": args.chi, "cutoff": args.cutoff, "layout": "interleaved",
              "precision": args.prec,
              "l2": f"flushed between timed steps (state capacity {args.n * 4 * args.chi * args.chi * 8 / 2**20:.1f} "
                    "MiB, L2-resident otherwise)"}
    if args.impl == "reference":
        if rank != 0:
            return
        config["precision"] = "f64 (the oracle)"
        done, sec, bonds = oracle_steps(args.n, args.chi, args.cutoff, args.steps, 120.0)
        value = done / sec
        line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus, "steps": done,
                "warmup": 0, "ms_per_step": sec * 1e3 / done, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config, "impl": "reference",
                "cpu_baseline": {"value": value, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                                 "blas_threads": blas_threads(),
                                 "sample": f"the first {done} Fresnel steps of the FP64 NumPy oracle from the "
                                           f"initial state (bounded at 120 s); final max bond {max(bonds)}"},
                "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    if args.workload == "batched":
        r = run_batched(args, local)
        value = args.items * args.steps * ws / (r["ms"] / 1e3)
        line = {"metric": "batched Fresnel MPO-MPS item-steps/s", "value": value, "unit": "item-steps/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "fp32" if r["prec"] == "fp32" else "bf16", "data": "synthetic",
                "config": {"workload": f"{args.items} interleaved wavefronts, Gaussian beam x Kolmogorov phase screen, "
                                       "n in 8..12, chi in {16,32,64}, one CUDA graph of all items launched once per "
                                       "step", "precision": r["prec"], "gemm_tiles_autotuned": r["tiles"],
                           "branches_autotuned": {"branches": r["branches"], "ms_per_step": r["branches_tuned_ms"]},
                           "eig_cluster_min": r["eig_cluster_min"],
                           "graph_build_s": r["build_s"],
                           "items": r["hist"], "cutoff": args.cutoff, "parallelism": f"replicas x{ws}",
                           "l2": "items stay L2-resident (no flush): the batch is one launch of one graph"},
                "clocks": r["clocks"], "gpu_launches": r["launches"], "e2e": None, "roofline": None}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "optics":
        r = run_optics(args, local, ws)
        value = args.items * args.steps * ws / (r["ms"] / 1e3)
        line = {"metric": "intensity-loss forward + mask gradient items/s", "value": value, "unit": "items/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "fp32",
                "data": "synthetic",
                "config": {"workload": f"{args.items} items per step: 4096x4096 interleaved field (n=12, chi=32, "
                                       "Gaussian beam x random rectangles), one smooth phase mask (chi=16) shared "
                                       "by the batch, rectangle targets; loss |I - I_t|^2 after one Fresnel step "
                                       "and its gradient with respect to the mask site tensors, summed over the "
                                       "items (all-reduced over the ranks)", "mask_bonds": r["mask_bonds"],
                           "cutoff": args.cutoff, "parallelism": f"items sharded x{ws}, mask gradient all-reduced", "launch": "eager, one engine, stream and host thread per item",
                           "l2": "states stay L2-resident (no flush)"},
                "clocks": r["clocks"], "gpu_launches": r["launches"], "e2e": None, "roofline": None}
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    arms = ["mixed", "fp32"] if args.prec == "both" else [args.prec]
    res = {p: run_ours(args, rank, ws, local, p) for p in arms}
    head = arms[0]
    r = res[head]
    steps_all = args.steps * ws
    value = steps_all / (r["total_ms"] / 1e3)
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["total_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32" if head == "fp32" else "bf16",
            "data": "synthetic", "config": config}
    line["config"]["precision"] = head if head == "fp32" else \
        "mixed: site contractions on tcgen05 tensor cores, BF16 operands split hi+lo (3 products), FP32 " \
        "accumulation; truncation SVD with FP64-accumulated Gram, FP32 rotations; FP64 bookkeeping"
    line["config"]["parallelism"] = f"replicas x{ws}"
    line["config"]["launch"] = "CUDA graph of one step (qtn_batch_create), replayed per step" if r["graph"] else \
        "eager (every kernel launched from the host)"
    line["config"]["mpo_bonds"] = {"qft": r["Qw"], "phase": r["Dw"]}
    line["config"]["state_bonds_initial"] = r["bonds0"]
    line["config"]["state_bonds_final"] = r["bonds"]
    line["clocks"] = r["clocks"]
    line["gpu_launches"] = r["launches"]
    line["e2e"] = None if r["e2e_ms"] is None else {
        "value": ws / (r["e2e_ms"] / 1e3), "unit": "steps/s", "h2d_bytes_per_step": r["h2d"],
        "d2h_bytes_per_step": r["h2d"]}
    if "fp32" in res and head != "fp32":
        p = res["fp32"]
        pv = steps_all / (p["total_ms"] / 1e3)
        from paper_2510_23089_gb300 import qtn
        import torch
        chk = qtn.Engine(n_sites=args.n, d=4, chi=args.chi, w=2, dense=0)
        a, b = r["final"], p["final"]
        d2 = chk.norm2(a) + chk.norm2(b) - 2 * chk.overlap(b, a).real
        line["fp32_plain"] = {
            "value": pv, "unit": "steps/s", "ms_per_step": p["total_ms"] / args.steps,
            "e2e": None if p["e2e_ms"] is None else {"value": ws / (p["e2e_ms"] / 1e3), "unit": "steps/s"},
            "state_bonds_final": p["bonds"], "clocks": p["clocks"], "gpu_launches": p["launches"],
            "roofline": roofline_line(p, json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                                      if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {},
                                      args.steps) if p["prof"] else None}
        line["mixed_over_plain"] = value / pv
        line["mixed_vs_plain_rel_l2"] = float(np.sqrt(max(d2, 0.0) / chk.norm2(b)))
        torch.cuda.synchronize()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    if r["prof"]:
        line["roofline"] = roofline_line(r, peaks, args.steps)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        try:
            line["cpu_baseline"] = cpu_baseline_line(args, 30.0)
        except Exception as ex:  # noqa: BLE001
            line["cpu_baseline"] = {"value": None, "unit": "steps/s", "kind": "oracle", "error": repr(ex)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
