"""World-size-2 runs of bench.py's multi-process path on CPU (gloo), as the bench runs it under torchrun.

A single MPS does not shard, so N > 1 means N independent replicas: the only collectives are the barrier
around the timed region and the max over ranks of the timed seconds.  These tests exercise both with two
gloo ranks, and check that the reference arm under torchrun prints exactly one JSON line (rank 0)."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    # no GPU for these ranks, so the bench's helpers take the gloo backend on any machine
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": "2", "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, ws, local = bench.dist_init()
    bench.barrier(ws)
    m = bench.max_over_ranks(1.5 + r, ws)          # the slower rank's time wins
    bench.barrier(ws)
    dist.destroy_process_group()
    out.put((r, ws, local, m))


def test_barrier_and_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 2, 0, 2.5), (1, 2, 1, 2.5)]


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_line_has_the_contract_keys():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT,
                       env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["unit"] == "steps/s" and line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["cores"] >= 1 and line["config"]["workload"]


def _grad_worker(rank, port, parts, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": "2", "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2510_23089_gb300 import optics
    dist.init_process_group("gloo", rank=rank, world_size=2)
    g = torch.from_numpy(parts[rank].copy())
    optics.sum_over_ranks_(g)
    loss = torch.tensor([float(rank + 1)], dtype=torch.float64)
    optics.sum_over_ranks_(loss)
    dist.destroy_process_group()
    out.put((rank, g.numpy(), float(loss.item())))


def test_sharded_batch_mask_gradient_is_the_sum_over_items():
    # the mask-learning batch shards by item: four items' gradients of the intensity loss with respect to one
    # shared mask (FP64 dense oracle, 8 x 8 fields), two per rank; the all-reduce gives every rank the sum over
    # all four items
    import numpy as np
    import synth
    from oracle import optics as OO
    rng = np.random.default_rng(61)
    n, c = 3, 0.4
    M = np.exp(1j * rng.uniform(-1, 1, (8, 8)))
    grads = []
    for i in range(4):
        E = synth.gaussian_beam_with_rectangles(n, seed=6100 + i, waist=0.3).astype(np.complex128)
        It = (rng.uniform(0, 1, (8, 8)) > 0.5).astype(np.float64)
        grads.append(OO.intensity_loss_grad_dense(E, M, It, c).astype(np.complex64))
    parts = [grads[0] + grads[1], grads[2] + grads[3]]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_grad_worker, args=(r, port, parts, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = sum(grads)
    for rank, g, loss in got:
        assert np.abs(g - total).max() <= 1e-6 * np.abs(total).max()
        assert loss == 3.0
