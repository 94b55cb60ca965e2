"""GPU parity of the batched Fresnel steps: all items of uneven n and chi advanced by one launch of one CUDA
graph (items split over parallel branches, longest first).

* Every item advanced by the batch agrees with the same item advanced by qtn_fresnel_step on its own (the
  same kernels; only the FP64 split-K accumulation order may differ: 1e-5), with items grouped several to a
  branch and GEMM tiles of both shapes.
* Items of the batched workload's sizes (n = 8, 10, 12 with chi = 16, 32, 64, Gaussian beams times Kolmogorov
  phase screens) against the FP64 oracle's step from the same initial state (built by the oracle and uploaded),
  in the FP32 and the mixed (tensor-core) precision, within 1e-5 and 3e-3 respectively on top of the truncation
  error, plus the status of the replays (qtn_batch_sync)."""
import numpy as np
import pytest
import torch

import synth
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS
from oracle import quantics as OQ

pytestmark = pytest.mark.gpu

CL = 25.3   # lambda z / dx^2 of one step, as in the large workload


def dist(a, b):
    na, nb = OS.norm2(a), OS.norm2(b)
    ab = OS.overlap(a, b)
    return np.sqrt(max(na + nb - 2 * ab.real, 0.0) / nb)


def gpu_ops(lib, eng, ns):
    ops = {}
    for n in ns:
        Q = eng.build_qft_mpo(n, False, 1e-12, w_cap=16)
        ops[n] = (Q, eng.mpo_dagger(Q), eng.build_phase_mpo(n, CL / (1 << n), 1e-12, w_cap=16))
    return ops


@pytest.mark.parametrize("tile", [64, 32])
def test_batched_steps_match_single_item_steps(lib, tile):
    specs = synth.batched_item_specs(count=6, n_choices=(5, 6), chi_choices=(16, 32))
    enc = lib.Engine(n_sites=6, d=4, chi=32, w=16, dense=1 << 12)
    ops = gpu_ops(lib, enc, sorted({s["n"] for s in specs}))
    items, engines, refs = [], [], []
    for sp in specs:
        n, chi = sp["n"], sp["chi"]
        psi = lib.MPS(n, 4, chi)
        enc.encode(torch.from_numpy(synth.batched_item_field(sp)).cuda(), n, "interleaved", psi, chi, 1e-10,
                   stats=False)
        items.append(psi)
        refs.append(psi.clone())
        e = lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=torch.cuda.Stream())
        e.set_gemm_tile(tile)
        engines.append(e)
    torch.cuda.synchronize()
    batch = lib.Batch(engines, items, [ops[s["n"]][0] for s in specs], [ops[s["n"]][1] for s in specs],
                      [ops[s["n"]][2] for s in specs], n_steps=1, chi_max=0, cutoff=1e-10, branches=2)
    batch.launch(2)
    batch.sync()
    for sp, ref in zip(specs, refs):
        Q, Qd, D = ops[sp["n"]]
        enc.fresnel_step(ref, "interleaved", Q, Qd, D, 2, sp["chi"], 1e-10, stats=False)
    torch.cuda.synchronize()
    for psi, ref in zip(items, refs):
        assert psi.canon == ref.canon
        a = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
        b = [A.astype(np.complex128) for A in ref.to_numpy_sites()]
        assert dist(a, b) < 1e-5
    batch.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("mixed", 3e-3)])
def test_workload_sized_items_match_oracle(lib, prec, tol):
    specs = [{"n": 8, "chi": 16, "r0": 0.1, "seed": 23100}, {"n": 10, "chi": 32, "r0": 0.07, "seed": 23101},
             {"n": 12, "chi": 64, "r0": 0.15, "seed": 23102}]
    enc = lib.Engine(n_sites=12, d=4, chi=64, w=16, dense=0)
    ops = gpu_ops(lib, enc, [s["n"] for s in specs])
    items, engines, sites0 = [], [], []
    for sp in specs:
        n, chi = sp["n"], sp["chi"]
        E = synth.batched_item_field(sp, dtype=np.complex128)
        sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, "interleaved"), n, 4, chi, 1e-10)
        sites0.append(sites)
        items.append(lib.MPS.from_numpy_sites(sites, chi, "left"))
        engines.append(lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=torch.cuda.Stream()))
    torch.cuda.synchronize()
    batch = lib.Batch(engines, items, [ops[s["n"]][0] for s in specs], [ops[s["n"]][1] for s in specs],
                      [ops[s["n"]][2] for s in specs], n_steps=1, chi_max=0, cutoff=1e-10, prec=prec, branches=3)
    batch.launch(1)
    batch.sync()
    for sp, psi, sites in zip(specs, items, sites0):
        n, chi = sp["n"], sp["chi"]
        c = CL / (1 << n)
        Qo = OM.qft_mpo_layers(n, 1e-12)
        ref, canon, disc = OF.fresnel_mps(sites, "interleaved", n, c, chi, 1e-10, canon="left", n_steps=1,
                                          ops=(Qo, OM.dagger(Qo), OM.phase_mpo(n, c, 1e-12)))
        got = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
        n2 = OS.norm2(sites)
        err = dist(got, ref)
        print(f"batched {prec} n={n} chi={chi}: rel {err:.2e}, oracle eps {disc / n2:.2e}, "
              f"bonds {psi.bonds()} vs {OS.bonds(ref)}")
        # the batch keeps no statistics: the GPU side's discarded weight is bounded by the oracle's plus the
        # distance of the two states
        assert err < tol + 2 * np.sqrt(disc / n2) + 1e-6
    batch.close()


def test_branch_tuner_and_shared_streams(lib, tmp_path):
    # items whose contexts share one stream (PyTorch's stream pool repeats after 32 streams); the tuner times
    # each branch count on copies, caches the choice, and the tuned batch (with range-path items, chi = 64,
    # whose two factorisation paths are conditional graph nodes) agrees with the single-item steps
    specs = [{"n": 6, "chi": 16, "r0": 0.1, "seed": 23110}, {"n": 7, "chi": 64, "r0": 0.07, "seed": 23111},
             {"n": 6, "chi": 32, "r0": 0.15, "seed": 23112}, {"n": 7, "chi": 64, "r0": 0.2, "seed": 23113}]
    enc = lib.Engine(n_sites=7, d=4, chi=64, w=16, dense=1 << 14)
    ops = gpu_ops(lib, enc, sorted({s["n"] for s in specs}))
    shared = torch.cuda.Stream()
    items, engines, refs = [], [], []
    for sp in specs:
        n, chi = sp["n"], sp["chi"]
        psi = lib.MPS(n, 4, chi)
        enc.encode(torch.from_numpy(synth.batched_item_field(sp)).cuda(), n, "interleaved", psi, chi, 1e-10,
                   stats=False)
        items.append(psi)
        refs.append(psi.clone())
        engines.append(lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=shared))
    torch.cuda.synchronize()
    Qs, Qds, Ds = ([ops[s["n"]][k] for s in specs] for k in range(3))
    cache = str(tmp_path / "tune.txt")
    copies = [it.clone() for it in items]
    br, ms = lib.tune_branches(engines, copies, Qs, Qds, Ds, 0, 1e-10, "fp32", [1, 2, 4], cache_path=cache)
    assert br in (1, 2, 4) and ms > 0
    br2, _ = lib.tune_branches(engines, copies, Qs, Qds, Ds, 0, 1e-10, "fp32", [1, 2, 4], cache_path=cache)
    assert br2 == br                                          # read back from the cache
    batch = lib.Batch(engines, items, Qs, Qds, Ds, n_steps=1, chi_max=0, cutoff=1e-10, branches=br)
    l0 = enc.launch_count()
    batch.launch(2)
    batch.sync()
    assert enc.launch_count() > l0
    for sp, ref in zip(specs, refs):
        Q, Qd, D = ops[sp["n"]]
        enc.fresnel_step(ref, "interleaved", Q, Qd, D, 2, sp["chi"], 1e-10, stats=False)
    torch.cuda.synchronize()
    for psi, ref in zip(items, refs):
        a = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
        b = [A.astype(np.complex128) for A in ref.to_numpy_sites()]
        assert dist(a, b) < 1e-5
    batch.close()
