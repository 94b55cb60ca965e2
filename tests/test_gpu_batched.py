"""GPU parity of the batched Fresnel steps (one CUDA graph per item, items on their own streams).

Items of mixed size (n in {5, 6}, chi in {16, 32}) built from Gaussian beams times Kolmogorov phase
screens, as in the batched workload at small sizes.  Every item advanced by the batch must agree with the
same item advanced by qtn_fresnel_step on its own (the same kernels; only the FP64 split-K accumulation
order may differ: 1e-5), and one item is checked against the FP64 oracle's truncated Fresnel step with the
tolerance of the single-item parity test."""
import numpy as np
import pytest
import torch

import synth
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS

pytestmark = pytest.mark.gpu

CL = 25.3   # lambda z / dx^2 of one step, as in the large workload


def dist(a, b):
    na, nb = OS.norm2(a), OS.norm2(b)
    ab = OS.overlap(a, b)
    return np.sqrt(max(na + nb - 2 * ab.real, 0.0) / nb)


def test_batched_steps_match_single_item_steps(lib):
    specs = synth.batched_item_specs(count=6, n_choices=(5, 6), chi_choices=(16, 32))
    enc = lib.Engine(n_sites=6, d=4, chi=32, w=16, dense=1 << 12)
    ops = {}
    for n in sorted({s["n"] for s in specs}):
        Q = enc.build_qft_mpo(n, False, 1e-12, w_cap=16)
        eng_p = lib.Engine(n_sites=n, d=2, chi=16, w=2, dense=1 << n)
        ops[n] = (Q, enc.mpo_dagger(Q), eng_p.build_phase_mpo(n, CL / (1 << n), 1e-12, w_cap=16))
    items, engines, refs = [], [], []
    for sp in specs:
        n, chi = sp["n"], sp["chi"]
        psi = lib.MPS(n, 4, chi)
        enc.encode(torch.from_numpy(synth.batched_item_field(sp)).cuda(), n, "interleaved", psi, chi, 1e-10,
                   stats=False)
        items.append(psi)
        refs.append(psi.clone())
        engines.append(lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=torch.cuda.Stream()))
    torch.cuda.synchronize()
    batch = lib.Batch(engines, items, [ops[s["n"]][0] for s in specs], [ops[s["n"]][1] for s in specs],
                      [ops[s["n"]][2] for s in specs], n_steps=1, chi_max=64, cutoff=1e-10)
    batch.launch(2)
    torch.cuda.synchronize()
    for sp, psi, ref in zip(specs, items, refs):
        Q, Qd, D = ops[sp["n"]]
        enc.fresnel_step(ref, "interleaved", Q, Qd, D, 2, sp["chi"], 1e-10, stats=False)
    torch.cuda.synchronize()
    for psi, ref in zip(items, refs):
        assert psi.canon == ref.canon
        a = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
        b = [A.astype(np.complex128) for A in ref.to_numpy_sites()]
        assert dist(a, b) < 1e-5
    batch.close()

    # one item against the oracle (two truncated steps from the same FP32 initial state)
    sp = specs[0]
    n, chi = sp["n"], sp["chi"]
    psi = lib.MPS(n, 4, chi)
    enc.encode(torch.from_numpy(synth.batched_item_field(sp)).cuda(), n, "interleaved", psi, chi, 1e-10, stats=False)
    sites = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
    c = CL / (1 << n)
    Qo = OM.qft_mpo_layers(n, 1e-12)
    ref, canon, disc = OF.fresnel_mps(sites, "interleaved", n, c, chi, 1e-10, canon=psi.canon, n_steps=2,
                                      ops=(Qo, OM.dagger(Qo), OM.phase_mpo(n, c, 1e-12)))
    eng = lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0, stream=torch.cuda.Stream())
    Q, Qd, D = ops[n]
    b2 = lib.Batch([eng], [psi], [Q], [Qd], [D], n_steps=2, chi_max=chi, cutoff=1e-10)
    b2.launch(1)
    torch.cuda.synchronize()
    got = [A.astype(np.complex128) for A in psi.to_numpy_sites()]
    n2 = OS.norm2(sites)
    assert dist(got, ref) < 1e-4 + 2.5 * np.sqrt(disc / n2) * 2
    b2.close()
