"""Independent mask-gradient items driven from host threads give the results of a sequential run.

Each item has its own engine (context, stream, workspace); the library keeps process-wide host state (the
launch counter, the profiling pool, the per-device set-up), so the same items are run one after another on
one thread and concurrently on three threads, and every item's loss and mask gradient are compared.  The
split-K FP64 accumulation of the Gram matrices sums in a hardware-dependent order, so the two runs agree to
FP32 rounding, not bit for bit: loss within 1e-6 relative, gradient within 1e-5 relative."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def make_items(lib, optics, count, n=7, chi=32, chi_m=8, cutoff=1e-10):
    c = 25.3 / (1 << n)
    enc = lib.Engine(n_sites=n, d=4, chi=64, w=32, dense=1 << (2 * n))
    items = []
    for i in range(count):
        E = torch.from_numpy(synth.gaussian_beam_with_rectangles(n, seed=8101 + 3 * i, waist=0.15)).cuda()
        Em = lib.MPS(n, 4, chi)
        enc.encode(E, n, "interleaved", Em, chi, cutoff, stats=False)
        mx, my = synth.smooth_random_phase_mask_factors(n, seed=8102 + 3 * i, strength=0.5)
        X, Y = lib.MPS(n, 2, 8), lib.MPS(n, 2, 8)
        enc.encode(torch.from_numpy(mx.astype(np.complex64)).cuda(), n, "1d", X, 8, 1e-12, stats=False)
        enc.encode(torch.from_numpy(my.astype(np.complex64)).cuda(), n, "1d", Y, 8, 1e-12, stats=False)
        M = lib.MPS(n, 4, 64)
        enc.kron_interleave(X, Y, M)
        enc.truncate(M, chi_m, cutoff, stats=False)
        It = torch.from_numpy(synth.rectangles_target(n, seed=8103 + 3 * i).astype(np.complex64)).cuda()
        Itm = lib.MPS(n, 4, chi_m)
        enc.encode(It, n, "interleaved", Itm, chi_m, cutoff, stats=False)
        eng = lib.Engine(n_sites=n, d=4, chi=64, w=32, dense=0, stream=torch.cuda.Stream())
        prob = optics.IntensityLossProblem(eng, n, c, chi=chi, cutoff=cutoff, w_cap=16)
        items.append((eng, prob, Em, M, Itm))
    torch.cuda.synchronize()
    return items


def run_item(it):
    eng, prob, Em, M, Itm = it
    with torch.cuda.stream(eng.stream):
        loss, cache = prob.forward(Em.clone(), M, Itm)
        _, H = prob.backward(Em, M, cache)
        H = H.clone()
    eng.stream.synchronize()
    return loss, H.cpu().numpy()


def test_threaded_items_match_sequential_run(lib):
    from paper_2510_23089_gb300 import optics
    items = make_items(lib, optics, 3)
    seq = [run_item(it) for it in items]
    with ThreadPoolExecutor(max_workers=len(items)) as pool:
        par = list(pool.map(run_item, items))
    for (l0, h0), (l1, h1) in zip(seq, par):
        assert abs(l1 - l0) <= 1e-6 * abs(l0)
        assert np.linalg.norm(h1 - h0) <= 1e-5 * np.linalg.norm(h0)


def test_batch_loss_and_gradient_is_the_sum_over_items(lib):
    # one mask for a batch of fields and targets: the batch loss and its mask gradient are the sums of the
    # items' (a single process: the all-reduce over ranks is the identity)
    from paper_2510_23089_gb300 import optics
    items = make_items(lib, optics, 3)
    eng, prob, _, M, _ = items[0]
    fields, targets = [it[2] for it in items], [it[4] for it in items]
    loss, H = optics.batch_loss_and_gradient(prob, fields, targets, M)
    ref_loss, ref_H = 0.0, None
    with torch.cuda.stream(eng.stream):
        for E, It in zip(fields, targets):
            val, cache = prob.forward(E, M, It)
            _, h = prob.backward(E, M, cache)
            ref_loss += val
            ref_H = h.clone() if ref_H is None else ref_H + h
    eng.stream.synchronize()
    H, ref_H = H.cpu().numpy(), ref_H.cpu().numpy()
    assert abs(loss - ref_loss) <= 1e-6 * abs(ref_loss)
    assert np.linalg.norm(H - ref_H) <= 1e-5 * np.linalg.norm(ref_H)
