"""qtn_amplitudes, qtn_overlap and qtn_norm2 (Sec. III decompression: one amplitude is a product of site
matrices, O(N chi^2); an overlap is a chain of transfer matrices, O(N d chi^3)) against the FP64 oracle on
seeded states whose bonds span several warps and a ragged tail."""
import numpy as np
import pytest
import torch

import synth
from oracle import mps as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=12, d=4, chi=64, w=8, dense=1 << 16)


@pytest.mark.parametrize("d,bonds", [(4, [1, 4, 16, 45, 33, 16, 4, 1]), (2, [1, 2, 4, 8, 16, 8, 4, 2, 1])])
def test_amplitudes_match_oracle(eng, lib, d, bonds):
    sites = synth.random_mps_sites(bonds, d, seed=41 + d)
    psi = lib.MPS.from_numpy_sites(sites, 64)
    ref_sites = psi.to_numpy_sites()                      # the complex64 values the GPU holds
    rng = np.random.default_rng(7)
    N = len(sites)
    digits = rng.integers(0, d, size=(300, N))
    got = eng.amplitudes(psi, torch.from_numpy(digits.astype(np.int32))).cpu().numpy()
    ref = np.array([OS.amplitude(ref_sites, list(dg)) for dg in digits])
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * scale
    # empty request: nothing launched, nothing written
    assert eng.amplitudes(psi, torch.zeros((0, N), dtype=torch.int32)).numel() == 0


def test_overlap_and_norm_match_oracle(eng, lib):
    a = synth.random_mps_sites([1, 4, 16, 37, 16, 4, 1], 4, seed=51)
    b = synth.random_mps_sites([1, 4, 11, 29, 13, 4, 1], 4, seed=52)
    A = lib.MPS.from_numpy_sites(a, 64)
    B = lib.MPS.from_numpy_sites(b, 64)
    a32, b32 = A.to_numpy_sites(), B.to_numpy_sites()
    ref = OS.overlap(a32, b32)
    got = eng.overlap(A, B)
    assert abs(got - ref) <= 1e-10 * np.sqrt(OS.norm2(a32) * OS.norm2(b32))     # FP64 accumulation
    assert abs(eng.norm2(A) - OS.norm2(a32)) <= 1e-10 * OS.norm2(a32)
    # <a|b> = conj(<b|a>)
    assert abs(eng.overlap(B, A) - np.conj(got)) <= 1e-10 * abs(ref) + 1e-12
