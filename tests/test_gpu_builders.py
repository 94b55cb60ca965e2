"""GPU parity of the state builders (interleaved Kronecker product, direct sum)
and of the truncation sweep on non-canonical, rank-deficient inputs such as
direct sums, against the FP64 oracle, through the C ABI.

States are compared through FP64 overlaps (never densified):
    dist(a, b) = |a - b| / |b|.
Tolerances as in the other parity tests: 1e-5 + sqrt(eps_gpu) + sqrt(eps_orc)
for truncated results (eps = relative discarded weight)."""
import numpy as np
import pytest
import torch

import synth
from oracle import mps as OS

pytestmark = pytest.mark.gpu


def f64(psi):
    return [A.astype(np.complex128) for A in psi.to_numpy_sites()]


def dist(a, b):
    na, nb = OS.norm2(a), OS.norm2(b)
    ab = OS.overlap(a, b)
    return np.sqrt(max(na + nb - 2 * ab.real, 0.0) / nb)


@pytest.fixture(scope="module")
def eng_big(lib):
    # chi 192: m = 4 * 192 = 768 rows, the 16-column block Gram-Schmidt of the range finder
    return lib.Engine(n_sites=10, d=4, chi=192, w=2, dense=1 << 10)


def test_kron_interleave_matches_oracle(lib, eng_big):
    n = 10
    X = synth.random_mps_sites([1, 2, 4, 6, 7, 6, 5, 4, 3, 2, 1], 2, seed=401, decay=0.2)
    Y = synth.random_mps_sites([1, 2, 4, 5, 5, 5, 4, 4, 3, 2, 1], 2, seed=402, decay=0.2)
    gx, gy = lib.MPS.from_numpy_sites(X, 32, "none"), lib.MPS.from_numpy_sites(Y, 32, "none")
    out = lib.MPS(n, 4, 192)
    eng_big.kron_interleave(gx, gy, out)
    ref = OS.kron_interleave(X, Y)
    assert out.bonds() == OS.bonds(ref)
    assert dist(f64(out), ref) < 1e-6


def test_add_matches_direct_sum(lib, eng_big):
    a = synth.random_mps_sites([1, 4, 16, 30, 41, 30, 16, 9, 7, 4, 1], 4, seed=403, decay=0.05)
    b = synth.random_mps_sites([1, 4, 12, 25, 33, 40, 22, 11, 6, 3, 1], 4, seed=404, decay=0.05)
    ga, gb = lib.MPS.from_numpy_sites(a, 64, "none"), lib.MPS.from_numpy_sites(b, 64, "none")
    out = lib.MPS(10, 4, 192)
    eng_big.add(ga, gb, out)
    ref = OS.direct_sum(a, b)
    assert out.bonds() == OS.bonds(ref)
    assert dist(f64(out), ref) < 1e-6


def canonical_term(lib, eng, fx, gy, n, cap, cutoff):
    """f(x) g(y) as an interleaved MPS, right-canonical.  The FP32 sweeps over a direct sum stay accurate
    only when its parts are in the same canonical form: with a left-canonical part the unswept environment
    is not an isometry and amplifies the rounding of every factorisation (measured 1e-4 instead of 2e-5)."""
    X, Y = lib.MPS(n, 2, 32), lib.MPS(n, 2, 32)
    eng.encode(torch.from_numpy(fx.astype(np.complex64)).cuda(), n, "1d", X, 32, cutoff, stats=False)
    eng.encode(torch.from_numpy(gy.astype(np.complex64)).cuda(), n, "1d", Y, 32, cutoff, stats=False)
    term = lib.MPS(n, 4, cap)
    eng.kron_interleave(X, Y, term)
    eng.truncate(term, cap, 1e-13, stats=False)
    return term


def separable_sum(lib, eng, n, terms, cap):
    """GPU state sum_r f_r(x) g_r(y) from 1-D encodes, interleaving and direct sums (no truncation)."""
    fx, gy = synth.separable_phase_factors(n, rank=terms)
    acc = None
    for r in range(terms):
        term = canonical_term(lib, eng, fx[r], gy[r], n, cap, 1e-12)
        if acc is None:
            acc = term
        else:
            s = lib.MPS(n, 4, cap)
            eng.add(acc, term, s)
            acc = s
    return acc


@pytest.mark.parametrize("terms", [2, 3])
def test_exact_truncation_of_a_direct_sum_is_lossless(lib, eng_big, terms):
    # a sum of separable terms is rank-deficient at every bond; the exact sweeps must lose nothing
    psi = separable_sum(lib, eng_big, 10, terms, 192)
    ref = f64(psi)
    eng_big.truncate(psi, 192, 1e-13)
    assert dist(f64(psi), ref) < 2e-5
    assert psi.canon == "right"


def test_truncation_of_a_direct_sum_matches_oracle(lib, eng_big):
    psi = separable_sum(lib, eng_big, 10, 3, 192)
    sites = f64(psi)
    n2 = OS.norm2(sites)
    ref, eps = OS.truncate(sites, 48, 1e-10)
    st = eng_big.truncate(psi, 48, 1e-10)
    tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert dist(f64(psi), ref) < tol
    assert abs(st.discarded - sum(eps)) <= 1e-6 * sum(eps) + 1e-6 * n2


def test_sequential_sum_and_truncation_matches_oracle(lib, eng_big):
    # the recipe of the separable rank-8 input: add one interleaved term at a time and truncate (chi 128,
    # cutoff 1e-10); every stage is compared with the oracle's truncation of the same GPU sum
    n, terms = 10, 6
    fx, gy = synth.separable_phase_factors(n, rank=terms)
    acc = None
    for r in range(terms):
        term = canonical_term(lib, eng_big, fx[r], gy[r], n, 192, 1e-10)
        if acc is None:
            acc = term
            continue
        s = lib.MPS(n, 4, 192)
        eng_big.add(acc, term, s)
        sites = f64(s)
        n2 = OS.norm2(sites)
        ref, eps = OS.truncate(sites, 128, 1e-10)
        st = eng_big.truncate(s, 128, 1e-10)
        tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
        assert dist(f64(s), ref) < tol, r
        acc = s


@pytest.mark.parametrize("m,n,rank", [(272, 68, 68), (512, 100, 60), (768, 150, 150), (200, 40, 25)])
def test_tsvd_tall_rank_deficient(lib, eng_big, m, n, rank):
    # m > 160 rows (range finder) with fewer columns than the sketch width, exact rank below both
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, rank)) + 1j * rng.standard_normal((m, rank))
    B = rng.standard_normal((rank, n)) + 1j * rng.standard_normal((rank, n))
    s = np.exp(-0.05 * np.arange(rank))
    T = ((A * s[None, :]) @ B).astype(np.complex64)
    U, C, st = eng_big.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, 1e-12)
    U, C = U.cpu().numpy().astype(np.complex128), C.cpu().numpy().astype(np.complex128)
    T64 = T.astype(np.complex128)
    assert np.linalg.norm(U @ C - T64) / np.linalg.norm(T64) < 2e-6
    assert U.shape[1] <= rank + 2
