"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (FP32 path): relative L2 of dense results within
    1e-5 + sqrt(eps_gpu) + sqrt(eps_orc)
with eps the relative discarded weights each side reports (a truncated result
differs from the exact one by at most the square root of what it discarded,
so two independent truncations differ by at most the sum); untruncated
results within 1e-5; relative discarded weights (discarded / |psi|^2, the
quantity the cutoff rule bounds) within 1e-6 of the oracle's.
Inputs are seeded; sizes span several 64-wide tiles and ragged bonds."""
import numpy as np
import pytest
import torch

import synth
from oracle import apply as OA
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS
from oracle import quantics as OQ

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def eng(lib):
    # states up to 16 sites with chi 64 (m = 256 > 160 exercises the range finder), dense up to 4^8
    return lib.Engine(n_sites=16, d=4, chi=64, w=32, dense=1 << 16)


@pytest.fixture(scope="module")
def eng_small(lib):
    # chi 32: m = 128 <= 160, every factorisation takes the shared-memory Jacobi path
    return lib.Engine(n_sites=16, d=4, chi=32, w=16, dense=1 << 16)


# ----------------------------------------------------------------------------- encode (TT-SVD)

def test_encode_of_smooth_factors_matches_oracle(lib):
    # 1-D encodes of the smooth phase factors of the 2^16 workload (fast-decaying spectra, most eigenvalues
    # at the rounding level of the Gram): bonds and relative discarded weight of the oracle's TT-SVD
    n = 16
    fx, gy = synth.separable_phase_factors(n)
    e = lib.Engine(n_sites=n, d=2, chi=32, w=2, dense=1 << n)
    for v in (fx[0], fx[1], gy[0], gy[1]):
        X = lib.MPS(n, 2, 32)
        st = e.encode(torch.from_numpy(v.astype(np.complex64)).cuda(), n, "1d", X, 32, 1e-10)
        v64 = v.astype(np.complex128)
        n2 = float(np.vdot(v64, v64).real)
        ref, eps = OS.tt_svd(OQ.dense_to_quantics(v64, "1d"), n, 2, 32, 1e-10)
        assert max(abs(a - b) for a, b in zip(X.bonds(), OS.bonds(ref))) <= 1, (X.bonds(), OS.bonds(ref))
        assert abs(st.discarded - sum(eps)) / n2 <= 1e-6 * sum(eps) / n2 + 1e-9
        got = [A.astype(np.complex128) for A in X.to_numpy_sites()]
        tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
        d2 = OS.norm2(got) + OS.norm2(ref) - 2 * OS.overlap(got, ref).real
        assert np.sqrt(max(d2, 0.0) / OS.norm2(ref)) < tol


@pytest.mark.parametrize("layout,n", [("interleaved", 4), ("serial", 4), ("1d", 10), ("interleaved", 6)])
def test_encode_untruncated_reconstructs(eng, lib, layout, n):
    E = synth.gaussian_beam_with_rectangles(n, seed=200 + n, waist=0.2) if layout != "1d" else \
        (np.random.default_rng(5).standard_normal(1 << n) + 1j * np.random.default_rng(6).standard_normal(1 << n)).astype(np.complex64)
    N, d = OQ.n_sites(n, layout), OQ.phys_dim(layout)
    psi = lib.MPS(N, d, 64)
    st = eng.encode(torch.from_numpy(E).cuda(), n, layout, psi, 64, 1e-12)
    got = eng.to_dense(psi, layout, n).cpu().numpy()
    assert rel(got, E) < 1e-5
    assert psi.canon == "left"
    # left isometries
    for A in psi.to_numpy_sites()[:-1]:
        a, dd, b = A.shape
        M = A.reshape(a * dd, b)
        assert np.abs(M.conj().T @ M - np.eye(b)).max() < 1e-5
    assert abs(st.norm2 - np.linalg.norm(E.astype(np.complex128)) ** 2) < 1e-5 * np.linalg.norm(E) ** 2


@pytest.mark.parametrize("chi", [4, 9, 16])
def test_encode_truncated_matches_oracle(eng, lib, chi):
    n = 5
    E = synth.gaussian_beam_with_rectangles(n, seed=210, waist=0.25)
    psi = lib.MPS(n, 4, 64)
    st = eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, chi, 1e-10)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    sites, eps = OS.tt_svd(OQ.dense_to_quantics(E.astype(np.complex128), "interleaved"), n, 4, chi, 1e-10)
    ref = OQ.quantics_to_dense(OS.to_vector(sites), n, "interleaved")
    n2 = np.linalg.norm(E.astype(np.complex128)) ** 2
    tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert rel(got, ref) < tol
    assert psi.bonds() == OS.bonds(sites)
    assert abs(st.discarded - sum(eps)) <= 1e-6 * n2
    # exact error bookkeeping: ||E - E~||^2 = discarded
    assert abs(np.linalg.norm(got - E) ** 2 - st.discarded) <= 2e-6 * n2


# ----------------------------------------------------------------------------- MPO builders

@pytest.mark.parametrize("n", [4, 6, 9])
def test_qft_mpo_matches_bit_reversed_dft(eng, n):
    Q = eng.build_qft_mpo(n, False, 1e-14)
    dense = OM.to_dense(Q.to_numpy_cores())
    ref = OM.qft_noswap_dense(n)
    # operator error relative to the unitary's Frobenius norm, and entrywise
    assert np.linalg.norm(dense - ref) / np.linalg.norm(ref) < 1e-5
    assert np.abs(dense - ref).max() < 1e-5 * np.abs(ref).max()
    assert Q.w_max <= max(OM.bonds(OM.qft_mpo_layers(n, 1e-14)))
    Qi = eng.build_qft_mpo(n, True, 1e-14)
    assert np.linalg.norm(OM.to_dense(Qi.to_numpy_cores()) - ref.conj().T) / np.linalg.norm(ref) < 1e-5


@pytest.mark.parametrize("n,c", [(6, 0.37), (10, 2.048), (12, 25.3 / 4096)])
def test_phase_mpo_matches_transfer_function(eng, n, c):
    D = eng.build_phase_mpo(n, c, 1e-14, w_cap=64)
    cores = D.to_numpy_cores()
    vec = OS.to_vector([np.stack([cc[:, 0, 0, :], cc[:, 1, 1, :]], axis=1) for cc in cores])
    ref = OM.phase_vector(n, c, True)
    assert np.abs(vec - ref).max() < 1e-5
    assert np.linalg.norm(vec - ref) / np.linalg.norm(ref) < 1e-5
    for cc in cores:
        assert np.abs(cc[:, 0, 1, :]).max() == 0 and np.abs(cc[:, 1, 0, :]).max() == 0


# ----------------------------------------------------------------------------- zip-up

@pytest.mark.parametrize("layout,axis", [("interleaved", 0), ("interleaved", 1), ("serial", 1), ("1d", 0)])
@pytest.mark.parametrize("canon", ["right", "left"])
@pytest.mark.parametrize("which", ["small", "range"])
def test_untruncated_apply_equals_exact_product(eng, eng_small, lib, layout, axis, canon, which):
    cap = 32 if which == "small" else 64
    eng = eng_small if which == "small" else eng
    n = 5
    N, d = OQ.n_sites(n, layout), OQ.phys_dim(layout)
    # exact product bonds stay below the capacity: rank of every unfolding <= d * bond * w <= cap
    bmax = 4 if which == "small" else 8
    bonds = [min(d ** k, d ** (N - k), bmax) for k in range(N + 1)]
    sites = synth.random_mps_sites(bonds, d, seed=300 + axis)
    sites = OS.right_canonicalize(sites) if canon == "right" else OS.left_canonicalize(sites)
    Qo = OM.qft_mpo_layers(n, 1e-14)
    Wfull = OM.embed(Qo, layout, axis, n)
    ref = OM.to_dense(Wfull) @ OS.to_vector(sites)
    psi = lib.MPS.from_numpy_sites(sites, cap, canon)
    W = lib.MPO.from_numpy_cores(Qo, 16)
    eng.apply_mpo(W, axis, psi, cap, 1e-12)
    got = OS.to_vector(psi.to_numpy_sites())
    assert rel(got, ref) < 1e-5
    assert psi.canon == ("left" if canon == "right" else "right")


@pytest.mark.parametrize("chi", [6, 20])
@pytest.mark.parametrize("which", ["small", "range"])
def test_truncated_zipup_matches_oracle_zipup(eng, eng_small, lib, chi, which):
    cap = 32 if which == "small" else 64
    eng = eng_small if which == "small" else eng
    n = 5
    bonds = [1, 4, 16, 16, 4, 1]
    sites = OS.right_canonicalize(synth.random_mps_sites(bonds, 4, seed=310, decay=0.08))
    Qo = OM.qft_mpo_layers(n, 1e-14)
    Wx = OM.embed(Qo, "interleaved", 0, n)
    ref_sites, eps = OA.zipup(Wx, sites, chi, 1e-12, "lr")
    psi = lib.MPS.from_numpy_sites(sites, cap, "right")
    st = eng.apply_mpo(lib.MPO.from_numpy_cores(Qo, 16), 0, psi, chi, 1e-12)
    got = OS.to_vector(psi.to_numpy_sites())
    ref = OS.to_vector(ref_sites)
    n2 = OS.norm2(sites)
    tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert rel(got, ref) < tol
    assert abs(st.discarded - sum(eps)) <= 1e-6 * n2
    assert psi.bonds() == OS.bonds(ref_sites)


def test_range_finder_path_matches_oracle(eng, lib):
    # m = 4 * 64 = 256 rows > 160: the randomised range finder + Rayleigh-Ritz path
    n = 6
    bonds = [1, 4, 16, 64, 16, 4, 1]
    sites = OS.right_canonicalize(synth.random_mps_sites(bonds, 4, seed=320, decay=0.06))
    Qo = OM.qft_mpo_layers(n, 1e-14)
    Wx = OM.embed(Qo, "interleaved", 0, n)
    chi = 40
    ref_sites, eps = OA.zipup(Wx, sites, chi, 0.0, "lr")
    psi = lib.MPS.from_numpy_sites(sites, 64, "right")
    st = eng.apply_mpo(lib.MPO.from_numpy_cores(Qo, 16), 0, psi, chi, 0.0)
    got = OS.to_vector(psi.to_numpy_sites())
    n2 = OS.norm2(sites)
    tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert rel(got, OS.to_vector(ref_sites)) < tol
    assert abs(st.discarded - sum(eps)) <= 1e-6 * n2


# ----------------------------------------------------------------------------- truncate

def test_truncate_is_eckart_young_and_matches_oracle(eng, lib):
    bonds = [1, 4, 16, 48, 16, 4, 1]
    sites = synth.random_mps_sites(bonds, 4, seed=330, decay=0.1)
    ref_sites, eps = OS.truncate(sites, 10, 0.0)
    psi = lib.MPS.from_numpy_sites(sites, 64, "none")
    st = eng.truncate(psi, 10, 0.0)
    got = OS.to_vector(psi.to_numpy_sites())
    v = OS.to_vector(sites)
    n2 = np.linalg.norm(v) ** 2
    assert rel(got, OS.to_vector(ref_sites)) < 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert abs(st.discarded - sum(eps)) <= 1e-6 * n2
    assert abs(np.linalg.norm(got - v) ** 2 - st.discarded) <= 1e-5 * n2
    assert psi.canon == "right"


# ----------------------------------------------------------------------------- Fresnel step

@pytest.mark.parametrize("layout", ["interleaved", "serial"])
def test_fresnel_step_untruncated_equals_dense(eng, lib, layout):
    n, c = 5, 0.3
    E = synth.gaussian_beam_with_rectangles(n, seed=340, waist=0.2)
    N, d = OQ.n_sites(n, layout), OQ.phys_dim(layout)
    psi = lib.MPS(N, d, 64)
    eng.encode(torch.from_numpy(E).cuda(), n, layout, psi, 64, 1e-12)
    Q = eng.build_qft_mpo(n, False, 1e-14)
    Qd = eng.mpo_dagger(Q)
    D = eng.build_phase_mpo(n, c, 1e-14, w_cap=32)
    st = eng.fresnel_step(psi, layout, Q, Qd, D, 1, 64, 1e-12)
    got = eng.to_dense(psi, layout, n).cpu().numpy()
    ref = OF.fresnel_dense(E.astype(np.complex128), c)
    assert rel(got, ref) < 1e-5
    assert abs(st.norm2 / np.linalg.norm(E.astype(np.complex128)) ** 2 - 1) < 1e-5


def test_fresnel_step_truncated_matches_oracle(eng, lib):
    n, c, chi = 5, 0.3, 12
    E = synth.gaussian_beam_with_rectangles(n, seed=350, waist=0.2)
    psi = lib.MPS(n, 4, 64)
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 64, 1e-12)
    Q = eng.build_qft_mpo(n, False, 1e-14)
    Qd = eng.mpo_dagger(Q)
    D = eng.build_phase_mpo(n, c, 1e-14, w_cap=32)
    st = eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, chi, 0.0)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    sites, _ = OS.tt_svd(OQ.dense_to_quantics(E.astype(np.complex128), "interleaved"), n, 4, 64, 1e-12)
    ops = OF.step_operators(n, c, qft=OM.qft_mpo_layers(n, 1e-14), phase_cutoff=1e-14)
    out, canon, disc = OF.fresnel_mps(sites, "interleaved", n, c, chi, 0.0, canon="left", ops=ops)
    ref = OQ.quantics_to_dense(OS.to_vector(out), n, "interleaved")
    n2 = np.linalg.norm(E.astype(np.complex128)) ** 2
    tol = 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(disc / n2)
    assert rel(got, ref) < tol
    assert abs(st.discarded - disc) <= 1e-6 * n2
