"""GPU parity of the single-matrix truncated SVD (qtn_tsvd) against LAPACK in FP64.

The factorisation is the building block of every truncation (Sec. IV, App. A).
Checked: reconstruction |T - U C| against the exact Eckart-Young error, the
isometry of U, the rank rule, and the discarded weight, on seeded matrices
whose spectra decay at controlled rates; shapes cover the shared-memory
eigensolver path (m <= 160) and the range-finder path (m > 160)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def make(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    T = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) * np.exp(-decay * np.arange(n))[None, :]
    return T.astype(np.complex64)


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=4, d=4, chi=128, w=8, dense=0)


@pytest.mark.parametrize("m,n,decay", [(4, 4, 0.0), (16, 33, 0.0), (48, 48, 0.3), (64, 96, 0.1), (128, 256, 0.05),
                                       (160, 200, 0.05), (37, 300, 0.0)])
def test_untruncated_reconstruction(eng, m, n, decay):
    T = make(m, n, decay, seed=m + n)
    U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, 1e-12)
    U, C = U.cpu().numpy().astype(np.complex128), C.cpu().numpy().astype(np.complex128)
    T64 = T.astype(np.complex128)
    assert np.linalg.norm(U @ C - T64) / np.linalg.norm(T64) < 2e-6
    assert np.abs(U.conj().T @ U - np.eye(U.shape[1])).max() < 2e-6
    assert np.abs(C - U.conj().T @ T64).max() < 2e-6 * np.linalg.norm(T64)


@pytest.mark.parametrize("m,n,decay,chi", [(64, 96, 0.1, 20), (128, 256, 0.05, 40), (96, 200, 0.02, 64),
                                           (256, 384, 0.05, 64), (512, 768, 0.02, 128),
                                           (300, 260, 0.05, 40)])   # range finder of 72 columns: partial last block
def test_truncated_matches_eckart_young(eng, m, n, decay, chi):
    T = make(m, n, decay, seed=7 * m + n)
    U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), chi, 0.0)
    U, C = U.cpu().numpy().astype(np.complex128), C.cpu().numpy().astype(np.complex128)
    T64 = T.astype(np.complex128)
    s = np.linalg.svd(T64, compute_uv=False)
    exact = float((s[chi:] ** 2).sum())
    n2 = float((s ** 2).sum())
    assert U.shape[1] == chi
    err2 = np.linalg.norm(U @ C - T64) ** 2
    assert abs(err2 - st.discarded) <= 1e-5 * n2                  # reported weight is the actual error
    assert np.abs(U.conj().T @ U - np.eye(chi)).max() < 2e-6
    # optimality: the relative discarded weight within 1e-6 of the Eckart-Young optimum
    assert abs(st.discarded - exact) <= 1e-6 * n2


@pytest.mark.parametrize("cutoff", [1e-1, 1e-2, 1e-4])
def test_cutoff_rule(eng, cutoff):
    T = make(64, 80, 0.08, seed=3)
    U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, cutoff)
    s = np.linalg.svd(T.astype(np.complex128), compute_uv=False)
    w = s ** 2
    k = 1
    while k < len(w) and w[k:].sum() > cutoff * w.sum():
        k += 1
    assert U.shape[1] == k


def test_rank_deficient_and_zero(eng):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((40, 5)) + 1j * rng.standard_normal((40, 5))
    B = rng.standard_normal((5, 70)) + 1j * rng.standard_normal((5, 70))
    T = (A @ B).astype(np.complex64)
    U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, 0.0)
    assert U.shape[1] == 5
    # a rank-deficient matrix on the range-finder path: the sketch keeps its five live columns
    A = rng.standard_normal((300, 5)) + 1j * rng.standard_normal((300, 5))
    B = rng.standard_normal((5, 420)) + 1j * rng.standard_normal((5, 420))
    T = (A @ B).astype(np.complex64)
    U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, 0.0)
    U, C = U.cpu().numpy().astype(np.complex128), C.cpu().numpy().astype(np.complex128)
    T64 = T.astype(np.complex128)
    assert U.shape[1] == 5
    assert np.linalg.norm(U @ C - T64) / np.linalg.norm(T64) < 2e-6
    assert np.abs(U.conj().T @ U - np.eye(5)).max() < 2e-6
    Z = np.zeros((12, 9), np.complex64)
    U, C, st = eng.tsvd(torch.from_numpy(Z).cuda(), 10 ** 6, 0.0)
    assert U.shape[1] == 1 and st.discarded == 0.0


@pytest.mark.parametrize("cluster_min", [2, 161])   # every order on the cluster solver / on the single CTA
@pytest.mark.parametrize("m,n,decay,chi", [(12, 40, 0.1, 8), (33, 70, 0.0, 20), (48, 48, 0.3, 30),
                                           (128, 256, 0.05, 40), (160, 200, 0.05, 64), (512, 768, 0.02, 128)])
def test_both_eigen_solvers_meet_eckart_young(eng, cluster_min, m, n, decay, chi):
    T = make(m, n, decay, seed=11 * m + n)
    T64 = T.astype(np.complex128)
    s = np.linalg.svd(T64, compute_uv=False)
    n2 = float((s ** 2).sum())
    eng.set_eig_cluster_min(cluster_min)
    try:
        U, C, st = eng.tsvd(torch.from_numpy(T).cuda(), chi, 0.0)
        Uf, Cf, stf = eng.tsvd(torch.from_numpy(T).cuda(), 10 ** 6, 1e-12)
    finally:
        eng.set_eig_cluster_min(32)
    U, C = U.cpu().numpy().astype(np.complex128), C.cpu().numpy().astype(np.complex128)
    assert U.shape[1] == chi
    assert np.abs(U.conj().T @ U - np.eye(chi)).max() < 2e-6
    assert abs(np.linalg.norm(U @ C - T64) ** 2 - st.discarded) <= 1e-5 * n2
    assert abs(st.discarded - float((s[chi:] ** 2).sum())) <= 1e-6 * n2
    if min(m, n) <= 160:   # beyond, the range finder keeps a 160-dimensional subspace
        Uf, Cf = Uf.cpu().numpy().astype(np.complex128), Cf.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(Uf @ Cf - T64) / np.linalg.norm(T64) < 2e-6
