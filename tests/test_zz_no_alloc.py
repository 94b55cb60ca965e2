"""qtn_tsvd_noalloc (truncated SVD on the library's fixed scratch array) against
qtn_tsvd (caller workspace), called through the C ABI.

The calls come in a row on one device, so the later ones run on whatever the
earlier ones left in the shared array; each result must still match the
workspace entry point within the tolerances of the qtn_tsvd tests.  Shapes
cover the shared-memory eigensolver path (m <= 160) and the range-finder path
(m > 160).  This file is collected last and also runs alone."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def make(m, n, decay, seed):
    rng = np.random.default_rng(seed)
    T = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) * np.exp(-decay * np.arange(n))[None, :]
    return T.astype(np.complex64)


def tsvd_noalloc(qtn, T, chi_max, cutoff, k_cap):
    lib = qtn.load_library()
    m, n = T.shape
    U = torch.zeros((m, k_cap), dtype=torch.complex64, device="cuda")
    C = torch.zeros((k_cap, n), dtype=torch.complex64, device="cuda")
    k = ctypes.c_int()
    st = qtn.c_stats()
    tr = qtn.c_trunc(chi_max, cutoff, 0, 0)
    code = lib.qtn_tsvd_noalloc(ctypes.c_void_p(T.data_ptr()), m, n, tr, ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(C.data_ptr()), k_cap, ctypes.byref(k), ctypes.byref(st),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, U[:, :k.value], C[:k.value], st


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=4, d=4, chi=64, w=8, dense=0)


# (m, n, decay, chi_max): range-finder path, shared-memory path, then the first case again
CASES = [(200, 300, 0.05, 64), (64, 96, 0.1, 20), (200, 300, 0.05, 64)]


def test_noalloc_matches_workspace_entry_point(lib, eng):
    for i, (m, n, decay, chi) in enumerate(CASES):
        Th = make(m, n, decay, seed=5 * m + n)
        T = torch.from_numpy(Th).cuda()
        code, U1, C1, st1 = tsvd_noalloc(lib, T, chi, 0.0, min(m, n))
        assert code == 0, lib.STATUS.get(code, code)
        U0, C0, st0 = eng.tsvd(T, chi, 0.0)
        torch.cuda.synchronize()
        U1, C1 = U1.cpu().numpy().astype(np.complex128), C1.cpu().numpy().astype(np.complex128)
        U0, C0 = U0.cpu().numpy().astype(np.complex128), C0.cpu().numpy().astype(np.complex128)
        T64 = Th.astype(np.complex128)
        n2 = float(np.linalg.norm(T64) ** 2)
        assert U1.shape == U0.shape == (m, chi), (i, U1.shape, U0.shape)
        # same factorisation: reconstructions, kept singular values and discarded weight agree
        assert np.linalg.norm(U1 @ C1 - U0 @ C0) / np.sqrt(n2) < 2e-6, i
        s1 = np.sort(np.linalg.norm(C1, axis=1))
        s0 = np.sort(np.linalg.norm(C0, axis=1))
        assert np.abs(s1 - s0).max() <= 2e-6 * s0.max(), i
        assert abs(st1.discarded - st0.discarded) <= 1e-6 * st0.discarded + 1e-7 * n2, i
        assert np.abs(U1.conj().T @ U1 - np.eye(chi)).max() < 2e-6, i
        # and both against the optimum of LAPACK's FP64 SVD (Eckart-Young)
        s = np.linalg.svd(T64, compute_uv=False)
        exact = float((s[chi:] ** 2).sum())
        assert abs(st1.discarded - exact) <= 1e-6 * n2, i
        assert abs(np.linalg.norm(U1 @ C1 - T64) ** 2 - exact) <= 1e-5 * n2, i


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    T = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    U = torch.zeros((8, 8), dtype=torch.complex64, device="cuda")
    lib_ = lib.load_library()
    k = ctypes.c_int()
    tr = lib.c_trunc(8, 0.0, 0, 0)
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ctypes.c_void_p(T.data_ptr())
    q = ctypes.c_void_p(U.data_ptr())
    # sizes are checked on the host before any device work, so the small buffers are never touched
    assert lib_.qtn_tsvd_noalloc(p, 257, 8, tr, q, q, 8, ctypes.byref(k), None, s) == 3      # QTN_ERR_CAPACITY
    assert lib_.qtn_tsvd_noalloc(p, 8, 2049, tr, q, q, 8, ctypes.byref(k), None, s) == 3
    assert lib_.qtn_tsvd_noalloc(p, 0, 8, tr, q, q, 8, ctypes.byref(k), None, s) == 1        # QTN_ERR_ARG
