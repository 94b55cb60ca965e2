"""Failure paths of the C ABI on the GPU, made on the host side: a solve capped at one sweep, a NaN in the
input field, a truncation rule that asks for more directions than the state can hold, and a batch item in
no canonical form.  Each returns the status the header promises, both from a call that fills statistics
and through the sticky status word read by qtn_check.  Nothing here faults, traps or waits without bound:
every device loop is bounded by its sweep limit or its size."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=8, d=4, chi=64, w=16, dense=1 << 16)


def make(m, n, seed):
    rng = np.random.default_rng(seed)
    T = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) * np.exp(-0.05 * np.arange(n))[None, :]
    return torch.from_numpy(T.astype(np.complex64)).cuda()


def test_one_sweep_cap_reports_no_convergence(eng, lib):
    eng.check()
    with pytest.raises(lib.QtnError) as ei:
        U = torch.zeros((96, 96), dtype=torch.complex64, device="cuda")
        C = torch.zeros((96, 128), dtype=torch.complex64, device="cuda")
        k = ctypes.c_int()
        st = lib.c_stats()
        T = make(96, 128, 1)
        code = eng.lib.qtn_tsvd(eng.ctx, ctypes.c_void_p(T.data_ptr()), 96, 128, lib.Engine.trunc(96, 0.0, "fp32", 1),
                                ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(C.data_ptr()), 96, ctypes.byref(k),
                                ctypes.byref(st), *eng._ws())
        assert st.flags & 1
        lib._check(code, "qtn_tsvd")
    assert ei.value.code == 4                                       # QTN_ERR_NOCONV
    with pytest.raises(lib.QtnError) as ei:                         # the sticky word saw it too
        eng.check()
    assert ei.value.code == 4
    eng.check()                                                      # and was cleared


def test_nan_input_reports_nonfinite(eng, lib):
    n = 4
    E = synth.gaussian_beam_with_rectangles(n, seed=3, waist=0.3)
    E[3, 5] = np.nan
    psi = lib.MPS(n, 4, 64)
    with pytest.raises(lib.QtnError) as ei:
        eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 64, 1e-12)
    assert ei.value.code == 5                                       # QTN_ERR_NONFINITE
    with pytest.raises(lib.QtnError):
        eng.check()
    # asynchronous call (no statistics): only the sticky word reports it
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 64, 1e-12, stats=False)
    with pytest.raises(lib.QtnError) as ei:
        eng.check()
    assert ei.value.code == 5
    eng.check()


def test_rank_above_capacity_reports_capacity(eng, lib):
    # a random 4-site d = 4 state has Schmidt rank 16 at the middle bond; a capacity of 8 cannot hold it
    n = 4
    rng = np.random.default_rng(9)
    E = (rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))).astype(np.complex64)
    psi = lib.MPS(n, 4, 8)
    with pytest.raises(lib.QtnError) as ei:
        eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 1000, 0.0)
    assert ei.value.code == 3                                       # QTN_ERR_CAPACITY
    assert max(psi.bonds()) == 8                                    # clamped, not overflowed
    with pytest.raises(lib.QtnError):
        eng.check()
    # chi_max equal to the capacity is a request, not an overflow
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 8, 0.0)
    eng.check()


def test_batch_rejects_an_item_in_no_canonical_form(eng, lib):
    n = 4
    psi = lib.MPS(n, 4, 16)
    psi.c.canon = 0
    e2 = lib.Engine(n_sites=n, d=4, chi=16, w=16, dense=0, stream=torch.cuda.Stream())
    Q = eng.build_qft_mpo(n, False, 1e-12)
    Qd = eng.mpo_dagger(Q)
    D = eng.build_phase_mpo(n, 0.3, 1e-12, w_cap=16)
    with pytest.raises(lib.QtnError) as ei:
        lib.Batch([e2], [psi], [Q], [Qd], [D], n_steps=1, chi_max=16, cutoff=1e-10)
    assert ei.value.code == 1                                       # QTN_ERR_ARG


def test_unknown_precision_is_rejected(eng, lib):
    psi = lib.MPS.from_numpy_sites(synth.random_mps_sites([1, 2, 4, 2, 1], 4, seed=77), 8)
    tr = lib.c_trunc(8, 1e-10, 7, 0)                                 # neither QTN_PLAIN_FP32 nor QTN_MIXED
    code = eng.lib.qtn_truncate(eng.ctx, ctypes.byref(psi.c), tr, None, *eng._ws())
    assert code == 1                                                 # QTN_ERR_ARG
