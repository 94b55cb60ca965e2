"""GPU parity of the FP64-built operators against the oracle: the lattice-dispersion propagator
U(t) = diag(exp(-i t cos(2 pi k / L))) as the closed-form Bessel MPO (Sec. VI.B.4) and as the Pauli-Z
circuit (Sec. VI.B.3), in both site orders, and one propagation step Q^dagger U(t) Q per axis on a field,
compared with the dense transfer-function propagation.  The operators are built in FP64 and rounded once to
complex64, so their entries agree with the oracle's to the FP32 tolerance of 1e-5."""
import numpy as np
import pytest
import torch

import synth
from oracle import fresnel as OF
from oracle import mpo as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=12, d=4, chi=64, w=32, dense=1 << 12)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("n,t,p_max", [(6, 1.0, 14), (12, 1.0, 14), (10, 4.0, 14), (8, 2.0, 5)])
@pytest.mark.parametrize("bit_reversed", [True, False])
def test_bessel_mpo_matches_oracle(eng, n, t, p_max, bit_reversed):
    W = eng.build_bessel_mpo(n, t, p_max, w_cap=32, bit_reversed=bit_reversed)
    assert W.w_max == 2 * p_max + 1 and W.bonds()[0] == 1 and W.bonds()[-1] == 1
    got = OM.diag_of(W.to_numpy_cores())
    ref = OM.diag_of(OM.bessel_mpo(n, t, p_max, bit_reversed))
    assert np.abs(got - ref).max() < 1e-5
    if p_max == 14 and t == 1.0:       # and the exact operator, as the closed form promises
        assert np.abs(got - OM.lattice_diagonal(n, t, bit_reversed)).max() < 1e-5


@pytest.mark.parametrize("n,t,gate_cut", [(6, 1.0, 1e-6), (8, 1.0, 1e-6), (8, 2.0, 1e-4), (10, 1.0, 1e-8)])
def test_pauliz_circuit_mpo_matches_oracle(eng, n, t, gate_cut):
    W = eng.build_pauliz_mpo(n, t, gate_cut, cutoff=1e-13, w_cap=32)
    got = OM.diag_of(W.to_numpy_cores())
    ref = OM.diag_of(OM.pauliz_mpo(n, t, gate_cut, cutoff=1e-13))
    assert np.abs(got - ref).max() < 1e-5
    # error against the exact propagator within the dropped-gate bound (plus FP32 rounding)
    L = 1 << n
    c = OM.walsh_coefficients(np.cos(2 * np.pi * np.arange(L) / L))
    bound = t * np.abs(c[1:][np.abs(c[1:]) < gate_cut]).sum()
    assert np.abs(got - OM.lattice_diagonal(n, t)).max() <= bound + 1e-5


def test_lattice_step_equals_dense_transfer(eng, lib):
    # Q^dagger U(t) Q on x then y (Fig. fig_mpo_mpo with the lattice dispersion): untruncated, equals the dense
    # propagation with the transfer function exp(-i t cos(2 pi k / L)) per axis
    n, t = 5, 2.0
    E = synth.gaussian_beam_with_rectangles(n, seed=611, waist=0.2)
    psi = lib.MPS(n, 4, 64)
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 64, 1e-12)
    Q = eng.build_qft_mpo(n, False, 1e-13)
    Qd = eng.mpo_dagger(Q)
    U = eng.build_bessel_mpo(n, t, 14)
    eng.fresnel_step(psi, "interleaved", Q, Qd, U, 1, 64, 1e-12)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    L = 1 << n
    ref = OF.transfer_dense(E.astype(np.complex128), np.exp(-1j * t * np.cos(2 * np.pi * np.arange(L) / L)))
    assert rel(got, ref) < 1e-5
