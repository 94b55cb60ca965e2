"""GPU parity of the imaging pipelines of Sec. V and the angular-spectrum step of Sec. VI.A against the dense
FP64 oracle, through the C ABI:

* the point spread function (Eq. psf_eq): |phi> = U_qft |E_0> normalised, ||PSF>> = |phi> (.) |phi>^*, read out in
  natural (and centred) frequency order after the site reversal, with ||PSF||_L1 = 1;
* image formation (Eq. convolution_eq): the circular convolution of a scene with the PSF, "exactly equivalent" on
  the finite grid to the FFT computation (the oracle sums the shifts);
* the angular-spectrum transfer function (Eq. eq_astf), which does not factor over the axes: encoded as an
  interleaved MPS and applied in Fourier space, paraxial and evanescent cases.

Tolerance (FP32 path): relative L2 within 1e-5 + sqrt(eps), eps the relative discarded weight reported."""
import numpy as np
import pytest
import torch

import synth
from oracle import optics as OO
from oracle import quantics as OQ

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def eng(lib):
    # zip-up bonds of the focal field near the chain end may reach the state's capacity: the products that use
    # it as an operator need MPO bonds up to 64
    return lib.Engine(n_sites=6, d=4, chi=64, w=64, dense=1 << 12)


@pytest.fixture(scope="module")
def ops(eng):
    Q = eng.build_qft_mpo(5, False, 1e-13)
    return Q, eng.mpo_dagger(Q)


def encode(eng, lib, E, n, chi=64, cut=1e-13):
    psi = lib.MPS(n, 4, chi)
    st = eng.encode(torch.from_numpy(np.ascontiguousarray(E).astype(np.complex64)).cuda(), n, "interleaved", psi,
                    chi, cut)
    return psi, st


@pytest.mark.parametrize("centre", [False, True])
def test_psf_matches_dense(eng, lib, ops, centre):
    n = 5
    E = synth.pupil_field(n)
    phi, st0 = encode(eng, lib, E, n)
    psf = lib.MPS(n, 4, 64)
    st = eng.psf(phi, ops[0], psf, 64, 1e-13, centre=centre)
    got = eng.to_dense(psf, "interleaved", n).cpu().numpy()
    ref = OO.psf_dense(E.astype(np.complex128), centre)
    eps = st.discarded + st0.discarded / float(np.linalg.norm(E.astype(np.complex128)) ** 2)
    assert rel(got, ref) < 1e-5 + np.sqrt(eps)
    assert abs(got.real.sum() - 1.0) < 1e-5 + eps                  # ||PSF||_L1 = <phi|phi> = 1
    assert np.abs(got.imag).max() < 1e-5 * np.abs(got).max()
    # the normalised focal field itself, in natural (and centred) frequency order
    from oracle import mpo as OM
    F = OM.dft_matrix(1 << n)
    Ef = F @ E.astype(np.complex128) @ F.T
    Ef = Ef / np.linalg.norm(Ef)
    if centre:
        Ef = np.roll(np.roll(Ef, 16, axis=0), 16, axis=1)
    assert rel(eng.to_dense(phi, "interleaved", n).cpu().numpy(), Ef) < 1e-5 + np.sqrt(eps)


def test_image_formation_convolves_the_scene_with_the_psf(eng, lib, ops):
    # Eq. convolution_eq: U_iqft(U_qft ||PSF>> (.) U_qft |S>) with the PSF of the aberrated pupil
    n = 5
    E = synth.pupil_field(n)
    phi, _ = encode(eng, lib, E, n)
    psf = lib.MPS(n, 4, 64)
    eng.psf(phi, ops[0], psf, 64, 1e-13, centre=True)
    S = synth.gaussian_random_field_image(n)
    img, st0 = encode(eng, lib, S, n)
    st = eng.convolve(psf, img, ops[0], ops[1], 64, 1e-13)
    got = eng.to_dense(img, "interleaved", n).cpu().numpy()
    ref = OO.convolve_dense(OO.psf_dense(E.astype(np.complex128), True), S)
    n2 = float(np.linalg.norm(S) ** 2)
    assert rel(got, ref) < 1e-5 + np.sqrt((st.discarded + st0.discarded) / n2)


@pytest.mark.parametrize("z_over_lambda,lambda_over_dx", [(2000.0, 0.0633), (3.0, 1.5), (0.0, 0.5)])
def test_angular_spectrum_step_matches_dense(eng, lib, ops, z_over_lambda, lambda_over_dx):
    n = 5
    L = 1 << n
    Tgpu = eng.astf_field(n, z_over_lambda, lambda_over_dx, bit_reversed=True).cpu().numpy()
    Tref = OO.astf_transfer(n, z_over_lambda, lambda_over_dx)
    rev = np.array([OQ.bit_reverse(i, n) for i in range(L)])
    assert np.abs(Tgpu - Tref[np.ix_(rev, rev)]).max() < 1e-6
    T, _ = encode(eng, lib, Tgpu, n)
    E = synth.gaussian_beam_with_rectangles(n, seed=811, waist=0.2)
    psi, st0 = encode(eng, lib, E, n)
    st = eng.transfer_step(psi, ops[0], ops[1], T, 64, 1e-13)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    ref = OO.propagate_dense_2d(E.astype(np.complex128), Tref)
    n2 = float(np.linalg.norm(E.astype(np.complex128)) ** 2)
    print(f"ASTF z/lambda={z_over_lambda} lambda/dx={lambda_over_dx}: rel {rel(got, ref):.2e}, "
          f"transfer bonds {T.bonds()}")
    assert rel(got, ref) < 1e-5 + np.sqrt((st.discarded + st0.discarded) / n2)
