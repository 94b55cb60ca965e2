"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute-force loops, closed forms, counting identities, invariants and special
cases that reduce to a textbook routine.  CPU only."""
import numpy as np
import pytest

import synth
from oracle import apply as OA
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS
from oracle import quantics as OQ


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


# ----------------------------------------------------------------------------- quantics map (Sec. III)

@pytest.mark.parametrize("layout", ["serial", "interleaved"])
def test_quantics_map_matches_bitwise_definition(layout):
    n = 3
    L = 1 << n
    E = np.arange(L * L).reshape(L, L)
    v = OQ.dense_to_quantics(E, layout)
    for a in range(L):
        for b in range(L):
            assert v[OQ.quantics_index(a, b, n, layout)] == E[a, b]
    assert np.array_equal(OQ.quantics_to_dense(v, n, layout), E)


def test_interleaved_digit_is_two_x_plus_y():
    # pixel (a, b) = (5, 3) on L = 8: x bits 101, y bits 011 -> mu = (2, 1, 3)
    n = 3
    idx = OQ.quantics_index(5, 3, n, "interleaved")
    assert OQ.site_digits(idx, n, 4) == [2 * 1 + 0, 2 * 0 + 1, 2 * 1 + 1]


# ----------------------------------------------------------------------------- TT-SVD (Sec. IV, App. A)

def test_untruncated_tt_svd_is_exact_and_has_page_ranks():
    rng = np.random.default_rng(1)
    N = 10
    v = rng.standard_normal(2 ** N) + 1j * rng.standard_normal(2 ** N)
    sites, eps = OS.tt_svd(v, N, 2)
    assert rel(OS.to_vector(sites), v) < 1e-12
    assert OS.bonds(sites) == [min(2 ** k, 2 ** (N - k)) for k in range(N + 1)]
    # Sec. IV: a generic binary MPS has D_max = 8/3 * 2^N parameters (exactly 8 (2^N - 1) / 3 for even N)
    D = sum(A.size for A in sites)
    assert D == 8 * (2 ** N - 1) // 3
    assert max(eps) < 1e-20


@pytest.mark.parametrize("chi,cutoff", [(6, 0.0), (64, 1e-3), (5, 1e-2)])
def test_tt_svd_discarded_weights_add_up(chi, cutoff):
    rng = np.random.default_rng(2)
    N, d = 6, 4
    v = rng.standard_normal(d ** N) + 1j * rng.standard_normal(d ** N)
    v *= np.exp(-0.002 * np.arange(d ** N))
    sites, eps = OS.tt_svd(v, N, d, chi, cutoff)
    err2 = np.linalg.norm(OS.to_vector(sites) - v) ** 2
    assert abs(err2 - sum(eps)) <= 1e-10 * np.linalg.norm(v) ** 2
    assert max(OS.bonds(sites)) <= chi


def test_two_site_truncation_is_eckart_young():
    # One bond: the canonical truncation is the best rank-k approximation, whose
    # squared error is the sum of the discarded eigenvalues of M M^dagger.
    rng = np.random.default_rng(3)
    M = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    sites = [M.reshape(1, 16, 16), np.eye(16, dtype=complex).reshape(16, 16, 1)]
    k = 5
    out, eps = OS.truncate(sites, k, 0.0)
    lam = np.sort(np.linalg.eigvalsh(M @ M.conj().T))[::-1]
    err2 = np.linalg.norm(OS.to_vector(out) - M.reshape(-1)) ** 2
    assert abs(err2 - lam[k:].sum()) < 1e-10 * lam.sum()
    assert abs(eps[0] - lam[k:].sum()) < 1e-10 * lam.sum()


def test_canonical_truncation_norm_bookkeeping():
    sites = synth.random_mps_sites([1, 4, 16, 32, 16, 4, 1], 4, seed=4, decay=0.1)
    v = OS.to_vector(sites)
    out, eps = OS.truncate(sites, 8, 0.0)
    w = OS.to_vector(out)
    n2 = np.linalg.norm(v) ** 2
    assert abs(np.linalg.norm(v - w) ** 2 - sum(eps)) < 1e-10 * n2
    assert abs(np.linalg.norm(w) ** 2 - (n2 - sum(eps))) < 1e-10 * n2
    assert OS.is_right_canonical(out)


def test_keep_rank_rule_brute_force():
    s = np.array([3.0, 2.0, 1.0, 0.5, 0.1])
    w = s ** 2
    for cutoff in [0.0, 1e-4, 0.002, 0.01, 0.05, 0.2, 1.0]:
        for chi in [1, 2, 3, 10]:
            k = 1
            while k < len(s) and w[k:].sum() > cutoff * w.sum():
                k += 1
            assert OS.keep_rank(s, chi, cutoff) == min(k, chi)


def test_canonical_forms_and_overlaps():
    sites = synth.random_mps_sites([1, 2, 4, 8, 4, 2, 1], 2, seed=5)
    v = OS.to_vector(sites)
    L_ = OS.left_canonicalize(sites)
    R_ = OS.right_canonicalize(sites)
    assert OS.is_left_canonical(L_) and OS.is_right_canonical(R_)
    assert rel(OS.to_vector(L_), v) < 1e-13 and rel(OS.to_vector(R_), v) < 1e-13
    other = synth.random_mps_sites([1, 2, 3, 3, 3, 2, 1], 2, seed=6)
    assert abs(OS.overlap(other, sites) - np.vdot(OS.to_vector(other), v)) < 1e-12 * np.linalg.norm(v)
    digits = [1, 0, 1, 1, 0, 1]
    flat = int("".join(map(str, digits)), 2)
    assert abs(OS.amplitude(sites, digits) - v[flat]) < 1e-13


def test_elementwise_sum_and_kron():
    A = synth.random_mps_sites([1, 3, 5, 3, 1], 4, seed=7)
    B = synth.random_mps_sites([1, 2, 4, 2, 1], 4, seed=8)
    va, vb = OS.to_vector(A), OS.to_vector(B)
    assert rel(OS.to_vector(OS.hadamard_product(A, B)), va * vb) < 1e-13
    assert rel(OS.to_vector(OS.hadamard_product(A, B, conj_b=True)), va * vb.conj()) < 1e-13
    assert rel(OS.to_vector(OS.direct_sum(A, B)), va + vb) < 1e-13
    X = synth.random_mps_sites([1, 2, 3, 2, 1], 2, seed=9)
    Y = synth.random_mps_sites([1, 3, 2, 2, 1], 2, seed=10)
    E = np.outer(OS.to_vector(X), OS.to_vector(Y))
    assert rel(OS.to_vector(OS.kron_interleave(X, Y)), OQ.dense_to_quantics(E, "interleaved")) < 1e-13


# ----------------------------------------------------------------------------- DFT / QFT (Sec. V)

def test_dft_matrix_brute_force_and_fft_witness():
    n = 5
    L = 1 << n
    rng = np.random.default_rng(11)
    v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    brute = np.array([sum(v[j] * np.exp(2j * np.pi * j * k / L) for j in range(L)) for k in range(L)]) / np.sqrt(L)
    assert rel(OM.dft_matrix(L) @ v, brute) < 1e-13
    # library FFT as a third witness: exp(+2 pi i jk/L) is L * ifft
    assert rel(brute, np.fft.ifft(v) * np.sqrt(L)) < 1e-13


def test_qft_circuit_layers_give_bit_reversed_dft():
    # The uncompressed product of the n circuit layers is the swap-free QFT:
    # row rev(k) holds DFT row k.
    n = 5
    W = OM.identity(n)
    for j in range(n):
        W = OM.product(OM.qft_layer(n, j), W)
    Q = OM.to_dense(W)
    L = 1 << n
    for k in range(L):
        r = OQ.bit_reverse(k, n)
        for j in range(L):
            assert abs(Q[r, j] - np.exp(2j * np.pi * j * k / L) / np.sqrt(L)) < 1e-13


@pytest.mark.parametrize("n", [4, 6, 8])
def test_qft_mpo_constructions_agree_and_are_low_rank(n):
    dense = OM.qft_noswap_dense(n)
    Wd = OM.qft_mpo_dense(n, 1e-20)
    Wl = OM.qft_mpo_layers(n, 1e-20)
    assert np.abs(OM.to_dense(Wd) - dense).max() < 1e-10
    assert np.abs(OM.to_dense(Wl) - dense).max() < 1e-10
    # C1 reading: cutoff 1e-10 keeps bond <= 8
    assert max(OM.bonds(OM.qft_mpo_layers(n, 1e-10))) <= 8
    Q = OM.to_dense(Wl)
    assert np.abs(Q.conj().T @ Q - np.eye(1 << n)).max() < 1e-10


def test_qft_rank_stays_bounded_with_n():
    # Sec. V: the QFT has a finite-rank MPO; the bond does not grow with n.
    ranks = [max(OM.bonds(OM.qft_mpo_layers(n, 1e-12))) for n in (8, 10, 12, 14)]
    assert max(ranks) <= 8 and len(set(ranks)) == 1


def fwht(v):
    """Fast Walsh-Hadamard transform, orthonormal (own butterfly code)."""
    v = np.array(v, dtype=np.complex128)
    h = 1
    while h < len(v):
        for i in range(0, len(v), 2 * h):
            a = v[i:i + h].copy()
            b = v[i + h:i + 2 * h].copy()
            v[i:i + h] = a + b
            v[i + h:i + 2 * h] = a - b
        h *= 2
    return v / np.sqrt(len(v))


def test_hadamard_mpo_is_rank_one_walsh_transform():
    n = 6
    sites = synth.random_mps_sites([1, 2, 4, 8, 4, 2, 1], 2, seed=12)
    sites = OS.right_canonicalize(sites)
    H = OM.hadamard_mpo(n)
    out, eps = OA.zipup(H, sites, 1 << 20, 0.0, "lr")
    assert rel(OS.to_vector(out), fwht(OS.to_vector(sites))) < 1e-12
    assert OM.bonds(H) == [1] * (n + 1)


def test_phase_mpo_matches_transfer_function():
    n, c = 8, 0.37
    W = OM.phase_mpo(n, c, 1e-20)
    Dm = OM.to_dense(W)
    L = 1 << n
    for idx in range(L):
        k = OQ.bit_reverse(idx, n)
        kf = k if k < L // 2 else k - L
        assert abs(Dm[idx, idx] - np.exp(-1j * np.pi * c * kf * kf / L)) < 1e-10
    assert np.abs(Dm - np.diag(np.diag(Dm))).max() < 1e-10
    assert max(OM.bonds(OM.phase_mpo(n, 0.0, 1e-14))) == 1


# ----------------------------------------------------------------------------- zip-up (Sec. V, Fig. fig_mpo)

@pytest.mark.parametrize("direction", ["lr", "rl"])
def test_untruncated_zipup_equals_exact_product(direction):
    n = 6
    sites = synth.random_mps_sites([1, 2, 4, 8, 4, 2, 1], 2, seed=13)
    sites = OS.right_canonicalize(sites) if direction == "lr" else OS.left_canonicalize(sites)
    W = OM.qft_mpo_layers(n, 1e-20)
    out, eps = OA.zipup(W, sites, 1 << 20, 0.0, direction)
    assert rel(OS.to_vector(out), OM.to_dense(W) @ OS.to_vector(sites)) < 1e-12
    check = OS.is_left_canonical if direction == "lr" else OS.is_right_canonical
    assert check(out)


def test_zipup_with_unitary_product_operator_is_sequential_svd():
    # With a bond-1 MPO of unitaries the right environment of every cut is an
    # isometry, so each zip-up truncation is the exact SVD of the current
    # unfolding: the result is TT-SVD of the exactly applied state.
    n = 6
    sites = OS.right_canonicalize(synth.random_mps_sites([1, 4, 16, 64, 16, 4, 1], 4, seed=14, decay=0.05))
    U = synth.random_unitary_sites(n, seed=15, dim=4)
    W = [u.reshape(1, 4, 4, 1) for u in U]
    out, eps = OA.zipup(W, sites, 10, 0.0, "lr")
    ref, eps_ref = OS.tt_svd(OM.to_dense(W) @ OS.to_vector(sites), n, 4, 10, 0.0)
    assert rel(OS.to_vector(out), OS.to_vector(ref)) < 1e-10
    assert np.allclose(eps, eps_ref, rtol=1e-9, atol=1e-14)


# ----------------------------------------------------------------------------- Fresnel (Sec. VI.A)

def test_dense_fresnel_matches_fft_and_is_unitary():
    E = synth.gaussian_beam_with_rectangles(5, seed=16, waist=0.2).astype(complex)
    a, b = OF.fresnel_dense(E, 0.3), OF.fresnel_fft(E, 0.3)
    assert rel(a, b) < 1e-13
    assert abs(np.linalg.norm(a) - np.linalg.norm(E)) < 1e-12 * np.linalg.norm(E)


@pytest.mark.parametrize("layout", ["interleaved", "serial"])
def test_untruncated_mps_fresnel_equals_dense(layout):
    n, c = 5, 0.3
    E = synth.gaussian_beam_with_rectangles(n, seed=17, waist=0.2).astype(complex)
    sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, layout), OQ.n_sites(n, layout), OQ.phys_dim(layout))
    ops = OF.step_operators(n, c, qft=OM.qft_mpo_layers(n, 1e-20), phase_cutoff=1e-20)
    out, canon, disc = OF.fresnel_mps(sites, layout, n, c, 1 << 20, 0.0, canon="left", ops=ops)
    Ez = OQ.quantics_to_dense(OS.to_vector(out), n, layout)
    assert rel(Ez, OF.fresnel_dense(E, c)) < 1e-11
    assert abs(np.linalg.norm(Ez) - np.linalg.norm(E)) < 1e-11 * np.linalg.norm(E)


@pytest.mark.parametrize("layout", ["interleaved", "serial"])
def test_matched_operator_form_untruncated_equals_dense(layout):
    # operators in the canonical form of each pass's sweep direction: the same operators, so without
    # truncation the step is still the dense propagator
    n, c = 5, 0.3
    E = synth.gaussian_beam_with_rectangles(n, seed=17, waist=0.2).astype(complex)
    sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, layout), OQ.n_sites(n, layout), OQ.phys_dim(layout))
    ops = OF.step_operators(n, c, qft=OM.qft_mpo_layers(n, 1e-20), phase_cutoff=1e-20)
    for W in ops:
        for side in ("left", "right"):
            Wc = OF.operator_canonical(W, side)
            assert np.abs(OM.to_dense(Wc) - OM.to_dense(W)).max() < 1e-12
    out, canon, disc = OF.fresnel_mps(sites, layout, n, c, 1 << 20, 0.0, canon="left", ops=ops,
                                      operator_form="matched")
    assert rel(OQ.quantics_to_dense(OS.to_vector(out), n, layout), OF.fresnel_dense(E, c)) < 1e-11


def test_matched_operator_form_depends_on_the_operator_only():
    # the matched form re-canonicalises the operators, so any representation of the same operator (here a
    # right-canonical MPO put through random non-unitary changes of gauge) gives the same truncated step,
    # within the truncation budget of the dense propagation
    n, c, chi = 6, 0.45, 10
    E = synth.gaussian_beam_with_rectangles(n, seed=19, waist=0.2).astype(complex)
    sites, eps0 = OS.tt_svd(OQ.dense_to_quantics(E, "interleaved"), n, 4, 1 << 20, 1e-14)
    Q = OM.qft_mpo_layers(n, 1e-14)
    rng = np.random.default_rng(7)
    G = [np.eye(1)] + [np.eye(Q[p].shape[3]) + 0.3 * rng.standard_normal((Q[p].shape[3],) * 2)
                       for p in range(n - 1)] + [np.eye(1)]
    Qg = [np.einsum("ia,atsb,bj->itsj", np.linalg.inv(G[p]), Q[p], G[p + 1]) for p in range(n)]
    assert np.abs(OM.to_dense(Qg) - OM.to_dense(Q)).max() < 1e-12
    D = OM.phase_mpo(n, c, 1e-14)
    runs = []
    for W in (Q, Qg):
        runs.append(OF.fresnel_mps(sites, "interleaved", n, c, chi, 1e-12, canon="left",
                                   ops=(W, OM.dagger(W), D), operator_form="matched"))
    (a, _, da), (b, _, db) = runs
    assert rel(OS.to_vector(b), OS.to_vector(a)) < 1e-10 and abs(da - db) < 1e-10 * OS.norm2(sites)
    exact = OF.fresnel_dense(E, c)
    got = OQ.quantics_to_dense(OS.to_vector(a), n, "interleaved")
    n2 = np.linalg.norm(E) ** 2
    assert da > 0.0
    assert np.linalg.norm(got - exact) <= np.sqrt(2 * 6 * da) + 1e-10 * np.sqrt(n2)


def test_fresnel_group_properties():
    n = 4
    E = synth.gaussian_beam_with_rectangles(n, seed=18, waist=0.3).astype(complex)
    sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, "interleaved"), n, 4)
    Q = OM.qft_mpo_layers(n, 1e-20)

    def step(s, c, canon="left"):
        ops = (Q, OM.dagger(Q), OM.phase_mpo(n, c, 1e-20))
        return OF.fresnel_mps(s, "interleaved", n, c, 1 << 20, 0.0, canon=canon, ops=ops)

    v0 = OS.to_vector(sites)
    a, ca, _ = step(sites, 0.0)
    assert rel(OS.to_vector(a), v0) < 1e-11                      # c = 0 is the identity
    b, cb, _ = step(*step(sites, 0.4)[:1], -0.4, canon="right")
    assert rel(OS.to_vector(b), v0) < 1e-11                      # forward then backward
    two = step(step(sites, 0.25)[0], 0.25, canon="right")[0]
    one = step(sites, 0.5)[0]
    assert rel(OS.to_vector(two), OS.to_vector(one)) < 1e-11     # z1 + z2 composes


def test_x_and_y_passes_commute():
    n = 4
    E = synth.gaussian_beam_with_rectangles(n, seed=19, waist=0.3).astype(complex)
    v = OQ.dense_to_quantics(E, "interleaved")
    Q = OM.qft_mpo_layers(n, 1e-20)
    Wx, Wy = OM.embed(Q, "interleaved", 0, n), OM.embed(Q, "interleaved", 1, n)
    Dx, Dy = OM.to_dense(Wx), OM.to_dense(Wy)
    assert np.abs(Dx @ Dy - Dy @ Dx).max() < 1e-12
    # acting on x alone is the 1-D transform of every column
    Qd = OM.to_dense(Q)
    assert rel(OQ.quantics_to_dense(Dx @ v, n, "interleaved"), Qd @ E) < 1e-12


def test_fourier_space_phase_identity():
    # Q psi_out = D (Q psi_in): the step is diagonal in (bit-reversed) Fourier space.
    n, c = 5, 0.7
    L = 1 << n
    rng = np.random.default_rng(20)
    v = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    out = OF.fresnel_dense_1d(v, c)
    Q = OM.qft_noswap_dense(n)
    D = OM.phase_vector(n, c, True)
    assert rel(Q @ out, D * (Q @ v)) < 1e-12


def test_hilbert_transform_pipeline():
    # Sec. VI.C: Q^dagger (-i Z_n) Q with a bond-1 diagonal is the periodic
    # Hilbert-type transform: multiply frequency k by -i for k < L/2, +i otherwise.
    n = 6
    L = 1 << n
    sites = OS.right_canonicalize(synth.random_mps_sites([1, 2, 4, 8, 4, 2, 1], 2, seed=21))
    v = OS.to_vector(sites)
    Q = OM.qft_mpo_layers(n, 1e-20)
    A, canon, _ = OF.apply_sequence([Q, OM.hilbert_diag_mpo(n), OM.dagger(Q)], sites, "right", 1 << 20, 0.0)
    F = OM.dft_matrix(L)
    sgn = np.where(np.arange(L) < L // 2, -1j, 1j)
    assert rel(OS.to_vector(A), F.conj().T @ (sgn * (F @ v))) < 1e-11


def test_gaussian_beam_closed_form_1d():
    # Textbook Fresnel propagation of a Gaussian (not in the paper); the grid
    # is fine enough and wide enough that sampling and wrap-around are < 1e-10.
    n = 10
    L = 1 << n
    x = np.arange(L) - L / 2
    w = 0.06 * L
    lz = 0.8 * L                                 # lambda z / dx^2 in pixel units
    c = lz / L
    v = np.exp(-x * x / (w * w))
    sites, _ = OS.tt_svd(np.roll(v, 0), n, 2, 1 << 20, 1e-24)
    out, canon, _ = OF.fresnel_mps(sites, "1d", n, c, 1 << 20, 1e-24, canon="left",
                                   ops=OF.step_operators(n, c, qft=OM.qft_mpo_layers(n, 1e-22), phase_cutoff=1e-24))
    got = OS.to_vector(out)
    ref = OF.gaussian_closed_form(x, w, lz)
    assert np.abs(got - ref).max() < 1e-9


def test_c1_image_qft_against_brute_force_dft():
    # C1: 64x64 image, serial 12 sites, TT-SVD chi 16, QFT MPO cutoff 1e-10.
    # Q is unitary, so ||Q psi~ - Q psi|| = ||psi~ - psi|| = sqrt(sum eps).
    n = 6
    L = 1 << n
    img = synth.gaussian_random_field_image(n)
    v = OQ.dense_to_quantics(img, "serial")
    sites, eps = OS.tt_svd(v, 2 * n, 2, 16, 0.0)
    Q = OM.qft_mpo_layers(n, 1e-10)
    out, canon, _ = OF.apply_sequence([OM.embed(Q, "serial", 0, n), OM.embed(Q, "serial", 1, n)],
                                      sites, "left", 1 << 20, 0.0)
    F = OM.dft_matrix(L)
    ref = F @ img @ F.T
    perm = [OQ.bit_reverse(k, n) for k in range(L)]
    ref_br = np.empty_like(ref)
    ref_br[np.ix_(perm, perm)] = ref
    got = OQ.quantics_to_dense(OS.to_vector(out), n, "serial")
    err = np.linalg.norm(got - ref_br)
    assert err <= np.sqrt(sum(eps)) + 1e-6 * np.linalg.norm(img)
    assert max(OS.bonds(sites)) <= 16


# ----------------------------------------------------------------------------- intensity loss and its adjoint

def test_intensity_loss_gradient_matches_finite_differences():
    # central differences of the dense loss in the real and imaginary part of single mask values: they pin
    # the conjugate-Wirtinger gradient G (dL = 2 Re conj(G) dM) without using its formula
    from oracle import optics as OO
    rng = np.random.default_rng(61)
    n = 3
    L = 1 << n
    E = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    M = np.exp(1j * 0.3 * rng.standard_normal((L, L)))
    It = rng.uniform(0, 2, size=(L, L))
    c = 0.7
    G = OO.intensity_loss_grad_dense(E, M, It, c)
    h = 1e-6
    for (i, j) in [(0, 0), (3, 5), (7, 2)]:
        for unit in (1.0, 1j):
            Mp, Mm = M.copy(), M.copy()
            Mp[i, j] += h * unit
            Mm[i, j] -= h * unit
            fd = (OO.intensity_loss_dense(E, Mp, It, c) - OO.intensity_loss_dense(E, Mm, It, c)) / (2 * h)
            pred = 2 * np.real(np.conj(G[i, j]) * unit)
            assert abs(fd - pred) <= 1e-6 * max(1.0, abs(pred))


# ----------------------------------------------------------------------------- exact / naive MPO application

def brute_force_apply(W, vec):
    """y[s'] = sum_s O[s', s] vec[s] with O[s', s] = prod_p W_p[:, s'_p, s_p, :] written out per index
    string (loops over all digit strings; independent of the oracle's contractions)."""
    n = len(W)
    dim = 2 ** n
    y = np.zeros(dim, dtype=np.complex128)
    for out_idx in range(dim):
        so = [(out_idx >> (n - 1 - p)) & 1 for p in range(n)]
        for in_idx in range(dim):
            si = [(in_idx >> (n - 1 - p)) & 1 for p in range(n)]
            m = np.ones((1, 1), dtype=np.complex128)
            for p in range(n):
                m = m @ W[p][:, so[p], si[p], :]
            y[out_idx] += m[0, 0] * vec[in_idx]
    return y


def test_apply_exact_and_dense_match_brute_force():
    n = 4
    W = OM.qft_mpo_layers(n, 1e-14)
    sites = synth.random_mps_sites([1, 2, 4, 2, 1], 2, seed=901)
    v = OS.to_vector(sites)
    ref = brute_force_apply(W, v)
    assert rel(OS.to_vector(OA.apply_exact(W, sites)), ref) < 1e-12
    assert rel(OA.apply_dense(W, v), ref) < 1e-12
    # bonds multiply
    assert OS.bonds(OA.apply_exact(W, sites)) == [a * b for a, b in zip(OM.bonds(W), OS.bonds(sites))]


def test_apply_naive_two_sites_is_eckart_young():
    # two sites: the naive truncation is one SVD of the 4 x 4 reshaped product, the optimum by Eckart-Young
    W = OM.qft_mpo_layers(2, 1e-14)
    sites = synth.random_mps_sites([1, 2, 1], 2, seed=902)
    y = OA.apply_dense(W, OS.to_vector(sites))
    s = np.linalg.svd(y.reshape(2, 2), compute_uv=False)
    out, eps = OA.apply_naive(W, sites, 1, 0.0)
    assert abs(sum(eps) - s[1] ** 2) < 1e-12 * (s ** 2).sum()
    assert abs(np.linalg.norm(OS.to_vector(out) - y) ** 2 - s[1] ** 2) < 1e-12 * (s ** 2).sum()


def test_apply_naive_error_equals_discarded_weight():
    # canonical truncation of the exact product: squared error = sum of the per-bond discarded weights
    n = 5
    W = OM.qft_mpo_layers(n, 1e-14)
    sites = synth.random_mps_sites([1, 2, 4, 4, 2, 1], 2, seed=903, decay=0.2)
    y = OA.apply_dense(W, OS.to_vector(sites))
    out, eps = OA.apply_naive(W, sites, 3, 0.0)
    assert max(OS.bonds(out)) <= 3
    assert abs(np.linalg.norm(OS.to_vector(out) - y) ** 2 - sum(eps)) < 1e-12 * np.linalg.norm(y) ** 2


def test_zipup_factorised_weights_of_an_isometric_chain_equal_the_norm():
    # the identity operator on a canonical state: everything left of a bond is an isometry (the new sites)
    # and everything right of it too (the untouched canonical sites), so every factorised two-site matrix
    # carries exactly the squared norm of the state; its discarded parts are parts of that weight
    n = 6
    ident = OM.identity(n)
    raw = synth.random_mps_sites([1, 2, 4, 8, 4, 2, 1], 2, seed=905, decay=0.3)
    n2 = OS.norm2(raw)
    for direction, canon in (("lr", OS.right_canonicalize), ("rl", OS.left_canonicalize)):
        totals = []
        out, eps = OA.zipup(ident, canon(raw), 1 << 10, 0.0, direction, totals)
        assert len(totals) == n - 1
        assert np.allclose(totals, n2, rtol=1e-12, atol=0.0)
        assert rel(OS.to_vector(out), OS.to_vector(raw)) < 1e-12
    # with truncation the discarded weights stay within the factorised weights
    totals = []
    out, eps = OA.zipup(ident, OS.right_canonicalize(raw), 2, 0.0, "lr", totals)
    assert all(0.0 <= e <= t for e, t in zip(eps, totals)) and sum(eps) > 0.0


def test_schmidt_spectra_match_dense_unfoldings():
    # the Schmidt values at bond k are the singular values of the (d^k) x (d^(N-k)) unfolding of the vector
    bonds = [1, 4, 9, 7, 3, 1]
    sites = synth.random_mps_sites(bonds, 3, seed=904)
    v = OS.to_vector(sites)
    spec = OS.schmidt_spectra(sites)
    N, d = 5, 3
    for k in range(1, N):
        s_ref = np.linalg.svd(v.reshape(d ** k, d ** (N - k)), compute_uv=False)
        s = np.sort(spec[k - 1])[::-1]
        r = len(s)
        assert np.allclose(s, s_ref[:r], rtol=0, atol=1e-12 * s_ref[0])
        assert np.all(s_ref[r:] < 1e-12 * s_ref[0])


# ----------------------------------------------------------------------------- lattice dispersion (Sec. VI.B)

@pytest.mark.parametrize("n", [4, 6, 8])
@pytest.mark.parametrize("bit_reversed", [True, False])
def test_bessel_mpo_reaches_1e10_at_pmax_14(n, bit_reversed):
    # Sec. VI.B.4, Fig. fig_error_mpo: at p_max = 14 (bond 29) the operator error is below 1e-10 for t = 1
    W = OM.bessel_mpo(n, 1.0, 14, bit_reversed)
    assert max(OM.bonds(W)) == 29
    assert np.abs(OM.diag_of(W) - OM.lattice_diagonal(n, 1.0, bit_reversed)).max() < 1e-10


@pytest.mark.parametrize("p_max", [2, 4, 6])
def test_bessel_truncation_within_the_bessel_tail_bound(p_max):
    # delta(p_max) <= sum_{|p| > p_max} |J_p(t)| since every plane-wave term has unit modulus (Sec. VI.B.4)
    from scipy.special import jv
    t, n = 2.0, 6
    err = np.abs(OM.diag_of(OM.bessel_mpo(n, t, p_max)) - OM.lattice_diagonal(n, t)).max()
    tail = 2 * sum(abs(jv(p, t)) for p in range(p_max + 1, 60))
    assert err <= tail * (1 + 1e-9)
    assert err > 0.1 * tail          # and the bound is not loose by orders of magnitude


def test_walsh_coefficients_match_definition_and_product_formula():
    # Eq. coeff_trace by brute force, and the closed product form Eq. eq_cs:
    # c_S = 2^-n Re prod_j (1 + (-1)^[j in S] e^{i theta_j}), theta_j = 2 pi / 2^j, qubit j = bit n-j of k
    n = 5
    L = 1 << n
    eps = np.cos(2 * np.pi * np.arange(L) / L)
    c = OM.walsh_coefficients(eps)
    for S in range(L):
        brute = sum(eps[s] * (-1) ** bin(S & s).count("1") for s in range(L)) / L
        prod = 1.0 + 0j
        for j in range(1, n + 1):
            inS = (S >> (n - j)) & 1
            prod *= 1 + (-1) ** inS * np.exp(2j * np.pi / 2 ** j)
        assert abs(c[S] - brute) < 1e-14
        assert abs(c[S] - prod.real / L) < 1e-14


@pytest.mark.parametrize("gate_cutoff", [0.0, 1e-6, 1e-3])
def test_pauliz_circuit_error_within_the_dropped_gate_bound(gate_cutoff):
    # ||U - U_trunc|| <= t sum_{dropped} |c_S| (Sec. VI.B.3); with every gate kept the circuit is exact
    n, t = 8, 1.0
    L = 1 << n
    c = OM.walsh_coefficients(np.cos(2 * np.pi * np.arange(L) / L))
    dropped = np.abs(c[1:][np.abs(c[1:]) < gate_cutoff]).sum()
    W = OM.pauliz_mpo(n, t, gate_cutoff, cutoff=0.0)
    err = np.abs(OM.diag_of(W) - OM.lattice_diagonal(n, t)).max()
    assert err <= t * dropped + 1e-12
    if gate_cutoff == 0.0:
        assert err < 1e-12


def test_lattice_transfer_reduces_to_fresnel_near_zero_frequency():
    # Sec. VI.B.1: cos k ~ 1 - k^2/2, so exp(-i t cos(2 pi k / L)) ~ exp(-i t) exp(+i t (2 pi k / L)^2 / 2) near k = 0
    n, t = 8, 3.0
    L = 1 << n
    k = np.arange(8)
    D = OM.lattice_diagonal(n, t, False)[k]
    approx = np.exp(-1j * t) * np.exp(1j * t * (2 * np.pi * k / L) ** 2 / 2)
    assert np.abs(D - approx).max() < t * (2 * np.pi * 8 / L) ** 4 / 24 + 1e-12


# ----------------------------------------------------------------------------- imaging and angular spectrum

def test_psf_of_a_box_aperture_is_the_dirichlet_kernel():
    # |sum_{j<w} e^{2 pi i j k / L}|^2 = sin^2(pi w k / L) / sin^2(pi k / L): the PSF of a w x w box pupil factors
    from oracle import optics as OO
    n, w = 5, 7
    L = 1 << n
    E = np.zeros((L, L), complex)
    E[:w, :w] = 1.0
    k = np.arange(L)
    with np.errstate(divide="ignore", invalid="ignore"):
        dk = np.where(k == 0, w * w, np.sin(np.pi * w * k / L) ** 2 / np.sin(np.pi * k / L) ** 2)
    ref = np.outer(dk, dk)
    ref = ref / ref.sum()
    assert np.abs(OO.psf_dense(E) - ref).max() < 1e-14
    c = OO.psf_dense(E, centre=True)
    assert abs(c.sum() - 1) < 1e-12 and np.argmax(c) == (L // 2) * L + L // 2


def test_circular_convolution_matches_fft_witness():
    # the paper's pin for Eq. convolution_eq: on the finite grid it is the FFT computation (library witness)
    from oracle import optics as OO
    rng = np.random.default_rng(5)
    a = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    b = rng.standard_normal((16, 16))
    ref = np.fft.ifft2(np.fft.fft2(a) * np.fft.fft2(b))
    assert np.abs(OO.convolve_dense(a, b) - ref).max() < 1e-12


def test_astf_reduces_to_fresnel_in_the_paraxial_limit_and_decays_when_evanescent():
    # Sec. VI.A: sqrt(1 - u) ~ 1 - u/2 gives exp(-i pi lambda z f^2) per axis, the Fresnel transfer function;
    # the neglected term is (z/lambda) 2 pi u^2 / 8 at most
    from oracle import optics as OO
    n = 6
    L = 1 << n
    zl, ld = 40.0, 0.0633
    T = OO.astf_transfer(n, zl, ld)
    kf = OM.fftfreq_int(L).astype(float)
    c = zl * ld * ld / L                      # lambda z / (L dx^2)
    Tf = np.exp(-1j * np.pi * c * kf ** 2 / L)
    u_max = 2 * (ld / 2) ** 2
    assert np.abs(T - np.outer(Tf, Tf)).max() <= 2 * np.pi * zl * u_max ** 2 / 8 * 1.01
    assert np.allclose(np.abs(T), 1.0)
    Te = OO.astf_transfer(n, 3.0, 1.5)       # lambda = 1.5 dx: the outer frequencies are evanescent
    lf = 1.5 * kf / L
    u = lf[:, None] ** 2 + lf[None, :] ** 2
    assert np.allclose(np.abs(Te[u <= 1]), 1.0)
    assert np.all(np.abs(Te[u > 1]) < 1.0)
    assert np.allclose(np.abs(Te[u > 1]), np.exp(-2 * np.pi * 3.0 * np.sqrt(u[u > 1] - 1)))


# ----------------------------------------------------------------------------- frozen-projector adjoint

def _frozen_case(n, chi):
    from oracle import optics as OO
    E = synth.gaussian_beam_with_rectangles(n, seed=931, waist=0.3).astype(np.complex128)
    E_sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, "interleaved"), n, 4, 64, 1e-14)
    mx, my = synth.smooth_random_phase_mask_factors(n, seed=932, strength=0.5)
    X, _ = OS.tt_svd(mx, n, 2, 64, 1e-14)
    Y, _ = OS.tt_svd(my, n, 2, 64, 1e-14)
    M_sites = OS.kron_interleave(X, Y)
    It = OQ.dense_to_quantics(synth.rectangles_target(n, seed=933).astype(np.float64), "interleaved")
    Q = OM.qft_mpo_layers(n, 1e-14)
    ops = (Q, OM.dagger(Q), OM.phase_mpo(n, 0.5, 1e-14))
    return OO, E_sites, M_sites, It, ops


def test_frozen_adjoint_matches_finite_differences_of_the_frozen_map():
    # with truncation active (chi 6 < the 4^2 bond of n = 4) the adjoint is the exact derivative of the map with
    # the recorded projectors held fixed: central differences along random directions
    n = 4
    OO, E_sites, M_sites, It, ops = _frozen_case(n, 6)
    L, G, pieces = OO.frozen_loss_and_grad(E_sites, M_sites, It, n, ops, 6, 0.0)
    m = OS.to_vector(M_sites)
    assert abs(OO.frozen_loss(m, pieces, It) - L) < 1e-12 * L
    rng = np.random.default_rng(3)
    for _ in range(4):
        dm = rng.standard_normal(m.shape) + 1j * rng.standard_normal(m.shape)
        h = 1e-6
        fd = (OO.frozen_loss(m + h * dm, pieces, It) - OO.frozen_loss(m - h * dm, pieces, It)) / (2 * h)
        assert abs(fd - 2 * np.real(np.vdot(G, dm))) < 1e-6 * np.abs(fd) + 1e-9


def test_frozen_adjoint_with_full_frames_is_the_true_gradient():
    # n = 2: every frame spans the whole space (bonds 4 = d), so every projector is the identity and the frozen
    # gradient is the dense gradient of the loss
    n = 2
    OO, E_sites, M_sites, It, ops = _frozen_case(n, 64)
    L, G, (P, K, e) = OO.frozen_loss_and_grad(E_sites, M_sites, It, n, ops, 64, 0.0)
    assert all(np.allclose(Pi, np.eye(16), atol=1e-12) for Pi in P)
    Ed = OQ.quantics_to_dense(OS.to_vector(E_sites), n, "interleaved")
    Md = OQ.quantics_to_dense(OS.to_vector(M_sites), n, "interleaved")
    Itd = OQ.quantics_to_dense(It, n, "interleaved")
    ref = OO.intensity_loss_grad_dense(Ed, Md, Itd, 0.5)
    assert abs(L - OO.intensity_loss_dense(Ed, Md, Itd, 0.5)) < 1e-9 * L
    assert np.linalg.norm(OQ.quantics_to_dense(G, n, "interleaved") - ref) < 1e-9 * np.linalg.norm(ref)
