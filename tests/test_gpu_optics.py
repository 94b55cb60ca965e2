"""GPU parity of the mask/intensity/loss/adjoint path against the FP64 oracle, through the C ABI.

Elementwise products (direct and by zip-up) against the oracle's Hadamard product, the overlap
derivative against brute force (the overlap is linear in every conjugated bra site), and the loss and its
gradient at n = 6 (64 x 64, capacities large enough that nothing is truncated) against the dense oracle; the gradient
with respect to the mask's site tensors is checked against central differences of the FP64 oracle loss.
Tolerances: 1e-6 for single products, 2e-5 for one zip-up, 1e-4 for the loss and 1e-3 for gradients
(several FP32 passes)."""
import numpy as np
import pytest
import torch

import synth
from oracle import mps as OS
from oracle import optics as OO
from oracle import quantics as OQ

pytestmark = pytest.mark.gpu


def f64(psi):
    return [A.astype(np.complex128) for A in psi.to_numpy_sites()]


def dist(a, b):
    na, nb = OS.norm2(a), OS.norm2(b)
    ab = OS.overlap(a, b)
    return np.sqrt(max(na + nb - 2 * ab.real, 0.0) / nb)


@pytest.fixture(scope="module")
def eng(lib):
    # room for n = 6 with no truncation anywhere: zip-up intermediates reach bond 128, the residual
    # I - I_t is a direct sum of bond 192, the intensity product uses the field (bond 128) as operator
    return lib.Engine(n_sites=6, d=4, chi=192, w=128, dense=1 << 14)


@pytest.mark.parametrize("conj_b", [False, True])
def test_hadamard_matches_oracle(lib, eng, conj_b):
    a = synth.random_mps_sites([1, 4, 8, 8, 4, 1], 4, seed=501, decay=0.1)
    b = synth.random_mps_sites([1, 3, 6, 5, 2, 1], 4, seed=502, decay=0.1)
    out = lib.MPS(5, 4, 64)
    eng.hadamard(lib.MPS.from_numpy_sites(a, 16), lib.MPS.from_numpy_sites(b, 16), out, conj_b)
    ref = OS.hadamard_product(a, b, conj_b)
    assert out.bonds() == OS.bonds(ref)
    assert dist(f64(out), ref) < 1e-6


@pytest.mark.parametrize("conj_b", [False, True])
def test_hadamard_zipup_untruncated_matches_oracle(lib, eng, conj_b):
    psi = OS.right_canonicalize(synth.random_mps_sites([1, 4, 12, 12, 4, 1], 4, seed=503, decay=0.1))
    b = synth.random_mps_sites([1, 4, 5, 5, 3, 1], 4, seed=504, decay=0.1)
    g = lib.MPS.from_numpy_sites(psi, 64, "right")
    eng.hadamard_zipup(lib.MPS.from_numpy_sites(b, 16), g, 64, 1e-13, conj_b=conj_b)
    assert dist(f64(g), OS.hadamard_product(psi, b, conj_b)) < 2e-5


def test_overlap_grad_matches_brute_force(lib, eng):
    a = synth.random_mps_sites([1, 4, 6, 4, 1], 4, seed=505)
    b = synth.random_mps_sites([1, 3, 5, 3, 1], 4, seed=506)
    H = eng.overlap_grad(lib.MPS.from_numpy_sites(a, 8), lib.MPS.from_numpy_sites(b, 8)).cpu().numpy()
    for p, A in enumerate(a):
        k_, d_, m_ = A.shape
        ref = np.zeros_like(A)
        for k in range(k_):
            for s in range(d_):
                for m in range(m_):
                    unit = [x.copy() for x in a]
                    unit[p] = np.zeros_like(A)
                    unit[p][k, s, m] = 1.0
                    ref[k, s, m] = OS.overlap(unit, b)   # linear in conj(a_p): the derivative itself
        got = H[p, :k_, :, :m_].astype(np.complex128)
        assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref), p


def mask_problem(lib, eng):
    """n = 6 field, smooth phase mask and rectangle target as MPS (exact bonds), plus the problem."""
    from paper_2510_23089_gb300 import optics
    n, c = 6, 0.5
    E = synth.gaussian_beam_with_rectangles(n, seed=611, waist=0.2).astype(np.complex64)
    Em = lib.MPS(n, 4, 128)
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", Em, 128, 1e-14, stats=False)
    mx, my = synth.smooth_random_phase_mask_factors(n, seed=612, strength=0.5)
    X, Y = lib.MPS(n, 2, 32), lib.MPS(n, 2, 32)
    eng.encode(torch.from_numpy(mx.astype(np.complex64)).cuda(), n, "1d", X, 32, 1e-14, stats=False)
    eng.encode(torch.from_numpy(my.astype(np.complex64)).cuda(), n, "1d", Y, 32, 1e-14, stats=False)
    M = lib.MPS(n, 4, 64)
    eng.kron_interleave(X, Y, M)
    It = synth.rectangles_target(n, seed=613).astype(np.complex64)
    Itm = lib.MPS(n, 4, 64)
    eng.encode(torch.from_numpy(It).cuda(), n, "interleaved", Itm, 64, 1e-14, stats=False)
    prob = optics.IntensityLossProblem(eng, n, c, chi=128, cutoff=1e-13)
    dense = lambda psi: eng.to_dense(psi, "interleaved", n).cpu().numpy().astype(np.complex128)
    return prob, Em, M, Itm, dense(Em), dense(M), dense(Itm).real, c


def test_loss_and_field_gradient_match_dense_oracle(lib, eng):
    prob, Em, M, Itm, Ed, Md, Itd, c = mask_problem(lib, eng)
    loss, cache = prob.forward(Em, M, Itm)
    ref = OO.intensity_loss_dense(Ed, Md, Itd, c)
    assert abs(loss - ref) <= 1e-4 * ref
    G, H = prob.backward(Em, M, cache)
    Gd = eng.to_dense(G, "interleaved", 6).cpu().numpy().astype(np.complex128)
    Gref = OO.intensity_loss_grad_dense(Ed, Md, Itd, c)
    assert np.linalg.norm(Gd - Gref) <= 1e-3 * np.linalg.norm(Gref)


def test_site_gradient_matches_oracle_finite_differences(lib, eng):
    from paper_2510_23089_gb300 import optics
    prob, Em, M, Itm, Ed, Md, Itd, c = mask_problem(lib, eng)
    sites = M.sites.clone()
    x = sites.clone().requires_grad_(True)
    loss = optics.FresnelIntensityLoss.apply(x, prob, Em, M, Itm)
    loss.backward()
    grad = x.grad.cpu().numpy().astype(np.complex128)          # PyTorch convention: 2 dL/d conj(site)
    bonds = M.bonds()
    base = [A.astype(np.complex128) for A in M.to_numpy_sites()]

    def oracle_loss(ss):
        Mv = OQ.quantics_to_dense(OS.to_vector(ss), 6, "interleaved")
        return OO.intensity_loss_dense(Ed, Mv, Itd, c)

    h = 1e-6
    rng = np.random.default_rng(7)
    checked = 0
    for p in (0, 2, 3, 5):
        a, d, b = base[p].shape
        for _ in range(2):
            k, s, m = rng.integers(a), rng.integers(d), rng.integers(b)
            for unit in (1.0, 1j):
                sp = [A.copy() for A in base]
                sm = [A.copy() for A in base]
                sp[p][k, s, m] += h * unit
                sm[p][k, s, m] -= h * unit
                fd = (oracle_loss(sp) - oracle_loss(sm)) / (2 * h)
                pred = np.real(np.conj(grad[p, k, s, m]) * unit)
                assert abs(fd - pred) <= 1e-3 * np.abs(grad).max() + 1e-3 * abs(fd), (p, k, s, m, unit)
                checked += 1
    assert checked == 16 and bonds[0] == 1


# ----------------------------------------------------------------------------- adjoints at a truncated size

def truncated_case(lib, eng, chi):
    """n = 6 problem whose passes truncate (chi below the full bond 64); inputs built by the oracle side and
    uploaded, so both sides start from the same field, mask and target."""
    from paper_2510_23089_gb300 import optics
    from oracle import mpo as OM
    n, c = 6, 0.5
    E = synth.gaussian_beam_with_rectangles(n, seed=621, waist=0.2).astype(np.complex128)
    E_sites, _ = OS.tt_svd(OQ.dense_to_quantics(E, "interleaved"), n, 4, 64, 1e-14)
    mx, my = synth.smooth_random_phase_mask_factors(n, seed=622, strength=0.5)
    X, _ = OS.tt_svd(mx, n, 2, 64, 1e-14)
    Y, _ = OS.tt_svd(my, n, 2, 64, 1e-14)
    M_sites = OS.kron_interleave(X, Y)
    It = synth.rectangles_target(n, seed=623).astype(np.float64)
    Em = lib.MPS.from_numpy_sites(E_sites, 128, "left")
    M = lib.MPS.from_numpy_sites(M_sites, 64, "none")
    Itm = lib.MPS(n, 4, 64)
    eng.encode(torch.from_numpy(It.astype(np.complex64)).cuda(), n, "interleaved", Itm, 64, 1e-14, stats=False)
    Q = OM.qft_mpo_layers(n, 1e-12)
    ops = (Q, OM.dagger(Q), OM.phase_mpo(n, c, 1e-12))
    probs = {a: optics.IntensityLossProblem(eng, n, c, chi=chi, cutoff=1e-12, chi_intensity=128, adjoint=a)
             for a in ("frozen", "exact")}
    return probs, Em, M, Itm, E_sites, M_sites, OQ.dense_to_quantics(It, "interleaved"), ops, n


def test_frozen_adjoint_matches_oracle_frozen_gradient(lib, eng):
    from oracle import optics as OO
    chi = 12
    probs, Em, M, Itm, E_sites, M_sites, It, ops, n = truncated_case(lib, eng, chi)
    loss, cache = probs["frozen"].forward(Em, M, Itm)
    G, H = probs["frozen"].backward(Em, M, cache)
    L_o, G_o, _ = OO.frozen_loss_and_grad(E_sites, M_sites, It, n, ops, chi, 1e-12)
    got = eng.to_dense(G, "interleaved", n).cpu().numpy().astype(np.complex128)
    ref = OQ.quantics_to_dense(G_o, n, "interleaved")
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"frozen adjoint at chi {chi}: loss rel {abs(loss - L_o) / L_o:.2e}, gradient rel {err:.2e}")
    assert abs(loss - L_o) <= 1e-3 * L_o
    assert err <= 1e-3


def test_exact_adjoint_against_finite_differences_of_the_truncated_map(lib, eng):
    # the oracle recomputes every truncation for each perturbed mask: central differences of the truncated
    # forward map along single site entries, against the site gradient of the "exact" adjoint
    from oracle import optics as OO
    chi = 12
    probs, Em, M, Itm, E_sites, M_sites, It, ops, n = truncated_case(lib, eng, chi)
    sites = M.sites.clone()
    x = sites.clone().requires_grad_(True)
    from paper_2510_23089_gb300 import optics
    loss = optics.FresnelIntensityLoss.apply(x, probs["exact"], Em, M, Itm)
    loss.backward()
    grad = x.grad.cpu().numpy().astype(np.complex128)

    def oracle_loss(ms):
        L, _, _ = OO.frozen_loss_and_grad(E_sites, ms, It, n, ops, chi, 1e-12)
        return L

    base = [A.copy() for A in M_sites]
    rng = np.random.default_rng(11)
    h = 1e-6
    errs = []
    for p in (1, 3, 4):
        a, d, b = base[p].shape
        for _ in range(2):
            k, s, m = rng.integers(a), rng.integers(d), rng.integers(b)
            sp = [A.copy() for A in base]
            sm = [A.copy() for A in base]
            sp[p][k, s, m] += h
            sm[p][k, s, m] -= h
            fd = (oracle_loss(sp) - oracle_loss(sm)) / (2 * h)
            pred = np.real(grad[p, k, s, m])
            errs.append(abs(fd - pred) / np.abs(grad).max())
    print(f"exact adjoint vs finite differences of the truncated map (chi {chi}): max rel {max(errs):.2e}")
    assert max(errs) <= 1e-2
