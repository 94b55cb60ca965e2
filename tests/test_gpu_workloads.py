"""Parity of the CUDA path with the FP64 oracle at the sizes of the benchmark workloads.

* 1024 x 1024 wavefront (n = 10 interleaved sites, chi = 64, c = 2.048, Gaussian beam through random
  rectangles): TT-SVD encode and one Fresnel step, dense comparison with the oracle's zip-up step.
* 2^16 x 2^16 wavefront (n = 16, chi = 128, lambda z / dx^2 = 25.3, the separable rank-8 field): one and three
  Fresnel steps from the same recipe on both sides, compared without densifying through qtn_overlap
  (||a - b||^2 = |a|^2 + |b|^2 - 2 Re <a|b>, FP64 accumulation), and point amplitudes through
  qtn_amplitudes.
* 2^16 x 2^16 Gaussian beam: one step against the textbook closed form of a Gaussian under the Fresnel
  transfer function, sampled by qtn_amplitudes (P9; aliasing and wrap-around terms are below 1e-10 here).

Tolerance (FP32 path): relative L2 within 1e-5 + sqrt(eps_gpu) + sqrt(eps_orc), eps the relative
discarded weights each side reports; discarded weights agree within 1e-6 relative.  Each local discarded
weight of a zip-up is part of the weight of the two-site matrix it is taken from, and an FP32 factorisation
resolves it to 1e-6 of that matrix's weight (the Eckart-Young check of the single factorisation); the zip-up's
environments are not isometric, so those weights can exceed |psi|^2 many times (the 1024^2 step at chi = 64
factorises matrices of up to ~60 |psi|^2).  The sums are compared within 1e-6 of |psi|^2 plus the weights of
the oracle's factorised matrices."""
import os
import sys

import numpy as np
import pytest
import torch

import synth
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS
from oracle import quantics as OQ

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402  (the workload recipes: build_state_gpu / oracle_state)

pytestmark = pytest.mark.gpu

LZ = 25.3


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def digits_of(a, b, n):
    """Interleaved site digits mu_p = 2 x_p + y_p of pixel (a, b), most significant bit first."""
    return [2 * ((a >> (n - 1 - p)) & 1) + ((b >> (n - 1 - p)) & 1) for p in range(n)]


def test_fresnel_step_1024(lib):
    n, chi, c, cut = 10, 64, 2.048, 1e-10
    E = synth.gaussian_beam_with_rectangles(n)
    E64 = E.astype(np.complex128)
    n2 = float(np.linalg.norm(E64) ** 2)
    # zip-up bonds near the chain end may exceed the exact Schmidt rank: room for the dense contraction
    eng = lib.Engine(n_sites=n, d=4, chi=chi, w=32, dense=1 << (2 * n + 4))
    psi = lib.MPS(n, 4, chi)
    st_e = eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, chi, cut)
    Q = eng.build_qft_mpo(n, False, 1e-12)
    Qd = eng.mpo_dagger(Q)
    D = eng.build_phase_mpo(n, c, 1e-12, w_cap=32)
    st = eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, chi, cut)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()

    sites, eps_e = OS.tt_svd(OQ.dense_to_quantics(E64, "interleaved"), n, 4, chi, cut)
    ops = OF.step_operators(n, c, qft=OM.qft_mpo_layers(n, 1e-12), phase_cutoff=1e-12)
    totals = []
    out, canon, disc = OF.fresnel_mps(sites, "interleaved", n, c, chi, cut, canon="left", ops=ops, totals=totals)
    ref = OQ.quantics_to_dense(OS.to_vector(out), n, "interleaved")
    eg = (st_e.discarded + st.discarded) / n2
    eo = (sum(eps_e) + disc) / n2
    err = rel(got, ref)
    print(f"n=10 step: rel {err:.3e} eps_gpu {eg:.2e} eps_orc {eo:.2e} bonds {psi.bonds()} vs {OS.bonds(out)}")
    assert err <= 1e-5 + np.sqrt(eg) + np.sqrt(eo)
    assert abs(st_e.discarded - sum(eps_e)) <= 1e-6 * n2
    print(f"n=10 step: discarded gpu {st.discarded:.6f} oracle {disc:.6f}, factorised weight {sum(totals):.1f}")
    assert abs(st.discarded - disc) <= 1e-6 * (n2 + sum(totals))
    # against the exact dense propagation (matrix DFTs): the truncated step stays within its own budget
    exact = OF.fresnel_dense(E64, c)
    print(f"n=10 step vs exact dense: gpu {rel(got, exact):.3e}, oracle {rel(ref, exact):.3e}")


def test_encode_4096_matches_oracle(lib):
    # the 4096 x 4096 field of the mask-learning workload (n = 12 interleaved sites, chi = 32, cutoff 1e-10):
    # the first unfoldings are 4 x 4^11 and 16 x 4^10 (long, HBM-streamed Gram products)
    n, chi, cut = 12, 32, 1e-10
    E = synth.gaussian_beam_with_rectangles(n, seed=7001, waist=0.1)
    E64 = E.astype(np.complex128)
    n2 = float(np.linalg.norm(E64) ** 2)
    # room for the read-out: every intermediate 4^p x bond[p] of the dense contraction fits the buffers
    eng = lib.Engine(n_sites=n, d=4, chi=64, w=32, dense=1 << (2 * n + 2))
    psi = lib.MPS(n, 4, chi)
    st = eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, chi, cut)
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    sites, eps = OS.tt_svd(OQ.dense_to_quantics(E64, "interleaved"), n, 4, chi, cut)
    ref = OQ.quantics_to_dense(OS.to_vector(sites), n, "interleaved")
    err = rel(got, ref)
    print(f"4096^2 encode: rel {err:.3e} eps_gpu {st.discarded / n2:.2e} eps_orc {sum(eps) / n2:.2e} "
          f"bonds {psi.bonds()} vs {OS.bonds(sites)}")
    assert max(abs(a - b) for a, b in zip(psi.bonds(), OS.bonds(sites))) <= 1
    assert err <= 1e-5 + np.sqrt(st.discarded / n2) + np.sqrt(sum(eps) / n2)
    assert abs(st.discarded - sum(eps)) <= 1e-6 * n2


@pytest.fixture(scope="module")
def n16(lib):
    n, chi, cut = 16, 128, 1e-10
    c = LZ / (1 << n)
    psi = bench.build_state_gpu(lib, n, chi, cut)
    eng_b = lib.Engine(n_sites=n, d=4, chi=16, w=16, dense=0)
    Q = eng_b.build_qft_mpo(n, False, 1e-12, w_cap=16)
    Qd = eng_b.mpo_dagger(Q)
    eng_p = lib.Engine(n_sites=n, d=2, chi=16, w=2, dense=1 << n)
    D = eng_p.build_phase_mpo(n, c, 1e-12, w_cap=16)
    eng = lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=1 << 16)
    sites = bench.oracle_state(n, chi, cut)
    ops = (OM.qft_mpo_layers(n, 1e-12), None, OM.phase_mpo(n, c, 1e-12))
    ops = (ops[0], OM.dagger(ops[0]), ops[2])
    return dict(n=n, chi=chi, cut=cut, c=c, psi=psi, Q=Q, Qd=Qd, D=D, eng=eng, sites=sites, ops=ops)


def overlap_rel(eng, lib, psi, sites, chi):
    """||psi - ref|| / ||ref|| by overlaps (never densified), ref the oracle's sites in complex64."""
    ref = lib.MPS.from_numpy_sites(sites, chi)
    a2, b2 = eng.norm2(psi), eng.norm2(ref)
    ab = eng.overlap(ref, psi)
    return np.sqrt(max(a2 + b2 - 2 * ab.real, 0.0) / b2), a2, b2


def test_fresnel_steps_2p16_match_oracle(lib, n16):
    eng, psi, chi = n16["eng"], n16["psi"], n16["chi"]
    n2 = eng.norm2(psi)
    sites, canon = n16["sites"], "right"
    eps_g = eps_o = 0.0
    for step in range(3):
        st = eng.fresnel_step(psi, "interleaved", n16["Q"], n16["Qd"], n16["D"], 1, chi, n16["cut"])
        sites, canon, disc = OF.fresnel_mps(sites, "interleaved", n16["n"], n16["c"], chi, n16["cut"], canon=canon,
                                            n_steps=1, ops=n16["ops"])
        eps_g += st.discarded / n2
        eps_o += disc / n2
        err, a2, b2 = overlap_rel(eng, lib, psi, sites, chi)
        print(f"2^16 after {step + 1} step(s): rel {err:.3e} eps_gpu {eps_g:.2e} eps_orc {eps_o:.2e} "
              f"norm2 ratio {a2 / b2 - 1:.2e} bonds {psi.bonds()} vs {OS.bonds(sites)}")
        assert err <= 1e-5 + np.sqrt(eps_g) + np.sqrt(eps_o)
        assert abs(st.discarded - disc) <= 1e-6 * n2                # this step's relative discarded weight
    # point amplitudes of the GPU state, read by qtn_amplitudes, against the oracle's state at seeded pixels
    rng = np.random.default_rng(17)
    L = 1 << n16["n"]
    ab = rng.integers(int(0.35 * L), int(0.65 * L), size=(256, 2))
    dig = np.array([digits_of(int(a), int(b), n16["n"]) for a, b in ab], dtype=np.int32)
    got = eng.amplitudes(psi, torch.from_numpy(dig)).cpu().numpy()
    ref = np.array([OS.amplitude(sites, list(d)) for d in dig])
    # and against the amplitudes of the GPU's own sites contracted by the oracle (the read-out kernel alone)
    own = np.array([OS.amplitude(psi.to_numpy_sites(), list(d)) for d in dig])
    assert np.abs(got - own).max() <= 1e-5 * np.abs(own).max()
    print(f"2^16 amplitudes: sampled rel L2 vs oracle {rel(got, ref):.3e}")
    assert rel(got, ref) <= 1e-4 + 3 * (np.sqrt(eps_g) + np.sqrt(eps_o))


def test_gaussian_beam_2p16_closed_form(lib):
    n, chi, cut = 16, 128, 1e-10
    L = 1 << n
    c = LZ / L
    w = 0.1 * L                                                  # waist in pixels
    u = np.arange(L) + 0.5 - L / 2
    g = np.exp(-(u / w) ** 2)
    eng = lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=1 << n)
    X = lib.MPS(n, 2, 32)
    st_x = eng.encode(torch.from_numpy(g.astype(np.complex64)).cuda(), n, "1d", X, 32, 1e-12)
    psi = lib.MPS(n, 4, chi)
    eng.kron_interleave(X, X, psi)
    eng.truncate(psi, chi, 1e-13)
    Q = eng.build_qft_mpo(n, False, 1e-12, w_cap=16)
    Qd = eng.mpo_dagger(Q)
    eng_p = lib.Engine(n_sites=n, d=2, chi=16, w=2, dense=1 << n)
    D = eng_p.build_phase_mpo(n, c, 1e-12, w_cap=16)
    n2 = eng.norm2(psi)
    st = eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, chi, cut)
    rng = np.random.default_rng(23)
    ab = rng.integers(int(L / 2 - 2 * w), int(L / 2 + 2 * w), size=(512, 2))
    dig = np.array([digits_of(int(a), int(b), n) for a, b in ab], dtype=np.int32)
    got = eng.amplitudes(psi, torch.from_numpy(dig)).cpu().numpy()
    gz = OF.gaussian_closed_form(u, w, c * L)
    ref = gz[ab[:, 0]] * gz[ab[:, 1]]
    eps = st.discarded / n2 + 2 * st_x.discarded / float((g ** 2).sum())
    err = rel(got, ref)
    print(f"2^16 Gaussian closed form: sampled rel L2 {err:.3e}, eps {eps:.2e}, bonds {psi.bonds()}")
    assert err <= 1e-5 + np.sqrt(eps)
