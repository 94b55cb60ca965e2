"""The mixed-precision path: the zip-up site contraction on the tcgen05 tensor cores (split BF16 operands,
FP32 accumulation in tensor memory), the truncation as in the FP32 path.  Checked through the C ABI against the
FP64 oracle within the mixed-path tolerance of 3e-3 relative L2 (on top of the truncation error), and against
the plain FP32 path, on tiles that span several 128 x 128 CTA tiles with ragged edges (bonds that are not
multiples of 64) and in both sweep orientations."""
import numpy as np
import pytest
import torch

import synth
from oracle import fresnel as OF
from oracle import mpo as OM
from oracle import mps as OS
from oracle import quantics as OQ

pytestmark = pytest.mark.gpu

TOL_MIXED = 3e-3


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.fixture(scope="module")
def eng(lib):
    return lib.Engine(n_sites=10, d=4, chi=128, w=16, dense=1 << 16)


@pytest.mark.parametrize("canon", ["right", "left"])
def test_mixed_untruncated_apply_equals_exact_product(eng, lib, canon):
    n = 5
    bonds = [1, 4, 16, 16, 4, 1]
    sites = synth.random_mps_sites(bonds, 4, seed=701)
    sites = OS.right_canonicalize(sites) if canon == "right" else OS.left_canonicalize(sites)
    Qo = OM.qft_mpo_layers(n, 1e-14)
    ref = OM.to_dense(OM.embed(Qo, "interleaved", 0, n)) @ OS.to_vector(sites)
    W = lib.MPO.from_numpy_cores(Qo, 16)
    out = {}
    for prec in ("mixed", "fp32"):
        psi = lib.MPS.from_numpy_sites(sites, 128, canon)
        eng.apply_mpo(W, 0, psi, 128, 1e-12, prec=prec)
        out[prec] = OS.to_vector(psi.to_numpy_sites())
    e_mixed, e_plain = rel(out["mixed"], ref), rel(out["fp32"], ref)
    print(f"untruncated apply ({canon}): mixed {e_mixed:.2e}, fp32 {e_plain:.2e}")
    assert e_mixed < TOL_MIXED
    assert e_mixed < 1e-4            # the split operands keep the product near FP32 rounding


def test_mixed_contraction_spans_several_tiles(eng, lib):
    # carry rows chi' * w = 96 * 8 > 64 (two CTA rows), columns d * chi = 4 * 100 > 128 (four CTA columns),
    # K = chi = 100 (two 64-wide chunks per half-segment, the second ragged)
    n = 6
    bonds = [1, 4, 16, 100, 16, 4, 1]
    sites = OS.right_canonicalize(synth.random_mps_sites(bonds, 4, seed=702, decay=0.05))
    Qo = OM.qft_mpo_layers(n, 1e-14)
    W = lib.MPO.from_numpy_cores(Qo, 16)
    res = {}
    for prec in ("mixed", "fp32"):
        psi = lib.MPS.from_numpy_sites(sites, 128, "right")
        st = eng.apply_mpo(W, 0, psi, 128, 1e-10, prec=prec)
        res[prec] = (psi, st)
    a, b = res["mixed"][0], res["fp32"][0]
    d2 = eng.norm2(a) + eng.norm2(b) - 2 * eng.overlap(b, a).real
    diff = np.sqrt(max(d2, 0.0) / eng.norm2(b))
    print(f"mixed vs fp32 after one pass over 6 sites (chi up to 100): {diff:.2e}")
    assert diff < TOL_MIXED
    assert abs(res["mixed"][1].discarded - res["fp32"][1].discarded) <= 1e-6 * OS.norm2(sites)


def test_mixed_fresnel_step_matches_dense(eng, lib):
    n, c = 6, 0.4
    E = synth.gaussian_beam_with_rectangles(n, seed=703, waist=0.2)
    psi = lib.MPS(n, 4, 64)
    eng.encode(torch.from_numpy(E).cuda(), n, "interleaved", psi, 64, 1e-12)
    Q = eng.build_qft_mpo(n, False, 1e-13)
    Qd = eng.mpo_dagger(Q)
    D = eng.build_phase_mpo(n, c, 1e-13, w_cap=32)
    st = eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, 64, 1e-12, prec="mixed")
    got = eng.to_dense(psi, "interleaved", n).cpu().numpy()
    ref = OF.fresnel_dense(E.astype(np.complex128), c)
    err = rel(got, ref)
    print(f"mixed Fresnel step n=6: rel {err:.2e}")
    assert err < TOL_MIXED + np.sqrt(st.discarded / np.linalg.norm(E.astype(np.complex128)) ** 2)
    eng.check()


def test_mixed_step_at_2p16_matches_oracle(lib):
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    n, chi, cut = 16, 128, 1e-10
    c = 25.3 / (1 << n)
    psi = bench.build_state_gpu(lib, n, chi, cut)
    eng_b = lib.Engine(n_sites=n, d=4, chi=16, w=16, dense=0)
    Q = eng_b.build_qft_mpo(n, False, 1e-12)
    Qd = eng_b.mpo_dagger(Q)
    D = eng_b.build_phase_mpo(n, c, 1e-12, w_cap=16)
    eng = lib.Engine(n_sites=n, d=4, chi=chi, w=16, dense=0)
    n2 = eng.norm2(psi)
    st = eng.fresnel_step(psi, "interleaved", Q, Qd, D, 1, chi, cut, prec="mixed")
    sites = bench.oracle_state(n, chi, cut)
    ops = (OM.qft_mpo_layers(n, 1e-12), None, OM.phase_mpo(n, c, 1e-12))
    ops = (ops[0], OM.dagger(ops[0]), ops[2])
    out, _, disc = OF.fresnel_mps(sites, "interleaved", n, c, chi, cut, canon="right", ops=ops)
    ref = lib.MPS.from_numpy_sites(out, chi)
    d2 = eng.norm2(psi) + eng.norm2(ref) - 2 * eng.overlap(ref, psi).real
    err = np.sqrt(max(d2, 0.0) / eng.norm2(ref))
    print(f"mixed step 2^16: rel {err:.2e}, eps {st.discarded / n2:.2e} vs {disc / n2:.2e}")
    assert err < TOL_MIXED + np.sqrt(st.discarded / n2) + np.sqrt(disc / n2)
