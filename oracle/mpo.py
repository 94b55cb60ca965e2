"""Matrix product operators in FP64: QFT, quadratic phase, Hadamard, embedding.

Test infrastructure only (see the package docstring).

An MPO is a list of cores W[p] of shape (w_{p-1}, d_out, d_in, w_p) with
O[s'_1..s'_N, s_1..s_N] = W[1][:, s'_1, s_1, :] ... W[N][:, s'_N, s_N, :]
(Sec. V, Fig. fig_mpo).  Per-axis operators act on n sites of d = 2.

QFT convention (the paper only says "Fourier transform" and cites a finite-rank
QFT MPO, Sec. V): unitary kernel exp(+2 pi i j k / L) / sqrt(L), no final
bit-reversal swaps, so output site p carries frequency bit k_{n+1-p}.  The
swap-free operator is the one with a small MPO rank; the Fourier-space state
is therefore in bit-reversed frequency order, and the phase diagonal is built
in that order so that U_QFT^dagger brings the field back to natural order.
"""
from __future__ import annotations

import numpy as np

from . import mps as _mps
from .quantics import bit_reverse

H1 = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)


# ----------------------------------------------------------------------------- dense operators

def dft_matrix(L: int) -> np.ndarray:
    """Unitary DFT F[k, j] = exp(+2 pi i j k / L) / sqrt(L), written out."""
    j = np.arange(L)
    return np.exp(2j * np.pi * np.outer(j, j) / L) / np.sqrt(L)


def qft_noswap_dense(n: int) -> np.ndarray:
    """Swap-free QFT as a matrix on site-ordered indices: row rev(k), column j."""
    L = 1 << n
    F = dft_matrix(L)
    Q = np.empty_like(F)
    for k in range(L):
        Q[bit_reverse(k, n)] = F[k]
    return Q


def fftfreq_int(L: int) -> np.ndarray:
    """Signed integer frequency k_f of DFT bin k: k for k < L/2, else k - L."""
    k = np.arange(L)
    return np.where(k < L // 2, k, k - L)


def phase_vector(n: int, c: float, bit_reversed: bool = True) -> np.ndarray:
    """Fresnel transfer function on the grid, exp(-i pi c k_f^2 / L)
    (Sec. VI.A, T_z(f) = exp(-i pi lambda z f^2) with f = k_f / (L dx) and
    c = lambda z / (L dx^2)).  Indexed by the site-ordered flat index: entry
    idx holds the phase of frequency rev(idx) when ``bit_reversed``."""
    L = 1 << n
    kf = fftfreq_int(L).astype(np.float64)
    D = np.exp(-1j * np.pi * c * kf ** 2 / L)
    if not bit_reversed:
        return D
    out = np.empty_like(D)
    for idx in range(L):
        out[idx] = D[bit_reverse(idx, n)]
    return out


# ----------------------------------------------------------------------------- MPO <-> dense

def to_dense(W) -> np.ndarray:
    """Contract an MPO into its (prod d_out) x (prod d_in) matrix."""
    M = np.ones((1, 1, 1), dtype=np.complex128)      # (rows, cols, bond)
    for core in W:
        a, do, di, b = core.shape
        M = np.einsum("rca,atsb->rtcsb", M, core)
        R, _, C, _, _ = M.shape
        M = M.reshape(R * do, C * di, b)
    return M[:, :, 0]


def operator_tt_svd(O: np.ndarray, n: int, chi_max: int = 1 << 30, cutoff: float = 0.0):
    """MPO of a dense 2^n x 2^n operator by TT-SVD with interleaved (out, in)
    legs (Sec. VI.A, Fig. MPO_construction)."""
    t = O.reshape((2,) * n + (2,) * n)
    order = [ax for p in range(n) for ax in (p, n + p)]
    v = t.transpose(order).reshape(-1)
    sites, _ = _mps.tt_svd(v, n, 4, chi_max, cutoff)
    return [A.reshape(A.shape[0], 2, 2, A.shape[2]) for A in sites]


def as_mps(W):
    return [c.reshape(c.shape[0], c.shape[1] * c.shape[2], c.shape[3]) for c in W]


def from_mps(sites, d_out=2, d_in=2):
    return [A.reshape(A.shape[0], d_out, d_in, A.shape[2]) for A in sites]


def compress(W, cutoff: float, chi_max: int = 1 << 30):
    """Canonical SVD compression of an MPO viewed as an MPS with d = d_out d_in."""
    do, di = W[0].shape[1], W[0].shape[2]
    sites, _ = _mps.truncate(as_mps(W), chi_max, cutoff)
    return from_mps(sites, do, di)


def product(A, B):
    """Exact MPO product A . B (B applied first); bonds multiply."""
    out = []
    for a, b in zip(A, B):
        t = np.einsum("iuvj,kvsl->ikusjl", a, b)
        out.append(t.reshape(a.shape[0] * b.shape[0], a.shape[1], b.shape[2], a.shape[3] * b.shape[3]))
    return out


def bonds(W):
    return [1] + [c.shape[3] for c in W]


def dagger(W):
    """Hermitian conjugate: W^dagger[a, s', s, b] = conj(W[a, s, s', b])."""
    return [c.transpose(0, 2, 1, 3).conj().copy() for c in W]


def identity(n: int, d: int = 2):
    return [np.eye(d, dtype=np.complex128).reshape(1, d, d, 1) for _ in range(n)]


# ----------------------------------------------------------------------------- builders

def qft_layer(n: int, j: int):
    """Layer j (0-based) of the swap-free QFT circuit as an MPO of bond <= 2:
    H on qubit j, then controlled phases exp(i pi b s / 2^(k-j)) between
    qubit j (post-H bit b, carried on the bond) and every qubit k > j."""
    cores = []
    for p in range(n):
        if p < j:
            cores.append(np.eye(2, dtype=np.complex128).reshape(1, 2, 2, 1))
        elif p == j:
            wr = 2 if j < n - 1 else 1
            c = np.zeros((1, 2, 2, wr), dtype=np.complex128)
            for b in range(2):
                for s in range(2):
                    c[0, b, s, b if wr == 2 else 0] = H1[b, s]
            cores.append(c)
        else:
            wr = 2 if p < n - 1 else 1
            c = np.zeros((2, 2, 2, wr), dtype=np.complex128)
            for b in range(2):
                for s in range(2):
                    c[b, s, s, b if wr == 2 else 0] = np.exp(1j * np.pi * b * s / 2 ** (p - j))
            cores.append(c)
    return cores


def qft_mpo_layers(n: int, cutoff: float = 1e-12, chi_max: int = 1 << 30):
    """Swap-free QFT MPO as the product of its n circuit layers, compressed
    after every layer (works for any n)."""
    W = identity(n)
    for j in range(n):
        W = compress(product(qft_layer(n, j), W), cutoff, chi_max)
    return W


def qft_mpo_dense(n: int, cutoff: float = 1e-12, chi_max: int = 1 << 30):
    """Swap-free QFT MPO by operator TT-SVD of the dense matrix (n <= 12)."""
    return operator_tt_svd(qft_noswap_dense(n), n, chi_max, cutoff)


def diagonal_mpo(vec: np.ndarray, n: int, cutoff: float = 1e-12, chi_max: int = 1 << 30):
    """Diagonal MPO of a length-2^n vector: TT-SVD (d = 2), brought to right-canonical form (the form in which
    every operator here is delivered: the zip-up truncation depends on the gauge of the operator it applies,
    and right-canonical forms differ only by unitary bond transformations, to which it is blind), then
    delta(s', s)."""
    sites, _ = _mps.tt_svd(vec, n, 2, chi_max, cutoff)
    sites = _mps.right_canonicalize(sites)
    out = []
    for A in sites:
        a, _, b = A.shape
        c = np.zeros((a, 2, 2, b), dtype=np.complex128)
        c[:, 0, 0, :] = A[:, 0, :]
        c[:, 1, 1, :] = A[:, 1, :]
        out.append(c)
    return out


def phase_mpo(n: int, c: float, cutoff: float = 1e-12, chi_max: int = 1 << 30):
    """Quadratic-phase (Fresnel) diagonal MPO in bit-reversed frequency order."""
    return diagonal_mpo(phase_vector(n, c, True), n, cutoff, chi_max)


def hadamard_mpo(n: int):
    """H_1^{(x) n}: rank-1 MPO (Sec. V, Eq. hadamard)."""
    return [H1.reshape(1, 2, 2, 1).copy() for _ in range(n)]


def hilbert_diag_mpo(n: int):
    """-i Z_n as a bond-1 diagonal MPO (Sec. VI.C): Z on the last site, which in
    the swap-free Fourier order carries the most significant frequency bit."""
    W = identity(n)
    W[-1] = np.diag([1.0, -1.0]).astype(np.complex128).reshape(1, 2, 2, 1)
    W[0] = W[0] * (-1j)
    return W


# ----------------------------------------------------------------------------- embedding

def embed(W, layout: str, axis: int, n: int):
    """Per-axis MPO (n sites, d = 2) as an operator on the full state.

    interleaved: site p index mu = 2 x + y; axis 0 acts on the x bit (high),
                 axis 1 on the y bit (low), identity on the other bit.
    serial:      axis 0 acts on sites 1..n, axis 1 on sites n+1..2n, identity
                 (bond 1) elsewhere.
    1d:          the MPO itself."""
    I2 = np.eye(2, dtype=np.complex128)
    if layout == "1d":
        return [c.copy() for c in W]
    if layout == "interleaved":
        out = []
        for c in W:
            a, _, _, b = c.shape
            if axis == 0:
                t = np.einsum("atsb,uv->atusvb", c, I2)
            else:
                t = np.einsum("uv,atsb->autvsb", I2, c)
            out.append(t.reshape(a, 4, 4, b))
        return out
    if layout == "serial":
        ident = identity(n)
        return ([c.copy() for c in W] + ident) if axis == 0 else (ident + [c.copy() for c in W])
    raise ValueError(layout)


def mirror(W):
    """Reverse the chain and swap each core's left/right bonds."""
    return [c.transpose(3, 1, 2, 0).copy() for c in reversed(W)]


# ----------------------------------------------------------------------------- lattice dispersion (Sec. VI.B)
#
# U(t) = sum_s exp(-i t eps(s)) |s><s| with eps(s) = cos(2 pi x_s), x_s = k / L the frequency of the basis
# state (Sec. VI.B.2-4: the tight-binding dispersion of the discretised free particle).  Both builders return
# the diagonal MPO in the site order of the swap-free QFT output (site q carries bit q of k) when
# ``bit_reversed``, else in natural order (site q carries bit n-1-q).

def lattice_diagonal(n: int, t: float, bit_reversed: bool = True) -> np.ndarray:
    """The exact diagonal exp(-i t cos(2 pi k / L)), indexed by the site-ordered flat index."""
    L = 1 << n
    k = np.arange(L)
    D = np.exp(-1j * t * np.cos(2 * np.pi * k / L))
    if not bit_reversed:
        return D
    return np.array([D[bit_reverse(idx, n)] for idx in range(L)])


def bessel_mpo(n: int, t: float, p_max: int, bit_reversed: bool = True):
    """Closed-form diagonal MPO of U(t) (Sec. VI.B.4): the Jacobi-Anger expansion
    exp(-i t cos theta) = sum_p (-i)^p J_p(t) exp(i p theta), truncated to |p| <= p_max, with theta = 2 pi k / L
    = sum over bits; the core of site q is diagonal in the bond index p and carries exp(i p theta_q s_q), the
    left boundary vector is (-i)^p J_p(t) and the right one all ones.  Bond 2 p_max + 1."""
    from scipy.special import jv
    ps = np.arange(-p_max, p_max + 1)
    chi = len(ps)
    vl = np.array([(-1j) ** int(p) * jv(int(p), t) for p in ps])
    cores = []
    for q in range(n):
        theta = 2 * np.pi * (2.0 ** q) / (1 << n) if bit_reversed else 2 * np.pi / 2.0 ** (q + 1)
        c = np.zeros((chi, 2, 2, chi), dtype=np.complex128)
        for i, p in enumerate(ps):
            for s in (0, 1):
                c[i, s, s, i] = np.exp(1j * p * theta * s)
        cores.append(c)
    cores[0] = np.einsum("p,pstq->stq", vl, cores[0])[None]     # left boundary vector
    cores[-1] = cores[-1].sum(axis=3)[..., None]                 # right boundary vector of ones
    return cores


def walsh_coefficients(eps: np.ndarray) -> np.ndarray:
    """c_S = 2^-n sum_s eps(s) (-1)^popcount(S & s) (Sec. VI.B.3, Eq. coeff_trace), by the fast Walsh-Hadamard
    butterflies written out (bit b of S pairs with bit b of s)."""
    v = np.array(eps, dtype=np.float64).copy()
    N = len(v)
    h = 1
    while h < N:
        for i in range(0, N, 2 * h):
            a = v[i:i + h].copy()
            b = v[i + h:i + 2 * h].copy()
            v[i:i + h] = a + b
            v[i + h:i + 2 * h] = a - b
        h *= 2
    return v / N


def pauliz_mpo(n: int, t: float, gate_cutoff: float, cutoff: float = 1e-12, bit_reversed: bool = True):
    """Diagonal MPO of the Pauli-Z circuit (Sec. VI.B.3, Eq. U-product_1): the product over strings with
    |c_S| >= gate_cutoff of cos(t c_S) I - i sin(t c_S) P_S, times the global phase exp(-i t c_0).  The gates
    commute and each is diagonal, so the product is diag(exp(-i t H_trunc(k))) with H_trunc the kept Walsh
    expansion; its diagonal is compressed by TT-SVD at ``cutoff``."""
    L = 1 << n
    k = np.arange(L)
    c = walsh_coefficients(np.cos(2 * np.pi * k / L))
    keep = np.abs(c) >= gate_cutoff
    keep[0] = True
    ct = np.where(keep, c, 0.0)
    # H_trunc(k) = sum_S c_S (-1)^popcount(S & k): the same butterflies, unscaled
    H = walsh_coefficients(ct) * L
    D = np.exp(-1j * t * H)
    if bit_reversed:
        D = np.array([D[bit_reverse(idx, n)] for idx in range(L)])
    return diagonal_mpo(D, n, cutoff)


def diag_of(W) -> np.ndarray:
    """Diagonal of a diagonal MPO, by site-ordered flat index."""
    return np.diag(to_dense(W)).copy()
