"""Matrix product states in FP64: TT-SVD, canonical forms, truncation, overlaps.

Test infrastructure only (see the package docstring).

An MPS is a list of site tensors A[p] of shape (chi_{p-1}, d, chi_p) with
chi_0 = chi_N = 1, representing psi[s_1 .. s_N] = A[1][:, s_1, :] ... A[N][:, s_N, :]
(Sec. IV, MPS factorisation; App. A).

Truncation rule (the paper uses a relative ``cutoff`` without defining it, Sec.
VI.B.3): keep the smallest k >= 1 whose discarded weight sum_{i>=k} s_i^2 is at
most cutoff * sum_i s_i^2, then cap k at chi_max.
"""
from __future__ import annotations

import numpy as np


def keep_rank(s: np.ndarray, chi_max: int, cutoff: float) -> int:
    w = np.asarray(s, dtype=np.float64) ** 2
    total = w.sum()
    if total == 0.0:
        return 1
    tail = np.append(np.cumsum(w[::-1])[::-1], 0.0)   # tail[k] = sum_{i>=k} w_i
    k = int(np.argmax(tail <= cutoff * total))
    return max(1, min(k, chi_max))


def svd(M: np.ndarray):
    return np.linalg.svd(M, full_matrices=False)


def tt_svd(vec: np.ndarray, N: int, d: int, chi_max: int = 1 << 30, cutoff: float = 0.0):
    """Sequential truncated SVD, left to right (Sec. IV, Fig. MPS; App. A).

    At bond k the remainder is unfolded as (r_{k-1} d) x rest, factorised by
    SVD, the kept left singular vectors become site k and diag(s) V^dagger is
    carried to the next bond.  Returns (sites, eps) with eps[k] the discarded
    weight at bond k.  The result is left-canonical; its norm sits in the last
    site."""
    sites, eps = [], []
    M = np.asarray(vec, dtype=np.complex128).reshape(1, -1)
    r = 1
    for _ in range(N - 1):
        M = M.reshape(r * d, -1)
        U, s, Vh = svd(M)
        k = keep_rank(s, chi_max, cutoff)
        eps.append(float(np.sum(s[k:] ** 2)))
        sites.append(U[:, :k].reshape(r, d, k))
        M = s[:k, None] * Vh[:k]
        r = k
    sites.append(M.reshape(r, d, 1))
    return sites, eps


def to_vector(sites) -> np.ndarray:
    """Contract all sites into the flat vector (site 1 most significant)."""
    v = np.ones((1, 1), dtype=np.complex128)
    for A in sites:
        a, d, b = A.shape
        v = (v @ A.reshape(a, d * b)).reshape(-1, b)
    return v.reshape(-1)


def overlap(bra, ket) -> complex:
    """<bra|ket> by left transfer matrices."""
    E = np.ones((1, 1), dtype=np.complex128)
    for A, B in zip(bra, ket):
        E = np.einsum("ij,isk,jsl->kl", E, A.conj(), B)
    return complex(E[0, 0])


def norm2(sites) -> float:
    return float(overlap(sites, sites).real)


def amplitude(sites, digits) -> complex:
    v = np.ones((1, 1), dtype=np.complex128)
    for A, s in zip(sites, digits):
        v = v @ A[:, s, :]
    return complex(v[0, 0])


def bonds(sites):
    return [1] + [A.shape[2] for A in sites]


def left_canonicalize(sites):
    """QR sweep left to right: sites 1..N-1 become left isometries and the
    norm moves into site N (App. A, left Schmidt bases)."""
    out = [A.copy() for A in sites]
    for p in range(len(out) - 1):
        a, d, b = out[p].shape
        Q, R = np.linalg.qr(out[p].reshape(a * d, b))
        out[p] = Q.reshape(a, d, Q.shape[1])
        out[p + 1] = np.einsum("ij,jsk->isk", R, out[p + 1])
    return out


def right_canonicalize(sites):
    """LQ sweep right to left: sites 2..N become right isometries and the norm
    moves into site 1."""
    out = [A.copy() for A in sites]
    for p in range(len(out) - 1, 0, -1):
        a, d, b = out[p].shape
        Q, R = np.linalg.qr(out[p].reshape(a, d * b).conj().T)   # A^dagger = Q R  ->  A = R^dagger Q^dagger
        out[p] = Q.conj().T.reshape(Q.shape[1], d, b)
        out[p - 1] = np.einsum("isj,jk->isk", out[p - 1], R.conj().T)
    return out


def is_left_canonical(sites, tol=1e-10) -> bool:
    for A in sites[:-1]:
        a, d, b = A.shape
        M = A.reshape(a * d, b)
        if np.abs(M.conj().T @ M - np.eye(b)).max() > tol:
            return False
    return True


def is_right_canonical(sites, tol=1e-10) -> bool:
    for A in sites[1:]:
        a, d, b = A.shape
        M = A.reshape(a, d * b)
        if np.abs(M @ M.conj().T - np.eye(a)).max() > tol:
            return False
    return True


def truncate(sites, chi_max: int, cutoff: float):
    """Canonical SVD compression: left-canonicalise, then sweep right to left
    truncating every bond by the rule above.  Each truncation acts on a true
    Schmidt decomposition, so the discarded weights add up exactly to the
    squared error (Eckart-Young per bond).  Returns (right-canonical sites, eps)."""
    out = left_canonicalize(sites)
    eps = [0.0] * (len(out) - 1)
    for p in range(len(out) - 1, 0, -1):
        a, d, b = out[p].shape
        U, s, Vh = svd(out[p].reshape(a, d * b))
        k = keep_rank(s, chi_max, cutoff)
        eps[p - 1] = float(np.sum(s[k:] ** 2))
        out[p] = Vh[:k].reshape(k, d, b)
        out[p - 1] = np.einsum("isj,jk->isk", out[p - 1], U[:, :k] * s[None, :k])
    return out, eps


def schmidt_spectra(sites):
    """Schmidt values at every bond (gauge-invariant fingerprint of a state)."""
    out = left_canonicalize(sites)
    spectra = [None] * (len(out) - 1)
    for p in range(len(out) - 1, 0, -1):
        a, d, b = out[p].shape
        U, s, Vh = svd(out[p].reshape(a, d * b))
        spectra[p - 1] = s
        out[p] = Vh.reshape(-1, d, b)
        out[p - 1] = np.einsum("isj,jk->isk", out[p - 1], U * s[None, :])
    return spectra


def hadamard_product(A, B, conj_b: bool = False):
    """Elementwise product of two MPS in the same site basis: physical indices
    are contracted locally, bonds multiply (Sec. V, Eq. psf_eq, the local
    contraction written |phi> (.) |phi>^dagger)."""
    out = []
    for a, b in zip(A, B):
        if conj_b:
            b = b.conj()
        t = np.einsum("isj,ksl->iksjl", a, b)
        out.append(t.reshape(a.shape[0] * b.shape[0], a.shape[1], a.shape[2] * b.shape[2]))
    return out


def direct_sum(A, B):
    """MPS of the sum |A> + |B> (block-diagonal bonds; boundaries concatenated)."""
    N = len(A)
    if N == 1:
        return [A[0] + B[0]]
    out = []
    for p, (a, b) in enumerate(zip(A, B)):
        la, d, ra = a.shape
        lb, _, rb = b.shape
        if p == 0:
            t = np.concatenate([a, b], axis=2)
        elif p == N - 1:
            t = np.concatenate([a, b], axis=0)
        else:
            t = np.zeros((la + lb, d, ra + rb), dtype=np.complex128)
            t[:la, :, :ra] = a
            t[la:, :, ra:] = b
        out.append(t)
    return out


def kron_interleave(X, Y):
    """Interleaved d = 4 MPS of f(x) g(y) from 1-D MPS of f and g: site p holds
    mu_p = 2 x_p + y_p (Sec. III), so its tensor is the Kronecker product of the
    two 1-D site tensors with bonds multiplied."""
    out = []
    for a, b in zip(X, Y):
        t = np.einsum("isj,ktl->ikstjl", a, b)
        out.append(t.reshape(a.shape[0] * b.shape[0], 4, a.shape[2] * b.shape[2]))
    return out


def scale(sites, alpha):
    out = [A.copy() for A in sites]
    out[0] = out[0] * alpha
    return out


def mirror(sites):
    """Reverse the chain and swap each site's left/right bonds."""
    return [A.transpose(2, 1, 0).copy() for A in reversed(sites)]
