"""MPO x MPS application in FP64 (Sec. V, Fig. fig_mpo; cost O(n chi_1^2 chi_2^2)).

Test infrastructure only (see the package docstring).

The paper applies operators with ITensor's ``apply`` without naming the
algorithm; this oracle implements the zip-up contraction the hot path uses:

  left-to-right (input right-canonical): a carry C[x, a, j] (new bond x, MPO
  bond a, old bond j) starts as the 1x1x1 identity.  At site p

      T[x, t, b, k] = sum_{a, j, s} C[x, a, j] A_p[j, s, k] W_p[a, t, s, b]

  is unfolded as (x t) x (b k) and factorised by SVD; the kept left singular
  vectors become the new site p and diag(s) V^dagger (reshaped (r, b, k)) the
  next carry.  At the last site T itself is the new site.  The output is
  left-canonical.

  right-to-left (input left-canonical) is the same sweep on the mirrored chain
  (sites reversed, left and right bonds swapped); its output is right-canonical.

It also provides the exact product (bonds multiply) and a dense reference.
"""
from __future__ import annotations

import numpy as np

from . import mps as _mps
from . import mpo as _mpo


def zipup_lr(W, A, chi_max: int, cutoff: float, totals=None):
    """Left-to-right zip-up; when `totals` is a list, the squared Frobenius norm of every factorised
    two-site matrix is appended to it (the weight each local discarded weight is a part of)."""
    N = len(A)
    C = np.ones((1, 1, 1), dtype=np.complex128)
    out, eps = [], []
    for p in range(N):
        T = np.einsum("xaj,jsk,atsb->xtbk", C, A[p], W[p])
        x, t, b, k = T.shape
        if p == N - 1:
            out.append(T.reshape(x, t, b * k))
            break
        U, s, Vh = _mps.svd(T.reshape(x * t, b * k))
        r = _mps.keep_rank(s, chi_max, cutoff)
        eps.append(float(np.sum(s[r:] ** 2)))
        if totals is not None:
            totals.append(float(np.sum(s ** 2)))
        out.append(U[:, :r].reshape(x, t, r))
        C = (s[:r, None] * Vh[:r]).reshape(r, b, k)
    return out, eps


def zipup(W, A, chi_max: int, cutoff: float, direction: str, totals=None):
    """Zip-up in the given direction ('lr' needs a right-canonical input, 'rl'
    a left-canonical one).  Returns (sites, eps) with eps in bond order."""
    if direction == "lr":
        return zipup_lr(W, A, chi_max, cutoff, totals)
    if direction == "rl":
        out, eps = zipup_lr(_mpo.mirror(W), _mps.mirror(A), chi_max, cutoff, totals)
        return _mps.mirror(out), eps[::-1]
    raise ValueError(direction)


def apply_exact(W, A):
    """Exact MPO x MPS product, bond w*chi (no truncation)."""
    out = []
    for c, a in zip(W, A):
        t = np.einsum("atsb,isj->aitbj", c, a)
        out.append(t.reshape(c.shape[0] * a.shape[0], c.shape[1], c.shape[3] * a.shape[2]))
    return out


def apply_naive(W, A, chi_max: int, cutoff: float):
    """Exact product followed by canonical SVD compression (optimal sequential
    truncation; a bound for the zip-up result)."""
    return _mps.truncate(apply_exact(W, A), chi_max, cutoff)


def apply_dense(W, vec: np.ndarray) -> np.ndarray:
    return _mpo.to_dense(W) @ vec
