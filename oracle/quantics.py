"""Quantics index maps (Sec. III, quantics representation).

Test infrastructure only (see the package docstring).

A pixel coordinate a in [0, 2^n) is split into bits a = sum_p x_p 2^(n-p),
x_1 the most significant ("coarse features in high-order qubits", Sec. III;
the same weights as x_s = sum_j s_j 2^-j in Sec. VI.B.2).  Sites are listed
most-significant first, so the flat index of a quantics tensor is its
row-major index.

Layouts:
  * ``serial``      2n sites of d = 2: (x_1 .. x_n, y_1 .. y_n)  -> flat = a*2^n + b
  * ``interleaved`` n sites of d = 4:  mu_p = (x_p y_p)_2 = 2 x_p + y_p
  * ``1d``          n sites of d = 2 for a single axis.
"""
from __future__ import annotations

import numpy as np


def n_sites(n: int, layout: str) -> int:
    return {"serial": 2 * n, "interleaved": n, "1d": n}[layout]


def phys_dim(layout: str) -> int:
    return {"serial": 2, "interleaved": 4, "1d": 2}[layout]


def dense_to_quantics(E: np.ndarray, layout: str) -> np.ndarray:
    """Flat quantics vector (site 1 most significant) of a 2^n x 2^n field E[a, b]
    (row a = x, column b = y), or of a length-2^n vector for ``1d``."""
    E = np.asarray(E)
    if layout == "1d":
        return E.reshape(-1).copy()
    L = E.shape[0]
    n = L.bit_length() - 1
    if layout == "serial":
        return E.reshape(-1).copy()
    if layout == "interleaved":
        t = E.reshape((2,) * n + (2,) * n)              # axes x_1..x_n, y_1..y_n
        order = [ax for p in range(n) for ax in (p, n + p)]  # x_1, y_1, x_2, y_2, ...
        return t.transpose(order).reshape(-1).copy()
    raise ValueError(layout)


def quantics_to_dense(v: np.ndarray, n: int, layout: str) -> np.ndarray:
    """Inverse of :func:`dense_to_quantics`."""
    v = np.asarray(v)
    L = 1 << n
    if layout == "1d":
        return v.reshape(L).copy()
    if layout == "serial":
        return v.reshape(L, L).copy()
    if layout == "interleaved":
        t = v.reshape((2,) * (2 * n))                   # x_1, y_1, x_2, y_2, ...
        order = [2 * p for p in range(n)] + [2 * p + 1 for p in range(n)]
        return t.transpose(order).reshape(L, L).copy()
    raise ValueError(layout)


def quantics_index(a: int, b: int, n: int, layout: str) -> int:
    """Flat quantics index of pixel (a, b), written bit by bit (used to pin the
    reshape-based maps above on small grids)."""
    if layout == "serial":
        return (a << n) | b
    if layout == "interleaved":
        idx = 0
        for p in range(1, n + 1):
            xp = (a >> (n - p)) & 1
            yp = (b >> (n - p)) & 1
            idx = idx * 4 + (2 * xp + yp)
        return idx
    raise ValueError(layout)


def bit_reverse(k: int, n: int) -> int:
    r = 0
    for _ in range(n):
        r = (r << 1) | (k & 1)
        k >>= 1
    return r


def site_digits(flat: int, N: int, d: int):
    """Per-site digits (s_1 .. s_N), s_1 most significant."""
    out = []
    for _ in range(N):
        out.append(flat % d)
        flat //= d
    return out[::-1]
