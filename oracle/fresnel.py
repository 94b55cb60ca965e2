"""Fresnel propagation: dense definition and the quantics-MPS step, in FP64.

Test infrastructure only (see the package docstring).

Dense definition (Sec. VI.A): E_z = F^{-1}[ F[E_0] . T(k_x) T(k_y) ] with the
paraxial factorisation T(k) = exp(-i pi c k_f^2 / L), c = lambda z / (L dx^2),
unitary DFTs written out as matrix products, periodic boundaries.  The global
factor exp(i k z) is dropped.

MPS step (Fig. fig_mpo_mpo, U_QFT^dagger U(z) U_QFT, applied per axis because
both factors are separable, Sec. VI.A and Fig. fig_psf_mps "first in the x then
y direction"):  Q_x, Q_y, D_x, D_y, Q_x^dagger, Q_y^dagger, each by zip-up.
Zip-up directions alternate so that every pass finds the canonical form it
needs: a left-canonical input starts right-to-left, a right-canonical one
left-to-right, and an input in no canonical form is left-canonicalised first.
"""
from __future__ import annotations

import numpy as np

from . import mps as _mps
from . import mpo as _mpo
from . import apply as _apply


def transfer_dense(E: np.ndarray, Dk: np.ndarray) -> np.ndarray:
    """Brute-force 2-D propagation by a separable transfer function: E_z = F^-1[F[E] Dk(k_x) Dk(k_y)] with the
    unitary matrix DFT F (Sec. VI.A; Dk indexed by the natural frequency bin k)."""
    E = np.asarray(E, dtype=np.complex128)
    L = E.shape[0]
    F = _mpo.dft_matrix(L)
    Ehat = F @ E @ F.T
    Ehat = Dk[:, None] * Ehat * Dk[None, :]
    Fi = F.conj().T
    return Fi @ Ehat @ Fi.T


def fresnel_dense(E: np.ndarray, c: float) -> np.ndarray:
    """Brute-force 2-D Fresnel transfer-function propagation (matrix DFTs)."""
    L = np.asarray(E).shape[0]
    kf = _mpo.fftfreq_int(L).astype(np.float64)
    return transfer_dense(E, np.exp(-1j * np.pi * c * kf ** 2 / L))


def fresnel_dense_1d(v: np.ndarray, c: float) -> np.ndarray:
    v = np.asarray(v, dtype=np.complex128)
    L = v.shape[0]
    F = _mpo.dft_matrix(L)
    kf = _mpo.fftfreq_int(L).astype(np.float64)
    D = np.exp(-1j * np.pi * c * kf ** 2 / L)
    return F.conj().T @ (D * (F @ v))


def fresnel_fft(E: np.ndarray, c: float) -> np.ndarray:
    """Cross-check of :func:`fresnel_dense` with the library FFT (the transfer
    function is even in k, so the FFT sign convention does not matter)."""
    E = np.asarray(E, dtype=np.complex128)
    L = E.shape[0]
    kf = _mpo.fftfreq_int(L).astype(np.float64)
    D = np.exp(-1j * np.pi * c * kf ** 2 / L)
    return np.fft.ifft2(np.fft.fft2(E) * D[:, None] * D[None, :])


def gaussian_closed_form(x: np.ndarray, w: float, lambda_z: float) -> np.ndarray:
    """Textbook Fresnel propagation of exp(-x^2/w^2) under exp(-i pi lambda z f^2):
    (w / W) exp(-x^2 / W^2) with W^2 = w^2 + i lambda z / pi.  Not in the paper."""
    W2 = w * w + 1j * lambda_z / np.pi
    return (w / np.sqrt(W2)) * np.exp(-x * x / W2)


def step_operators(n: int, c: float, qft_cutoff: float = 1e-12, phase_cutoff: float = 1e-12,
                   qft=None):
    """(Q, Q^dagger, D) per-axis MPOs for one Fresnel step."""
    Q = qft if qft is not None else (_mpo.qft_mpo_dense(n, qft_cutoff) if n <= 10
                                     else _mpo.qft_mpo_layers(n, qft_cutoff))
    return Q, _mpo.dagger(Q), _mpo.phase_mpo(n, c, phase_cutoff)


def step_passes(layout: str, n: int, Q, Qd, D):
    """The six embedded operators of one step, in application order."""
    axes = (0,) if layout == "1d" else (0, 1)
    passes = []
    for op in (Q, D, Qd):
        for ax in axes:
            passes.append(_mpo.embed(op, layout, ax, n))
    return passes


def operator_canonical(W, side: str):
    """An MPO (cores (a, s', s, b)) in left- or right-canonical form, as an MPS of the (s', s) pairs
    (the same operator; exact QR sweeps)."""
    as_mps = [w.reshape(w.shape[0], w.shape[1] * w.shape[2], w.shape[3]) for w in W]
    m = _mps.left_canonicalize(as_mps) if side == "left" else _mps.right_canonicalize(as_mps)
    return [x.reshape(x.shape[0], W[p].shape[1], W[p].shape[2], x.shape[2]) for p, x in enumerate(m)]


def apply_sequence(passes, sites, canon: str, chi_max: int, cutoff: float, totals=None, passes_left=None):
    """Apply embedded MPOs in order by zip-up with alternating directions.
    Returns (sites, canon, total discarded weight); `totals` (a list) collects
    the squared norms of the factorised matrices.  With `passes_left` (the same
    operators in left-canonical form), a right-to-left pass applies the
    left-canonical form and a left-to-right pass the right-canonical one
    (`passes`), so that every operator is canonical in the direction of its sweep."""
    A = sites
    if canon == "none":
        A = _mps.left_canonicalize(A)
        canon = "left"
    disc = 0.0
    for i, W in enumerate(passes):
        direction = "rl" if canon == "left" else "lr"
        if passes_left is not None and direction == "rl":
            W = passes_left[i]
        A, eps = _apply.zipup(W, A, chi_max, cutoff, direction, totals)
        disc += sum(eps)
        canon = "right" if direction == "rl" else "left"
    return A, canon, disc


def fresnel_mps(sites, layout: str, n: int, c: float, chi_max: int, cutoff: float,
                canon: str = "none", n_steps: int = 1, ops=None, totals=None, operator_form: str = "right"):
    """n_steps Fresnel steps on an MPS.  Returns (sites, canon, discarded).

    operator_form "right": every pass applies the right-canonical operators the
    builders deliver; "matched": each pass applies its operator in the canonical
    form of its sweep direction (left-canonical for right-to-left passes)."""
    Q, Qd, D = ops if ops is not None else step_operators(n, c)
    passes_left = None
    if operator_form == "matched":
        Q, Qd, D = (operator_canonical(op, "right") for op in (Q, Qd, D))
        passes_left = step_passes(layout, n, *(operator_canonical(op, "left") for op in (Q, Qd, D)))
    elif operator_form != "right":
        raise ValueError(operator_form)
    passes = step_passes(layout, n, Q, Qd, D)
    disc = 0.0
    A = sites
    for _ in range(n_steps):
        A, canon, d = apply_sequence(passes, A, canon, chi_max, cutoff, totals, passes_left)
        disc += d
    return A, canon, disc
