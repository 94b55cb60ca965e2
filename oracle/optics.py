"""FP64 dense oracle of the intensity-loss pipeline on a phase mask (test infrastructure only).

Not in the paper: the mask product, the intensity of the propagated field, the loss against a target
intensity and its adjoint follow the reading of the differentiation workload (a field E multiplied
elementwise by a mask M, one Fresnel step, intensity I = |E'|^2, loss sum (I - I_t)^2), with the
Fresnel step of Sec. VI.A written densely by fresnel_dense.

Gradient convention: for the real loss L of the complex mask values M,
    dL = 2 Re sum_x conj(G(x)) dM(x),   G = dL/d conj(M)  (conjugate Wirtinger derivative).
"""
import numpy as np

from .fresnel import fresnel_dense


def intensity_loss_dense(E, M, It, c):
    """L = sum_x (|U (E M)|^2 - It)^2 with U the Fresnel step of parameter c."""
    Fp = fresnel_dense(np.asarray(E) * np.asarray(M), c)
    R = np.abs(Fp) ** 2 - np.asarray(It, dtype=np.float64)
    return float((R ** 2).sum())


def intensity_loss_grad_dense(E, M, It, c):
    """G = dL/d conj(M): with F' = U (E M) and R = |F'|^2 - It,
    dL/d conj(F') = 2 R F', the step is unitary so dL/d conj(E M) = U^dagger (2 R F'), and the product
    rule gives G = conj(E) U^dagger (2 R F').  U^dagger is the step with -c (the transfer function's
    conjugate)."""
    E = np.asarray(E, dtype=np.complex128)
    Fp = fresnel_dense(E * np.asarray(M), c)
    R = np.abs(Fp) ** 2 - np.asarray(It, dtype=np.float64)
    Gf = fresnel_dense(2.0 * R * Fp, -c)
    return np.conj(E) * Gf
