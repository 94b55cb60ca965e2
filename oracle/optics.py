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


# ----------------------------------------------------------------------------- imaging (Sec. V)

def psf_dense(E0, centre: bool = False):
    """PSF = |F(E_0)|^2 normalised to unit sum (Sec. V, Eq. psf_eq, ||PSF||_L1 = 1), with the unitary matrix DFT
    F[k, j] = exp(+2 pi i j k / L) / sqrt(L) on both axes, natural frequency order; ``centre`` moves frequency
    k to k + L/2 (mod L) on both axes."""
    from .mpo import dft_matrix
    E0 = np.asarray(E0, dtype=np.complex128)
    L = E0.shape[0]
    F = dft_matrix(L)
    Ef = F @ E0 @ F.T
    P = np.abs(Ef) ** 2
    P = P / P.sum()
    if centre:
        P = np.roll(np.roll(P, L // 2, axis=0), L // 2, axis=1)
    return P


def convolve_dense(a, b):
    """Circular convolution (a * b)[x, y] = sum_{m, n} a[m, n] b[x - m, y - n] (indices mod L), by the sum over
    shifts written out (Sec. V, I_img = I_obj * PSF on the periodic grid)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    L = a.shape[0]
    out = np.zeros((L, L), dtype=np.complex128)
    for m in range(L):
        for n in range(L):
            if a[m, n] != 0:
                out += a[m, n] * np.roll(np.roll(b, m, axis=0), n, axis=1)
    return out


# ----------------------------------------------------------------------------- angular spectrum (Sec. VI.A)

def astf_transfer(n: int, z_over_lambda: float, lambda_over_dx: float):
    """Angular-spectrum transfer function (Eq. eq_astf) on the L x L grid of frequency bins (natural order), with
    the constant exp(2 pi i z / lambda) divided out: exp(2 pi i (z/lambda)(sqrt(1 - u) - 1)),
    u = (lambda f_x)^2 + (lambda f_y)^2, lambda f = (lambda/dx) k_f / L; for u > 1 the square root is i sqrt(u - 1)
    (evanescent decay)."""
    from .mpo import fftfreq_int
    L = 1 << n
    lf = lambda_over_dx * fftfreq_int(L).astype(np.float64) / L
    u = lf[:, None] ** 2 + lf[None, :] ** 2
    root = np.sqrt((1.0 - u).astype(np.complex128))       # i sqrt(u - 1) for u > 1
    return np.exp(2j * np.pi * z_over_lambda * (root - 1.0))


def propagate_dense_2d(E, T):
    """E_z = F^-1[F[E] T] with a non-separable transfer function T (natural frequency bins), matrix DFTs."""
    from .mpo import dft_matrix
    E = np.asarray(E, dtype=np.complex128)
    F = dft_matrix(E.shape[0])
    Ehat = (F @ E @ F.T) * T
    Fi = F.conj().T
    return Fi @ Ehat @ Fi.T


# ----------------------------------------------------------------------------- fixed-rank (frozen-projector) adjoint
#
# Not in the paper.  A zip-up pass (Sec. V) that applies K writes N - 1 isometric sites (the frame V) and a centre
# c = V^dagger K psi, so with its truncation frozen it is the linear map psi -> V V^dagger K psi.  The forward
# computation of the intensity loss (mask product by zip-up, then the six passes of a Fresnel step) is then
# F(m) = P_6 K_6 ... P_1 K_1 P_0 diag(e) m with P_i = V_i V_i^dagger, and its adjoint takes the cotangent g of
# F back as conj(e) . P_0 K_1^dagger P_1 ... K_6^dagger P_6 g.  Dense, for small n.

def frame_isometry(sites, canon: str) -> np.ndarray:
    """Dense isometry V of a zip-up output: every site but the centre contracted, the centre's indices open.
    canon 'left': the centre is the last site, V[(r, s), (k, s')] = L[r, k] delta(s, s');
    canon 'right': the centre is the first site, V[(s, r), (s', k)] = delta(s, s') R[k, r]."""
    d = sites[0].shape[1]
    if canon == "left":
        L = np.ones((1, 1), dtype=np.complex128)
        for A in sites[:-1]:
            a, dd, b = A.shape
            L = (L @ A.reshape(a, dd * b)).reshape(-1, b)
        return np.kron(L, np.eye(d))
    R = np.ones((1, 1), dtype=np.complex128)
    for A in reversed(sites[1:]):
        a, dd, b = A.shape
        R = (A.reshape(a * dd, b) @ R).reshape(a, -1)
    return np.kron(np.eye(d), R.T)


def diag_operator(sites):
    """An MPS seen as an operator diagonal in the site index: W[a, s', s, b] = delta(s', s) A[a, s, b]."""
    out = []
    for A in sites:
        a, d, b = A.shape
        W = np.zeros((a, d, d, b), dtype=np.complex128)
        for s in range(d):
            W[:, s, s, :] = A[:, s, :]
        out.append(W)
    return out


def frozen_forward(E_sites, M_sites, n: int, ops, chi: int, cutoff: float):
    """The forward computation with every zip-up output recorded: the mask product (the mask as a diagonal
    operator applied by zip-up to the left-canonical field) and the six passes Q_x, Q_y, D_x, D_y, Q^dagger_x,
    Q^dagger_y.  Returns [(sites, canon)] after the mask product and after each pass, and the embedded operators."""
    from .apply import zipup
    from .fresnel import step_passes
    from .mpo import dagger
    Q, Qd, D = ops
    frames = []
    A, eps = zipup(diag_operator(M_sites), E_sites, chi, cutoff, "rl")
    canon = "right"
    frames.append((A, canon))
    passes = step_passes("interleaved", n, Q, Qd, D)
    for W in passes:
        direction = "rl" if canon == "left" else "lr"
        A, _ = zipup(W, A, chi, cutoff, direction)
        canon = "right" if direction == "rl" else "left"
        frames.append((A, canon))
    return frames, passes


def frozen_loss_and_grad(E_sites, M_sites, It_site_order, n: int, ops, chi: int, cutoff: float):
    """Loss L = sum (|F|^2 - I_t)^2 of the recorded forward pass and G = dL/d conj(m) of the frozen-projector map
    (site-ordered dense vectors).  Also returns the dense pieces for finite differences."""
    from .mpo import to_dense
    from .mps import to_vector
    frames, passes = frozen_forward(E_sites, M_sites, n, ops, chi, cutoff)
    P = []
    for sites, canon in frames:
        V = frame_isometry(sites, canon)
        P.append(V @ V.conj().T)
    K = [to_dense(W) for W in passes]
    e = to_vector(E_sites)
    psi = to_vector(frames[-1][0])
    R = np.abs(psi) ** 2 - np.asarray(It_site_order, dtype=np.float64)
    h = P[6] @ (2.0 * R * psi)
    for i in range(6, 0, -1):
        h = P[i - 1] @ (K[i - 1].conj().T @ h)
    G = np.conj(e) * h
    return float((R ** 2).sum()), G, (P, K, e)


def frozen_loss(m, pieces, It_site_order):
    """L(m) of the frozen-projector map F(m) = P_6 K_6 ... P_1 K_1 P_0 (e . m)."""
    P, K, e = pieces
    f = P[0] @ (e * m)
    for i in range(6):
        f = P[i + 1] @ (K[i] @ f)
    R = np.abs(f) ** 2 - np.asarray(It_site_order, dtype=np.float64)
    return float((R ** 2).sum())
