"""Seeded generators of images, wavefronts and random tensors.

The shapes and value distributions follow the workloads of the paper:
natural-image-like random fields with a power-law spectrum (Sec. II reports
natural images with roughly 1/f spectra), Gaussian beams through binary
apertures (Sec. V, Fig. fig_aperture uses apertures carrying a phase), and
smooth aberration phases (Sec. V, Eq. field).  The Kolmogorov phase screen is
the textbook turbulence model; it is not in the paper.

Nothing here encodes, compresses or propagates: outputs are plain samples.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 23089

# Wavelength and pixel pitch used for every propagation example (Sec. VI.A).
LAMBDA_M = 633e-9
PITCH_M = 10e-6


def physical_constants(n: int, z_m: float) -> dict:
    """Dimensionless Fresnel constant for an L = 2**n grid at distance z.

    Returns ``lambda_z_over_dx2`` (= lambda z / dx^2) and ``c`` (= lambda z /
    (L dx^2)); the transfer-function phase on the grid is -pi c k_f^2 / L.
    """
    L = 1 << n
    lz = LAMBDA_M * z_m / PITCH_M ** 2
    return {"lambda_z_over_dx2": lz, "c": lz / L, "L": L}


def gaussian_random_field_image(n: int = 6, seed: int = SEED_BASE + 0) -> np.ndarray:
    """Real 2^n x 2^n image: complex white noise shaped to a 1/f^2 power
    spectrum (amplitude 1/|f|, DC removed), real part of the inverse transform,
    min-max normalised to [0, 1].  float64."""
    L = 1 << n
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    f = np.fft.fftfreq(L) * L
    fr = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    amp = np.zeros_like(fr)
    amp[fr > 0] = 1.0 / fr[fr > 0]
    img = np.fft.ifft2(noise * amp).real
    img = (img - img.min()) / (img.max() - img.min())
    return img


def gaussian_beam_with_rectangles(n: int = 10, seed: int = SEED_BASE + 1,
                                  waist: float = 0.1, n_rect: int = 6,
                                  dtype=np.complex64) -> np.ndarray:
    """Complex field exp(-r^2/w^2) (w = waist * field width, centred) times the
    union of ``n_rect`` seeded axis-aligned rectangles (sides U[0.05, 0.3] W,
    centres U[0.25, 0.75] W).  Row index = x, column index = y."""
    L = 1 << n
    rng = np.random.default_rng(seed)
    u = (np.arange(L) + 0.5) / L - 0.5
    g = np.exp(-(u / waist) ** 2)
    field = np.outer(g, g)
    mask = np.zeros((L, L), dtype=bool)
    for _ in range(n_rect):
        sx, sy = rng.uniform(0.05, 0.3, size=2)
        cx, cy = rng.uniform(0.25, 0.75, size=2)
        x0, x1 = int((cx - sx / 2) * L), int((cx + sx / 2) * L)
        y0, y1 = int((cy - sy / 2) * L), int((cy + sy / 2) * L)
        mask[max(x0, 0):min(x1, L), max(y0, 0):min(y1, L)] = True
    return (field * mask).astype(dtype)


def separable_phase_factors(n: int = 16, seed: int = SEED_BASE + 2, rank: int = 8,
                            waist: float = 0.1):
    """Per-axis samples of a Gaussian beam times a rank-``rank`` smooth phase:

        E0(x, y) = G(x) G(y) * sum_r c_r u_r(x) v_r(y),
        u_r(x) = exp(i a_r cos(2 pi p_r x + theta_r)),  v_r likewise,

    a_r ~ U[0.5, 2], p_r in {1..4}, theta_r ~ U[0, 2 pi), c_r complex normal
    normalised so sum |c_r| = 1.  Returns (fx, gy), each (rank, 2^n) complex128,
    with E0 = sum_r outer(fx[r], gy[r]); fx carries c_r and G, gy carries G.
    The 2-D field is never formed."""
    L = 1 << n
    rng = np.random.default_rng(seed)
    x = (np.arange(L) + 0.5) / L
    G = np.exp(-((x - 0.5) / waist) ** 2)
    c = rng.standard_normal(rank) + 1j * rng.standard_normal(rank)
    c = c / np.abs(c).sum()
    fx = np.empty((rank, L), np.complex128)
    gy = np.empty((rank, L), np.complex128)
    for r in range(rank):
        a1, a2 = rng.uniform(0.5, 2.0, size=2)
        p1, p2 = rng.integers(1, 5, size=2)
        t1, t2 = rng.uniform(0, 2 * np.pi, size=2)
        fx[r] = c[r] * G * np.exp(1j * a1 * np.cos(2 * np.pi * p1 * x + t1))
        gy[r] = G * np.exp(1j * a2 * np.cos(2 * np.pi * p2 * x + t2))
    return fx, gy


def kolmogorov_phase_screen(n: int, r0_frac: float, rng: np.random.Generator) -> np.ndarray:
    """Kolmogorov phase screen (radians) on a 2^n grid by FFT filtering of complex
    Gaussian noise with phase PSD 0.023 r0^(-5/3) f^(-11/3) (f in cycles per
    field width, r0 in field widths; DC removed).  Textbook turbulence model."""
    L = 1 << n
    f = np.fft.fftfreq(L) * L
    fr = np.sqrt(f[:, None] ** 2 + f[None, :] ** 2)
    psd = np.zeros_like(fr)
    nz = fr > 0
    psd[nz] = 0.023 * r0_frac ** (-5.0 / 3.0) * fr[nz] ** (-11.0 / 3.0)
    noise = rng.standard_normal((L, L)) + 1j * rng.standard_normal((L, L))
    screen = np.fft.ifft2(noise * np.sqrt(psd)).real * L
    return screen


def batched_item_specs(count: int = 256, seed: int = SEED_BASE + 3,
                       n_choices=(8, 9, 10, 11, 12), chi_choices=(16, 32, 64)):
    """Per-item (n, chi, r0_frac, seed) for the batched workload."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        specs.append({
            "n": int(rng.choice(n_choices)),
            "chi": int(rng.choice(chi_choices)),
            "r0": float(rng.uniform(0.05, 0.2)),
            "seed": seed + 1 + i,
        })
    return specs


def batched_item_field(spec: dict, waist: float = 0.15, dtype=np.complex64) -> np.ndarray:
    """Gaussian beam (w = waist * W) times exp(i * Kolmogorov screen)."""
    n = spec["n"]
    L = 1 << n
    rng = np.random.default_rng(spec["seed"])
    u = (np.arange(L) + 0.5) / L - 0.5
    g = np.exp(-(u / waist) ** 2)
    phase = kolmogorov_phase_screen(n, spec["r0"], rng)
    return (np.outer(g, g) * np.exp(1j * phase)).astype(dtype)


def rectangles_target(n: int, seed: int, n_rect: int = 3, dtype=np.float32) -> np.ndarray:
    """Binary intensity target: union of seeded axis-aligned rectangles."""
    L = 1 << n
    rng = np.random.default_rng(seed)
    t = np.zeros((L, L), dtype=dtype)
    for _ in range(n_rect):
        sx, sy = rng.uniform(0.05, 0.25, size=2)
        cx, cy = rng.uniform(0.3, 0.7, size=2)
        x0, x1 = int((cx - sx / 2) * L), int((cx + sx / 2) * L)
        y0, y1 = int((cy - sy / 2) * L), int((cy + sy / 2) * L)
        t[max(x0, 0):min(x1, L), max(y0, 0):min(y1, L)] = 1
    return t


def smooth_random_phase_mask_factors(n: int, seed: int, strength: float = 0.1, n_modes: int = 4):
    """Per-axis samples of a smooth random phase exp(i * strength * phi(x)) with
    phi a seeded sum of ``n_modes`` low-frequency cosines of unit-normal weights.
    Returns (mx, my), each 2^n complex128; the mask is outer(mx, my)."""
    L = 1 << n
    rng = np.random.default_rng(seed)
    x = (np.arange(L) + 0.5) / L
    out = []
    for _ in range(2):
        phi = np.zeros(L)
        for m in range(1, n_modes + 1):
            phi += rng.standard_normal() * np.cos(2 * np.pi * m * x + rng.uniform(0, 2 * np.pi))
        out.append(np.exp(1j * strength * phi))
    return out[0], out[1]


def random_mps_sites(bonds, d: int, seed: int, decay: float = 0.0):
    """Random complex site tensors (bonds[p], d, bonds[p+1]) with unit-normal
    entries; ``decay`` > 0 scales the j-th right-bond column by exp(-decay*j) so
    that Schmidt spectra decay and truncation ranks are well separated."""
    rng = np.random.default_rng(seed)
    sites = []
    for p in range(len(bonds) - 1):
        a, b = bonds[p], bonds[p + 1]
        t = rng.standard_normal((a, d, b)) + 1j * rng.standard_normal((a, d, b))
        if decay > 0:
            t = t * np.exp(-decay * np.arange(b))[None, None, :]
        sites.append(t / np.sqrt(a * d))
    return sites


def random_unitary_sites(n: int, seed: int, dim: int = 2):
    """n Haar-like random dim x dim unitaries (QR of complex Gaussian matrices)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        z = rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))
        q, r = np.linalg.qr(z)
        q = q * (np.diag(r) / np.abs(np.diag(r)))[None, :]
        out.append(q)
    return out


def pupil_field(n: int, alpha: float = 0.001, r0: float = 0.5, dtype=np.complex64) -> np.ndarray:
    """Aberrated pupil E_0 = A(r) exp(-i Phi(u, v)) on (u, v) in [-1, 1)^2 (Sec. V, Eq. field): a soft-edged
    disk A(r) = 1 / (1 + exp((r - r0) / alpha)) and the paper's test phase
    Phi(u, v) = cos(u) cos(u) + cos(2u + 5v) + sin(u v) + cos(2u + 2v)^13.  Row index = u, column index = v."""
    L = 1 << n
    t = (np.arange(L) + 0.5) / L * 2.0 - 1.0
    u, v = np.meshgrid(t, t, indexing="ij")
    r = np.sqrt(u * u + v * v)
    A = 0.5 * (1.0 - np.tanh((r - r0) / (2.0 * alpha)))    # = 1 / (1 + exp((r - r0)/alpha)), overflow-free
    phi = np.cos(u) * np.cos(u) + np.cos(2 * u + 5 * v) + np.sin(u * v) + np.cos(2 * u + 2 * v) ** 13
    return (A * np.exp(-1j * phi)).astype(dtype)
