"""Python binding of the C ABI in include/qtn.h (argument marshalling only).

Device memory and streams come from PyTorch; every computation runs in
libqtn.so.  The entry points keep the C names without the ``qtn_`` prefix:
``encode``, ``apply_mpo``, ``truncate``, ``fresnel_step``, ``to_dense``,
``build_qft_mpo``, ``build_phase_mpo``, ``mpo_dagger``, ``norm2``,
``overlap``, ``amplitudes``.

There is no fallback: if the library is missing or no CUDA device is present,
loading raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqtn.so")

LAYOUTS = {"serial": 0, "interleaved": 1, "1d": 2}
PRECISIONS = {"fp32": 0, "plain": 0, "mixed": 1}
CANON = {0: "none", 1: "left", 2: "right"}
STATUS = {
    0: "QTN_OK", 1: "QTN_ERR_ARG", 2: "QTN_ERR_SHAPE", 3: "QTN_ERR_CAPACITY", 4: "QTN_ERR_NOCONV",
    5: "QTN_ERR_NONFINITE", 6: "QTN_ERR_TIMEOUT", 7: "QTN_ERR_CUDA", 8: "QTN_ERR_BOUNDS", 9: "QTN_ERR_WORKSPACE",
}

# Every symbol include/qtn.h declares (checked by the CPU test-suite).
EXPORTS = (
    "qtn_create", "qtn_destroy", "qtn_set_stream", "qtn_status_string", "qtn_version", "qtn_workspace_size",
    "qtn_encode", "qtn_build_qft_mpo", "qtn_build_phase_mpo", "qtn_mpo_dagger", "qtn_apply_mpo", "qtn_truncate",
    "qtn_fresnel_step", "qtn_to_dense", "qtn_norm2", "qtn_overlap", "qtn_amplitudes", "qtn_tsvd",
    "qtn_kron_interleave", "qtn_add", "qtn_launch_count", "qtn_profile", "qtn_profile_read", "qtn_tsvd_noalloc",
    "qtn_hadamard", "qtn_scale", "qtn_hadamard_zipup", "qtn_overlap_grad",
    "qtn_batch_create", "qtn_batch_launch", "qtn_batch_destroy", "qtn_batch_sync",
    "qtn_workspace_init", "qtn_check", "qtn_build_bessel_mpo", "qtn_build_pauliz_mpo",
    "qtn_reverse_sites", "qtn_psf", "qtn_convolve", "qtn_astf_field", "qtn_transfer_step", "qtn_project_apply",
    "qtn_batch_stream", "qtn_set_gemm_tile", "qtn_tune_gemm_tile", "qtn_batch_tune_branches",
    "qtn_set_eig_cluster_min",
)


class QtnError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


class c_mps(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int), ("d", ctypes.c_int), ("chi_cap", ctypes.c_int), ("canon", ctypes.c_int),
                ("bond", ctypes.c_void_p), ("sites", ctypes.c_void_p)]


class c_mpo(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int), ("w_cap", ctypes.c_int), ("w_max", ctypes.c_int),
                ("bond", ctypes.c_void_p), ("sites", ctypes.c_void_p)]


class c_trunc(ctypes.Structure):
    _fields_ = [("chi_max", ctypes.c_int), ("cutoff", ctypes.c_double), ("prec", ctypes.c_int),
                ("max_sweeps", ctypes.c_int)]


class c_stats(ctypes.Structure):
    _fields_ = [("discarded", ctypes.c_double), ("norm2", ctypes.c_double), ("max_bond", ctypes.c_int),
                ("sweeps_used", ctypes.c_int), ("flags", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libqtn.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_2510_23089_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    LL = ctypes.c_longlong
    mp, op, tr, st = ctypes.POINTER(c_mps), ctypes.POINTER(c_mpo), c_trunc, ctypes.POINTER(c_stats)
    sig = {
        "qtn_create": [ctypes.POINTER(P), P], "qtn_destroy": [P], "qtn_set_stream": [P, P],
        "qtn_workspace_size": [P, I, I, I, I, LL, ctypes.POINTER(S)],
        "qtn_encode": [P, P, I, I, tr, mp, st, P, S],
        "qtn_build_qft_mpo": [P, I, I, D, op, P, S],
        "qtn_build_phase_mpo": [P, I, D, I, D, op, P, S],
        "qtn_build_bessel_mpo": [P, I, D, I, I, op, P, S],
        "qtn_build_pauliz_mpo": [P, I, D, D, I, D, op, P, S],
        "qtn_mpo_dagger": [P, op, op],
        "qtn_apply_mpo": [P, op, I, mp, tr, st, P, S],
        "qtn_truncate": [P, mp, tr, st, P, S],
        "qtn_fresnel_step": [P, mp, I, op, op, op, I, tr, st, P, S],
        "qtn_to_dense": [P, mp, I, P, LL, P, S],
        "qtn_norm2": [P, mp, ctypes.POINTER(D), P, S],
        "qtn_overlap": [P, mp, mp, ctypes.POINTER(D), P, S],
        "qtn_amplitudes": [P, mp, P, I, P, P, S],
        "qtn_tsvd": [P, P, I, I, tr, P, P, I, ctypes.POINTER(I), st, P, S],
        "qtn_tsvd_noalloc": [P, I, I, tr, P, P, I, ctypes.POINTER(I), st, P],
        "qtn_kron_interleave": [P, mp, mp, mp],
        "qtn_add": [P, mp, mp, mp],
        "qtn_hadamard": [P, mp, mp, I, mp],
        "qtn_scale": [P, mp, D, D],
        "qtn_hadamard_zipup": [P, mp, I, mp, tr, st, P, S],
        "qtn_overlap_grad": [P, mp, mp, P, P, S],
        "qtn_batch_create": [I, ctypes.POINTER(P), mp, op, op, op, I, tr, ctypes.POINTER(P), ctypes.POINTER(S),
                             I, ctypes.POINTER(P)],
        "qtn_batch_stream": [P, ctypes.POINTER(P)],
        "qtn_batch_tune_branches": [I, ctypes.POINTER(P), mp, op, op, op, tr, ctypes.POINTER(P), ctypes.POINTER(S),
                                    ctypes.POINTER(I), I, ctypes.c_char_p, ctypes.POINTER(I), ctypes.POINTER(D)],
        "qtn_set_gemm_tile": [P, I],
        "qtn_set_eig_cluster_min": [I],
        "qtn_tune_gemm_tile": [P, mp, op, op, op, tr, P, S, ctypes.c_char_p, ctypes.POINTER(I), ctypes.POINTER(D)],
        "qtn_batch_launch": [P, I],
        "qtn_batch_sync": [P],
        "qtn_reverse_sites": [P, mp],
        "qtn_project_apply": [P, op, I, mp, mp, P, S],
        "qtn_psf": [P, mp, op, I, tr, mp, st, P, S],
        "qtn_convolve": [P, mp, mp, op, op, tr, st, P, S],
        "qtn_astf_field": [P, I, D, D, I, P, LL],
        "qtn_transfer_step": [P, mp, op, op, mp, tr, st, P, S],
        "qtn_workspace_init": [P, P, S],
        "qtn_check": [P, P, S],
        "qtn_batch_destroy": [P],
        "qtn_profile": [P, I, P, S],
        "qtn_profile_read": [P, I, ctypes.POINTER(D), ctypes.POINTER(LL), ctypes.POINTER(D), P, S],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = I
    lib.qtn_status_string.argtypes = [I]
    lib.qtn_status_string.restype = ctypes.c_char_p
    lib.qtn_version.argtypes = []
    lib.qtn_version.restype = I
    lib.qtn_launch_count.argtypes = []
    lib.qtn_launch_count.restype = LL
    _lib = lib
    return lib


def _check(code: int, where: str):
    if code != 0:
        raise QtnError(code, where)


@dataclass
class Stats:
    discarded: float
    norm2: float
    max_bond: int
    sweeps_used: int
    flags: int


def _stats(s: c_stats) -> Stats:
    return Stats(s.discarded, s.norm2, s.max_bond, s.sweeps_used, s.flags)


class MPS:
    """Device MPS in the padded layout of include/qtn.h (torch-owned memory)."""

    def __init__(self, n_sites: int, d: int, chi_cap: int, device="cuda"):
        self.sites = torch.zeros((n_sites, chi_cap, d, chi_cap), dtype=torch.complex64, device=device)
        self.bond = torch.ones(n_sites + 1, dtype=torch.int32, device=device)
        self.c = c_mps(n_sites, d, chi_cap, 0, self.bond.data_ptr(), self.sites.data_ptr())

    @property
    def n_sites(self):
        return self.c.n_sites

    @property
    def d(self):
        return self.c.d

    @property
    def chi_cap(self):
        return self.c.chi_cap

    @property
    def canon(self) -> str:
        return CANON[self.c.canon]

    def bonds(self):
        return [int(b) for b in self.bond.cpu()]

    def to_numpy_sites(self):
        """Compact site tensors (bond[p], d, bond[p+1]) as complex128 numpy arrays."""
        b = self.bonds()
        S = self.sites.cpu().numpy()
        return [S[p, :b[p], :, :b[p + 1]].astype("complex128") for p in range(self.n_sites)]

    @classmethod
    def from_numpy_sites(cls, sites, chi_cap: int, canon: str = "none", device="cuda"):
        N, d = len(sites), sites[0].shape[1]
        m = cls(N, d, chi_cap, device)
        host = torch.zeros((N, chi_cap, d, chi_cap), dtype=torch.complex64)
        bonds = [1]
        for p, A in enumerate(sites):
            a, _, b = A.shape
            host[p, :a, :, :b] = torch.from_numpy(A.astype("complex64"))
            bonds.append(b)
        m.sites.copy_(host)
        m.bond.copy_(torch.tensor(bonds, dtype=torch.int32))
        m.c.canon = {"none": 0, "left": 1, "right": 2}[canon]
        return m

    def clone(self):
        m = MPS(self.n_sites, self.d, self.chi_cap, self.sites.device)
        m.sites.copy_(self.sites)
        m.bond.copy_(self.bond)
        m.c.canon = self.c.canon
        return m


class MPO:
    """Device per-axis MPO (n sites, d = 2) in the padded layout of include/qtn.h."""

    def __init__(self, n_sites: int, w_cap: int, device="cuda"):
        self.sites = torch.zeros((n_sites, w_cap, 2, 2, w_cap), dtype=torch.complex64, device=device)
        self.bond = torch.ones(n_sites + 1, dtype=torch.int32, device=device)
        self.c = c_mpo(n_sites, w_cap, 1, self.bond.data_ptr(), self.sites.data_ptr())

    @property
    def n_sites(self):
        return self.c.n_sites

    @property
    def w_max(self):
        return self.c.w_max

    def bonds(self):
        return [int(b) for b in self.bond.cpu()]

    def to_numpy_cores(self):
        b = self.bonds()
        S = self.sites.cpu().numpy()
        return [S[p, :b[p], :, :, :b[p + 1]].astype("complex128") for p in range(self.n_sites)]

    @classmethod
    def from_numpy_cores(cls, cores, w_cap: int, device="cuda"):
        m = cls(len(cores), w_cap, device)
        host = torch.zeros((len(cores), w_cap, 2, 2, w_cap), dtype=torch.complex64)
        bonds = [1]
        for p, c in enumerate(cores):
            a, _, _, b = c.shape
            host[p, :a, :, :, :b] = torch.from_numpy(c.astype("complex64"))
            bonds.append(b)
        m.sites.copy_(host)
        m.bond.copy_(torch.tensor(bonds, dtype=torch.int32))
        m.c.w_max = max(bonds)
        return m


class Engine:
    """A library context on the current torch stream plus a workspace sized for
    states of up to ``n_sites`` sites, dimension ``d``, bonds ``chi`` and MPO
    bonds ``w``, and dense inputs of ``dense`` entries."""

    def __init__(self, n_sites: int, d: int, chi: int, w: int, dense: int = 0, stream=None):
        self.lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the qtn library has no CPU path")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        ctx = ctypes.c_void_p()
        _check(self.lib.qtn_create(ctypes.byref(ctx), ctypes.c_void_p(self.stream.cuda_stream)), "qtn_create")
        self.ctx = ctx
        nbytes = ctypes.c_size_t()
        _check(self.lib.qtn_workspace_size(ctx, n_sites, d, chi, w, dense, ctypes.byref(nbytes)),
               "qtn_workspace_size")
        self.ws = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self.ws_bytes = int(nbytes.value)
        _check(self.lib.qtn_workspace_init(ctx, *self._ws()), "qtn_workspace_init")

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.lib.qtn_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    def _ws(self):
        return ctypes.c_void_p(self.ws.data_ptr()), ctypes.c_size_t(self.ws_bytes)

    @staticmethod
    def trunc(chi_max: int, cutoff: float, prec: str = "fp32", max_sweeps: int = 0) -> c_trunc:
        return c_trunc(int(chi_max), float(cutoff), PRECISIONS[prec], int(max_sweeps))

    # --------------------------------------------------------------- entry points
    def encode(self, dense: torch.Tensor, n: int, layout: str, out: MPS, chi_max: int, cutoff: float,
               prec: str = "fp32", stats: bool = True):
        assert dense.is_cuda and dense.dtype == torch.complex64 and dense.is_contiguous()
        st = c_stats()
        _check(self.lib.qtn_encode(self.ctx, ctypes.c_void_p(dense.data_ptr()), n, LAYOUTS[layout],
                                   self.trunc(chi_max, cutoff, prec), ctypes.byref(out.c),
                                   ctypes.byref(st) if stats else None, *self._ws()), "qtn_encode")
        return _stats(st) if stats else None

    def build_qft_mpo(self, n: int, inverse: bool, cutoff: float, w_cap: int = 16) -> MPO:
        m = MPO(n, w_cap)
        _check(self.lib.qtn_build_qft_mpo(self.ctx, n, int(inverse), cutoff, ctypes.byref(m.c), *self._ws()),
               "qtn_build_qft_mpo")
        return m

    def build_phase_mpo(self, n: int, c: float, cutoff: float, w_cap: int = 64, bit_reversed: bool = True) -> MPO:
        m = MPO(n, w_cap)
        _check(self.lib.qtn_build_phase_mpo(self.ctx, n, float(c), int(bit_reversed), cutoff, ctypes.byref(m.c),
                                            *self._ws()), "qtn_build_phase_mpo")
        return m

    def build_bessel_mpo(self, n: int, t: float, p_max: int, w_cap: int = 32, bit_reversed: bool = True) -> MPO:
        m = MPO(n, w_cap)
        _check(self.lib.qtn_build_bessel_mpo(self.ctx, n, float(t), int(p_max), int(bit_reversed), ctypes.byref(m.c),
                                             *self._ws()), "qtn_build_bessel_mpo")
        return m

    def build_pauliz_mpo(self, n: int, t: float, gate_cutoff: float, cutoff: float = 1e-12, w_cap: int = 32,
                         bit_reversed: bool = True) -> MPO:
        m = MPO(n, w_cap)
        _check(self.lib.qtn_build_pauliz_mpo(self.ctx, n, float(t), float(gate_cutoff), int(bit_reversed),
                                             float(cutoff), ctypes.byref(m.c), *self._ws()), "qtn_build_pauliz_mpo")
        return m

    def mpo_dagger(self, W: MPO) -> MPO:
        out = MPO(W.n_sites, W.c.w_cap)
        _check(self.lib.qtn_mpo_dagger(self.ctx, ctypes.byref(W.c), ctypes.byref(out.c)), "qtn_mpo_dagger")
        return out

    def apply_mpo(self, W: MPO, axis: int, psi: MPS, chi_max: int, cutoff: float, prec: str = "fp32",
                  stats: bool = True):
        st = c_stats()
        _check(self.lib.qtn_apply_mpo(self.ctx, ctypes.byref(W.c), axis, ctypes.byref(psi.c),
                                      self.trunc(chi_max, cutoff, prec), ctypes.byref(st) if stats else None,
                                      *self._ws()), "qtn_apply_mpo")
        return _stats(st) if stats else None

    def truncate(self, psi: MPS, chi_max: int, cutoff: float, prec: str = "fp32", stats: bool = True):
        st = c_stats()
        _check(self.lib.qtn_truncate(self.ctx, ctypes.byref(psi.c), self.trunc(chi_max, cutoff, prec),
                                     ctypes.byref(st) if stats else None, *self._ws()), "qtn_truncate")
        return _stats(st) if stats else None

    def fresnel_step(self, psi: MPS, layout: str, Q: MPO, Qd: MPO, D: MPO, n_steps: int, chi_max: int,
                     cutoff: float, prec: str = "fp32", stats: bool = True):
        st = c_stats()
        _check(self.lib.qtn_fresnel_step(self.ctx, ctypes.byref(psi.c), LAYOUTS[layout], ctypes.byref(Q.c),
                                         ctypes.byref(Qd.c), ctypes.byref(D.c), n_steps,
                                         self.trunc(chi_max, cutoff, prec), ctypes.byref(st) if stats else None,
                                         *self._ws()), "qtn_fresnel_step")
        return _stats(st) if stats else None

    def to_dense(self, psi: MPS, layout: str, n: int) -> torch.Tensor:
        L = 1 << n
        out = torch.empty((L,) if layout == "1d" else (L, L), dtype=torch.complex64, device="cuda")
        _check(self.lib.qtn_to_dense(self.ctx, ctypes.byref(psi.c), LAYOUTS[layout], ctypes.c_void_p(out.data_ptr()),
                                     out.numel(), *self._ws()), "qtn_to_dense")
        return out

    def norm2(self, psi: MPS) -> float:
        v = ctypes.c_double()
        _check(self.lib.qtn_norm2(self.ctx, ctypes.byref(psi.c), ctypes.byref(v), *self._ws()), "qtn_norm2")
        return v.value

    def overlap(self, a: MPS, b: MPS) -> complex:
        v = (ctypes.c_double * 2)()
        _check(self.lib.qtn_overlap(self.ctx, ctypes.byref(a.c), ctypes.byref(b.c), v, *self._ws()), "qtn_overlap")
        return complex(v[0], v[1])

    def tsvd(self, T: torch.Tensor, chi_max: int, cutoff: float, k_cap: int = None, prec: str = "fp32"):
        """Truncated SVD of one m x n matrix: returns (U[:, :k], C[:k], stats) with T ~ U C."""
        assert T.is_cuda and T.dtype == torch.complex64 and T.dim() == 2
        T = T.contiguous()
        m, n = T.shape
        k_cap = k_cap or min(m, n)
        U = torch.zeros((m, k_cap), dtype=torch.complex64, device="cuda")
        C = torch.zeros((k_cap, n), dtype=torch.complex64, device="cuda")
        k = ctypes.c_int()
        st = c_stats()
        _check(self.lib.qtn_tsvd(self.ctx, ctypes.c_void_p(T.data_ptr()), m, n, self.trunc(chi_max, cutoff, prec),
                                 ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(C.data_ptr()), k_cap,
                                 ctypes.byref(k), ctypes.byref(st), *self._ws()), "qtn_tsvd")
        return U[:, :k.value], C[:k.value], _stats(st)

    def kron_interleave(self, x: MPS, y: MPS, out: MPS) -> MPS:
        _check(self.lib.qtn_kron_interleave(self.ctx, ctypes.byref(x.c), ctypes.byref(y.c), ctypes.byref(out.c)),
               "qtn_kron_interleave")
        return out

    def hadamard(self, a: MPS, b: MPS, out: MPS, conj_b: bool = False) -> MPS:
        _check(self.lib.qtn_hadamard(self.ctx, ctypes.byref(a.c), ctypes.byref(b.c), int(conj_b), ctypes.byref(out.c)),
               "qtn_hadamard")
        return out

    def hadamard_zipup(self, b: MPS, psi: MPS, chi_max: int, cutoff: float, conj_b: bool = False,
                       stats: bool = True):
        """psi <- truncate(psi (.) b) by zip-up (b conjugated when conj_b)."""
        st = c_stats()
        _check(self.lib.qtn_hadamard_zipup(self.ctx, ctypes.byref(b.c), int(conj_b), ctypes.byref(psi.c),
                                           self.trunc(chi_max, cutoff), ctypes.byref(st) if stats else None,
                                           *self._ws()), "qtn_hadamard_zipup")
        return _stats(st) if stats else None

    def overlap_grad(self, a: MPS, b: MPS) -> torch.Tensor:
        """d<a|b>/d conj(a's site tensors), same layout as a.sites."""
        g = torch.empty_like(a.sites)
        _check(self.lib.qtn_overlap_grad(self.ctx, ctypes.byref(a.c), ctypes.byref(b.c), ctypes.c_void_p(g.data_ptr()),
                                         *self._ws()), "qtn_overlap_grad")
        return g

    def scale(self, psi: MPS, z: complex) -> MPS:
        _check(self.lib.qtn_scale(self.ctx, ctypes.byref(psi.c), float(z.real), float(z.imag)), "qtn_scale")
        return psi

    def add(self, a: MPS, b: MPS, out: MPS) -> MPS:
        _check(self.lib.qtn_add(self.ctx, ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(out.c)), "qtn_add")
        return out

    def project_apply(self, W, axis: int, ket: MPS, frame: MPS) -> MPS:
        """frame <- V V^dagger W ket: the frame's centre replaced (qtn_project_apply; W None = identity)."""
        _check(self.lib.qtn_project_apply(self.ctx, ctypes.byref(W.c) if W is not None else None, int(axis),
                                          ctypes.byref(ket.c), ctypes.byref(frame.c), *self._ws()),
               "qtn_project_apply")
        return frame

    def reverse_sites(self, psi: MPS) -> MPS:
        _check(self.lib.qtn_reverse_sites(self.ctx, ctypes.byref(psi.c)), "qtn_reverse_sites")
        return psi

    def psf(self, phi: MPS, Q: MPO, psf: MPS, chi_max: int, cutoff: float, centre: bool = False,
            stats: bool = True):
        """phi <- normalised U_qft phi (natural frequency order); psf <- |phi|^2 as an MPS (qtn_psf)."""
        st = c_stats()
        _check(self.lib.qtn_psf(self.ctx, ctypes.byref(phi.c), ctypes.byref(Q.c), int(centre),
                                self.trunc(chi_max, cutoff), ctypes.byref(psf.c), ctypes.byref(st) if stats else None,
                                *self._ws()), "qtn_psf")
        return _stats(st) if stats else None

    def convolve(self, a: MPS, b: MPS, Q: MPO, Qd: MPO, chi_max: int, cutoff: float, stats: bool = True):
        """b <- a (*) b (circular convolution); a is overwritten by its transform (qtn_convolve)."""
        st = c_stats()
        _check(self.lib.qtn_convolve(self.ctx, ctypes.byref(a.c), ctypes.byref(b.c), ctypes.byref(Q.c),
                                     ctypes.byref(Qd.c), self.trunc(chi_max, cutoff),
                                     ctypes.byref(st) if stats else None, *self._ws()), "qtn_convolve")
        return _stats(st) if stats else None

    def astf_field(self, n: int, z_over_lambda: float, lambda_over_dx: float, bit_reversed: bool = True):
        L = 1 << n
        out = torch.empty((L, L), dtype=torch.complex64, device="cuda")
        _check(self.lib.qtn_astf_field(self.ctx, n, float(z_over_lambda), float(lambda_over_dx), int(bit_reversed),
                                       ctypes.c_void_p(out.data_ptr()), out.numel()), "qtn_astf_field")
        return out

    def transfer_step(self, psi: MPS, Q: MPO, Qd: MPO, T: MPS, chi_max: int, cutoff: float, stats: bool = True):
        st = c_stats()
        _check(self.lib.qtn_transfer_step(self.ctx, ctypes.byref(psi.c), ctypes.byref(Q.c), ctypes.byref(Qd.c),
                                          ctypes.byref(T.c), self.trunc(chi_max, cutoff),
                                          ctypes.byref(st) if stats else None, *self._ws()), "qtn_transfer_step")
        return _stats(st) if stats else None

    def set_eig_cluster_min(self, r_min: int):
        """Smallest problem order solved by the cluster eigen-solver (process-wide; 161 disables it)."""
        _check(self.lib.qtn_set_eig_cluster_min(int(r_min)), "qtn_set_eig_cluster_min")

    def set_gemm_tile(self, tile: int):
        _check(self.lib.qtn_set_gemm_tile(self.ctx, int(tile)), "qtn_set_gemm_tile")

    def tune_gemm_tile(self, item: MPS, Q: MPO, Qd: MPO, D: MPO, chi_max: int, cutoff: float, prec: str = "fp32",
                       cache_path: str | None = None):
        """(tile, ms per step) chosen by qtn_tune_gemm_tile; `item` is advanced by the trial steps."""
        t, ms = ctypes.c_int(), ctypes.c_double()
        _check(self.lib.qtn_tune_gemm_tile(self.ctx, ctypes.byref(item.c), ctypes.byref(Q.c), ctypes.byref(Qd.c),
                                           ctypes.byref(D.c), self.trunc(chi_max, cutoff, prec), *self._ws(),
                                           cache_path.encode() if cache_path else None, ctypes.byref(t),
                                           ctypes.byref(ms)), "qtn_tune_gemm_tile")
        return t.value, ms.value

    def check(self):
        """Raises QtnError for any device-side failure since the last check (qtn_check)."""
        _check(self.lib.qtn_check(self.ctx, *self._ws()), "qtn_check")

    def launch_count(self) -> int:
        return int(self.lib.qtn_launch_count())

    def profile(self, enable: bool):
        _check(self.lib.qtn_profile(self.ctx, int(enable), *self._ws()), "qtn_profile")

    def profile_read(self, kernel_class: int):
        """(total ms, launches, algorithmic FLOPs) of a kernel class: 0 GEMM, 1 eigensolver."""
        ms, n, fl = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        _check(self.lib.qtn_profile_read(self.ctx, kernel_class, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                         *self._ws()), "qtn_profile_read")
        return ms.value, n.value, fl.value

    def amplitudes(self, psi: MPS, digits: torch.Tensor) -> torch.Tensor:
        digits = digits.to(device="cuda", dtype=torch.int32).contiguous()
        out = torch.empty(digits.shape[0], dtype=torch.complex64, device="cuda")
        _check(self.lib.qtn_amplitudes(self.ctx, ctypes.byref(psi.c), ctypes.c_void_p(digits.data_ptr()),
                                       digits.shape[0], ctypes.c_void_p(out.data_ptr()), *self._ws()),
               "qtn_amplitudes")
        return out


def tune_branches(engines, items, Qs, Qds, Ds, chi_max: int, cutoff: float, prec: str, candidates,
                  cache_path: str | None = None):
    """(branches, ms per step) chosen by qtn_batch_tune_branches; the items are advanced by the trial steps."""
    lib = load_library()
    n = len(items)
    ctxs = (ctypes.c_void_p * n)(*[e.ctx.value for e in engines])
    its = (c_mps * n)(*[it.c for it in items])
    qa = (c_mpo * n)(*[q.c for q in Qs])
    qda = (c_mpo * n)(*[q.c for q in Qds])
    da = (c_mpo * n)(*[q.c for q in Ds])
    wss = (ctypes.c_void_p * n)(*[e.ws.data_ptr() for e in engines])
    wsb = (ctypes.c_size_t * n)(*[e.ws_bytes for e in engines])
    cand = (ctypes.c_int * len(candidates))(*candidates)
    best, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib.qtn_batch_tune_branches(n, ctxs, its, qa, qda, da, Engine.trunc(chi_max, cutoff, prec), wss, wsb, cand,
                                       len(candidates), cache_path.encode() if cache_path else None,
                                       ctypes.byref(best), ctypes.byref(ms)), "qtn_batch_tune_branches")
    for it, c in zip(items, its):
        it.c.canon = c.canon
    return best.value, ms.value


class Batch:
    """Fresnel steps of many independent interleaved items recorded as ONE CUDA graph (qtn_batch_create) of
    `branches` parallel branches and launched with one call per step (qtn_batch_launch): item i uses
    engines[i]'s workspace, GEMM tile and operators (Qs[i], Qds[i], Ds[i]); the branches run on the streams of
    the first `branches` engines."""

    def __init__(self, engines, items, Qs, Qds, Ds, n_steps: int, chi_max: int, cutoff: float, prec: str = "fp32",
                 branches: int = 0):
        lib = load_library()
        self.lib, self.count = lib, len(items)
        self._keep = (engines, items, Qs, Qds, Ds)
        n = self.count
        ctxs = (ctypes.c_void_p * n)(*[e.ctx.value for e in engines])
        its = (c_mps * n)(*[it.c for it in items])
        qa = (c_mpo * n)(*[q.c for q in Qs])
        qda = (c_mpo * n)(*[q.c for q in Qds])
        da = (c_mpo * n)(*[q.c for q in Ds])
        wss = (ctypes.c_void_p * n)(*[e.ws.data_ptr() for e in engines])
        wsb = (ctypes.c_size_t * n)(*[e.ws_bytes for e in engines])
        h = ctypes.c_void_p()
        _check(lib.qtn_batch_create(n, ctxs, its, qa, qda, da, n_steps, Engine.trunc(chi_max, cutoff, prec), wss, wsb,
                                    int(branches), ctypes.byref(h)), "qtn_batch_create")
        self.handle = h
        self.stream = engines[0].stream

    def launch(self, repeats: int = 1):
        _check(self.lib.qtn_batch_launch(self.handle, repeats), "qtn_batch_launch")

    def sync(self):
        """Waits for every item and raises for any device-side failure of their replays (qtn_batch_sync)."""
        _check(self.lib.qtn_batch_sync(self.handle), "qtn_batch_sync")

    def close(self):
        if getattr(self, "handle", None) is not None:
            self.lib.qtn_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
