"""Plain, slow, FP64 CPU oracle of the quantics-MPS Fresnel hot path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import anything from here; the
library path never does, and this package imports nothing from the library.

Everything is NumPy complex128 with LAPACK SVD/QR as library steps.  Each
function states the passage of arXiv:2510.23089 it follows:

* quantics index maps ............ Sec. III (quantics representation, mu_p = (x_p y_p)_2)
* TT-SVD, canonical forms ........ Sec. IV (MPS factorisation), App. A (Schmidt decomposition per bond)
* MPO x MPS, Hadamard ............ Sec. V (Fig. fig_mpo, Eq. hadamard)
* QFT MPO ........................ Sec. V (QFT as a finite-rank MPO); Sec. VI.A (MPO by SVD of a dense operator, Fig. MPO_construction)
* Fresnel transfer function ...... Sec. VI.A (paraxial factorisation T_z(f) = exp(-i pi lambda z f^2)),
                                   Fig. fig_mpo_mpo (U_QFT^dagger U(z) U_QFT)
* elementwise product ............ Sec. V (Eq. psf_eq, local contraction of physical indices)
* Hilbert transform .............. Sec. VI.C (U_QFT^dagger (-i Z_n) U_QFT)
"""
from . import quantics, mps, mpo, apply, fresnel  # noqa: F401
