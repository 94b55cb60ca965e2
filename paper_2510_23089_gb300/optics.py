"""Phase-mask optimisation through one Fresnel step, on quantics MPS.

The differentiation workload: a field E is multiplied elementwise by a mask M, propagated by one Fresnel
step U (Sec. VI.A), its intensity I = |U(E M)|^2 is compared with a target I_t, and the loss
L = sum_x (I - I_t)^2 is differentiated with respect to the mask.  The mask product and the intensity are
elementwise products of MPS (Sec. V, Eq. psf_eq), applied by zip-up with truncation.

The adjoint is taken at fixed truncation ranks (the truncations are treated as the identity): with
F' = U (E M) and R = I - I_t,
    dL/d conj(F') = 2 R F',   dL/d conj(E M) = U^dagger (2 R F'),   G = dL/d conj(M) = conj(E) U^dagger (2 R F'),
where U^dagger is the Fresnel step with the conjugate transfer function (parameter -c).  The gradient with
respect to the mask's site tensors follows from G by the overlap derivative (qtn_overlap_grad).  Nothing
here stores site environments between the passes: the backward pass recomputes what it needs.

Every product, propagation, truncation and contraction runs in libqtn through the C ABI; this module only
sequences the calls and holds the intermediate states.
"""
from __future__ import annotations

import torch

from . import qtn


class IntensityLossProblem:
    """Operators and truncation settings of the loss for interleaved fields of n sites per axis."""

    def __init__(self, eng: "qtn.Engine", n: int, c: float, chi: int, cutoff: float = 1e-10, w_cap: int = 16,
                 chi_intensity: int | None = None):
        self.eng, self.n, self.c, self.chi, self.cutoff = eng, n, c, chi, cutoff
        self.chi_i = chi_intensity or chi
        self.Q = eng.build_qft_mpo(n, False, 1e-12, w_cap=w_cap)
        self.Qd = eng.mpo_dagger(self.Q)
        # the phase builders need a 2^n dense scratch of their own
        eng_p = qtn.Engine(n_sites=n, d=2, chi=16, w=2, dense=1 << n)
        self.D = eng_p.build_phase_mpo(n, c, 1e-12, w_cap=w_cap)
        self.Dadj = eng_p.build_phase_mpo(n, -c, 1e-12, w_cap=w_cap)

    def _right_canonical(self, psi: "qtn.MPS", chi: int):
        if psi.canon != "right":
            self.eng.truncate(psi, chi, self.cutoff, stats=False)

    def forward(self, E: "qtn.MPS", M: "qtn.MPS", It: "qtn.MPS"):
        """Returns (loss, cache) with cache = (F', R) for the backward pass."""
        eng = self.eng
        F = E.clone()
        eng.hadamard_zipup(M, F, self.chi, self.cutoff, stats=False)                     # E (.) M
        eng.fresnel_step(F, "interleaved", self.Q, self.Qd, self.D, 1, self.chi, self.cutoff, stats=False)
        I = F.clone()
        eng.hadamard_zipup(F, I, self.chi_i, self.cutoff, conj_b=True, stats=False)      # |F'|^2
        self._right_canonical(I, self.chi_i)
        neg = It.clone()
        self._right_canonical(neg, neg.chi_cap)
        eng.scale(neg, -1.0)
        R = qtn.MPS(self.n, 4, I.chi_cap + neg.chi_cap)
        eng.add(I, neg, R)
        eng.truncate(R, self.chi_i, self.cutoff, stats=False)                           # R = I - I_t
        return eng.norm2(R), (F, R)

    def backward(self, E: "qtn.MPS", M: "qtn.MPS", cache):
        """Returns (G, H): G = dL/d conj(M) as an MPS, H = dL/d conj(site tensors of M) (M's layout)."""
        eng = self.eng
        F, R = cache
        G = R.clone()
        eng.scale(G, 2.0)
        eng.hadamard_zipup(F, G, self.chi, self.cutoff, stats=False)                     # 2 R (.) F'
        eng.fresnel_step(G, "interleaved", self.Q, self.Qd, self.Dadj, 1, self.chi, self.cutoff, stats=False)
        eng.hadamard_zipup(E, G, self.chi, self.cutoff, conj_b=True, stats=False)        # conj(E) (.) U^dag(...)
        return G, eng.overlap_grad(M, G)


class FresnelIntensityLoss(torch.autograd.Function):
    """L(mask site tensors) for a fixed field and target; backward by the adjoint above.

    forward(mask_sites, problem, E, M, It): mask_sites is a complex64 tensor in M's padded site layout
    (M provides the bonds); returns the loss as a float64 scalar.  The gradient follows PyTorch's complex
    convention (twice the conjugate Wirtinger derivative for a real loss)."""

    @staticmethod
    def forward(ctx, mask_sites, problem, E, M, It):
        M.sites.copy_(mask_sites)
        loss, cache = problem.forward(E, M, It)
        ctx.problem, ctx.E, ctx.M, ctx.cache = problem, E, M, cache
        return torch.tensor(loss, dtype=torch.float64, device=mask_sites.device)

    @staticmethod
    def backward(ctx, grad_out):
        _, H = ctx.problem.backward(ctx.E, ctx.M, ctx.cache)
        return 2.0 * grad_out.to(H.dtype) * H, None, None, None, None
