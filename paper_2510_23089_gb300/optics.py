"""Phase-mask optimisation through one Fresnel step, on quantics MPS.

The differentiation workload: a field E is multiplied elementwise by a mask M, propagated by one Fresnel
step U (Sec. VI.A), its intensity I = |U(E M)|^2 is compared with a target I_t, and the loss
L = sum_x (I - I_t)^2 is differentiated with respect to the mask.  The mask product and the intensity are
elementwise products of MPS (Sec. V, Eq. psf_eq), applied by zip-up with truncation.

Each zip-up pass applies an operator K and writes N - 1 isometric sites (its frame V) and a centre; the
forward pass records the state after the mask product and after each of the six passes of the step
(Q_x, Q_y, D_x, D_y, Q^dagger_x, Q^dagger_y).  With F' the output and R = I - I_t,
    dL/d conj(F') = 2 R F'.
Two adjoints of the step, both at the truncation ranks of the forward pass:

* "frozen": every pass is taken as the linear map psi -> V V^dagger K psi with its recorded frame held fixed;
  the cotangent is projected onto each recorded frame and taken back through K^dagger
  (qtn_project_apply), ending at conj(E) . (V_0 V_0^dagger g).  This is the exact derivative of the forward
  map with the truncation subspaces frozen; the frames span the ranges of the state's unfoldings, so it is
  the gradient restricted to the recorded subspaces.
* "exact": the cotangent is taken back through K^dagger pass by pass by zip-up (the step with the conjugate
  transfer function, -c) with the same truncation rule; when nothing is truncated this is the full gradient
  conj(E) U^dagger (2 R F').

The gradient with respect to the mask's site tensors follows from the mask-field gradient by the overlap
derivative (qtn_overlap_grad).  The backward pass keeps no site environments between passes: each
projection and each overlap derivative recomputes the transfer matrices it needs.

Every product, propagation, projection, truncation and contraction runs in libqtn through the C ABI; this
module only sequences the calls and holds the intermediate states.
"""
from __future__ import annotations

import torch

from . import qtn


class IntensityLossProblem:
    """Operators and truncation settings of the loss for interleaved fields of n sites per axis."""

    def __init__(self, eng: "qtn.Engine", n: int, c: float, chi: int, cutoff: float = 1e-10, w_cap: int = 16,
                 chi_intensity: int | None = None, adjoint: str = "exact"):
        if adjoint not in ("exact", "frozen"):
            raise ValueError(adjoint)
        self.eng, self.n, self.c, self.chi, self.cutoff = eng, n, c, chi, cutoff
        self.chi_i = chi_intensity or chi
        self.adjoint = adjoint
        self.Q = eng.build_qft_mpo(n, False, 1e-12, w_cap=w_cap)
        self.Qd = eng.mpo_dagger(self.Q)
        self.D = eng.build_phase_mpo(n, c, 1e-12, w_cap=w_cap)
        self.Dd = eng.mpo_dagger(self.D)
        self.Dadj = eng.build_phase_mpo(n, -c, 1e-12, w_cap=w_cap)
        # the six passes of the step and the adjoint operator of each
        self.passes = [(self.Q, 0), (self.Q, 1), (self.D, 0), (self.D, 1), (self.Qd, 0), (self.Qd, 1)]
        self.adjoints = [(self.Qd, 0), (self.Qd, 1), (self.Dd, 0), (self.Dd, 1), (self.Q, 0), (self.Q, 1)]

    def _right_canonical(self, psi: "qtn.MPS", chi: int):
        if psi.canon != "right":
            self.eng.truncate(psi, chi, self.cutoff, stats=False)

    def forward(self, E: "qtn.MPS", M: "qtn.MPS", It: "qtn.MPS"):
        """Returns (loss, cache); cache holds the output F', the residual R and the recorded frames."""
        eng = self.eng
        F = E.clone()
        eng.hadamard_zipup(M, F, self.chi, self.cutoff, stats=False)                     # E (.) M
        frames = [F.clone()] if self.adjoint == "frozen" else None
        for W, axis in self.passes:
            eng.apply_mpo(W, axis, F, self.chi, self.cutoff, stats=False)
            if frames is not None:
                frames.append(F.clone())
        I = F.clone()
        eng.hadamard_zipup(F, I, self.chi_i, self.cutoff, conj_b=True, stats=False)      # |F'|^2
        self._right_canonical(I, self.chi_i)
        neg = It.clone()
        self._right_canonical(neg, neg.chi_cap)
        eng.scale(neg, -1.0)
        R = qtn.MPS(self.n, 4, I.chi_cap + neg.chi_cap)
        eng.add(I, neg, R)
        eng.truncate(R, self.chi_i, self.cutoff, stats=False)                           # R = I - I_t
        return eng.norm2(R), (F, R, frames)

    def backward(self, E: "qtn.MPS", M: "qtn.MPS", cache):
        """Returns (G, H): G = dL/d conj(M) as an MPS, H = dL/d conj(site tensors of M) (M's layout)."""
        eng = self.eng
        F, R, frames = cache
        G = R.clone()
        eng.scale(G, 2.0)
        eng.hadamard_zipup(F, G, self.chi_i, self.cutoff, stats=False)                   # 2 R (.) F'
        if self.adjoint == "frozen":
            H = frames[6].clone()
            eng.project_apply(None, 0, G, H)                                             # V_6 V_6^dagger g
            for i in range(6, 0, -1):
                W, axis = self.adjoints[i - 1]
                Hn = frames[i - 1].clone()
                eng.project_apply(W, axis, H, Hn)                                        # V V^dagger K_i^dagger h
                H = Hn
            G = H
        else:
            eng.fresnel_step(G, "interleaved", self.Q, self.Qd, self.Dadj, 1, self.chi, self.cutoff, stats=False)
        eng.hadamard_zipup(E, G, self.chi_i, self.cutoff, conj_b=True, stats=False)      # conj(E) (.) ...
        return G, eng.overlap_grad(M, G)


def sum_over_ranks_(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sums `t` in place over the ranks of `group` (the default process group when None) and returns it; a
    no-op without an initialised process group of more than one rank.

    The batch of the mask-learning workload shards by item (every rank holds some of the fields and
    targets, all ranks the same mask); the gradient of the batch loss with respect to the shared mask is
    the sum of the per-item gradients, so this all-reduce (one mask gradient, ~100 KB at chi = 16) is the
    only exchange between ranks.  Complex tensors are reduced through their real view."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) <= 1:
        return t
    dist.all_reduce(torch.view_as_real(t) if t.is_complex() else t, op=dist.ReduceOp.SUM, group=group)
    return t


def batch_loss_and_gradient(problem: "IntensityLossProblem", fields, targets, M: "qtn.MPS", group=None):
    """Loss summed over this rank's items (fields[i], targets[i]) for the shared mask M, and its gradient
    with respect to M's site tensors (M's padded layout), both summed over the ranks of `group`."""
    total, H_sum = 0.0, None
    with torch.cuda.stream(problem.eng.stream):     # the sums follow the engine's work on its stream
        for E, It in zip(fields, targets):
            loss, cache = problem.forward(E, M, It)
            _, H = problem.backward(E, M, cache)
            total += loss
            H_sum = H.clone() if H_sum is None else H_sum.add_(H)
        loss_t = torch.tensor([total], dtype=torch.float64, device=H_sum.device)
        sum_over_ranks_(loss_t, group)
        sum_over_ranks_(H_sum, group)
        value = float(loss_t.item())
    return value, H_sum


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
