"""Differentiable measurement and sparsity operators and an unrolled SDMM.

* ``PhiFn`` / ``PhiAdjFn``: y = Phi x and x = Phi^H y (§5 eq. opmodel) as
  ``torch.autograd.Function``s; the backward of each is the other one (the
  adjoint CUDA kernels), which is the vector-Jacobian product of a complex
  linear map under PyTorch's conjugate-Wirtinger convention.
* ``PsiAdjFn`` / ``PsiFn``: the SARA analysis and synthesis (§3.3), each the
  backward of the other.
* ``SDMMUnrolled``: K iterations of Algorithm 1 for the weighted problem
  min ||W Psi^H x||_1 s.t. ||y_w - Phi_w x||_2 <= eps, x >= 0, with
  per-visibility weights w (Phi_w = diag(w) Phi, y_w = diag(w) y; the
  weighting matrices §5 says fold into the measurement operator) and SARA
  weights omega.  The forward keeps the SDMM state every ``checkpoint``
  iterations; the backward recomputes one segment at a time from its
  checkpoint and back-propagates through it, so memory holds one segment's
  graph, not K iterations'.  The x-update is the conjugate-gradient method
  truncated at k steps and is differentiated exactly as run (including its
  data-dependent step sizes), not through the implicit-function shortcut.
  gamma is a constant of the forward (held fixed for the derivative).

The linear operators run in the CUDA library; the entrywise parts (prox,
projections, CG vector updates) are torch operations.
"""
from __future__ import annotations

import torch

from . import binding


class PhiFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return op.phi(x.contiguous().reshape(-1)).clone()

    @staticmethod
    def backward(ctx, gy):
        op = ctx.op
        return op.phi_adj(gy.contiguous()).reshape(op.n, op.n).clone(), None


class PhiAdjFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, op):
        ctx.op = op
        return op.phi_adj(y.contiguous()).reshape(op.n, op.n).clone()

    @staticmethod
    def backward(ctx, gx):
        return ctx.op.phi(gx.contiguous().reshape(-1)).clone(), None


class PsiAdjFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, op):
        ctx.op = op
        return op.sara_analysis(x.contiguous().reshape(-1)).clone()

    @staticmethod
    def backward(ctx, ga):
        op = ctx.op
        return op.sara_synthesis(ga.contiguous().reshape(-1)).reshape(op.n, op.n).clone(), None


class PsiFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, op):
        ctx.op = op
        return op.sara_synthesis(a.contiguous().reshape(-1)).reshape(op.n, op.n).clone()

    @staticmethod
    def backward(ctx, gx):
        return ctx.op.sara_analysis(gx.contiguous().reshape(-1)).clone(), None


def _cdot(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Re <a, b> accumulated in FP64."""
    return (a.real.double() * b.real.double() + a.imag.double() * b.imag.double()).sum()


def _soft(a: torch.Tensor, lam: torch.Tensor) -> torch.Tensor:
    """a / |a| (|a| - lam)^+ with a derivative that stays finite at a = 0."""
    mag = torch.sqrt(a.real * a.real + a.imag * a.imag + 1e-30)
    return a * (torch.relu(mag - lam) / mag)


class _Problem:
    """Operators and data of one weighted problem."""

    def __init__(self, op: binding.Context, y: torch.Tensor, eps: float, gamma: float, cg_iters: int):
        self.op, self.y, self.eps, self.gamma, self.cg_iters = op, y, float(eps), float(gamma), int(cg_iters)

    def phi_w(self, x, wv):
        return wv * PhiFn.apply(x, self.op)

    def phi_w_adj(self, v, wv):
        return PhiAdjFn.apply(wv * v, self.op)

    def iterate(self, state, wv, omega):
        """One pass of Algorithm 1 steps 5-9 (torch, differentiable)."""
        x_hat, z1, z2, z3, x1, x2, x3 = state
        op = self.op

        def apply_q(v):
            return self.phi_w_adj(self.phi_w(v, wv), wv) + 2.0 * v

        # step 5: CG from the previous x_hat, k steps (standard CG, FP64 inner products)
        b = x1 + x2 + x3
        x = x_hat
        r = b - apply_q(x)
        p = r
        rho = _cdot(r, r)
        for _ in range(self.cg_iters):
            q = apply_q(p)
            pq = _cdot(p, q)
            alpha = torch.where(pq > 0, rho / torch.where(pq > 0, pq, torch.ones_like(pq)), torch.zeros_like(pq))
            x = x + alpha.to(torch.float32) * p
            r = r - alpha.to(torch.float32) * q
            rho_new = _cdot(r, r)
            beta = torch.where(rho > 0, rho_new / torch.where(rho > 0, rho, torch.ones_like(rho)), torch.zeros_like(rho))
            p = r + beta.to(torch.float32) * p
            rho = rho_new
        x_hat = x
        # i = 1: weighted soft threshold on Psi^H x_hat
        s1 = PsiAdjFn.apply(x_hat, op).reshape(z1.shape)
        a1 = s1 + z1
        r1 = _soft(a1, self.gamma * omega)
        z1 = a1 - r1
        x1 = PsiFn.apply(r1 - z1, op)
        # i = 2: projection onto the l2 ball around y_w
        yw = wv * self.y
        s2 = self.phi_w(x_hat, wv)
        a2 = s2 + z2
        d = a2 - yw
        nd = torch.sqrt(_cdot(d, d))
        scale = torch.clamp(self.eps / nd, max=1.0).to(torch.float32)
        r2 = yw + scale * d
        z2 = a2 - r2
        x2 = self.phi_w_adj(r2 - z2, wv)
        # i = 3: positive orthant
        a3 = x_hat + z3
        r3 = torch.complex(torch.relu(a3.real), torch.zeros_like(a3.real))
        z3 = a3 - r3
        x3 = r3 - z3
        return (x_hat, z1, z2, z3, x1, x2, x3)


def initial_state(op: binding.Context) -> tuple:
    dev = op.device
    zi = torch.zeros((op.n, op.n), dtype=torch.complex64, device=dev)
    return (zi, torch.zeros((op.q, op.n, op.n), dtype=torch.complex64, device=dev),
            torch.zeros(op.M, dtype=torch.complex64, device=dev), zi.clone(), zi.clone(), zi.clone(), zi.clone())


def penalty(op: binding.Context, y: torch.Tensor, wv: torch.Tensor, beta: float = 1e-3) -> float:
    """gamma = beta ||Psi^H Phi_w^H y_w||_inf (§4.4)."""
    with torch.no_grad():
        d = op.phi_adj((wv * wv * y).contiguous())
        return float(beta * op.sara_analysis(d.reshape(-1)).abs().max().item())


class SDMMUnrolled(torch.autograd.Function):
    """x_K of K SDMM iterations as a function of (w, omega), with checkpointing."""

    @staticmethod
    def forward(ctx, wv, omega, problem: _Problem, K: int, checkpoint: int):
        state = initial_state(problem.op)
        saved = []
        with torch.no_grad():
            for t in range(K):
                if t % checkpoint == 0:
                    saved.append(tuple(s.clone() for s in state))
                state = problem.iterate(state, wv, omega)
        ctx.problem, ctx.K, ctx.checkpoint = problem, K, checkpoint
        ctx.saved_states = saved
        ctx.save_for_backward(wv, omega)
        return state[0].clone()

    @staticmethod
    def backward(ctx, g_x):
        wv, omega = ctx.saved_tensors
        problem, K, C = ctx.problem, ctx.K, ctx.checkpoint
        g_w = torch.zeros_like(wv)
        g_om = torch.zeros_like(omega)
        # adjoint of the state after iteration K: only x_hat is an output
        adj = None
        for seg in reversed(range(len(ctx.saved_states))):
            t0 = seg * C
            t1 = min(K, t0 + C)
            with torch.enable_grad():
                st = tuple(s.detach().requires_grad_(True) for s in ctx.saved_states[seg])
                w_ = wv.detach().requires_grad_(True)
                o_ = omega.detach().requires_grad_(True)
                cur = st
                for _ in range(t0, t1):
                    cur = problem.iterate(cur, w_, o_)
                if adj is None:
                    outs, grads = [cur[0]], [g_x]
                else:
                    outs = [c for c, a in zip(cur, adj) if a is not None]
                    grads = [a for a in adj if a is not None]
                got = torch.autograd.grad(outs, list(st) + [w_, o_], grads, allow_unused=True)
            adj = list(got[:len(st)])
            if got[len(st)] is not None:
                g_w += got[len(st)]
            if got[len(st) + 1] is not None:
                g_om += got[len(st) + 1]
        ctx.saved_states = None
        return g_w, g_om, None, None, None


def sdmm_unrolled(op: binding.Context, y: torch.Tensor, eps: float, wv: torch.Tensor, omega: torch.Tensor,
                  K: int = 20, cg_iters: int = 10, checkpoint: int = 5, gamma: float | None = None) -> torch.Tensor:
    """x_K as a differentiable function of the visibility weights wv (M, real)
    and the SARA weights omega (q, n, n, real)."""
    if gamma is None:
        gamma = penalty(op, y, wv.detach())
    problem = _Problem(op, y, eps, gamma, cg_iters)
    return SDMMUnrolled.apply(wv, omega, problem, int(K), int(checkpoint))
