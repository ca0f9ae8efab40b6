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
  weights omega.  Each iteration is the library's purify_diff_iteration
  (CUDA kernels; the CG step sizes in FP64 on the host) and its backward
  the library's purify_diff_iteration_vjp: CG reversed from the step sizes
  and vectors on the tape, and the Jacobians of the soft threshold, the
  l2-ball projection and the positivity projection.  The forward keeps the
  SDMM state every ``checkpoint`` iterations; the backward re-runs one
  segment at a time from its checkpoint (with tapes) and reverses it, so
  memory holds one segment's tapes, not K iterations'.  The x-update is
  the conjugate-gradient method truncated at k steps and is differentiated
  exactly as run (including its data-dependent step sizes), not through the
  implicit-function shortcut.  gamma is a constant of the forward (held
  fixed for the derivative).

Every arithmetic step runs in the CUDA library; torch holds the tensors and
the autograd graph.
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


def initial_state(op: binding.Context) -> list:
    """Algorithm 1 steps 1-3 with x_hat(0) = 0: every state array zero."""
    return [torch.zeros(n, dtype=torch.complex64, device=op.device) for n in op.diff_state_shapes()]


def penalty(op: binding.Context, y: torch.Tensor, wv: torch.Tensor, beta: float = 1e-3) -> float:
    """gamma = beta ||Psi^H Phi_w^H y_w||_inf (§4.4), on the device."""
    return op.diff_penalty(y.contiguous(), wv.detach().contiguous(), beta)


class _Problem:
    """Operators and data of one weighted problem."""

    def __init__(self, op: binding.Context, y: torch.Tensor, eps: float, gamma: float, cg_iters: int):
        self.op, self.y, self.eps, self.gamma, self.cg_iters = op, y.contiguous(), float(eps), float(gamma), int(cg_iters)

    def step(self, state, wv, omega, tape):
        """One iteration of Algorithm 1 (purify_diff_iteration), its tape filled."""
        out = [torch.empty_like(t) for t in state]
        self.op.diff_iteration(self.y, wv, omega, self.gamma, self.eps, self.cg_iters, state, out, tape)
        return out

    def step_vjp(self, state, tape, bar_out, wv, omega, w_bar, om_bar):
        """Adjoints of one iteration's inputs (purify_diff_iteration_vjp); adds to w_bar, om_bar."""
        bar_in = [torch.empty_like(t) for t in state]
        self.op.diff_iteration_vjp(self.y, wv, omega, self.gamma, self.eps, self.cg_iters, state, tape, bar_out,
                                   bar_in, w_bar, om_bar)
        return bar_in


class SDMMUnrolled(torch.autograd.Function):
    """x_K of K SDMM iterations as a function of (w, omega), with checkpointing.

    Forward: K calls of the library's differentiable iteration, keeping the
    state every ``checkpoint`` iterations.  Backward: per segment (last
    first), the iterations are re-run from the segment's checkpoint with
    their tapes kept, then reversed one by one with the hand-written
    vector-Jacobian product of the library (CG reversed from its stored step
    sizes and vectors, the Jacobians of the three proximity operators).
    Memory holds one segment's states and tapes, not K iterations'."""

    @staticmethod
    def forward(ctx, wv, omega, problem: _Problem, K: int, checkpoint: int):
        wv_c = wv.detach().contiguous()
        om_c = omega.detach().contiguous().reshape(-1)
        state = initial_state(problem.op)
        tape = problem.op.diff_tape(problem.cg_iters)
        saved = []
        for t in range(K):
            if t % checkpoint == 0:
                saved.append([s.clone() for s in state])
            state = problem.step(state, wv_c, om_c, tape)
        ctx.problem, ctx.K, ctx.checkpoint = problem, K, checkpoint
        ctx.saved_states = saved
        ctx.save_for_backward(wv, omega)
        n = problem.op.n
        return state[0].reshape(n, n).clone()

    @staticmethod
    def backward(ctx, g_x):
        wv, omega = ctx.saved_tensors
        problem, K, C = ctx.problem, ctx.K, ctx.checkpoint
        op = problem.op
        wv_c = wv.detach().contiguous()
        om_c = omega.detach().contiguous().reshape(-1)
        w_bar = torch.zeros_like(wv_c)
        om_bar = torch.zeros_like(om_c)
        # adjoint of the state after iteration K: only x_hat is an output
        bar = [torch.zeros(n, dtype=torch.complex64, device=op.device) for n in op.diff_state_shapes()]
        bar[0] = g_x.detach().to(torch.complex64).contiguous().reshape(-1).clone()
        for seg in reversed(range(len(ctx.saved_states))):
            t0 = seg * C
            t1 = min(K, t0 + C)
            states, tapes = [], []
            cur = ctx.saved_states[seg]
            for _ in range(t0, t1):
                tape = op.diff_tape(problem.cg_iters)
                states.append(cur)
                tapes.append(tape)
                cur = problem.step(cur, wv_c, om_c, tape)
            for st, tape in zip(reversed(states), reversed(tapes)):
                bar = problem.step_vjp(st, tape, bar, wv_c, om_c, w_bar, om_bar)
            del states, tapes
        ctx.saved_states = None
        return w_bar.reshape(wv.shape), om_bar.reshape(omega.shape), None, None, None


def sdmm_unrolled(op: binding.Context, y: torch.Tensor, eps: float, wv: torch.Tensor, omega: torch.Tensor,
                  K: int = 20, cg_iters: int = 10, checkpoint: int = 5, gamma: float | None = None) -> torch.Tensor:
    """x_K as a differentiable function of the visibility weights wv (M, real)
    and the SARA weights omega (q, n, n, real)."""
    if gamma is None:
        gamma = penalty(op, y, wv.detach())
    problem = _Problem(op, y, eps, gamma, cg_iters)
    return SDMMUnrolled.apply(wv, omega, problem, int(K), int(checkpoint))
