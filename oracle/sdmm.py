"""SDMM for the reweighted analysis problem (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Problem (§3.3 eq. delta): min ||W Psi^H x||_1  s.t. ||y - Phi x||_2 <= eps,
x in R_+^N.  §4.3 eq. cvx2 splits it into f1(L1 x) + f2(L2 x) + f3(L3 x)
with L1 = Psi^H, L2 = Phi, L3 = I, f1 = ||W .||_1, f2 = indicator of the
l2 ball B around y, f3 = indicator of the positive orthant.  Algorithm 1
(S = 3), step by step:

  1  gamma > 0, x_hat(0), z_i(0) = 0
  2  r_i(0) = L_i x_hat(0)
  3  x_i(0) = L_i^H r_i(0)
  4  for t = 1..T:
  5      x_hat(t) = Q^{-1} sum_i x_i(t-1)                  (CG, ``cg``)
  6      for i = 1..3:
  7          r_i(t) = prox_{gamma f_i}(L_i x_hat(t) + z_i(t-1))
  8          z_i(t) = z_i(t-1) + L_i x_hat(t) - r_i(t)
  9          x_i(t) = L_i^H (r_i(t) - z_i(t))
 11      stop if the halting test holds

Readings of what the paper leaves open (the choices made here):

* x is kept complex, as in eq. cvx2 (x in C^N); the image is Re x_hat.
* x_hat(0) = 0, so r_i(0) = 0 and x_i(0) = 0.
* gamma = beta ||Psi^H Phi^H y||_inf with beta = 1e-3 (§4.4), the complex
  modulus inside the max norm, computed once before t = 1.
* Halting test of §4.4: zeta = |f1(t) - f1(t-1)| / |f1(t-1)| < xi = 1e-3 and
  nu = ||y - Phi x_hat(t)|| / eps in [1 - tau, 1 + tau], tau = 0.1, with
  f1(t) = f1(L1 x_hat(t)).  zeta is +inf while f1(t-1) = 0.  Parity runs use
  a fixed T (``stop=False``); the quantities are still recorded.
* CG: warm start from x_hat(t-1), ``cg_iters`` fixed steps.
* Reweighting (§3.3 defers the rule to Candes et al. 2008): round 0 uses
  w = 1; round r >= 1 uses w_j = delta_r / (delta_r + |alpha_j|) with
  alpha = Psi^H x_hat at the end of round r-1 and
  delta_r = max(10^-r ||alpha||_inf, 1e-6 ||alpha||_inf).  All SDMM state
  (x_hat, z_i, x_i, gamma) carries over between rounds.

Pinned by ``tests/test_oracle_sdmm.py``: the fixed point satisfies the
constraints, and on a tiny problem the result approaches an independent
constrained-minimisation solution of eq. delta.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np

from . import cg as cg_mod
from . import prox
from . import tv as tv_mod

BETA = 1e-3
XI = 1e-3
TAU = 0.1


@dataclasses.dataclass
class Operators:
    """The linear operators of eq. cvx2 (callables on complex128 arrays)."""

    phi: Callable[[np.ndarray], np.ndarray]       # L2: C^N -> C^M
    phi_adj: Callable[[np.ndarray], np.ndarray]   # L2^H
    psi_adj: Callable[[np.ndarray], np.ndarray]   # L1 = Psi^H: C^N -> C^D
    psi: Callable[[np.ndarray], np.ndarray]       # L1^H = Psi


@dataclasses.dataclass
class State:
    """SDMM variables after iteration ``t``."""

    x_hat: np.ndarray
    z1: np.ndarray
    z2: np.ndarray
    z3: np.ndarray
    x1: np.ndarray
    x2: np.ndarray
    x3: np.ndarray
    gamma: float
    t: int = 0
    f1_prev: float = 0.0
    history: list = dataclasses.field(default_factory=list)


def penalty(ops: Operators, y: np.ndarray, beta: float = BETA) -> float:
    """gamma = beta ||Psi^H Phi^H y||_inf (§4.4)."""
    return float(beta * np.max(np.abs(ops.psi_adj(ops.phi_adj(y)))))


def init_state(ops: Operators, y: np.ndarray, image_shape, beta: float = BETA) -> State:
    """Algorithm 1 steps 1-3 with x_hat(0) = 0."""
    x0 = np.zeros(image_shape, dtype=np.complex128)
    r1 = ops.psi_adj(x0)
    r2 = ops.phi(x0)
    r3 = x0.copy()
    return State(x_hat=x0, z1=np.zeros_like(r1), z2=np.zeros_like(r2), z3=np.zeros_like(r3),
                 x1=ops.psi(r1), x2=ops.phi_adj(r2), x3=r3.copy(),
                 gamma=penalty(ops, y, beta))


def sdmm_iteration(ops: Operators, st: State, y: np.ndarray, eps: float, w: np.ndarray,
                   cg_iters: int) -> dict:
    """One pass of Algorithm 1 steps 5-9; updates ``st`` in place."""
    def apply_q(v):
        return ops.phi_adj(ops.phi(v)) + 2.0 * v

    # step 5
    b = st.x1 + st.x2 + st.x3
    st.x_hat, cg_res = cg_mod.cg(apply_q, b, st.x_hat, cg_iters)
    # steps 7-9, i = 1 (L1 = Psi^H, f1 = ||W .||_1)
    s1 = ops.psi_adj(st.x_hat)
    r1 = prox.soft_threshold(s1 + st.z1, st.gamma * w)
    st.z1 = st.z1 + s1 - r1
    st.x1 = ops.psi(r1 - st.z1)
    # i = 2 (L2 = Phi, f2 = indicator of the l2 ball around y)
    s2 = ops.phi(st.x_hat)
    r2 = prox.project_l2_ball(s2 + st.z2, y, eps)
    st.z2 = st.z2 + s2 - r2
    st.x2 = ops.phi_adj(r2 - st.z2)
    # i = 3 (L3 = I, f3 = indicator of the positive orthant)
    s3 = st.x_hat
    r3 = prox.project_positive(s3 + st.z3)
    st.z3 = st.z3 + s3 - r3
    st.x3 = r3 - st.z3
    # halting quantities (§4.4)
    f1 = float(np.sum(w * np.abs(s1)))
    zeta = abs(f1 - st.f1_prev) / abs(st.f1_prev) if st.f1_prev != 0.0 else np.inf
    nu = float(np.linalg.norm(y - s2) / eps)
    st.f1_prev = f1
    st.t += 1
    rec = {"t": st.t, "f1": f1, "zeta": zeta, "nu": nu, "cg_residual": cg_res}
    st.history.append(rec)
    return rec


def halted(rec: dict, xi: float = XI, tau: float = TAU) -> bool:
    """The halting test of §4.4."""
    return rec["zeta"] < xi and (1.0 - tau) <= rec["nu"] <= (1.0 + tau)


def reweight(ops: Operators, x_hat: np.ndarray, round_index: int) -> np.ndarray:
    """Weights of reweighting round ``round_index`` >= 1 (rule in the module docstring)."""
    alpha = np.abs(ops.psi_adj(x_hat))
    amax = float(alpha.max())
    delta = max(10.0 ** (-round_index) * amax, 1e-6 * amax)
    if delta == 0.0:
        return np.ones_like(alpha)
    return delta / (delta + alpha)


def solve(ops: Operators, y: np.ndarray, eps: float, image_shape, coeff_shape,
          iters: int, cg_iters: int, rounds: int = 1, stop: bool = False,
          beta: float = BETA, weights: np.ndarray | None = None) -> State:
    """``rounds`` reweighting rounds of ``iters`` SDMM iterations each."""
    st = init_state(ops, y, image_shape, beta)
    w = np.ones(coeff_shape) if weights is None else np.asarray(weights, dtype=np.float64)
    for rnd in range(rounds):
        if rnd > 0:
            w = reweight(ops, st.x_hat, rnd)
        for _ in range(iters):
            rec = sdmm_iteration(ops, st, y, eps, w, cg_iters)
            if stop and halted(rec):
                break
    st.weights = w
    return st


# ---------------------------------------------------------------------------
# Distributed-block form (§4.5 eqs. blocks, dbp1, dbp2)
# ---------------------------------------------------------------------------
# y and Phi are cut into R row blocks y_i, Phi_i (eq. blocks), each with its
# own bound eps_i (eq. dbp1).  Eq. dbp2 is Algorithm 1 with S = R + 2:
# f1 = ||W .||_1 with L1 = Psi^H, f2 = positivity with L2 = I, and f_{i+2}
# the indicator of the ball B_i with L_{i+2} = Phi_i.  Q = sum_i L_i^H L_i =
# Psi Psi^H + I + sum_i Phi_i^H Phi_i = Phi^H Phi + 2I, the same as for one
# ball.  Each block's x_{i+2} = Phi_i^H (r_{i+2} - z_{i+2}) is formed on its
# own (Phi_i^H v_i is Phi^H of v_i placed in block i, zeros elsewhere).
# Halting reading: every nu_i = ||y_i - Phi_i x_hat|| / eps_i in the band.


@dataclasses.dataclass
class BlockState:
    """SDMM variables of eq. dbp2 after iteration ``t`` (per-block lists for f_{i+2})."""

    x_hat: np.ndarray
    z1: np.ndarray
    x1: np.ndarray
    z2: np.ndarray            # positivity (L2 = I)
    x2: np.ndarray
    zb: list                  # z_{i+2}, one array of M_i per block
    xb: list                  # x_{i+2} = Phi_i^H (r_{i+2} - z_{i+2}), images
    gamma: float
    t: int = 0
    f1_prev: float = 0.0
    history: list = dataclasses.field(default_factory=list)


def _block_adj(ops: Operators, v: np.ndarray, offsets, i: int, M: int) -> np.ndarray:
    """Phi_i^H v for v in C^{M_i}."""
    full = np.zeros(M, dtype=np.complex128)
    full[offsets[i]:offsets[i + 1]] = v
    return ops.phi_adj(full)


def init_state_blocks(ops: Operators, y: np.ndarray, offsets, image_shape, beta: float = BETA) -> BlockState:
    """Algorithm 1 steps 1-3 for eq. dbp2 with x_hat(0) = 0 (so every r_i(0), x_i(0) = 0)."""
    x0 = np.zeros(image_shape, dtype=np.complex128)
    R = len(offsets) - 1
    M = int(offsets[-1])
    z1 = np.zeros_like(ops.psi_adj(x0))
    return BlockState(x_hat=x0, z1=z1, x1=ops.psi(z1), z2=x0.copy(), x2=x0.copy(),
                      zb=[np.zeros(offsets[i + 1] - offsets[i], dtype=np.complex128) for i in range(R)],
                      xb=[_block_adj(ops, np.zeros(offsets[i + 1] - offsets[i]), offsets, i, M)
                          for i in range(R)],
                      gamma=penalty(ops, y, beta))


def sdmm_iteration_blocks(ops: Operators, st: BlockState, y: np.ndarray, eps, offsets, w: np.ndarray,
                          cg_iters: int) -> dict:
    """One pass of Algorithm 1 steps 5-9 for eq. dbp2; updates ``st`` in place."""
    def apply_q(v):
        return ops.phi_adj(ops.phi(v)) + 2.0 * v

    R = len(eps)
    M = int(offsets[-1])
    # step 5
    b = st.x1 + st.x2
    for i in range(R):
        b = b + st.xb[i]
    st.x_hat, cg_res = cg_mod.cg(apply_q, b, st.x_hat, cg_iters)
    # f1: L1 = Psi^H
    s1 = ops.psi_adj(st.x_hat)
    r1 = prox.soft_threshold(s1 + st.z1, st.gamma * w)
    st.z1 = st.z1 + s1 - r1
    st.x1 = ops.psi(r1 - st.z1)
    # f2: L2 = I, positivity
    r2 = prox.project_positive(st.x_hat + st.z2)
    st.z2 = st.z2 + st.x_hat - r2
    st.x2 = r2 - st.z2
    # f_{i+2}: L = Phi_i, ball B_i
    s = ops.phi(st.x_hat)
    nus = []
    for i in range(R):
        sl = slice(offsets[i], offsets[i + 1])
        si = s[sl]
        ri = prox.project_l2_ball(si + st.zb[i], y[sl], eps[i])
        st.zb[i] = st.zb[i] + si - ri
        st.xb[i] = _block_adj(ops, ri - st.zb[i], offsets, i, M)
        nus.append(float(np.linalg.norm(y[sl] - si) / eps[i]))
    f1 = float(np.sum(w * np.abs(s1)))
    zeta = abs(f1 - st.f1_prev) / abs(st.f1_prev) if st.f1_prev != 0.0 else np.inf
    st.f1_prev = f1
    st.t += 1
    rec = {"t": st.t, "f1": f1, "zeta": zeta, "nu": max(nus), "nu_min": min(nus), "nu_blocks": nus,
           "cg_residual": cg_res}
    st.history.append(rec)
    return rec


def halted_blocks(rec: dict, xi: float = XI, tau: float = TAU) -> bool:
    """The halting test of §4.4 with every block's nu_i in the band."""
    return rec["zeta"] < xi and rec["nu"] <= 1.0 + tau and rec["nu_min"] >= 1.0 - tau


def solve_blocks(ops: Operators, y: np.ndarray, eps, offsets, image_shape, coeff_shape, iters: int,
                 cg_iters: int, beta: float = BETA, weights: np.ndarray | None = None) -> BlockState:
    """``iters`` SDMM iterations of eq. dbp2 (one reweighting round, fixed count)."""
    st = init_state_blocks(ops, y, offsets, image_shape, beta)
    w = np.ones(coeff_shape) if weights is None else np.asarray(weights, dtype=np.float64)
    for _ in range(iters):
        sdmm_iteration_blocks(ops, st, y, eps, offsets, w, cg_iters)
    return st


# ---------------------------------------------------------------------------
# TV prior (§3.3 eq. tvproblem with the positivity of §6's "TV", §5 weighted TV)
# ---------------------------------------------------------------------------
# Algorithm 1 with S = 3: L1 = I and f1 = ||W grad .||_1 (prox by FGP,
# ``tv.prox_tv``), L2 = Phi with the l2 ball, L3 = I with positivity.  Q is
# again Phi^H Phi + 2I.  Readings: gamma = beta max_j |grad(Phi^H y)|_j (the
# l1 rule of §4.4 with the TV operator in place of Psi^H); the TV weights of
# reweighting round r are delta_r / (delta_r + |grad x_hat|) with delta_r as
# for SARA.


def penalty_tv(ops: Operators, y: np.ndarray, beta: float = BETA) -> float:
    """gamma = beta max |grad(Phi^H y)|."""
    return float(beta * np.max(tv_mod.grad_magnitude(ops.phi_adj(y))))


def init_state_tv(ops: Operators, y: np.ndarray, image_shape, beta: float = BETA) -> State:
    """Algorithm 1 steps 1-3 for the TV problem with x_hat(0) = 0."""
    x0 = np.zeros(image_shape, dtype=np.complex128)
    return State(x_hat=x0, z1=x0.copy(), z2=np.zeros_like(ops.phi(x0)), z3=x0.copy(), x1=x0.copy(),
                 x2=ops.phi_adj(np.zeros_like(ops.phi(x0))), x3=x0.copy(), gamma=penalty_tv(ops, y, beta))


def sdmm_iteration_tv(ops: Operators, st: State, y: np.ndarray, eps: float, w: np.ndarray | None,
                      cg_iters: int, fgp_iters: int = tv_mod.FGP_ITERS) -> dict:
    """One pass of Algorithm 1 steps 5-9 for the (weighted) TV problem."""
    def apply_q(v):
        return ops.phi_adj(ops.phi(v)) + 2.0 * v

    b = st.x1 + st.x2 + st.x3
    st.x_hat, cg_res = cg_mod.cg(apply_q, b, st.x_hat, cg_iters)
    # i = 1 (L1 = I, f1 = ||W grad .||_1)
    r1 = tv_mod.prox_tv(st.x_hat + st.z1, st.gamma, w, fgp_iters)
    st.z1 = st.z1 + st.x_hat - r1
    st.x1 = r1 - st.z1
    # i = 2 (l2 ball), i = 3 (positivity): as for SARA
    s2 = ops.phi(st.x_hat)
    r2 = prox.project_l2_ball(s2 + st.z2, y, eps)
    st.z2 = st.z2 + s2 - r2
    st.x2 = ops.phi_adj(r2 - st.z2)
    r3 = prox.project_positive(st.x_hat + st.z3)
    st.z3 = st.z3 + st.x_hat - r3
    st.x3 = r3 - st.z3
    f1 = tv_mod.tv_norm(st.x_hat, w)
    zeta = abs(f1 - st.f1_prev) / abs(st.f1_prev) if st.f1_prev != 0.0 else np.inf
    nu = float(np.linalg.norm(y - s2) / eps)
    st.f1_prev = f1
    st.t += 1
    rec = {"t": st.t, "f1": f1, "zeta": zeta, "nu": nu, "cg_residual": cg_res}
    st.history.append(rec)
    return rec


def reweight_tv(x_hat: np.ndarray, round_index: int) -> np.ndarray:
    """TV weights of reweighting round ``round_index`` >= 1."""
    g = tv_mod.grad_magnitude(x_hat)
    gmax = float(g.max())
    delta = max(10.0 ** (-round_index) * gmax, 1e-6 * gmax)
    if delta == 0.0:
        return np.ones_like(g)
    return delta / (delta + g)


def solve_tv(ops: Operators, y: np.ndarray, eps: float, image_shape, iters: int, cg_iters: int,
             rounds: int = 1, fgp_iters: int = tv_mod.FGP_ITERS, beta: float = BETA) -> State:
    """``rounds`` reweighting rounds (TV, then RWTV) of ``iters`` SDMM iterations each."""
    st = init_state_tv(ops, y, image_shape, beta)
    w = np.ones(image_shape)
    for rnd in range(rounds):
        if rnd > 0:
            w = reweight_tv(st.x_hat, rnd)
        for _ in range(iters):
            sdmm_iteration_tv(ops, st, y, eps, w, cg_iters, fgp_iters)
    st.weights = w
    return st
