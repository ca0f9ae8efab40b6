"""Writes the stored expected values of the full-size parity tests.

Only the FP64 oracle (``oracle/``) and the seeded input recipe
(``paper_1307_4370_gb300/inputs.py``) are called here: nothing comes from the
CUDA path.  The oracle takes minutes at these sizes, too long to rerun inside
every GPU test, so its results are kept as small .npz files next to this
script: the final iterate at a seeded sample of pixels, its l2 norm and the
halting quantities of §4.4.

    python tests/golden/make_golden.py sdmm256_rounds   # Algorithm 1, 2 x 30 iterations, one reweighting
    python tests/golden/make_golden.py sdmm1024_k10     # Algorithm 1, 2 iterations of 10 CG steps
    python tests/golden/make_golden.py diff256_fd       # central differences of an unrolled 20-iteration loss
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import measurement as me, sara, sdmm, simulate  # noqa: E402
from paper_1307_4370_gb300 import inputs  # noqa: E402

SAMPLE = 16384      # pixels of the final image kept
SAMPLE_SEED = 4370  # seed of the pixel sample


def data(name):
    """The workload's image, coverage and noisy visibilities (complex64-rounded), and eps."""
    p = inputs.make_problem(name)
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db)
    return p, y.astype(np.complex64).astype(np.complex128), eps


def sample_index(N: int) -> np.ndarray:
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(N, min(SAMPLE, N), replace=False))


def save(name: str, st, **extra):
    x = st.x_hat.ravel()
    idx = sample_index(x.size)
    last = st.history[-1]
    np.savez_compressed(os.path.join(HERE, name + ".npz"), idx=idx, x=x[idx], x_norm=np.linalg.norm(x),
                        nu=last["nu"], f1=last["f1"], zeta=last["zeta"], gamma=st.gamma,
                        t=st.t, **extra)


def sdmm256_rounds():
    """256^2, M = 65536, J = 6: two reweighting rounds of 30 iterations, k = 10 (§4.4, §3.3)."""
    p, y, eps = data("sdmm256")
    w = p.workload
    st = sdmm.solve(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), (9, w.n, w.n),
                    iters=30, cg_iters=10, rounds=2)
    round0 = st.history[29]
    save("sdmm256_rounds", st, nu_round0=round0["nu"], f1_round0=round0["f1"])


def sdmm1024_k10():
    """1024^2, M = 2^21 with radial arcs, J = 6: two iterations of 10 CG steps each."""
    p, y, eps = data("sdmm1024")
    w = p.workload
    st = sdmm.solve(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), (9, w.n, w.n),
                    iters=2, cg_iters=10)
    save("sdmm1024_k10", st)


# Differentiation workload (256^2, M = 65536, J = 6): loss ||x_K - x_true||^2
# after K = 20 iterations of 10 CG steps of the weighted problem (visibility
# weights w fold into Phi and y), as a function of w and of the SARA weights
# omega; central differences of the oracle's loss along one seeded direction
# of each, h = 1e-5.  The loss is only piecewise smooth (the soft threshold
# switches entries on and off), and along omega the differences move by a
# few 1e-3 relative between h = 1e-3 and 1e-4 as thresholds are crossed; at
# h = 1e-5 they have settled, and the FP64 round-off of the difference
# (~1e-16 loss / h) stays near 1e-11.
DIFF_K, DIFF_CG, DIFF_H, DIFF_SEED = 20, 10, 1e-5, 2024


def diff_inputs(M: int, n: int):
    """Seeded base weights (near 1) and directions, rounded to float32."""
    rng = np.random.default_rng(DIFF_SEED)
    wv0 = (1.0 + 0.1 * rng.uniform(-1, 1, M)).astype(np.float32).astype(np.float64)
    om0 = (1.0 + 0.1 * rng.uniform(-1, 1, (9, n, n))).astype(np.float32).astype(np.float64)
    dw = rng.standard_normal(M).astype(np.float32).astype(np.float64)
    dom = rng.standard_normal((9, n, n)).astype(np.float32).astype(np.float64)
    return wv0, om0, dw, dom


def weighted_loss(p, y, eps, wv, omega, gamma, K, cg_iters):
    """||x_K - x_true||^2 of the oracle's Algorithm 1 on the weighted problem."""
    w = p.workload
    ops = sdmm.Operators(
        phi=lambda x: wv * me.phi(x, p.uv, w.J),
        phi_adj=lambda v: me.phi_adj(wv * v, p.uv, w.n, w.J),
        psi_adj=lambda x: sara.sara_analysis(x, 4),
        psi=lambda a: sara.sara_synthesis(a, 4))
    yw = wv * y
    st = sdmm.init_state(ops, yw, (w.n, w.n))
    st.gamma = gamma
    for _ in range(K):
        sdmm.sdmm_iteration(ops, st, yw, eps, omega, cg_iters)
    return float(np.sum(np.abs(st.x_hat - p.x_true) ** 2))


def diff256_fd():
    p, y, eps = data("diff256")
    w = p.workload
    wv0, om0, dw, dom = diff_inputs(w.M, w.n)
    gamma = 1e-3 * float(np.max(np.abs(sara.sara_analysis(me.phi_adj(wv0 * wv0 * y, p.uv, w.n, w.J), 4))))
    L = lambda wv, om: weighted_loss(p, y, eps, wv, om, gamma, DIFF_K, DIFF_CG)  # noqa: E731
    L0 = L(wv0, om0)
    fd_w = (L(wv0 + DIFF_H * dw, om0) - L(wv0 - DIFF_H * dw, om0)) / (2 * DIFF_H)
    fd_om = (L(wv0, om0 + DIFF_H * dom) - L(wv0, om0 - DIFF_H * dom)) / (2 * DIFF_H)
    np.savez_compressed(os.path.join(HERE, "diff256_fd.npz"), loss=L0, fd_w=fd_w, fd_om=fd_om, gamma=gamma,
                        eps=eps, K=DIFF_K, cg_iters=DIFF_CG, h=DIFF_H, seed=DIFF_SEED)


CASES = {"sdmm256_rounds": sdmm256_rounds, "sdmm1024_k10": sdmm1024_k10, "diff256_fd": diff256_fd}

if __name__ == "__main__":
    for name in sys.argv[1:] or sorted(CASES):
        CASES[name]()
        print("wrote", name)
