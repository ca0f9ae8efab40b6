"""Writes the stored expected values of the full-size parity tests.

Only the FP64 oracle (``oracle/``) and the seeded input recipe
(``paper_1307_4370_gb300/inputs.py``) are called here: nothing comes from the
CUDA path.  The oracle takes minutes at these sizes, too long to rerun inside
every GPU test, so its results are kept as small .npz files next to this
script: the final iterate at a seeded sample of pixels, its l2 norm and the
halting quantities of §4.4.

    python tests/golden/make_golden.py sdmm256_rounds   # Algorithm 1, 2 x 30 iterations, one reweighting
    python tests/golden/make_golden.py sdmm1024_k10     # Algorithm 1, 2 iterations of 10 CG steps
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import sdmm, simulate  # noqa: E402
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


CASES = {"sdmm256_rounds": sdmm256_rounds, "sdmm1024_k10": sdmm1024_k10}

if __name__ == "__main__":
    for name in sys.argv[1:] or sorted(CASES):
        CASES[name]()
        print("wrote", name)
