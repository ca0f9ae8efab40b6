"""One SDMM iteration launched kernel by kernel, for kernel profilers.

    python -m paper_1307_4370_gb300.profile_step sdmm1024 [steps]

Builds the named workload's context and state (the data vector is seeded
random visibilities: the kernels' work does not depend on the values), runs
`steps` SDMM iterations without the CUDA graph (so a profiler sees every
launch under its own name) and synchronises.  Launch order of one iteration:
per CG step the forward row and column passes, the Gram gridding and the
inverse column and row passes; then the forward passes of Phi x_hat, the
SARA analysis levels (prior branch) with the degridding, l2 update and
gridding (data branch), the SARA synthesis levels and the inverse passes.
"""
from __future__ import annotations

import math
import sys

import numpy as np
import torch

from . import binding, inputs


def main(argv: list[str]) -> None:
    name = argv[0] if argv else "sdmm1024"
    steps = int(argv[1]) if len(argv) > 1 else 1
    w = inputs.WORKLOADS[name]
    p = inputs.make_problem(w)
    torch.cuda.set_device(0)
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J, tile=32 if w.n >= 512 else 16)
    rng = np.random.default_rng(1)
    y = torch.tensor((rng.standard_normal(w.M) + 1j * rng.standard_normal(w.M)).astype(np.complex64),
                     device="cuda")
    st = ctx.sdmm_state()
    st.init(y, 0.5 * math.sqrt(w.M), cg_iters=w.cg_iters, use_graph=False)
    for _ in range(steps):
        st.step()
    torch.cuda.synchronize()
    print(f"{name}: {steps} SDMM iteration(s) launched kernel by kernel")


if __name__ == "__main__":
    main(sys.argv[1:])
