"""Batched SDMM over uneven problems (needs a GB300).

Problems of different image sides, visibility counts and kernel supports,
advanced together by purify_batch_step, must follow exactly the iterates each
would have alone (the batch only changes the schedule), and the small one must
match the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import sdmm as osdmm, simulate
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

SPECS = [(64, 1500, 4, 11), (96, 6000, 6, 12), (128, 3000, 4, 13), (192, 30000, 6, 14)]


def make(spec):
    n, M, J, seed = spec
    w = inputs.Workload(f"b{n}", n=n, M=M, J=J, n_src=10, diffuse=False, seed=seed)
    p = inputs.make_problem(w)
    y, eps = simulate.visibilities(p.x_true, p.uv, J, p.noise_unit, 30.0)
    return w, p, y.astype(np.complex64).astype(np.complex128), eps


def test_batch_matches_single_problems_and_oracle():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    iters = 6
    probs = [make(s) for s in SPECS]
    ctxs, states = [], []
    for w, p, y, eps in probs:
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps)
        ctxs.append(ctx)
        states.append(st)
    batch = binding.Batch(states)
    batch.step(iters)
    assert batch.kernels_per_iteration() > 0
    torch.cuda.synchronize()
    xb = [host(st.get_image()) for st in states]
    for k, (w, p, y, eps) in enumerate(probs):
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps)
        for _ in range(iters):
            st.step()
        assert rel_err(xb[k], host(st.get_image())) <= 1e-6
        assert st.report()["iters"] == iters and states[k].report()["iters"] == iters
    w, p, y, eps = probs[0]
    ref = osdmm.solve(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), (9, w.n, w.n),
                      iters=iters, cg_iters=w.cg_iters)
    assert rel_err(xb[0], ref.x_hat) <= 1e-4
    batch.close()


def test_batch_rejects_shared_context():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    w, p, y, eps = make(SPECS[0])
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    a, b = ctx.sdmm_state(), ctx.sdmm_state()
    with pytest.raises(binding.PurifyError):
        binding.Batch([a, b])


def test_batch_with_mixed_forms():
    """One batch of problems that use the options of the state: the TV prior,
    the distributed data blocks, the Gaussian kernel with a primary beam; each
    follows the iterates it has alone."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    iters = 5
    probs = [make(s) for s in SPECS[:3]]

    def build(k, w, p, y, eps):
        kernel = "gauss" if k == 2 else "kb"
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J, kernel=kernel)
        if k == 2:
            ctx.set_beam(np.linspace(0.5, 1.0, w.n * w.n).reshape(w.n, w.n))
        st = ctx.sdmm_state()
        if k == 0:
            st.set_prior("tv", fgp_iters=10)
        st.init(dev(y, torch), eps)
        if k == 1:
            st.set_blocks([0, w.M // 3, w.M], [eps * 0.6, eps * 0.8])
        return ctx, st

    made = [build(k, *pr) for k, pr in enumerate(probs)]
    batch = binding.Batch([st for _, st in made])
    batch.step(iters)
    torch.cuda.synchronize()
    xb = [host(st.get_image()) for _, st in made]
    for k, pr in enumerate(probs):
        _, st = build(k, *pr)
        for _ in range(iters):
            st.step()
        assert rel_err(xb[k], host(st.get_image())) <= 1e-6
    batch.close()
