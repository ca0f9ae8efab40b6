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


def test_batch_recaptures_after_state_changes():
    """A batch step after purify_sdmm_set_blocks / set_prior / set_data_bf16 on
    one of its states must run the new form of that problem (its graph is
    re-captured), matching the problem stepped on its own."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    probs = [make(s) for s in SPECS[:2]]

    def fresh(w, p, y, eps):
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps)
        return ctx, st

    made = [fresh(*pr) for pr in probs]
    batch = binding.Batch([st for _, st in made])
    batch.step(2)
    # change the form of every problem between batch steps
    w0, p0, y0, eps0 = probs[0]
    made[0][1].set_blocks([0, w0.M // 2, w0.M], [eps0 * 0.7, eps0 * 0.75])
    made[1][1].set_prior("tv", fgp_iters=8)
    made[1][1].init(dev(probs[1][2], torch), probs[1][3])   # the prior is chosen before init
    batch.step(2)
    w1, p1, y1, eps1 = probs[1]
    made[1][1].set_data_bf16(dev(y1, torch))
    batch.step(1)
    torch.cuda.synchronize()
    xb = [host(st.get_image()) for _, st in made]
    # the same sequence, stepped problem by problem
    solo = [fresh(*pr) for pr in probs]
    for _ in range(2):
        for _, st in solo:
            st.step()
    solo[0][1].set_blocks([0, w0.M // 2, w0.M], [eps0 * 0.7, eps0 * 0.75])
    solo[1][1].set_prior("tv", fgp_iters=8)
    solo[1][1].init(dev(probs[1][2], torch), probs[1][3])
    for _ in range(2):
        for _, st in solo:
            st.step()
    solo[1][1].set_data_bf16(dev(y1, torch))
    for _, st in solo:
        st.step()
    for k in range(2):
        assert rel_err(xb[k], host(solo[k][1].get_image())) <= 1e-6
    batch.close()


def test_batch_with_the_largest_batched_sizes():
    """A batch holding an n = 384 problem (768 x 768 grid, radix 3) and an
    n = 512 one, the two largest image sides of the 32-problem workload: each
    follows its solo iterates, and the n = 384 one matches the FP64 oracle."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    iters = 3
    probs = [make(s) for s in [(384, 40000, 6, 21), (512, 80000, 4, 22)]]
    made = []
    for w, p, y, eps in probs:
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps)
        made.append((ctx, st))
    batch = binding.Batch([st for _, st in made])
    batch.step(iters)
    torch.cuda.synchronize()
    xb = [host(st.get_image()) for _, st in made]
    for k, (w, p, y, eps) in enumerate(probs):
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps)
        for _ in range(iters):
            st.step()
        assert rel_err(xb[k], host(st.get_image())) <= 1e-6
    w, p, y, eps = probs[0]
    ref = osdmm.solve(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), (9, w.n, w.n),
                      iters=iters, cg_iters=w.cg_iters)
    assert rel_err(xb[0], ref.x_hat) <= 1e-4
    batch.close()
