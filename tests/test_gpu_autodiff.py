"""Differentiation through Phi, Psi and the unrolled SDMM (needs a GB300).

* The autograd backward of Phi (and Psi^H) is the adjoint kernel: the
  gradient of Re <v, Phi x> with respect to x is Phi^H v (oracle).
* Directional derivatives of ||x_K - x_true||^2 with respect to the
  per-visibility weights w and the SARA weights omega, from the checkpointed
  reverse pass on the GPU, match central finite differences of the FP64
  oracle's K-iteration SDMM to 1e-3 relative.  The map is only piecewise
  smooth (soft threshold, ball projection): on this problem central
  differences with h = 1e-3 themselves move by ~1e-3 relative from their
  h -> 0 limit (measured with the oracle), so the differences use h = 1e-4.
* On the 256 x 256, M = 65536, K = 20 problem the checkpointed gradient equals
  the one-segment gradient and needs less memory.
"""
import numpy as np
import pytest

from oracle import measurement as me, sara as osara, sdmm as osdmm, simulate
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def test_operator_backward_is_the_adjoint():
    torch = require_gpu()
    from paper_1307_4370_gb300 import autodiff, binding

    n, M, J = 32, 900, 6
    rng = np.random.default_rng(3)
    uv = inputs.uniform_uv(M, rng)
    op = binding.Context(n, uv.astype(np.float32), J=J)
    x = dev(inputs.random_image(n, rng), torch).requires_grad_(True)
    v = inputs.random_vis(M, rng)
    y = autodiff.PhiFn.apply(x, op)
    loss = (torch.conj(dev(v, torch)) * y).real.sum()
    (gx,) = torch.autograd.grad(loss, x)
    assert rel_err(host(gx), me.phi_adj(v, uv, n, J)) <= 1e-5
    a = autodiff.PsiAdjFn.apply(x, op)
    bcoef = rng.standard_normal((9, n, n)) + 1j * rng.standard_normal((9, n, n))
    loss = (torch.conj(dev(bcoef, torch)) * a).real.sum()
    (gx,) = torch.autograd.grad(loss, x)
    assert rel_err(host(gx), osara.sara_synthesis(bcoef.astype(np.complex64).astype(np.complex128), 4)) <= 1e-5


def oracle_loss(p, y, eps, wv, omega, gamma, K, cg_iters):
    w = p.workload
    ops = osdmm.Operators(
        phi=lambda x: wv * me.phi(x, p.uv, w.J),
        phi_adj=lambda v: me.phi_adj(wv * v, p.uv, w.n, w.J),
        psi_adj=lambda x: osara.sara_analysis(x, 4),
        psi=lambda a: osara.sara_synthesis(a, 4))
    yw = wv * y
    st = osdmm.init_state(ops, yw, (w.n, w.n))
    st.gamma = gamma
    for _ in range(K):
        osdmm.sdmm_iteration(ops, st, yw, eps, omega, cg_iters)
    return float(np.sum(np.abs(st.x_hat - p.x_true) ** 2))


def test_sdmm_gradients_against_oracle_finite_differences():
    torch = require_gpu()
    from paper_1307_4370_gb300 import autodiff, binding

    w = inputs.Workload("fd", n=32, M=1024, J=4, n_src=6, diffuse=False, seed=77)
    p = inputs.make_problem(w)
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, 30.0)
    y = y.astype(np.complex64).astype(np.complex128)
    K, cg_iters, C = 6, 8, 2
    rng = np.random.default_rng(5)
    wv0 = (1.0 + 0.1 * rng.uniform(-1, 1, w.M)).astype(np.float32).astype(np.float64)
    om0 = (1.0 + 0.1 * rng.uniform(-1, 1, (9, w.n, w.n))).astype(np.float32).astype(np.float64)
    op = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    yt = dev(y, torch)
    wt = torch.tensor(wv0, dtype=torch.float32, device="cuda", requires_grad=True)
    ot = torch.tensor(om0, dtype=torch.float32, device="cuda", requires_grad=True)
    gamma = autodiff.penalty(op, yt, wt.detach())
    xk = autodiff.sdmm_unrolled(op, yt, eps, wt, ot, K=K, cg_iters=cg_iters, checkpoint=C, gamma=gamma)
    xt = torch.tensor(p.x_true.astype(np.complex64), device="cuda")
    loss = ((xk - xt).abs() ** 2).sum()
    loss.backward()
    gw = wt.grad.double().cpu().numpy()
    go = ot.grad.double().cpu().numpy()
    L0 = oracle_loss(p, y, eps, wv0, om0, gamma, K, cg_iters)
    assert float(loss.item()) == pytest.approx(L0, rel=1e-3)
    h = 1e-4
    for k in range(2):
        dw = rng.standard_normal(w.M)
        fd = (oracle_loss(p, y, eps, wv0 + h * dw, om0, gamma, K, cg_iters)
              - oracle_loss(p, y, eps, wv0 - h * dw, om0, gamma, K, cg_iters)) / (2 * h)
        assert float(np.dot(gw, dw)) == pytest.approx(fd, rel=1e-3)
        do = rng.standard_normal(om0.shape)
        fd = (oracle_loss(p, y, eps, wv0, om0 + h * do, gamma, K, cg_iters)
              - oracle_loss(p, y, eps, wv0, om0 - h * do, gamma, K, cg_iters)) / (2 * h)
        assert float(np.sum(go * do)) == pytest.approx(fd, rel=1e-3)


def test_checkpointed_gradient_full_size():
    torch = require_gpu()
    from paper_1307_4370_gb300 import autodiff, binding

    p = inputs.make_problem("diff256")
    w = p.workload
    op = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    x_true = torch.tensor(p.x_true.astype(np.complex64), device="cuda")
    y0 = op.phi(x_true)
    sig = float(torch.linalg.vector_norm(y0).item()) / np.sqrt(w.M) * 10 ** (-w.isnr_db / 20)
    y = y0 + sig * torch.tensor(p.noise_unit.astype(np.complex64), device="cuda")
    eps = simulate.l2_bound(w.M, sig)
    grads, peaks = [], []
    for C in (5, 20):
        wt = torch.ones(w.M, dtype=torch.float32, device="cuda", requires_grad=True)
        ot = torch.ones((9, w.n, w.n), dtype=torch.float32, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        xk = autodiff.sdmm_unrolled(op, y, eps, wt, ot, K=w.T, cg_iters=w.cg_iters, checkpoint=C)
        loss = ((xk - x_true).abs() ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated() - base)
        grads.append((wt.grad.double().cpu().numpy(), ot.grad.double().cpu().numpy()))
    for a, b in zip(grads[0], grads[1]):
        assert np.all(np.isfinite(a)) and np.linalg.norm(a) > 0
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)
    assert peaks[0] < peaks[1]


def _fd_check(fwd, a, abar, rbar, h=1e-6, rng=None):
    """<abar, da> against central differences of Re<rbar, fwd(a)> (FP64)."""
    da = (rng.standard_normal(a.shape) + 1j * rng.standard_normal(a.shape))
    L = lambda z: float(np.real(np.vdot(rbar, fwd(z))))  # noqa: E731
    fd = (L(a + h * da) - L(a - h * da)) / (2 * h)
    an = float(np.real(np.vdot(da, abar)))
    return an, fd


def test_prox_vjps_against_oracle_differences():
    """The vector-Jacobian products of the three proximity operators of §4.4
    (soft threshold, l2-ball projection, positivity), on the GPU, against
    central differences of the oracle's operators in FP64."""
    torch = require_gpu()
    from oracle import prox as oprox
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(9)
    n = 4000
    a = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64).astype(np.complex128)
    rb = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64).astype(np.complex128)
    wts = rng.uniform(0.2, 2.0, n).astype(np.float32).astype(np.float64)
    gamma = 0.7
    # soft threshold with weights (about half the entries thresholded to 0)
    wbar = torch.zeros(n, dtype=torch.float32, device="cuda")
    ab = host(binding.vjp_soft_threshold(dev(a, torch), dev(wts, torch), gamma, dev(rb, torch), wbar=wbar))
    an, fd = _fd_check(lambda z: oprox.soft_threshold(z, gamma * wts), a, ab, rb, rng=rng)
    assert an == pytest.approx(fd, rel=1e-4)
    dwt = rng.standard_normal(n)
    Lw = lambda ww: float(np.real(np.vdot(rb, oprox.soft_threshold(a, gamma * ww))))  # noqa: E731
    h = 1e-6
    fdw = (Lw(wts + h * dwt) - Lw(wts - h * dwt)) / (2 * h)
    assert float(np.dot(wbar.double().cpu().numpy(), dwt)) == pytest.approx(fdw, rel=1e-4)
    # positivity
    ab = host(binding.vjp_positive(dev(a, torch), dev(rb, torch)))
    an, fd = _fd_check(oprox.project_positive, a, ab, rb, rng=rng)
    assert an == pytest.approx(fd, rel=1e-5)
    # l2 ball around y: outside (projection active) and inside (identity)
    op = binding.Context(16, inputs.uniform_uv(n, rng).astype(np.float32), J=4)
    y = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64).astype(np.complex128)
    for eps in (0.3 * np.linalg.norm(a - y), 3.0 * np.linalg.norm(a - y)):
        abar, ybar = op.vjp_l2ball(dev(a, torch), dev(y, torch), eps, dev(rb, torch))
        an, fd = _fd_check(lambda z: oprox.project_l2_ball(z, y, eps), a, host(abar), rb, rng=rng)
        assert an == pytest.approx(fd, rel=1e-4)
        an, fd = _fd_check(lambda z: oprox.project_l2_ball(a, z, eps), y, host(ybar), rb, rng=rng)
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-6 * np.linalg.norm(rb))


def test_sdmm_gradient_full_size_against_stored_differences(capsys):
    """256 x 256, M = 65536, K = 20 iterations of 10 CG steps, checkpoints
    every 5 (the differentiation workload): the loss and the directional
    derivatives along one seeded direction of w and of omega from the
    library's reverse pass, against central differences (h = 1e-4) of the
    FP64 oracle's loss stored by tests/golden/make_golden.py."""
    torch = require_gpu()
    import importlib.util
    import os
    from paper_1307_4370_gb300 import autodiff, binding

    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    g = dict(np.load(os.path.join(here, "golden", "diff256_fd.npz")))
    p = inputs.make_problem("diff256")
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db)
    y = y.astype(np.complex64).astype(np.complex128)
    assert eps == pytest.approx(float(g["eps"]), rel=1e-12)
    wv0, om0, dw, dom = mg.diff_inputs(w.M, w.n)
    op = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    wt = torch.tensor(wv0, dtype=torch.float32, device="cuda", requires_grad=True)
    ot = torch.tensor(om0, dtype=torch.float32, device="cuda", requires_grad=True)
    gamma_gpu = autodiff.penalty(op, dev(y, torch), wt.detach())
    assert gamma_gpu == pytest.approx(float(g["gamma"]), rel=1e-5)
    xk = autodiff.sdmm_unrolled(op, dev(y, torch), eps, wt, ot, K=int(g["K"]), cg_iters=int(g["cg_iters"]),
                                checkpoint=5, gamma=float(g["gamma"]))
    xt = torch.tensor(p.x_true.astype(np.complex64), device="cuda")
    loss = ((xk - xt).abs() ** 2).sum()
    loss.backward()
    dw_an = float(np.dot(wt.grad.double().cpu().numpy(), dw))
    dom_an = float(np.sum(ot.grad.double().cpu().numpy() * dom))
    with capsys.disabled():
        print(f"\ndiff256 K=20: loss {float(loss.item()):.6e} vs {float(g['loss']):.6e}; "
              f"d/dw {dw_an:.6e} vs FD {float(g['fd_w']):.6e}; d/domega {dom_an:.6e} vs FD {float(g['fd_om']):.6e}")
    assert float(loss.item()) == pytest.approx(float(g["loss"]), rel=1e-3)
    assert dw_an == pytest.approx(float(g["fd_w"]), rel=1e-3)
    assert dom_an == pytest.approx(float(g["fd_om"]), rel=1e-3)
