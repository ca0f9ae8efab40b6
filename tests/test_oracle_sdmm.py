"""Pins of the oracle's SDMM (Algorithm 1) and its set-up (no GPU).

* On tiny problems with one orthonormal basis, SDMM must reach the solution
  of eq. delta found by an independent solver (SLSQP on a split
  reformulation), in objective and constraint.
* At a fixed point of Algorithm 1, L_i x_hat = r_i, which with steps 5 and 9
  forces sum_i L_i^H z_i = 0; the dual variables must satisfy that.
* On the 64 x 64 workload the iterates approach the constraint set of §4.4
  (nu within [1 - tau, 1 + tau]), stay nearly real and non-negative, and SARA
  beats the Dirac basis in SNR, the ordering §6 reports.
* The noise model and l2 bound of §6.
"""
import numpy as np
import pytest
from scipy import optimize

from oracle import measurement as me, sara, sdmm, simulate, tv
from paper_1307_4370_gb300 import inputs


def tiny_problem(seed=11, n=8, J=4, M=40):
    rng = np.random.default_rng(seed)
    uv = inputs.uniform_uv(M, rng)
    x_true = np.zeros((n, n))
    idx = rng.choice(n * n, 5, replace=False)
    x_true.ravel()[idx] = rng.uniform(0.5, 1, 5)
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n, complex)
        e[k] = 1
        cols.append(me.phi(e.reshape(n, n), uv, J))
    A = np.array(cols).T
    y0 = A @ x_true.ravel()
    sig = simulate.noise_sigma(y0, 30.0)
    y = y0 + sig * inputs.unit_complex_noise(M, rng)
    return A, y, simulate.l2_bound(M, sig), n


def dense_ops(A, Wm, n, q):
    return sdmm.Operators(
        phi=lambda x: A @ x.ravel(),
        phi_adj=lambda v: (A.conj().T @ v).reshape(n, n),
        psi_adj=lambda x: (Wm @ x.ravel()).reshape(q, n, n),
        psi=lambda a: (Wm.T @ a.ravel()).reshape(n, n))


def slsqp_reference(A, y, eps, Wm):
    """min ||Wm x||_1 s.t. ||y - A x|| <= eps, x >= 0, with x = Wm^T (c+ - c-)."""
    D = Wm.shape[0]
    Ar = np.vstack([A.real, A.imag])
    yr = np.concatenate([y.real, y.imag])
    WT = Wm.T

    def l2(v):
        r = yr - Ar @ (WT @ (v[:D] - v[D:]))
        return eps ** 2 - r @ r

    res = optimize.minimize(lambda v: v.sum(), np.full(2 * D, 0.1), method="SLSQP",
                            bounds=[(0, None)] * (2 * D),
                            constraints=[{"type": "ineq", "fun": l2},
                                         {"type": "ineq", "fun": lambda v: WT @ (v[:D] - v[D:])}],
                            options={"maxiter": 3000, "ftol": 1e-14})
    # SLSQP may stop on a line-search message at the optimum; require feasibility instead.
    assert l2(res.x) >= -1e-9 * eps ** 2
    assert np.min(WT @ (res.x[:D] - res.x[D:])) >= -1e-9
    return res.fun


@pytest.mark.parametrize("bases,levels", [((0,), 4), ((2,), 2), ((1,), 3)])
def test_sdmm_reaches_constrained_minimum(bases, levels):
    A, y, eps, n = tiny_problem()
    Wm = np.array([sara.sara_analysis(np.eye(n * n)[k].reshape(n, n), levels, bases).ravel()
                   for k in range(n * n)]).T.real
    ops = dense_ops(A, Wm, n, len(bases))
    st = sdmm.init_state(ops, y, (n, n))
    w = np.ones((len(bases), n, n))
    for _ in range(3000):
        sdmm.sdmm_iteration(ops, st, y, eps, w, 10)
    x = st.x_hat
    assert np.max(np.abs(x.imag)) < 1e-8
    assert x.real.min() > -1e-8
    f_sdmm = np.abs(Wm @ x.real.ravel()).sum()
    f_ref = slsqp_reference(A, y, eps, Wm)
    assert f_sdmm == pytest.approx(f_ref, rel=1e-7)
    assert np.linalg.norm(y - A @ x.real.ravel()) <= eps * (1 + 1e-7)
    # fixed point: sum_i L_i^H z_i = 0
    kkt = ops.psi(st.z1) + ops.phi_adj(st.z2) + st.z3
    assert np.max(np.abs(kkt)) < 1e-6 * max(1.0, np.max(np.abs(st.z3)))


def test_first_iteration_closed_form():
    # x_hat(0) = 0 gives x_hat(1) = 0 (b = 0) and r2(1) = P_B(0): z2 = -P_B(0),
    # x2(1) = Phi^H (2 P_B(0)) with P_B(0) = (1 - eps/||y||) y.
    A, y, eps, n = tiny_problem()
    Wm = np.eye(n * n)
    ops = dense_ops(A, Wm, n, 1)
    st = sdmm.init_state(ops, y, (n, n))
    sdmm.sdmm_iteration(ops, st, y, eps, np.ones((1, n, n)), 10)
    assert np.all(st.x_hat == 0)
    pb0 = (1 - eps / np.linalg.norm(y)) * y
    assert np.allclose(st.z2, -pb0, atol=1e-15)
    assert np.allclose(st.x2, (A.conj().T @ (2 * pb0)).reshape(n, n), atol=1e-14)
    assert st.gamma == pytest.approx(1e-3 * np.max(np.abs(A.conj().T @ y)))


@pytest.fixture(scope="module")
def sdmm64_runs():
    p = inputs.make_problem("sdmm64")
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db)
    sa = sdmm.solve(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), (9, w.n, w.n),
                    iters=50, cg_iters=10)
    bp = sdmm.solve(simulate.operators(p.uv, w.n, w.J, bases=(0,)), y, eps, (w.n, w.n),
                    (1, w.n, w.n), iters=50, cg_iters=10)
    return p, sa, bp


@pytest.mark.slow
def test_sdmm64_constraint_and_ordering(sdmm64_runs):
    p, sa, bp = sdmm64_runs
    nus = [h["nu"] for h in sa.history]
    assert nus[0] > 10                       # starts far outside the ball
    assert all(0.85 <= v <= 1.1 for v in nus[-10:])
    assert max(h["cg_residual"] for h in sa.history[-5:]) < 1e-6
    x = sa.x_hat
    assert np.max(np.abs(x.imag)) < 1e-2 * np.max(np.abs(x.real))
    assert x.real.min() > -1e-2 * x.real.max()
    assert simulate.snr_db(p.x_true, x.real) > simulate.snr_db(p.x_true, bp.x_hat.real) + 3.0


def test_noise_model():
    rng = np.random.default_rng(5)
    M = 4096
    y0 = inputs.random_vis(M, rng) * 3.0
    sig = simulate.noise_sigma(y0, 30.0)
    norms = []
    for _ in range(200):
        n_ = sig * inputs.unit_complex_noise(M, rng)
        norms.append(np.linalg.norm(n_))
    norms = np.array(norms)
    # realised input SNR ~ 30 dB
    assert 20 * np.log10(np.linalg.norm(y0) / np.mean(norms)) == pytest.approx(30.0, abs=0.05)
    # eps^2 = (2M + 4 sqrt M) sigma^2 / 2 is the mean of ||n||^2 plus two standard deviations
    eps = simulate.l2_bound(M, sig)
    assert np.mean(norms <= eps) > 0.9
    assert eps ** 2 == pytest.approx(M * sig ** 2 + 2 * np.sqrt(M) * sig ** 2, rel=1e-12)


# ---------------------------------------------------------------------------
# Distributed-block form (§4.5 eqs. blocks, dbp1, dbp2)
# ---------------------------------------------------------------------------
def slsqp_blocks_reference(A, y, eps, offsets, Wm):
    """min ||Wm x||_1 s.t. ||y_i - A_i x|| <= eps_i for every block, x >= 0."""
    D = Wm.shape[0]
    WT = Wm.T
    cons = [{"type": "ineq", "fun": lambda v: WT @ (v[:D] - v[D:])}]
    for i in range(len(eps)):
        Ai = A[offsets[i]:offsets[i + 1]]
        Ar = np.vstack([Ai.real, Ai.imag])
        yr = np.concatenate([y[offsets[i]:offsets[i + 1]].real, y[offsets[i]:offsets[i + 1]].imag])

        def l2(v, Ar=Ar, yr=yr, e=eps[i]):
            r = yr - Ar @ (WT @ (v[:D] - v[D:]))
            return e ** 2 - r @ r
        cons.append({"type": "ineq", "fun": l2})
    res = optimize.minimize(lambda v: v.sum(), np.full(2 * D, 0.1), method="SLSQP",
                            bounds=[(0, None)] * (2 * D), constraints=cons,
                            options={"maxiter": 3000, "ftol": 1e-14})
    for c in cons[1:]:
        assert c["fun"](res.x) >= -1e-9 * max(eps) ** 2
    return res.fun


@pytest.mark.parametrize("offsets_frac", [(0, 0.5, 1.0), (0, 0.3, 0.55, 1.0)])
def test_block_sdmm_reaches_constrained_minimum(offsets_frac):
    A, y, eps, n = tiny_problem(seed=12)
    M = len(y)
    offsets = [int(round(f * M)) for f in offsets_frac]
    # per-block bounds: the single ball's budget split in proportion to M_i, tightened
    # so that the block constraints bind differently from the single ball
    eps_b = [eps * np.sqrt((offsets[i + 1] - offsets[i]) / M) * (0.9 if i == 0 else 1.05)
             for i in range(len(offsets) - 1)]
    Wm = np.eye(n * n)
    ops = dense_ops(A, Wm, n, 1)
    st = sdmm.init_state_blocks(ops, y, offsets, (n, n))
    w = np.ones((1, n, n))
    for _ in range(3000):
        rec = sdmm.sdmm_iteration_blocks(ops, st, y, eps_b, offsets, w, 10)
    x = st.x_hat
    assert np.max(np.abs(x.imag)) < 1e-8 and x.real.min() > -1e-8
    f_ref = slsqp_blocks_reference(A, y, eps_b, offsets, Wm)
    assert np.abs(x.real).sum() == pytest.approx(f_ref, rel=1e-6)
    for i, e in enumerate(eps_b):
        sl = slice(offsets[i], offsets[i + 1])
        assert np.linalg.norm(y[sl] - A[sl] @ x.real.ravel()) <= e * (1 + 1e-6)
    assert rec["nu"] == max(rec["nu_blocks"]) and rec["nu_min"] == min(rec["nu_blocks"])


def test_one_block_is_the_single_ball():
    p = inputs.make_problem(inputs.Workload("b32", n=32, M=800, J=4, n_src=5, diffuse=False, seed=4))
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, 30.0)
    ops = simulate.operators(p.uv, w.n, w.J)
    a = sdmm.solve(ops, y, eps, (w.n, w.n), (9, w.n, w.n), iters=8, cg_iters=10)
    b = sdmm.solve_blocks(ops, y, [eps], [0, w.M], (w.n, w.n), (9, w.n, w.n), iters=8, cg_iters=10)
    assert np.linalg.norm(a.x_hat - b.x_hat) <= 1e-12 * np.linalg.norm(a.x_hat)
    for ha, hb in zip(a.history, b.history):
        assert hb["nu"] == pytest.approx(ha["nu"], rel=1e-12)
        assert hb["f1"] == pytest.approx(ha["f1"], rel=1e-12)


def test_block_projection():
    rng = np.random.default_rng(3)
    M = 60
    offsets = [0, 20, 45, 60]
    y = inputs.random_vis(M, rng)
    r = y + 2.0 * inputs.random_vis(M, rng)
    eps = [0.5, 100.0, 1.0]
    out = sdmm.prox.project_l2_balls(r, y, eps, offsets)
    for i, e in enumerate(eps):
        sl = slice(offsets[i], offsets[i + 1])
        assert np.linalg.norm(out[sl] - y[sl]) <= e * (1 + 1e-14)
        assert np.allclose(out[sl], sdmm.prox.project_l2_ball(r[sl], y[sl], e), rtol=0, atol=0)
    assert np.array_equal(out[20:45], r[20:45])   # block 2 was inside its ball
    assert np.allclose(sdmm.prox.project_l2_balls(out, y, eps, offsets), out, rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# TV prior (§3.3 eq. tvproblem with positivity; prox by FGP)
# ---------------------------------------------------------------------------
def smoothed_tv_reference(A, y, eps, n, x0):
    """Independent solver: min sum sqrt(|grad x|^2 + mu^2) s.t. ||y - A x|| <= eps,
    x >= 0 (SLSQP on the smooth problem, mu continued down to 1e-5)."""
    Ar = np.vstack([A.real, A.imag])
    yr = np.concatenate([y.real, y.imag])
    v = np.maximum(x0, 0.0)
    for mu in (1e-2, 1e-3, 1e-4, 1e-5):
        def f(v, mu=mu):
            d1, d2 = tv.grad(v.reshape(n, n))
            return np.sum(np.sqrt(d1 ** 2 + d2 ** 2 + mu ** 2))
        v = optimize.minimize(f, v, method="SLSQP", bounds=[(0, None)] * (n * n),
                              constraints=[{"type": "ineq", "fun": lambda v: eps ** 2 - np.sum((yr - Ar @ v) ** 2)}],
                              options={"maxiter": 5000, "ftol": 1e-15}).x
    assert np.sum((yr - Ar @ v) ** 2) <= eps ** 2 * (1 + 1e-9) and v.min() >= -1e-12
    return v


def test_tv_sdmm_reaches_constrained_minimum():
    A, y, eps, n = tiny_problem(seed=13)
    ops = dense_ops(A, np.eye(n * n), n, 1)
    st = sdmm.init_state_tv(ops, y, (n, n))
    for _ in range(3000):
        sdmm.sdmm_iteration_tv(ops, st, y, eps, None, 10, 50)
    x = st.x_hat
    assert np.max(np.abs(x.imag)) < 1e-6 and x.real.min() > -1e-6
    assert np.linalg.norm(y - A @ x.real.ravel()) <= eps * (1 + 1e-6)
    v = smoothed_tv_reference(A, y, eps, n, x.real.ravel())
    tv_sdmm, tv_ref = tv.tv_norm(x.real), tv.tv_norm(v.reshape(n, n))
    assert tv_sdmm == pytest.approx(tv_ref, rel=2e-5)
    assert tv_sdmm <= tv_ref * (1 + 1e-6)
    assert st.gamma == pytest.approx(1e-3 * np.max(tv.grad_magnitude((A.conj().T @ y).reshape(n, n))))


def test_tv_reweighting_rule():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((8, 8))
    w = sdmm.reweight_tv(x, 2)
    g = tv.grad_magnitude(x)
    delta = 1e-2 * g.max()
    assert np.allclose(w, delta / (delta + g), rtol=1e-15, atol=0)
    assert np.all(sdmm.reweight_tv(np.ones((4, 4)), 1) == 1.0)


# ---------------------------------------------------------------------------
# Reweighting rule (§3.3, reading c14) and halting test (§4.4), pinned by
# hand-computed values rather than by the rule restated.
# ---------------------------------------------------------------------------
def _identity_planes_ops(scales):
    """Psi^H x = [s_0 x; s_1 x; ...] (planes in order), so alpha is known by hand."""
    return sdmm.Operators(phi=None, phi_adj=None,
                          psi_adj=lambda x: np.stack([s * x for s in scales]),
                          psi=None)


def test_reweight_hand_values():
    # |alpha| = (0, 1, 2, 4) in plane 0; max 4
    x = np.array([[0.0, 1.0], [-2.0, 4.0j]])
    ops = _identity_planes_ops([1.0])
    # round 1: delta = 0.4 -> 1, 2/7, 1/6, 1/11
    assert np.allclose(sdmm.reweight(ops, x, 1)[0], [[1.0, 2 / 7], [1 / 6, 1 / 11]], rtol=1e-15, atol=0)
    # round 2: delta = 0.04 -> 1, 1/26, 1/51, 1/101
    assert np.allclose(sdmm.reweight(ops, x, 2)[0], [[1.0, 1 / 26], [1 / 51, 1 / 101]], rtol=1e-15, atol=0)
    # round 7: 10^-7 * 4 is below the floor 1e-6 * 4 = 4e-6 -> delta = 4e-6
    d = 4e-6
    assert np.allclose(sdmm.reweight(ops, x, 7)[0], [[1.0, d / (d + 1)], [d / (d + 2), d / (d + 4)]],
                       rtol=1e-15, atol=0)
    # round 6 is exactly at the floor (10^-6 = 1e-6): same weights as round 7
    assert np.allclose(sdmm.reweight(ops, x, 6), sdmm.reweight(ops, x, 7), rtol=1e-15, atol=0)
    # weights are 1 where alpha = 0 and never exceed 1
    w = sdmm.reweight(ops, x, 3)
    assert w[0, 0, 0] == 1.0 and np.all(w <= 1.0)


def test_reweight_zero_image_and_plane_order():
    ops = _identity_planes_ops([1.0, 3.0])
    assert np.all(sdmm.reweight(ops, np.zeros((3, 3)), 1) == 1.0)
    # two planes: |alpha| = (1, 3) at one pixel, max 3; round 1: delta = 0.3
    x = np.zeros((2, 2), dtype=complex)
    x[1, 0] = 1.0
    w = sdmm.reweight(ops, x, 1)
    assert w.shape == (2, 2, 2)
    assert w[0, 1, 0] == pytest.approx(0.3 / 1.3, rel=1e-15)
    assert w[1, 1, 0] == pytest.approx(0.3 / 3.3, rel=1e-15)
    w[0, 1, 0] = w[1, 1, 0] = 1.0
    assert np.all(w == 1.0)


@pytest.mark.parametrize("zeta,nu,expect", [
    (0.5e-3, 1.0, True),        # inside the band, small change
    (1e-3, 1.0, False),         # zeta = xi is not below xi
    (0.999e-3, 0.9, True),      # nu = 1 - tau: band is closed
    (0.999e-3, 1.1, True),      # nu = 1 + tau
    (0.5e-3, 0.8999, False),    # below the band
    (0.5e-3, 1.1001, False),    # above the band
    (np.inf, 1.0, False),       # first iteration: f1(t-1) = 0
    (0.0, 1.05, True),
])
def test_halted_truth_table(zeta, nu, expect):
    assert sdmm.halted({"zeta": zeta, "nu": nu}) is expect


def test_halted_stops_solve_at_first_true_record():
    # the solve loop must stop right after the first iteration whose record halts
    p = inputs.make_problem(inputs.Workload("h32", n=32, M=900, J=4, n_src=6, diffuse=False, seed=8))
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, 30.0)
    ops = simulate.operators(p.uv, w.n, w.J)
    free = sdmm.solve(ops, y, eps, (w.n, w.n), (9, w.n, w.n), iters=200, cg_iters=10)
    first = next((h["t"] for h in free.history if sdmm.halted(h)), None)
    assert first is not None and first < 200
    stopped = sdmm.solve(ops, y, eps, (w.n, w.n), (9, w.n, w.n), iters=200, cg_iters=10, stop=True)
    assert stopped.t == first
    exact = sdmm.solve(ops, y, eps, (w.n, w.n), (9, w.n, w.n), iters=first, cg_iters=10)
    assert np.array_equal(stopped.x_hat, exact.x_hat)
