"""The weighted TV prior on the GPU against the FP64 oracle (§3.3 eq.
tvproblem with positivity, §5 weighted TV with the prox by fast gradient
projection).

* prox of lam ||W grad .||_1 after the same number of FGP iterations as the
  oracle agrees to 1e-5 relative l2; lam = 0 returns the input;
* SDMM with the TV prior (graph path), a fixed iteration count, matches the
  oracle's image to 1e-4, with gamma = beta max |grad Phi^H y| and the
  halting quantities; one reweighting round (RWTV) as well.
"""
import numpy as np
import pytest

from oracle import sdmm as osdmm, simulate, tv
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,iters", [(16, 20), (64, 20), (96, 100)])
def test_prox_tv(n, iters):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n)
    uv = inputs.uniform_uv(64, rng)
    ctx = binding.Context(n, uv.astype(np.float32), J=4)
    b = inputs.random_image(n, rng) + 0.5 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    b = b.astype(np.complex64).astype(np.complex128)
    w = rng.uniform(0.5, 1.5, (n, n)).astype(np.float32).astype(np.float64)
    lam = 0.2
    want = tv.prox_tv(b, lam, w, iters)
    got = host(ctx.prox_tv(dev(b, torch), torch.tensor(w, dtype=torch.float32, device="cuda"), lam, iters))
    assert rel_err(got, want) <= 1e-5
    want1 = tv.prox_tv(b, lam, None, iters)
    assert rel_err(host(ctx.prox_tv(dev(b, torch), None, lam, iters)), want1) <= 1e-5
    assert np.array_equal(host(ctx.prox_tv(dev(b, torch), None, 0.0, iters)), b.astype(np.complex64))


def tv_problem():
    p = inputs.make_problem("sdmm64")
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db)
    return p, y.astype(np.complex64).astype(np.complex128), eps


@pytest.mark.parametrize("rounds,iters", [(1, 30), (2, 10)])
def test_sdmm_tv(rounds, iters):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    p, y, eps = tv_problem()
    w = p.workload
    ref = osdmm.solve_tv(simulate.operators(p.uv, w.n, w.J), y, eps, (w.n, w.n), iters=iters,
                         cg_iters=w.cg_iters, rounds=rounds, fgp_iters=20)
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    st = ctx.sdmm_state()
    st.set_prior("tv", fgp_iters=20)
    st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
    assert st.report()["gamma"] == pytest.approx(ref.gamma, rel=1e-5)
    for rnd in range(rounds):
        if rnd > 0:
            st.reweight(rnd)
        for _ in range(iters):
            st.step()
    err = rel_err(host(st.get_image()), ref.x_hat)
    assert err <= 1e-4, err
    rep = st.report()
    last = ref.history[-1]
    assert rep["f1"] == pytest.approx(last["f1"], rel=1e-4)
    assert rep["nu"] == pytest.approx(last["nu"], rel=1e-4)
