"""The paper's Gaussian interpolation kernel and a primary beam B on the GPU
(Phi = G F D Z B, §5 eq. opmodel), against the FP64 oracle.

Phi and Phi^H with either kernel and a random positive beam agree with the
oracle to 1e-5 relative l2 (FP32 against FP64); clearing the beam restores
B = I exactly; and the SDMM iteration (graph path) with the Gaussian kernel
and a beam matches the oracle's image after a fixed iteration count to
1e-4, including when the beam is set after the state already captured its
iteration graph.
"""
import numpy as np
import pytest

from oracle import measurement as me, sdmm as osdmm, simulate
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.mark.parametrize("kernel", ["kb", "gauss"])
@pytest.mark.parametrize("n,M,J", [(32, 1000, 4), (64, 3000, 6), (96, 5000, 8)])
def test_phi_kernel_and_beam(kernel, n, M, J):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n + J)
    uv = inputs.uv_variable_density(M, n, rng).astype(np.float32).astype(np.float64)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    beam = rng.uniform(0.2, 1.0, (n, n)).astype(np.float32).astype(np.float64)
    ctx = binding.Context(n, uv.astype(np.float32), J=J, kernel=kernel)
    plain_y = host(ctx.phi(dev(x, torch)))
    plain_x = host(ctx.phi_adj(dev(v, torch)))
    assert rel_err(plain_y, me.phi(x, uv, J, kernel)) <= TOL
    assert rel_err(plain_x, me.phi_adj(v, uv, n, J, kernel)) <= TOL
    ctx.set_beam(beam)
    assert rel_err(host(ctx.phi(dev(x, torch))), me.phi(x, uv, J, kernel, beam)) <= TOL
    assert rel_err(host(ctx.phi_adj(dev(v, torch))), me.phi_adj(v, uv, n, J, kernel, beam)) <= TOL
    ctx.set_beam(None)
    assert np.array_equal(host(ctx.phi(dev(x, torch))), plain_y)
    assert np.array_equal(host(ctx.phi_adj(dev(v, torch))), plain_x)


def test_sdmm_gauss_kernel_with_beam():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    p = inputs.make_problem("sdmm64")
    w = p.workload
    rng = np.random.default_rng(11)
    beam = np.exp(-((np.arange(w.n) - w.n / 2) ** 2)[:, None] / (2 * (0.4 * w.n) ** 2)
                  - ((np.arange(w.n) - w.n / 2) ** 2)[None, :] / (2 * (0.4 * w.n) ** 2))
    beam = beam.astype(np.float32).astype(np.float64)
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db, kernel="gauss", beam=beam)
    y = y.astype(np.complex64).astype(np.complex128)
    iters = 30
    ref = osdmm.solve(simulate.operators(p.uv, w.n, w.J, kernel="gauss", beam=beam), y, eps, (w.n, w.n),
                      (9, w.n, w.n), iters=iters, cg_iters=w.cg_iters)
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J, kernel="gauss")
    st = ctx.sdmm_state()
    # one step without a beam captures the iteration graph; setting the beam
    # afterwards must make the next step re-capture it
    st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
    st.step()
    ctx.set_beam(beam)
    st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
    assert st.report()["gamma"] == pytest.approx(ref.gamma, rel=1e-5)
    for _ in range(iters):
        st.step()
    err = rel_err(host(st.get_image()), ref.x_hat)
    assert err <= 1e-4, err
    assert st.report()["nu"] == pytest.approx(ref.history[-1]["nu"], rel=1e-4)
