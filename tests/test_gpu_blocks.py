"""Distributed-block SDMM (§4.5 eqs. blocks, dbp1, dbp2) on one GPU against
the FP64 oracle: R consecutive blocks of visibilities, one l2 ball each.

After a fixed iteration count the image matches the oracle's eq. dbp2 run to
1e-4 and the largest / smallest block nu track the oracle's; one block gives
the single-ball iteration; returning to the single ball restores it exactly;
malformed block tables are refused before any work.
"""
import numpy as np
import pytest

from oracle import sdmm as osdmm, simulate
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu


def problem():
    p = inputs.make_problem("sdmm64")
    w = p.workload
    y, eps = simulate.visibilities(p.x_true, p.uv, w.J, p.noise_unit, w.isnr_db)
    sig = eps / np.sqrt(w.M + 2 * np.sqrt(w.M))  # sigma_n from the chi^2 bound eps
    return p, y.astype(np.complex64).astype(np.complex128), eps, sig


def test_blocks_match_oracle():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    p, y, eps, sig = problem()
    w = p.workload
    offsets = [0, 500, 1300, w.M]
    eps_b = [simulate.l2_bound(offsets[i + 1] - offsets[i], sig) for i in range(3)]
    iters = 30
    ref = osdmm.solve_blocks(simulate.operators(p.uv, w.n, w.J), y, eps_b, offsets, (w.n, w.n),
                             (9, w.n, w.n), iters=iters, cg_iters=w.cg_iters)
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    st = ctx.sdmm_state()
    st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
    st.set_blocks(offsets, eps_b)
    for _ in range(iters):
        st.step()
    rep = st.report()
    err = rel_err(host(st.get_image()), ref.x_hat)
    assert err <= 1e-4, err
    last = ref.history[-1]
    assert rep["nu"] == pytest.approx(last["nu"], rel=1e-4)
    assert rep["nu_min"] == pytest.approx(last["nu_min"], rel=1e-4)
    assert rep["f1"] == pytest.approx(last["f1"], rel=1e-4)


def test_one_block_and_back_to_single_ball():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    p, y, eps, _ = problem()
    w = p.workload
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)

    def run(blocks):
        st = ctx.sdmm_state()
        st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
        if blocks == "one":
            st.set_blocks([0, w.M], [eps])
        elif blocks == "toggle":
            st.set_blocks([0, 100, w.M], [eps, eps])
            st.step()                     # captured with blocks
            st.set_blocks(None)           # back to the single ball
            st.init(dev(y, torch), eps, cg_iters=w.cg_iters)
        for _ in range(12):
            st.step()
        return host(st.get_image()), st.report()

    x0, r0 = run(None)
    x1, r1 = run("one")
    assert rel_err(x1, x0) <= 1e-6
    assert r1["nu"] == pytest.approx(r0["nu"], rel=1e-6) and r1["nu_min"] == r1["nu"]
    x2, r2 = run("toggle")
    assert np.array_equal(x2, x0)
    assert r0["nu_min"] == r0["nu"]


def test_bad_block_tables():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    p, y, eps, _ = problem()
    w = p.workload
    ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J)
    st = ctx.sdmm_state()
    for off, e in [([0, 10, 10, w.M], [1.0, 1.0, 1.0]), ([1, w.M], [1.0]), ([0, w.M - 1], [1.0]),
                   ([0, 100, w.M], [1.0, 0.0])]:
        with pytest.raises(binding.PurifyError):
            st.set_blocks(off, e)
