"""GPU parity of the operators against the FP64 oracle (needs a GB300).

Phi, Phi^H (§5 eq. opmodel), Psi, Psi^H (§3.3) and the proximity operators
(§4.4) of the CUDA library, called through the C ABI, against the oracle on
the same seeded complex64 / float32 inputs.  Bound: relative l2 error <= 1e-5
for the FP32 operators; the prox outputs to FP32 rounding.
"""
import numpy as np
import pytest

from oracle import measurement as me, prox as oprox, sara as osara, cg as ocg
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5

# (n, M, J, coverage): several FFT tiles, radix-3 grids (2n = 192, 384), ragged M,
# the 64 x 64 and 256 x 256 workloads at full size.
PHI_CASES = [
    (8, 37, 2, "uniform"),
    (16, 500, 6, "uniform"),
    (32, 1000, 8, "uniform"),
    (64, 2048, 4, "sdmm64"),
    (96, 3001, 6, "gauss"),
    (192, 20000, 4, "gauss"),
    (256, 65536, 6, "sdmm256"),
]


def coverage(kind, n, M, rng):
    if kind == "uniform":
        return inputs.uniform_uv(M, rng)
    if kind == "gauss":
        return inputs.uv_variable_density(M, n, rng).astype(np.float32).astype(np.float64)
    return inputs.make_problem(kind).uv


@pytest.mark.parametrize("n,M,J,kind", PHI_CASES)
def test_phi_and_adjoint(n, M, J, kind):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n + M)
    uv = coverage(kind, n, M, rng)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    ctx = binding.Context(n, uv.astype(np.float32), J=J, levels=min(4, int(np.log2(n)) - 1))
    y = host(ctx.phi(dev(x, torch)))
    xa = host(ctx.phi_adj(dev(v, torch)))
    assert rel_err(y, me.phi(x, uv, J)) <= TOL
    assert rel_err(xa, me.phi_adj(v, uv, n, J)) <= TOL
    # repeated calls give the same result (the scratch grid is fully rewritten)
    y2 = host(ctx.phi(dev(x, torch)))
    assert rel_err(y2, y) <= 1e-6


def test_phi_large_sampled():
    """1024 x 1024, M = 2^21 (the mixed-precision workload's sizes), all outputs,
    for every tile side the autotuner may pick (dense arcs give multi-chunk
    tiles and the largest shared-memory footprints)."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import autotune, binding

    p = inputs.make_problem("sdmm1024")
    w = p.workload
    rng = np.random.default_rng(3)
    x = inputs.random_image(w.n, rng)
    idx = rng.choice(w.M, 20000, replace=False)
    want = me.phi(x, p.uv, w.J)
    v = inputs.random_vis(w.M, rng)
    want_adj = me.phi_adj(v, p.uv, w.n, w.J)
    for t in autotune.valid_tiles(w.n, w.J):
        ctx = binding.Context(w.n, p.uv.astype(np.float32), J=w.J, tile=t)
        y = host(ctx.phi(dev(x, torch)))
        assert rel_err(y, want) <= TOL
        assert rel_err(y[idx], want[idx]) <= TOL
        xa = host(ctx.phi_adj(dev(v, torch)))
        assert rel_err(xa, want_adj) <= TOL
        ctx.close()


# Sizes from 8^2 (filters longer than the deep bands) to 1024^2, basis subsets
# and level counts.
@pytest.mark.parametrize("n,levels,mask", [(16, 4, 0x1FF), (64, 4, 0x1FF), (96, 4, 0x1FF), (192, 4, 0x1FF),
                                           (256, 4, 0x1FF), (64, 3, 0x100), (32, 2, 0x001), (64, 4, 0x0F5),
                                           (8, 3, 0x1FF), (384, 4, 0x1FF), (512, 4, 0x1FF), (1024, 4, 0x1FF),
                                           (512, 2, 0x082), (1024, 3, 0x1FF)])
def test_sara(n, levels, mask):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n * 7 + levels)
    bases = tuple(b for b in range(9) if mask >> b & 1)
    uv = inputs.uniform_uv(16, rng)
    ctx = binding.Context(n, uv.astype(np.float32), J=4, levels=levels, bases_mask=mask)
    x = inputs.random_image(n, rng)
    al = host(ctx.sara_analysis(dev(x, torch)))
    assert al.shape == (len(bases), n, n)
    assert rel_err(al, osara.sara_analysis(x, levels, bases)) <= TOL
    b = rng.standard_normal((len(bases), n, n)) + 1j * rng.standard_normal((len(bases), n, n))
    b = b.astype(np.complex64).astype(np.complex128)
    xs = host(ctx.sara_synthesis(dev(b, torch)))
    assert rel_err(xs, osara.sara_synthesis(b, levels, bases)) <= TOL


def test_prox_operators():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(9)
    ctx = binding.Context(16, inputs.uniform_uv(8, rng).astype(np.float32), J=4)
    for count in (0, 1, 1000, 300001):
        a = inputs.random_vis(count, rng)
        w = rng.uniform(0, 2, count).astype(np.float32).astype(np.float64)
        gamma = 0.7
        if count == 0:
            continue
        got = host(ctx.prox_l1_reweighted(dev(a, torch), dev(w, torch), gamma))
        want = oprox.soft_threshold(a, np.float32(gamma) * w)
        assert np.max(np.abs(got - want)) <= 1e-6 * max(1.0, np.abs(a).max())
        got1 = host(ctx.prox_l1_reweighted(dev(a, torch), None, gamma))
        assert np.max(np.abs(got1 - oprox.soft_threshold(a, gamma))) <= 1e-6 * max(1.0, np.abs(a).max())
        y = inputs.random_vis(count, rng)
        for eps in (0.5 * np.sqrt(count), 10.0 * np.sqrt(count)):  # outside / inside the ball
            nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
            got = host(ctx.proj_l2ball(dev(a, torch), dev(y, torch), eps, norm_out=nrm))
            assert rel_err(got, oprox.project_l2_ball(a, y, eps)) <= 1e-6
            assert float(nrm.item()) == pytest.approx(np.linalg.norm(a - y), rel=1e-9)
        got = host(ctx.proj_positive(dev(a, torch)))
        assert np.array_equal(got, oprox.project_positive(a))


@pytest.mark.parametrize("n,M,J,iters", [(16, 300, 4, 40), (64, 2048, 4, 10), (256, 65536, 6, 10)])
def test_cg_solve(n, M, J, iters):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n + iters)
    uv = inputs.uniform_uv(M, rng)
    ctx = binding.Context(n, uv.astype(np.float32), J=J)
    b = inputs.random_image(n, rng)
    x0 = inputs.random_image(n, rng)
    x, res = ctx.cg_solve(dev(b, torch), dev(x0, torch), iters)
    want, want_res = ocg.cg(lambda v: me.phi_adj(me.phi(v, uv, J), uv, n, J) + 2.0 * v, b, x0, iters)
    assert rel_err(host(x).reshape(n, n), want) <= 1e-5
    assert float(res.item()) == pytest.approx(want_res, rel=1e-3, abs=1e-6 * np.linalg.norm(b))


@pytest.mark.parametrize("n,M,J", [(64, 2048, 4), (256, 65536, 6)])
def test_tile_schedules_agree(n, M, J, tmp_path):
    """Every tile side gives the same Phi / Phi^H (the schedule is not the method),
    and the autotuner picks one of them and caches it."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import autotune, binding

    rng = np.random.default_rng(n + 5)
    uv = inputs.uv_variable_density(M, n, rng).astype(np.float32).astype(np.float64)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    want_y = me.phi(x, uv, J)
    want_x = me.phi_adj(v, uv, n, J)
    for t in autotune.valid_tiles(n, J):
        ctx = binding.Context(n, uv.astype(np.float32), J=J, tile=t)
        assert rel_err(host(ctx.phi(dev(x, torch))), want_y) <= TOL
        assert rel_err(host(ctx.phi_adj(dev(v, torch))), want_x) <= TOL
    cache = str(tmp_path / "tune.json")
    entry = autotune.autotune_tile(n, uv, J, cache_path=cache, reps=3)
    assert entry["tile"] in autotune.valid_tiles(n, J)
    assert autotune.autotune_tile(n, uv, J, cache_path=cache)["tile"] == entry["tile"]


# Power-of-two grids of the compile-time FFT engine (2n = 256 .. 4096), each
# against the oracle: both zero-padding prunings, every row and column pass.
@pytest.mark.parametrize("n,M,J", [(128, 4000, 4), (512, 20000, 6), (2048, 20000, 6)])
def test_phi_and_adjoint_power_of_two_grids(n, M, J):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n + 7)
    uv = inputs.uv_variable_density(M, n, rng).astype(np.float32).astype(np.float64)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    ctx = binding.Context(n, uv.astype(np.float32), J=J, levels=4)
    assert rel_err(host(ctx.phi(dev(x, torch))), me.phi(x, uv, J)) <= TOL
    assert rel_err(host(ctx.phi_adj(dev(v, torch))), me.phi_adj(v, uv, n, J)) <= TOL


@pytest.mark.parametrize("n,M,J,tile", [(64, 40000, 6, 16), (96, 60000, 4, 16), (128, 60000, 6, 32)])
def test_cg_solve_dense_tiles(n, M, J, tile):
    """Coverages dense enough (more than two list entries per grid cell in
    the central tiles) that the Gram pass applies G^T G from its stored
    per-cell stencils there and gathers elsewhere: CG against the oracle."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n + M)
    uv = inputs.uv_variable_density(M, n, rng).astype(np.float32).astype(np.float64)
    ctx = binding.Context(n, uv.astype(np.float32), J=J, tile=tile)
    b = inputs.random_image(n, rng)
    x0 = inputs.random_image(n, rng)
    x, _ = ctx.cg_solve(dev(b, torch), dev(x0, torch), 6)
    want, _ = ocg.cg(lambda v: me.phi_adj(me.phi(v, uv, J), uv, n, J) + 2.0 * v, b, x0, 6)
    assert rel_err(host(x).reshape(n, n), want) <= 1e-5


def test_sara_contexts_of_different_sizes():
    """Contexts of different sizes used in turn: a kernel's shared-memory
    limit is a property of the kernel, shared by every context of the
    process, so each launch must still get the size it needs."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(5)
    big = binding.Context(512, inputs.uniform_uv(64, rng).astype(np.float32), J=4, levels=4)
    small = binding.Context(64, inputs.uniform_uv(64, rng).astype(np.float32), J=4, levels=4)
    for ctx, n in ((big, 512), (small, 64), (big, 512)):
        x = inputs.random_image(n, rng)
        al = host(ctx.sara_analysis(dev(x, torch)))
        assert rel_err(al, osara.sara_analysis(x, 4)) <= TOL
        assert rel_err(host(ctx.sara_synthesis(dev(al, torch))).reshape(n, n), osara.sara_synthesis(al, 4)) <= TOL
