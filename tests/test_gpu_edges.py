"""Edge and degenerate cases of the operators on the GPU against the FP64 oracle.

* one visibility (every other tile empty);
* every visibility in one footprint start cell (the densest case: one tile
  split into many chunks merged in order, and the Gram form of CG on it);
* frequencies on exact grid lines and at the ends of [-pi, pi) (the floor
  rule of the footprint and the periodic wrap);
* the largest image side, n = 2048 (4096-point rows: 16 elements per thread);
* a 768 x 768 image (1536 = 3 * 2^9 rows and columns, radix 3).
"""
import numpy as np
import pytest

from oracle import cg as ocg, measurement as me
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu
TOL = 1e-5


def check_pair(n, uv, J, rng, tile=0):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    uv = np.asarray(uv, dtype=np.float32).astype(np.float64)
    M = uv.shape[0]
    ctx = binding.Context(n, uv.astype(np.float32), J=J, tile=tile)
    x = inputs.random_image(n, rng)
    v = inputs.random_vis(M, rng)
    assert rel_err(host(ctx.phi(dev(x, torch))), me.phi(x, uv, J)) <= TOL
    assert rel_err(host(ctx.phi_adj(dev(v, torch))), me.phi_adj(v, uv, n, J)) <= TOL
    return ctx


def test_single_visibility():
    rng = np.random.default_rng(1)
    check_pair(16, [[0.3, -1.2]], 4, rng)


@pytest.mark.parametrize("tile", [8, 16])
def test_all_visibilities_in_one_cell(tile):
    torch = require_gpu()
    rng = np.random.default_rng(2)
    n, J, M = 32, 6, 5000
    L = 2 * n
    # one start cell: kappa in [k, k + 1) on both axes
    k = 9
    kap = k + rng.uniform(0.05, 0.95, size=(M, 2))
    uv = (kap * 2 * np.pi / L).astype(np.float32).astype(np.float64)
    ctx = check_pair(n, uv, J, rng, tile=tile)
    # CG on Q = Phi^H Phi + 2I (its G^T G in the one-pass form)
    b = inputs.random_image(n, rng)
    x, _ = ctx.cg_solve(dev(b, torch), dev(np.zeros((n, n), dtype=np.complex128), torch), 4)
    want, _ = ocg.cg(lambda v: me.phi_adj(me.phi(v, uv, J), uv, n, J) + 2.0 * v, b, np.zeros((n, n)), 4)
    assert rel_err(host(x).reshape(n, n), want) <= TOL


def test_grid_line_and_boundary_frequencies():
    rng = np.random.default_rng(3)
    n, J = 32, 6
    L = 2 * n
    on_lines = (np.arange(-L // 2, L // 2, 3)[:, None] * 2 * np.pi / L) * np.ones((1, 2))
    ends = np.array([[-np.pi, -np.pi], [-np.pi, 0.5], [np.nextafter(np.float32(np.pi), np.float32(0)), 1.0],
                     [0.0, np.nextafter(np.float32(np.pi), np.float32(0))], [0.0, 0.0]])
    check_pair(n, np.concatenate([on_lines, ends]), J, rng)


def test_largest_image():
    rng = np.random.default_rng(4)
    n, J, M = 2048, 6, 100000
    check_pair(n, inputs.uniform_uv(M, rng), J, rng)


def test_radix3_large():
    rng = np.random.default_rng(5)
    n, J, M = 768, 4, 60000
    check_pair(n, inputs.uv_variable_density(M, n, rng), J, rng)
