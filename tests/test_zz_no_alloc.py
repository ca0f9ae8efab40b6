"""purify_phi_static, the entry point that allocates nothing (needs a GB300).

Callers that cannot allocate device memory when they need Phi (their GPU
memory is reserved by another allocator, or they cannot afford cudaMalloc in
a latency-critical loop) use purify_phi_static, whose scratch is a fixed
device array inside the library.  Its output must match purify_phi, the
context-based entry point, within the operator tolerance of the other GPU
tests, on two calls in a row (the second call reuses the array the first one
left behind), and it must match the FP64 oracle's Phi (§5 eq. opmodel) to
the same 1e-5.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import measurement as me
from paper_1307_4370_gb300 import inputs

from gpu_util import dev, host, rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.mark.parametrize("n,M,J", [(64, 2048, 4), (96, 3001, 6), (256, 65536, 6)])
def test_phi_static_matches_phi(n, M, J):
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(n * 31 + J)
    uv = inputs.uv_variable_density(M, n, rng).astype(np.float32)
    uv_t = torch.tensor(uv, device="cuda")
    ctx = binding.Context(n, uv, J=J, levels=4)
    for _ in range(2):  # two calls in a row, different images
        x_np = inputs.random_image(n, rng)
        x = dev(x_np, torch)
        want = host(ctx.phi(x))
        got = host(binding.phi_static(n, J, uv_t, x))
        torch.cuda.synchronize()
        assert rel_err(got, want) <= TOL
        assert rel_err(got, me.phi(x_np, uv.astype(np.float64), J)) <= TOL


def test_phi_static_size_change_rewrites_its_tables():
    """Calls alternating between two sizes: the tables the fixed array keeps
    from the previous call are rewritten for the new size."""
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    rng = np.random.default_rng(77)
    cases = []
    for n, M, J in [(64, 1000, 4), (96, 1500, 6)]:
        uv = inputs.uv_variable_density(M, n, rng).astype(np.float32)
        cases.append((n, J, uv, torch.tensor(uv, device="cuda")))
    for k in range(4):
        n, J, uv, uv_t = cases[k % 2]
        x_np = inputs.random_image(n, rng)
        got = host(binding.phi_static(n, J, uv_t, dev(x_np, torch)))
        assert rel_err(got, me.phi(x_np, uv.astype(np.float64), J)) <= TOL


def test_phi_static_rejects_sizes_beyond_the_limit():
    torch = require_gpu()
    from paper_1307_4370_gb300 import binding

    uv = torch.zeros((4, 2), dtype=torch.float32, device="cuda")
    x = torch.zeros(512 * 512, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.PurifyError) as e:
        binding.phi_static(512, 6, uv, x)
    assert e.value.status == -2
