"""Host checks of index arithmetic used by the CUDA kernels.

The gridding kernel divides small non-negative integers by the halo and key
widths with a rounded float reciprocal (`quot_small` in `csrc/common.cuh`):
floor(k / d) = trunc(rn(rn(k + 1/2) * rn(1/d))).  IEEE float32 arithmetic
with round-to-nearest is the same on the host (numpy) and the device
(`__fadd_rn`, `__fmul_rn`, correctly rounded division), so the identity is
checked here exhaustively over the whole stated domain."""
import numpy as np


def test_float_reciprocal_quotient_is_exact():
    k = np.arange(1 << 16, dtype=np.int64)
    kf = (k.astype(np.float32) + np.float32(0.5)).astype(np.float32)
    for d in range(1, 129):
        r = np.float32(1.0) / np.float32(d)
        q = np.trunc((kf * r).astype(np.float32)).astype(np.int64)
        assert np.array_equal(q, k // d), d


def test_slice_of_owner_step():
    """The fix-up of the gridding kernel finds the slice holding step x of a
    chunk's Wt steps, floor(x / Wt) for x = P * 256 with 0 <= P <= Wt < 2^16,
    as trunc(rn(float(x) * rn(1 / Wt))) corrected by one integer comparison
    each way (the quotient is at most 256, so the float product is within
    one of it).  Checked for every P at the extreme and a spread of Wt."""
    rng = np.random.default_rng(0)
    wts = np.unique(np.concatenate([np.arange(1, 2049), rng.integers(2049, 1 << 16, 3000), [(1 << 16) - 1]]))
    for wt in wts:
        P = np.arange(wt + 1, dtype=np.int64)
        x = P * 256
        inv = np.float32(1.0) / np.float32(wt)
        q = np.trunc((x.astype(np.float32) * inv).astype(np.float32)).astype(np.int64)
        q = np.where(q * wt > x, q - 1, np.where((q + 1) * wt <= x, q + 1, q))
        assert np.array_equal(q, x // wt), wt
