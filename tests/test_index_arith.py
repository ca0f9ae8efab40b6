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
