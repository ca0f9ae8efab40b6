"""Host checks of index arithmetic used by the CUDA kernels.

The gridding kernel divides small non-negative integers by the halo and key
widths with a rounded float reciprocal (`quot_small` in `csrc/common.cuh`):
floor(k / d) = trunc(rn(rn(k + 1/2) * rn(1/d))).  IEEE float32 arithmetic
with round-to-nearest is the same on the host (numpy) and the device
(`__fadd_rn`, `__fmul_rn`, correctly rounded division), so the identity is
checked here exhaustively over the whole stated domain.  The other checks
restate the index layouts the set-up writes and the kernels read (the owner
fix-up slices, the half G^T G stencil of dense tiles) and verify them on
small random cases."""
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


def test_half_stencil_gram_indexing():
    """The half (symmetric) G^T G stencil of a dense tile, in the index
    layout the set-up writes and the Gram kernel reads (offset slices
    s(d) for d >= 0 in lexicographic order, the tile extended by J - 1 rows
    above and J - 1 columns each side, the halo's first row R0 - (J - 1) and
    first column C0 - J), reproduces degrid-then-grid of random entries on
    random halo values: sum_{d>=0} H[s(d)][k] X(k+d) + sum_{d>0} H[s(d)][k-d] X(k-d)."""
    rng = np.random.default_rng(1)
    for J, T in [(6, 8), (4, 8), (2, 4), (8, 8)]:
        W, NDW = T + J - 1, 2 * J - 1
        NH, EW, EH = J + (J - 1) * NDW, T + 2 * (J - 1), T + J - 1
        HWS = T + 2 * J
        ne = 60
        kr, kc = rng.integers(0, W, ne), rng.integers(0, W, ne)  # footprint start + (J - 1), tile-relative
        wr, wc = rng.random((ne, J)), rng.random((ne, J))
        halo = rng.standard_normal((T + 2 * (J - 1), HWS)) + 1j * rng.standard_normal((T + 2 * (J - 1), HWS))
        ref = np.zeros((T, T), complex)
        H = np.zeros((NH, EH * EW))
        for m in range(ne):
            r0, c0 = kr[m] - (J - 1), kc[m] - (J - 1)
            w2 = np.outer(wr[m], wc[m])
            v = np.sum(w2 * halo[r0 + J - 1:r0 + 2 * J - 1, c0 + J:c0 + 2 * J])
            for a in range(J):
                for b in range(J):
                    if 0 <= r0 + a < T and 0 <= c0 + b < T:
                        ref[r0 + a, c0 + b] += w2[a, b] * v
                    er, ec = kr[m] + a, kc[m] + b
                    if er >= EH or ec >= EW:
                        continue
                    for a2 in range(a, J):
                        for b2 in range(b if a2 == a else 0, J):
                            dr, dc = a2 - a, b2 - b
                            sl = dc if dr == 0 else J + (dr - 1) * NDW + dc + J - 1
                            H[sl, er * EW + ec] += w2[a, b] * w2[a2, b2]
        hf = halo.reshape(-1)
        out = np.zeros((T, T), complex)
        for r in range(T):
            for c in range(T):
                e0, xk = (r + J - 1) * EW + c + J - 1, (r + J - 1) * HWS + c + J
                acc = H[0, e0] * hf[xk]
                for dc in range(1, J):
                    acc += H[dc, e0] * hf[xk + dc] + H[dc, e0 - dc] * hf[xk - dc]
                for dr in range(1, J):
                    for dc in range(-(J - 1), J):
                        sl = J + (dr - 1) * NDW + dc + J - 1
                        acc += H[sl, e0] * hf[xk + dr * HWS + dc]
                        acc += H[sl, e0 - dr * EW - dc] * hf[xk - dr * HWS - dc]
                out[r, c] = acc
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max(), (J, T)
