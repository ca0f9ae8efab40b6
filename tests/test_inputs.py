"""The seeded input recipe (stand-ins for the images and coverage of §6):
determinism, value ranges and the stated shapes of the draws."""
import numpy as np
import pytest

from paper_1307_4370_gb300 import inputs


def _is_f32(a):
    return np.array_equal(a, a.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("name", ["sdmm64", "sdmm256"])
def test_problem_is_seeded_and_in_storage_precision(name):
    p, q = inputs.make_problem(name), inputs.make_problem(name)
    w = p.workload
    assert np.array_equal(p.x_true, q.x_true) and np.array_equal(p.uv, q.uv)
    assert np.array_equal(p.noise_unit, q.noise_unit)
    assert p.x_true.shape == (w.n, w.n) and p.uv.shape == (w.M, 2) and p.noise_unit.shape == (w.M,)
    assert _is_f32(p.x_true) and _is_f32(p.uv)
    assert _is_f32(p.noise_unit.real) and _is_f32(p.noise_unit.imag)
    assert p.x_true.min() >= 0.0 and p.x_true.max() > 0.0
    # another seed gives another draw
    assert not np.array_equal(inputs.make_problem(name, seed=w.seed + 100).uv, p.uv)


@pytest.mark.parametrize("name", ["sdmm64", "sdmm256"])
def test_coverage_range_and_origin_suppression(name):
    p = inputs.make_problem(name)
    u = p.uv
    assert np.all(u >= -np.pi) and np.all(u < np.pi)
    # |u| >= 2 pi / n up to the float32 rounding of the stored values
    r = np.hypot(u[:, 0], u[:, 1])
    assert r.min() >= 2 * np.pi / p.workload.n * (1 - 1e-6)
    # Gaussian variable density, sigma = pi/4 per axis: the truncation to the
    # square and the origin hole barely change the second moment
    assert np.mean(u * u) == pytest.approx((np.pi / 4) ** 2, rel=0.05)


def test_unit_noise_variance():
    z = inputs.unit_complex_noise(1 << 16, np.random.default_rng(5))
    assert np.mean(np.abs(z) ** 2) == pytest.approx(1.0, abs=4 / np.sqrt(1 << 16))
    assert np.mean(z.real ** 2) == pytest.approx(0.5, abs=4 / np.sqrt(1 << 16))
    assert abs(np.mean(z)) < 4 / np.sqrt(1 << 16)


def test_radial_arcs():
    n, M, arcs = 256, 10000, 50
    u = inputs.uv_radial_arcs(M, n, arcs, np.random.default_rng(3))
    assert u.shape == (M, 2)
    r = np.hypot(u[:, 0], u[:, 1])
    assert r.min() >= 2 * np.pi / n * (1 - 1e-12) and r.max() < np.pi
    # points lie on at most `arcs` circles, as equally shared as the division allows
    radii, counts = np.unique(np.round(r, 9), return_counts=True)
    assert len(radii) <= arcs and counts.max() - counts.min() <= 1
    # each arc spans at most pi/2
    for rad in radii:
        on = np.isclose(r, rad)
        ang = np.sort(np.mod(np.arctan2(u[on, 1], u[on, 0]), 2 * np.pi))
        gaps = np.diff(np.concatenate([ang, ang[:1] + 2 * np.pi]))
        assert 2 * np.pi - gaps.max() <= np.pi / 2 + 1e-9


def test_batch_workloads():
    ws = inputs.batch_workloads()
    assert len(ws) == 32 and ws == inputs.batch_workloads()
    for w in ws:
        N = w.n * w.n
        assert w.n in (128, 192, 256, 384, 512) and w.J in (4, 6)
        assert 0.2 * N - 1 <= w.M <= 2 * N and w.T == 200
    assert len({w.n for w in ws}) >= 3
