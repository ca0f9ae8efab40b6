"""Seeded synthetic inputs shaped like the simulations of §6.

This module is shared by the FP64 oracle, the tests and the benchmark.  It
draws images, u-v coverages and unit-variance noise; it contains none of the
imaging method's arithmetic (no measurement operator, no wavelet, no prox).
Whatever the method needs from these draws (the clean visibilities, the noise
scale, the l2 bound epsilon) is computed by each implementation on its own.

Recipe (stand-ins for the M31 / 30Dor images and the AMI coverage of §6,
which are not available):

* Sky: a sum of elliptical Gaussian sources (centres uniform over the inner
  80 % of the field, major-axis width U[1, 6] pixels, axis ratio U[0.3, 1],
  position angle U[0, pi), amplitude log-uniform in [1e-3, 1]), optionally
  plus a non-negative diffuse field with a k^-2 power spectrum, min-shifted,
  scaled to peak 0.1 and tapered by a smooth circular window.
* Coverage: continuous frequencies u in [-pi, pi)^2 (radians per pixel)
  drawn from an isotropic Gaussian variable-density profile (sigma = pi/4,
  truncated to the square by rejection); the (0,0) component is suppressed
  by rejecting |u| < 2 pi / n (§6 suppresses the origin of the Fourier
  plane).  The radial-track variant puts half of the points on arcs of
  uniform-random radius and angle.
* Noise: i.i.d. complex Gaussian draws of unit variance (real and imaginary
  parts each N(0, 1/2)); the caller scales them to the input SNR of §6.

All values are rounded to the storage precision of the GPU path (float32 /
complex64) before they are returned, so the oracle and the CUDA path read
bit-identical inputs.
"""
from __future__ import annotations

import dataclasses

import numpy as np

# Seeds: 1307 + index of the workload in the table below.
SEED_BASE = 1307


@dataclasses.dataclass(frozen=True)
class Workload:
    """Sizes of one synthetic imaging problem."""

    name: str
    n: int                 # image side (N = n*n pixels)
    M: int                 # number of visibilities
    J: int                 # Kaiser-Bessel support (cells per axis)
    n_src: int             # number of Gaussian sources
    diffuse: bool          # add the k^-2 diffuse component
    arcs: int = 0          # number of radial-track arcs (0 = none)
    T: int = 50            # SDMM iterations per reweighting round
    rounds: int = 1        # reweighting rounds
    cg_iters: int = 10     # conjugate-gradient steps per SDMM iteration
    isnr_db: float = 30.0  # input SNR of the visibilities
    seed: int = SEED_BASE


# The five workloads: oracle-sized, the 256^2 FP32 problem, the 1024^2
# mixed-precision problem, and the two derived ones.
WORKLOADS = {
    "sdmm64": Workload("sdmm64", n=64, M=2048, J=4, n_src=20, diffuse=False,
                       T=50, rounds=1, seed=SEED_BASE + 0),
    "sdmm256": Workload("sdmm256", n=256, M=65536, J=6, n_src=200,
                        diffuse=True, T=60, rounds=5, seed=SEED_BASE + 1),
    "sdmm1024": Workload("sdmm1024", n=1024, M=2097152, J=6, n_src=5000,
                         diffuse=True, arcs=200, T=60, rounds=1,
                         seed=SEED_BASE + 2),
    "diff256": Workload("diff256", n=256, M=65536, J=6, n_src=200,
                        diffuse=True, T=20, rounds=1, seed=SEED_BASE + 4),
}


def gaussian_sources(n: int, n_src: int, rng: np.random.Generator) -> np.ndarray:
    """Sum of ``n_src`` elliptical Gaussians on an n x n grid (float64)."""
    r = np.arange(n, dtype=np.float64)[:, None]
    c = np.arange(n, dtype=np.float64)[None, :]
    img = np.zeros((n, n))
    cr = rng.uniform(0.1 * n, 0.9 * n, n_src)
    cc = rng.uniform(0.1 * n, 0.9 * n, n_src)
    sig_a = rng.uniform(1.0, 6.0, n_src)
    ratio = rng.uniform(0.3, 1.0, n_src)
    ang = rng.uniform(0.0, np.pi, n_src)
    amp = 10.0 ** rng.uniform(-3.0, 0.0, n_src)
    for k in range(n_src):
        # Evaluate on a window of +-5 sigma around the centre (the Gaussian is
        # below 4e-6 of its peak outside it).
        h = int(np.ceil(5.0 * sig_a[k])) + 1
        r0, r1 = max(0, int(cr[k]) - h), min(n, int(cr[k]) + h + 1)
        c0, c1 = max(0, int(cc[k]) - h), min(n, int(cc[k]) + h + 1)
        dr = r[r0:r1] - cr[k]
        dc = c[:, c0:c1] - cc[k]
        ca, sa = np.cos(ang[k]), np.sin(ang[k])
        p = ca * dr + sa * dc
        q = -sa * dr + ca * dc
        sb = sig_a[k] * ratio[k]
        img[r0:r1, c0:c1] += amp[k] * np.exp(-0.5 * (p * p / sig_a[k] ** 2 + q * q / sb ** 2))
    return img


def diffuse_field(n: int, rng: np.random.Generator, peak: float = 0.1) -> np.ndarray:
    """Non-negative Gaussian random field with a k^-2 power spectrum."""
    white = rng.standard_normal((n, n))
    k = np.fft.fftfreq(n)
    kk = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    kk[0, 0] = np.inf  # drop the mean
    field = np.real(np.fft.ifft2(np.fft.fft2(white) / kk))  # amplitude ~ k^-1
    field -= field.min()
    field *= peak / max(field.max(), 1e-300)
    rr = np.hypot(np.arange(n) - n / 2 + 0.5, (np.arange(n) - n / 2 + 0.5)[:, None]) / (n / 2)
    taper = np.where(rr < 1.0, np.cos(0.5 * np.pi * np.clip(rr, 0, 1)) ** 2, 0.0)
    return field * taper


def sky_image(w: Workload, rng: np.random.Generator) -> np.ndarray:
    """Ground-truth image (float32 values, returned as float64)."""
    img = gaussian_sources(w.n, w.n_src, rng)
    if w.diffuse:
        img += diffuse_field(w.n, rng)
    return img.astype(np.float32).astype(np.float64)


def uv_variable_density(M: int, n: int, rng: np.random.Generator,
                        sigma: float = np.pi / 4) -> np.ndarray:
    """M points of an isotropic Gaussian density truncated to [-pi, pi)^2.

    Points with |u| < 2 pi / n (inside the first image-frequency cell) are
    rejected, which suppresses the (0,0) component of the Fourier plane.
    """
    out = np.empty((0, 2))
    rmin = 2.0 * np.pi / n
    while out.shape[0] < M:
        need = M - out.shape[0]
        u = rng.normal(0.0, sigma, size=(2 * need + 64, 2))
        ok = np.all((u >= -np.pi) & (u < np.pi), axis=1) & (np.hypot(u[:, 0], u[:, 1]) >= rmin)
        out = np.concatenate([out, u[ok][:need]])
    return out


def uv_radial_arcs(M: int, n: int, n_arcs: int, rng: np.random.Generator) -> np.ndarray:
    """M points on ``n_arcs`` circular arcs centred on the origin.

    Radius U(2 pi / n, pi), start angle U[0, 2 pi), angular extent
    U[0, pi/2]; the points are spread evenly along each arc and the arcs
    share the points as equally as the division allows.
    """
    rad = rng.uniform(2.0 * np.pi / n, np.pi, n_arcs)
    start = rng.uniform(0.0, 2.0 * np.pi, n_arcs)
    ext = rng.uniform(0.0, np.pi / 2, n_arcs)
    counts = np.full(n_arcs, M // n_arcs)
    counts[: M - counts.sum()] += 1
    pts = []
    for a in range(n_arcs):
        t = start[a] + ext[a] * (np.arange(counts[a]) + 0.5) / counts[a]
        pts.append(np.stack([rad[a] * np.cos(t), rad[a] * np.sin(t)], axis=1))
    u = np.concatenate(pts)
    # Fold into [-pi, pi): radius < pi already keeps |u_i| < pi.
    return np.clip(u, -np.pi, np.nextafter(np.pi, 0.0))


def coverage(w: Workload, rng: np.random.Generator) -> np.ndarray:
    """u-v coverage of a workload, float32 values (returned as float64)."""
    if w.arcs > 0:
        m_arc = w.M // 2
        uv = np.concatenate([uv_variable_density(w.M - m_arc, w.n, rng),
                             uv_radial_arcs(m_arc, w.n, w.arcs, rng)])
        uv = uv[rng.permutation(w.M)]
    else:
        uv = uv_variable_density(w.M, w.n, rng)
    uv32 = uv.astype(np.float32)
    # float32 rounding must not push a point onto +pi.
    uv32 = np.where(uv32 >= np.float32(np.pi), np.nextafter(np.float32(np.pi), np.float32(0)), uv32)
    return uv32.astype(np.float64)


def unit_complex_noise(M: int, rng: np.random.Generator) -> np.ndarray:
    """i.i.d. complex Gaussian of unit variance (complex64 values)."""
    z = (rng.standard_normal(M) + 1j * rng.standard_normal(M)) / np.sqrt(2.0)
    return z.astype(np.complex64).astype(np.complex128)


@dataclasses.dataclass
class Problem:
    """Seeded draws of one workload (float64/complex128 arrays holding
    float32/complex64 values)."""

    workload: Workload
    x_true: np.ndarray     # (n, n) non-negative image
    uv: np.ndarray         # (M, 2) frequencies in radians per pixel
    noise_unit: np.ndarray # (M,) unit-variance complex noise


def make_problem(name_or_workload, seed: int | None = None) -> Problem:
    """Draw the image, coverage and unit noise of a workload."""
    w = WORKLOADS[name_or_workload] if isinstance(name_or_workload, str) else name_or_workload
    rng = np.random.default_rng(w.seed if seed is None else seed)
    x = sky_image(w, rng)
    uv = coverage(w, rng)
    nz = unit_complex_noise(w.M, rng)
    return Problem(w, x, uv, nz)


def random_image(n: int, rng: np.random.Generator, complex_: bool = True) -> np.ndarray:
    """Random test image (complex64 values) for operator-level tests."""
    x = rng.standard_normal((n, n))
    if complex_:
        x = x + 1j * rng.standard_normal((n, n))
        return x.astype(np.complex64).astype(np.complex128)
    return x.astype(np.float32).astype(np.float64)


def random_vis(M: int, rng: np.random.Generator) -> np.ndarray:
    """Random complex vector (complex64 values)."""
    return unit_complex_noise(M, rng)


def uniform_uv(M: int, rng: np.random.Generator) -> np.ndarray:
    """M frequencies uniform on [-pi, pi)^2 (float32 values)."""
    uv = rng.uniform(-np.pi, np.pi, size=(M, 2)).astype(np.float32)
    uv = np.where(uv >= np.float32(np.pi), np.nextafter(np.float32(np.pi), np.float32(0)), uv)
    return uv.astype(np.float64)


def batch_workloads(count: int = 32, seed: int = SEED_BASE + 3) -> list[Workload]:
    """Uneven independent problems: image side uniform in {128, 192, 256, 384,
    512}, M uniform in [0.2 N, 2 N], Kaiser-Bessel support 4 or 6, 200
    iterations each (each problem draws its own image and coverage)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice([128, 192, 256, 384, 512]))
        N = n * n
        M = int(rng.integers(int(0.2 * N), 2 * N + 1))
        J = int(rng.choice([4, 6]))
        out.append(Workload(f"batch{k}", n=n, M=M, J=J, n_src=max(20, n // 2), diffuse=True,
                            T=200, rounds=1, seed=seed * 100 + k))
    return out
