"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the projector or of the solvers.  It draws
random ellipse / ellipsoid phantoms, samples them at pixel centres and writes
their *analytic* line integrals (the continuous parallel-beam projection of
Sec. 2, evaluated in closed form for each ellipse) at the detector-bin centres,
then adds Poisson (Sec. 2, -ln normalisation of I/I0) or Gaussian noise.

Coordinate conventions (the same ones the projector uses):
  * pixel (ix, iy) is the unit square centred at x = ix + 1/2 - nx/2,
    y = iy + 1/2 - ny/2; the tomogram is stored (nz, ny, nx), x fastest;
  * bin k of angle theta sits at detector coordinate p = k + 1/2 - c
    (c = n_p/2 by default); the sinogram is stored (nz, n_theta, n_p);
  * the ray of (theta, p) is the line x cos(theta) + y sin(theta) = p.

Phantoms are point-sampled at pixel centres, and sinograms are the exact
projection of the continuous ellipses, so the data are not exactly in the
range of the discrete operator (like measured data).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# ----------------------------------------------------------------------------
# Workload table: the five synthetic workloads the library is exercised on.
# ----------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int            # nx = ny = n_p
    n_theta: int
    n_z: int          # slices per batch
    solver: str       # "sirt" | "sirt_bb" | "cgls" | "gd"
    iters: int
    noise: str        # "poisson" | "gaussian"
    noise_level: float
    phantom: str      # "ellipses2d" | "ellipsoids3d"
    values: str = "f32"
    seed: int = 0


WORKLOADS = {
    # one 128x128 slice, 180 angles, Poisson 1e5 photons/ray, SIRT 50
    "sirt_128x180_b1": Workload("sirt_128x180_b1", 128, 180, 1, "sirt", 50,
                                "poisson", 1e5, "ellipses2d", seed=12677 + 1),
    # 64 slices of 512x512, 360 angles, Poisson 1e4 photons/ray, SIRT 100
    "sirt_512x360_b64": Workload("sirt_512x360_b64", 512, 360, 64, "sirt", 100,
                                 "poisson", 1e4, "ellipsoids3d", seed=12677 + 2),
    # 16 slices of 2048x2048, 1024 angles, 5% Gaussian noise, CGLS 50, BF16 values
    "cgls_2048x1024_b16": Workload("cgls_2048x1024_b16", 2048, 1024, 16, "cgls", 50,
                                   "gaussian", 0.05, "ellipsoids3d", values="bf16",
                                   seed=12677 + 3),
    # 32 slices of 1024x1024, 720 angles, TV-regularised least squares by GD
    "gd_1024x720_b32": Workload("gd_1024x720_b32", 1024, 720, 32, "gd", 50,
                                "gaussian", 0.05, "ellipsoids3d", seed=12677 + 4),
}


# ----------------------------------------------------------------------------
# Phantom parameters
# ----------------------------------------------------------------------------

def random_ellipses(n: int, rng: np.random.Generator, count: int = 10) -> np.ndarray:
    """2-D random ellipses: rows (x0, y0, A, B, phi, rho).

    Centres uniform in a disk of radius 0.7*n/2 about the image centre,
    semi-axes U[0.05, 0.35]*n/2, orientation U[0, pi), density U[0, 1].
    """
    out = np.empty((count, 6))
    R = 0.7 * n / 2
    for e in range(count):
        rad = R * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * math.pi)
        out[e, 0] = rad * math.cos(ang)
        out[e, 1] = rad * math.sin(ang)
        out[e, 2] = rng.uniform(0.05, 0.35) * n / 2
        out[e, 3] = rng.uniform(0.05, 0.35) * n / 2
        out[e, 4] = rng.uniform(0, math.pi)
        out[e, 5] = rng.uniform(0, 1)
    return out


def random_ellipsoids(n: int, nz: int, rng: np.random.Generator, count: int = 16) -> np.ndarray:
    """3-D random ellipsoids rotated about z: rows (x0, y0, z0, A, B, C, phi, rho)."""
    out = np.empty((count, 8))
    R = 0.7 * n / 2
    for e in range(count):
        rad = R * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * math.pi)
        out[e, 0] = rad * math.cos(ang)
        out[e, 1] = rad * math.sin(ang)
        out[e, 2] = rng.uniform(-nz / 2, nz / 2)
        out[e, 3] = rng.uniform(0.05, 0.35) * n / 2
        out[e, 4] = rng.uniform(0.05, 0.35) * n / 2
        out[e, 5] = rng.uniform(0.25, 1.0) * max(nz, 1) / 2
        out[e, 6] = rng.uniform(0, math.pi)
        out[e, 7] = rng.uniform(0, 1)
    return out


def ellipsoid_section(ell3: np.ndarray, z: float) -> np.ndarray:
    """Cross-section of z-rotated ellipsoids at height z, as 2-D ellipses."""
    rows = []
    for x0, y0, z0, A, B, C, phi, rho in ell3:
        u = (z - z0) / C
        if abs(u) >= 1.0:
            continue
        f = math.sqrt(1.0 - u * u)
        rows.append((x0, y0, A * f, B * f, phi, rho))
    return np.array(rows, dtype=np.float64).reshape(-1, 6)


# ----------------------------------------------------------------------------
# Sampling and analytic projection
# ----------------------------------------------------------------------------

def rasterize(ell: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """Sum of ellipse densities at the pixel centres, shape (ny, nx), float64."""
    x = np.arange(nx) + 0.5 - nx / 2
    y = np.arange(ny) + 0.5 - ny / 2
    X, Y = np.meshgrid(x, y)
    img = np.zeros((ny, nx))
    for x0, y0, A, B, phi, rho in ell:
        c, s = math.cos(phi), math.sin(phi)
        u = (X - x0) * c + (Y - y0) * s
        v = -(X - x0) * s + (Y - y0) * c
        img += rho * ((u / A) ** 2 + (v / B) ** 2 <= 1.0)
    return img


def default_angles(n_theta: int) -> np.ndarray:
    """theta_m = m*pi/n_theta, m = 0..n_theta-1 (uniform over [0, pi))."""
    return np.arange(n_theta, dtype=np.float64) * math.pi / n_theta


def project_ellipses(ell: np.ndarray, angles: np.ndarray, n_p: int,
                     center: Optional[float] = None) -> np.ndarray:
    """Exact line integrals of the ellipses, shape (n_theta, n_p), float64.

    For an ellipse with semi-axes (A, B) rotated by phi, the chord of the line
    x cos(t) + y sin(t) = p has length 2AB sqrt(a^2 - s^2)/a^2 with
    a^2 = A^2 cos^2(t-phi) + B^2 sin^2(t-phi) and s the offset of p from the
    projected centre (Kak & Slaney, ch. 3).
    """
    c = n_p / 2 if center is None else center
    p = np.arange(n_p) + 0.5 - c
    ct = np.cos(angles)[:, None]
    st = np.sin(angles)[:, None]
    out = np.zeros((len(angles), n_p))
    for x0, y0, A, B, phi, rho in ell:
        a2 = A * A * np.cos(angles - phi) ** 2 + B * B * np.sin(angles - phi) ** 2
        s = p[None, :] - (x0 * ct + y0 * st)
        q = a2[:, None] - s * s
        out += np.where(q > 0, 2.0 * rho * A * B * np.sqrt(np.maximum(q, 0.0)) / a2[:, None], 0.0)
    return out


def poisson_sinogram(p: np.ndarray, I0: float, rng: np.random.Generator) -> np.ndarray:
    """Noisy line integrals from Poisson counts: b = -ln(max(N,1)/I0)/s.

    s = 2/max(p) rescales the slice so the lowest transmission is exp(-2);
    N ~ Poisson(I0 exp(-s p)).
    """
    pm = float(p.max())
    s = 2.0 / pm if pm > 0 else 1.0
    counts = rng.poisson(I0 * np.exp(-s * p))
    return -np.log(np.maximum(counts, 1) / I0) / s


def gaussian_sinogram(p: np.ndarray, rel: float, rng: np.random.Generator) -> np.ndarray:
    """b = p + rel * rms(p) * N(0, 1)."""
    rms = float(np.sqrt(np.mean(p * p)))
    return p + rel * rms * rng.standard_normal(p.shape)


# ----------------------------------------------------------------------------
# Whole cases
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Case:
    n: int
    n_theta: int
    n_z: int
    phantom: np.ndarray      # (nz, n, n) float32
    sino: np.ndarray         # (nz, n_theta, n) float32, noisy
    clean: np.ndarray        # (nz, n_theta, n) float32, noise-free analytic projection


def make_case(n: int, n_theta: int, n_z: int, seed: int, phantom: str = "ellipsoids3d",
              noise: str = "poisson", level: float = 1e4, slices: Optional[Sequence[int]] = None) -> Case:
    """Build a seeded case; `slices` restricts which slices are materialised."""
    rng = np.random.default_rng(seed)
    angles = default_angles(n_theta)
    sl = list(range(n_z)) if slices is None else list(slices)
    if phantom == "ellipses2d":
        ells = [random_ellipses(n, rng) for _ in range(n_z)]
        sections = [ells[s] for s in sl]
    else:
        e3 = random_ellipsoids(n, n_z, rng)
        sections = [ellipsoid_section(e3, s + 0.5 - n_z / 2) for s in sl]
    ph = np.stack([rasterize(e, n, n) for e in sections]).astype(np.float32)
    clean = np.stack([project_ellipses(e, angles, n) for e in sections])
    noise_rng = np.random.default_rng(seed + 7919)
    if noise == "poisson":
        noisy = np.stack([poisson_sinogram(c, level, noise_rng) for c in clean])
    elif noise == "gaussian":
        noisy = np.stack([gaussian_sinogram(c, level, noise_rng) for c in clean])
    else:
        noisy = clean.copy()
    return Case(n, n_theta, len(sl), ph, noisy.astype(np.float32), clean.astype(np.float32))


def workload_case(name: str, slices: Optional[Sequence[int]] = None) -> Case:
    w = WORKLOADS[name]
    return make_case(w.n, w.n_theta, w.n_z, w.seed, w.phantom, w.noise, w.noise_level, slices)


# the benchmark's 64-slice 512x512x360 data solved by the paper's SIRT (Hamming
# preconditioning, BB step), 30 iterations
WORKLOADS["sirt_bb_512x360_b64"] = Workload("sirt_bb_512x360_b64", 512, 360, 64, "sirt_bb", 30,
                                           "poisson", 1e4, "ellipsoids3d", seed=12677 + 2)

# the same data through the Fubini-Radon operator (Fourier slice theorem,
# Kaiser-Bessel gridding, kw = 6): one forward and one adjoint per iteration
WORKLOADS["fubini_512x360_b64"] = Workload("fubini_512x360_b64", 512, 360, 64, "fubini", 100,
                                          "poisson", 1e4, "ellipsoids3d", seed=12677 + 2)

# the same data solved by the paper's SIRT on the Fubini-Radon operator with
# its normal operator applied in one step (a 2n x 2n convolution), 30 iterations
WORKLOADS["fubini_normal_512x360_b64"] = Workload("fubini_normal_512x360_b64", 512, 360, 64, "fubini_normal", 30,
                                                 "poisson", 1e4, "ellipsoids3d", seed=12677 + 2)

# a profiling stand-in for cgls_2048x1024_b16: the same image, detector, slices
# and 16-bit values on 128 of the angles (one eighth of the matrix, a few GB),
# for hardware-counter captures that replay each launch many times
WORKLOADS["cgls_2048x128_b16"] = Workload("cgls_2048x128_b16", 2048, 128, 16, "cgls", 50,
                                         "gaussian", 0.05, "ellipsoids3d", values="bf16", seed=12677 + 3)

WORKLOADS["uneven_256"] = Workload("uneven_256", 2048, 1024, 0, "cgls", 30, "poisson", 1e5, "ellipses2d",
                                  values="bf16", seed=12677 + 5)


@dataclasses.dataclass
class Request:
    n: int
    n_theta: int
    n_z: int
    seed: int


def uneven_requests(count: int = 256, seed: int = 12677 + 5,
                    sizes: Sequence[int] = (256, 512, 1024, 2048),
                    angle_counts: Sequence[int] = (180, 360, 720, 1024),
                    max_slices: int = 32) -> List[Request]:
    """Seeded mix of reconstruction requests of uneven size and slice count."""
    rng = np.random.default_rng(seed)
    out = []
    for r in range(count):
        n = int(rng.choice(sizes))
        nt = int(rng.choice(angle_counts))
        nz = int(rng.integers(1, max_slices + 1))
        out.append(Request(n, nt, nz, seed + 1000 * (r + 1)))
    return out


def request_case(req: Request) -> Case:
    return make_case(req.n, req.n_theta, req.n_z, req.seed, "ellipses2d", "poisson", 1e5)


def random_slices(shape, seed: int) -> np.ndarray:
    """Plain seeded U[0,1) float32 data for operator tests."""
    return np.random.default_rng(seed).random(shape, dtype=np.float32)
