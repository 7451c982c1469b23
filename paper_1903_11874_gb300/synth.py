"""Seeded synthetic inputs: phantoms, noise and random test vectors.

This module holds none of the method's arithmetic (no projection, no BSGD
step); it only draws inputs, so that the tests can feed the same data to the
CUDA library and to the FP64 oracle. It imports nothing from either.

The paper's data (a Shepp-Logan phantom, the TIGRE skull) are replaced by
random ellipses / ellipsoids of the same kind:
  * 2D: n ellipses, drawn in the order cx, cy ~ U[-.6, .6]; a, b ~ U[.05, .4];
    phi ~ U[0, pi); rho ~ U[0, 1]; densities add up; sampled at pixel centres
    in normalised coordinates [-1, 1];
  * 3D: centres ~ U[-.6, .6]^3, semi-axes ~ U[.05, .4]^3, rotation about z by
    phi ~ U[0, pi), rho ~ U[0, 1].
"""
import math

import numpy as np


def _norm_coords(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * (2.0 / n) - 1.0


def ellipse_phantom(nx: int, ny: int, n_ellipses: int = 6, seed: int = 0) -> np.ndarray:
    """[ny, nx] float64 image of random ellipses."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(_norm_coords(nx), _norm_coords(ny), indexing="xy")
    img = np.zeros((ny, nx))
    for _ in range(n_ellipses):
        cx, cy = rng.uniform(-0.6, 0.6, size=2)
        a, b = rng.uniform(0.05, 0.4, size=2)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        c, s = math.cos(phi), math.sin(phi)
        xr = c * (X - cx) + s * (Y - cy)
        yr = -s * (X - cx) + c * (Y - cy)
        img[(xr / a) ** 2 + (yr / b) ** 2 <= 1.0] += rho
    return img


def ellipsoid_phantom(nx: int, ny: int, nz: int, n_ellipsoids: int = 10, seed: int = 0) -> np.ndarray:
    """[nz, ny, nx] float32 volume of random ellipsoids (built slice by slice to
    keep memory at one slice of float64)."""
    rng = np.random.default_rng(seed)
    params = []
    for _ in range(n_ellipsoids):
        ctr = rng.uniform(-0.6, 0.6, size=3)
        ax = rng.uniform(0.05, 0.4, size=3)
        phi = rng.uniform(0.0, math.pi)
        rho = rng.uniform(0.0, 1.0)
        params.append((ctr, ax, math.cos(phi), math.sin(phi), rho))
    X, Y = np.meshgrid(_norm_coords(nx), _norm_coords(ny), indexing="xy")
    zc = _norm_coords(nz)
    vol = np.zeros((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        sl = np.zeros((ny, nx))
        for ctr, ax, c, s, rho in params:
            dz = (zc[k] - ctr[2]) / ax[2]
            if dz * dz > 1.0:
                continue
            xr = c * (X - ctr[0]) + s * (Y - ctr[1])
            yr = -s * (X - ctr[0]) + c * (Y - ctr[1])
            sl[(xr / ax[0]) ** 2 + (yr / ax[1]) ** 2 + dz * dz <= 1.0] += rho
        vol[k] = sl
    return vol


def poisson_log_data(line_integrals: np.ndarray, i0: float, seed: int) -> np.ndarray:
    """Transmission data with Poisson counts: N ~ Poisson(I0 exp(-p)),
    y = -ln(max(N, 1) / I0). Returned as float32."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(i0 * np.exp(-np.asarray(line_integrals, dtype=np.float64)))
    return (-np.log(np.maximum(counts, 1) / i0)).astype(np.float32)


def gaussian_noise_at_snr(y: np.ndarray, snr_db: float, seed: int) -> np.ndarray:
    """y + e with white Gaussian e scaled so that 20 log10(||y|| / ||e||) = snr_db."""
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(y.shape)
    e *= np.linalg.norm(y) / (np.linalg.norm(e) * 10.0 ** (snr_db / 20.0))
    return y + e


def uniform_array(shape, seed: int, lo: float = 0.0, hi: float = 1.0, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape).astype(dtype)


def normal_array(shape, seed: int, dtype=np.float64) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(size=shape).astype(dtype)


# Reduced precision workload: the 512^3 / 720-view / 512^2-detector BSGD-TV
# set-up at 1/8 of its resolution in every dimension (the same 256 mm volume,
# 409.6 mm detector, DSO 500 / DSD 1000 mm), 16 x 16 blocks, one pair per
# iteration, uniform draws, lambda = 1e-3 with 20 FGP iterations per epoch,
# noise-free data of a kappa-scaled ellipsoid phantom, 10 epochs. The FP64
# oracle finishes it in a minute or two; its image after every epoch is kept at
# n_samples seeded voxels (sample_indices) for the bench's comparison.
PRECISION_REDUCED = dict(
    geometry=dict(kind="cone3d", nx=64, ny=64, nz=64, dx=4.0, dy=4.0, dz=4.0, n_views=90,
                  nu=64, nv=64, du=6.4, dv=6.4, dso=500.0, dsd=1000.0),
    M=16, N=16, tv_lambda=1e-3, tv_iters=20, epochs=10, seed=1, rho=0.25, power_iters=30,
    phantom_seed=0, n_ellipsoids=10, kappa=0.01, n_samples=512, sample_seed=11,
)


def precision_reduced_phantom() -> np.ndarray:
    w = PRECISION_REDUCED
    g = w["geometry"]
    return ellipsoid_phantom(g["nx"], g["ny"], g["nz"], w["n_ellipsoids"], w["phantom_seed"]) * w["kappa"]


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct voxel indices of [0, n), sorted."""
    return np.sort(np.random.default_rng(seed).choice(n, size=k, replace=False))
