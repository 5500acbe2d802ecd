"""Seeded synthetic fluorescence volumes (inputs only; no deconvolution arithmetic).

The paper's Richardson-Lucy example (Section 4, "Richardson-Lucy
deconvolution") runs on a confocal stack of Hoechst-stained nuclei with a
theoretical PSF of the same ZYX size; that data is not available, so these
volumes stand in for it: bright Gaussian blobs ("nuclei") on a flat background,
blurred circularly by a normalised anisotropic Gaussian (the microscope), then
Poisson shot noise.  Arrays are C-order [nz][ny][nx] float32; workload sizes
are quoted X x Y x Z.

This module is shared by the tests, the benchmark and the oracle's callers.
It holds none of the method's arithmetic: the blur is the library routine
``scipy.ndimage.fourier_gaussian`` applied through ``numpy.fft`` (a stand-in
for the optics), not the deconvolution's convolution, and the PSF handed to
the deconvolution is built elsewhere.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20251014

def _is_5smooth(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


#: the twenty 2^a 3^b 5^c lengths in [48, 160]
SMOOTH_48_160 = tuple(n for n in range(48, 161) if _is_5smooth(n))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic deconvolution problem family (sizes are X, Y, Z)."""
    name: str
    xyz: tuple
    n_blobs: int
    blob_sigma: tuple
    background: float
    psf_sigma_xy: float
    psf_sigma_z: float
    n_iter: int
    seed: int

    @property
    def shape(self) -> tuple:
        """numpy shape (nz, ny, nx)"""
        x, y, z = self.xyz
        return (z, y, x)

    @property
    def voxels(self) -> int:
        return int(np.prod(self.xyz))


# Plain single-volume workloads (64x64x32, 256x256x128, 1024x1024x128, 2560x2160x30).
SMALL = Workload("rl_64x64x32", (64, 64, 32), 12, (2.0, 4.0), 10.0, 1.5, 3.0, 20, SEED_BASE + 1)
MEDIUM = Workload("rl_256x256x128", (256, 256, 128), 400, (2.0, 5.0), 10.0, 2.0, 5.0, 100, SEED_BASE + 2)
LARGE = Workload("rl_1024x1024x128", (1024, 1024, 128), 20000, (2.0, 6.0), 20.0, 2.5, 6.0, 50,
                 SEED_BASE + 3)
# The paper's stack shape (ZYX 30 x 2160 x 2560, a PSF of the same size), with the large
# workload's blob density and PSF.
PAPER = Workload("rl_2560x2160x30", (2560, 2160, 30), round(20000 * 2560 * 2160 * 30 / (1024 * 1024 * 128)),
                 (2.0, 6.0), 20.0, 2.5, 6.0, 50, SEED_BASE + 5)
PLAIN = {w.name: w for w in (SMALL, MEDIUM, LARGE, PAPER)}

# Batched: 64 volumes, each axis drawn from SMOOTH_48_160, small-volume blob density.
BATCH_COUNT = 64
BATCH_ITERS = 50
# Differentiable: 16 volumes 128x128x64, data PSF (2, 5), gradient at (2.4, 6.0, 1.0).
GRAD_COUNT = 16
GRAD_XYZ = (128, 128, 64)
GRAD_ITERS = 30
GRAD_CKPT = 6
GRAD_DATA_PSF = (2.0, 5.0)
GRAD_EVAL_PSF = (2.4, 6.0, 1.0)


def render_blobs(shape, n_blobs: int, sigma_range, background: float,
                 rng: np.random.Generator) -> np.ndarray:
    """Ground-truth object: background + isotropic Gaussian blobs.

    Each blob has peak amplitude U[200, 1000], sigma U[lo, hi] voxels and a
    uniform random (sub-voxel) centre; it is rendered inside a box of radius
    ceil(4 sigma) with circular wrap-around.  float64 result.
    """
    nz, ny, nx = shape
    amp = rng.uniform(200.0, 1000.0, n_blobs)
    sig = rng.uniform(sigma_range[0], sigma_range[1], n_blobs)
    cen = rng.uniform(0.0, 1.0, (n_blobs, 3)) * np.array([nz, ny, nx], dtype=np.float64)
    rmax = int(math.ceil(4.0 * sigma_range[1]))
    # render into a padded canvas with plain slicing, then fold the margins back
    pz, py, px = (min(rmax, n) for n in (nz, ny, nx))
    canvas = np.zeros((nz + 2 * pz, ny + 2 * py, nx + 2 * px), np.float64)
    for a, s, (cz, cy, cx) in zip(amp, sig, cen):
        r = int(math.ceil(4.0 * s))
        prof = []
        lo = []
        for c, n, p in ((cz, nz, pz), (cy, ny, py), (cx, nx, px)):
            rr = min(r, p)
            i0 = int(math.floor(c)) - rr
            idx = np.arange(i0, i0 + 2 * rr + 1, dtype=np.float64)
            prof.append(np.exp(-0.5 * ((idx - c) / s) ** 2))
            lo.append(i0 + p)
        gz, gy, gx = prof
        blob = a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        z0, y0, x0 = lo
        canvas[z0:z0 + blob.shape[0], y0:y0 + blob.shape[1], x0:x0 + blob.shape[2]] += blob
    # fold the padding onto the opposite faces (circular wrap)
    for axis, (n, p) in enumerate(((nz, pz), (ny, py), (nx, px))):
        if p == 0:
            continue
        sl = [slice(None)] * 3
        core = canvas
        lo_pad = np.take(core, np.arange(0, p), axis=axis)
        hi_pad = np.take(core, np.arange(n + p, n + 2 * p), axis=axis)
        core = np.take(core, np.arange(p, n + p), axis=axis)
        sl[axis] = slice(n - p, n)
        core[tuple(sl)] += lo_pad
        sl[axis] = slice(0, p)
        core[tuple(sl)] += hi_pad
        canvas = core
    return canvas + background


def microscope_blur(obj: np.ndarray, sigma_xy: float, sigma_z: float) -> np.ndarray:
    """Circular blur by a normalised anisotropic Gaussian (library routine)."""
    from scipy import ndimage
    spec = np.fft.rfftn(obj)
    spec = ndimage.fourier_gaussian(spec, sigma=(sigma_z, sigma_xy, sigma_xy), n=obj.shape[-1])
    return np.fft.irfftn(spec, s=obj.shape, axes=(0, 1, 2))


def make_volume(shape, n_blobs: int, sigma_range, background: float, psf_sigma_xy: float,
                psf_sigma_z: float, seed: int):
    """(image d float32 with Poisson noise, ground truth float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    obj = render_blobs(shape, n_blobs, sigma_range, background, rng)
    blurred = np.maximum(microscope_blur(obj, psf_sigma_xy, psf_sigma_z), 0.0)
    d = rng.poisson(blurred).astype(np.float32)
    return d, obj.astype(np.float32)


def workload_volume(w: Workload):
    """(d, x_true) for a plain workload."""
    return make_volume(w.shape, w.n_blobs, w.blob_sigma, w.background, w.psf_sigma_xy,
                       w.psf_sigma_z, w.seed)


def batch_shapes(count: int = BATCH_COUNT, seed: int = SEED_BASE + 4):
    """Per-volume numpy shapes (nz, ny, nx), each axis drawn from SMOOTH_48_160."""
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = rng.integers(0, len(SMOOTH_48_160), size=(count, 3))
    return [tuple(int(SMOOTH_48_160[i]) for i in row) for row in idx]


def batch_volume(j: int, shape):
    """Volume j of the batched workload: small-volume parameters, density-scaled count."""
    v = int(np.prod(shape))
    n_blobs = max(1, int(round(SMALL.n_blobs * v / SMALL.voxels)))
    return make_volume(shape, n_blobs, SMALL.blob_sigma, SMALL.background, SMALL.psf_sigma_xy,
                       SMALL.psf_sigma_z, SEED_BASE * 100 + j)


def grad_volume(j: int):
    """Volume j of the differentiable workload (128x128x64)."""
    x, y, z = GRAD_XYZ
    return make_volume((z, y, x), 50, (2.0, 5.0), 10.0, GRAD_DATA_PSF[0], GRAD_DATA_PSF[1],
                       (SEED_BASE + 1) * 100 + j)


def random_field(shape, seed: int, lo: float = 0.5, hi: float = 1.5, dtype=np.float32):
    """Uniform positive field for kernel-level tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, shape).astype(dtype)


def random_complex(shape, seed: int, dtype=np.complex64):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
