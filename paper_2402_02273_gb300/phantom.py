"""Seeded synthetic inputs: a nested-ellipsoid head phantom and Gaussian seeds.

The paper builds its diffusion field from 29 MRI bitmaps of one author's head
(Sec. 3.1), thresholded into air / white matter / gray matter / skull, and sets
D to D_w = 0.13 or D_g = 0.013 mm^2/day in tissue and 0 elsewhere (Sec. 2,
Table 1).  Those scans are not available, so this module stands in for them
with a deterministic phantom of the same structure:

* labels 0 = background (air), 1 = CSF / skull shell and ventricle,
  2 = gray matter, 3 = white matter, on an Nz x Ny x Nx grid (x fastest);
* D per label (0, 0, D_g, D_w), optionally multiplied per tissue voxel by
  (1 + noise * U[-1, 1]) and always rounded to the nearest FP32 value, so the
  same D is exact in FP64 and FP32 storage;
* an initial density u0 = peak * exp(-r^2 / (2 sigma^2)) (sigma in voxels) or
  the maximum of several such blobs.

Random numbers come from a counter-based SplitMix64 stream written out below,
so the inputs are identical on every machine and numpy version.  This module
holds no arithmetic of the integrator: both the CUDA path and the CPU oracle
receive its arrays as plain inputs.
"""
from __future__ import annotations

import numpy as np

# Paper's Table 1 values (mm^2/day, 1/day).
D_WHITE = 0.13
D_GRAY = 0.013
RHO = 0.025

LABEL_BACKGROUND, LABEL_CSF, LABEL_GRAY, LABEL_WHITE = 0, 1, 2, 3

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea & Flood 2014), elementwise on uint64."""
    with np.errstate(over="ignore"):
        z = x.astype(np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from counter-based SplitMix64 (seed, stream, k)."""
    with np.errstate(over="ignore"):
        key = _splitmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        key = _splitmix64(np.array([key ^ np.uint64(stream & 0xFFFFFFFF)], dtype=np.uint64))[0]
        ctr = np.arange(n, dtype=np.uint64) * _GOLDEN + key
        bits = _splitmix64(ctr)
    return (bits >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _axes(shape):
    """Voxel-centre coordinates z, y, x as broadcastable (nz,1,1), (1,ny,1), (1,1,nx) arrays."""
    nz, ny, nx = shape
    return (np.arange(nz, dtype=np.float64).reshape(nz, 1, 1),
            np.arange(ny, dtype=np.float64).reshape(1, ny, 1),
            np.arange(nx, dtype=np.float64).reshape(1, 1, nx))


def _ellipsoid(shape, centre, radii):
    z, y, x = _axes(shape)
    q = ((x - centre[0]) / radii[0]) ** 2 + ((y - centre[1]) / radii[1]) ** 2 \
        + ((z - centre[2]) / radii[2]) ** 2
    return q <= 1.0


def head_labels(shape, seed: int = 0) -> np.ndarray:
    """Label map (uint8, shape (Nz, Ny, Nx)) of a jittered nested-ellipsoid head.

    Radii are fractions of the grid extent per axis (x, y, z): head
    (0.46, 0.42, 0.44), brain (0.40, 0.36, 0.38), white core (0.28, 0.24, 0.26),
    ventricle (0.05, 0.09, 0.05) displaced by +0.06 Ny in y; every radius gets a
    seeded +-3 % jitter.
    """
    nz, ny, nx = shape
    ext = np.array([nx, ny, nz], dtype=np.float64)
    c = (ext - 1.0) / 2.0
    fr = {
        "head": (0.46, 0.42, 0.44),
        "brain": (0.40, 0.36, 0.38),
        "white": (0.28, 0.24, 0.26),
        "vent": (0.05, 0.09, 0.05),
    }
    jit = 1.0 + 0.03 * (2.0 * uniform(seed, 1, 12) - 1.0)
    r = {}
    for i, key in enumerate(("head", "brain", "white", "vent")):
        r[key] = np.array(fr[key]) * ext * jit[3 * i:3 * i + 3]
    lab = np.zeros(shape, dtype=np.uint8)
    lab[_ellipsoid(shape, c, r["head"])] = LABEL_CSF
    lab[_ellipsoid(shape, c, r["brain"])] = LABEL_GRAY
    lab[_ellipsoid(shape, c, r["white"])] = LABEL_WHITE
    vc = c + np.array([0.0, 0.06 * ny, 0.0])
    lab[_ellipsoid(shape, vc, r["vent"])] = LABEL_CSF
    return lab


def diffusion_field(labels: np.ndarray, seed: int = 0, d_white: float = D_WHITE,
                    d_gray: float = D_GRAY, noise: float = 0.0,
                    scale: float = 1.0) -> np.ndarray:
    """Per-voxel D (float64, FP32-exact values) from a label map.

    Tissue voxels get D_w or D_g times `scale` times (1 + noise * U[-1, 1]);
    background and CSF get 0 (the paper's "D_w or D_g or 0", Table 1).
    """
    table = np.array([0.0, 0.0, d_gray, d_white], dtype=np.float64) * scale
    D = table[labels]
    if noise:
        u = uniform(seed, 2, labels.size).reshape(labels.shape)
        tissue = labels >= LABEL_GRAY
        D = np.where(tissue, D * (1.0 + noise * (2.0 * u - 1.0)), D)
    return D.astype(np.float32).astype(np.float64)


def gaussian_blob(shape, centre, peak: float = 0.8, sigma: float = 2.0) -> np.ndarray:
    """peak * exp(-|x - centre|^2 / (2 sigma^2)) on voxel centres (float64)."""
    z, y, x = _axes(shape)
    r2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    return peak * np.exp(-r2 / (2.0 * sigma * sigma))


def seed_centre(shape) -> tuple:
    """Default seed site: grid centre shifted by +0.15 Nx in x (inside the white core)."""
    nz, ny, nx = shape
    return ((nx - 1) / 2.0 + 0.15 * nx, (ny - 1) / 2.0, (nz - 1) / 2.0)


def random_white_sites(labels: np.ndarray, seed: int, count: int) -> list:
    """`count` distinct white-matter voxel centres (x, y, z) picked by the seeded stream."""
    flat = np.flatnonzero(labels.reshape(-1) == LABEL_WHITE)
    if flat.size == 0:
        raise ValueError("phantom has no white matter")
    picks = (uniform(seed, 3, count) * flat.size).astype(np.int64)
    nz, ny, nx = labels.shape
    out = []
    for p in flat[picks]:
        out.append((float(p % nx), float((p // nx) % ny), float(p // (nx * ny))))
    return out


def case(n, seed: int = 0, noise: float = 0.0, d_white: float = D_WHITE,
         d_gray: float = D_GRAY, peak: float = 0.8, sigma: float = 2.0):
    """(D, u0) for an n^3 (or (nz, ny, nx)) head phantom with one centred-off seed."""
    shape = (n, n, n) if np.isscalar(n) else tuple(n)
    lab = head_labels(shape, seed)
    D = diffusion_field(lab, seed, d_white=d_white, d_gray=d_gray, noise=noise)
    u0 = gaussian_blob(shape, seed_centre(shape), peak=peak, sigma=sigma)
    return D, u0


def batch_case(index: int, base_seed: int = 1000):
    """One instance of the many-patient workload: n in {96..160}, rho, D scale, 1-3 blobs."""
    seed = base_seed + index
    r = uniform(seed, 4, 4)
    n = (96, 112, 128, 144, 160)[int(r[0] * 5)]
    rho = 0.01 + 0.04 * r[1]
    dscale = 0.5 + 1.5 * r[2]
    nblobs = 1 + int(r[3] * 3)
    shape = (n, n, n)
    lab = head_labels(shape, seed)
    D = diffusion_field(lab, seed, noise=0.1, scale=dscale)
    u0 = np.zeros(shape)
    for c in random_white_sites(lab, seed, nblobs):
        u0 = np.maximum(u0, gaussian_blob(shape, c))
    return {"n": n, "rho": rho, "dscale": dscale, "D": D, "u0": u0, "seed": seed}
