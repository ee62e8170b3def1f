"""Seeded synthetic workloads for the three-grid IOFD Helmholtz solver.

This module is shared by the CPU oracle (``oracle/``) and the GPU library
(``paper_2608_22946_gb300``).  It holds only problem *inputs*: grid sizes,
velocity models, source and receiver positions.  It contains none of the
method's arithmetic (no stencil, no PML profile, no IOFD coefficient, no
Krylov step), so that the oracle and the CUDA path stay independent.

Conventions (paper Sec. 5: a mesh is named by its fine-grid interval count
n per direction, and every one of its (n+1)^3 nodes is an unknown):

* ``n`` intervals per direction including ``n_pml`` PML layers on each side;
  nodes ``i = 0..n``; physical box ``[0,1]^3`` spans ``n - 2 n_pml`` intervals,
  so ``h = 1/(n - 2 n_pml)``.
* Node ``i`` sits at normalised coordinate ``xbar = (i - n_pml)/(n - 2 n_pml)``.
* Arrays are indexed ``[iz, iy, ix]`` (x fastest in memory).
* ``omega = 2 pi c_min / (ppw h)`` puts ``ppw`` fine points in the shortest
  wavelength (Sec. 6.1, Sec. 4.1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20261202


@dataclasses.dataclass
class Workload:
    name: str
    n: int                      # intervals per direction incl. PML
    n_pml: int                  # PML layers per side on the fine grid
    h: float
    omega: float
    c: np.ndarray               # (n+1)^3 float64 velocity on all fine nodes
    sources: list               # list of (ix, iy, iz, amp complex)
    receivers: np.ndarray | None = None   # (nrec, 3) int node indices (ix, iy, iz)
    seed: int = 0
    gamma_max: float = 1.119058  # Table 4
    c_true: np.ndarray | None = None      # for the inversion workload

    @property
    def nodes(self) -> int:
        return self.n + 1

    @property
    def N(self) -> int:
        return (self.n + 1) ** 3


def grid_params(n: int, n_pml: int, c_min: float, ppw: float = 6.0):
    h = 1.0 / (n - 2 * n_pml)
    omega = 2.0 * math.pi * c_min / (ppw * h)
    return h, omega


def xbar(n: int, n_pml: int) -> np.ndarray:
    """Normalised coordinate of each node index 0..n."""
    return (np.arange(n + 1, dtype=np.float64) - n_pml) / (n - 2 * n_pml)


def _mesh(n, n_pml):
    xb = xbar(n, n_pml)
    Z, Y, X = np.meshgrid(xb, xb, xb, indexing="ij")
    return X, Y, Z


def homogeneous(n: int = 48, n_pml: int = 8, c0: float = 1.0, ppw: float = 6.0,
                src=None) -> Workload:
    """Constant wave speed with one unit point source at the centre node."""
    c = np.full((n + 1,) * 3, c0, dtype=np.float64)
    h, omega = grid_params(n, n_pml, c0, ppw)
    if src is None:
        src = [(n // 2, n // 2, n // 2, 1.0 + 0.0j)]
    return Workload("homogeneous", n, n_pml, h, omega, c, src, seed=0)


def gaussian_lens(n: int = 288, n_pml: int = 16, ppw: float = 6.0) -> Workload:
    """Background 1.0, Gaussian lens of peak 1.5 and sigma 0.15 of the side."""
    X, Y, Z = _mesh(n, n_pml)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    c = 1.0 + 0.5 * np.exp(-r2 / (2.0 * 0.15 ** 2))
    h, omega = grid_params(n, n_pml, 1.0, ppw)
    src = [(n // 2, n // 2, n // 2, 1.0 + 0.0j)]
    return Workload("gaussian_lens", n, n_pml, h, omega, c, src, seed=0)


def layered_inclusion(n: int = 224, n_pml: int = 16, nsrc: int = 16,
                      ppw: float = 6.0, seed: int = SEED_BASE + 3) -> Workload:
    """Five horizontal layers with velocities U[1.5, 4.5] and one spherical
    inclusion 10x faster than its host layer; sources on a random z plane."""
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.uniform(0.1, 0.9, size=4))
    vel = rng.uniform(1.5, 4.5, size=5)
    X, Y, Z = _mesh(n, n_pml)
    layer = np.searchsorted(depths, Z)
    c = vel[layer]
    centre = rng.uniform(0.2, 0.8, size=3)
    host = vel[np.searchsorted(depths, centre[2])]
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    c = np.where(r <= 0.08, 10.0 * host, c)
    cmin = float(c.min())
    h, omega = grid_params(n, n_pml, cmin, ppw)
    lo, hi = n_pml + 2, n - n_pml - 2
    zs = int(rng.integers(lo, hi + 1))
    xs = rng.integers(lo, hi + 1, size=nsrc)
    ys = rng.integers(lo, hi + 1, size=nsrc)
    src = [(int(xs[s]), int(ys[s]), zs, 1.0 + 0.0j) for s in range(nsrc)]
    return Workload("layered_inclusion", n, n_pml, h, omega, c, src, seed=seed)


def _smooth_noise_fft(shape, corr_nodes, rng):
    """White noise filtered by a Gaussian kernel of std ``corr_nodes`` nodes."""
    w = rng.standard_normal(shape)
    F = np.fft.rfftn(w)
    k = [np.fft.fftfreq(s) for s in shape[:-1]] + [np.fft.rfftfreq(shape[-1])]
    K = np.meshgrid(*k, indexing="ij")
    k2 = sum(kk ** 2 for kk in K)
    F *= np.exp(-2.0 * (math.pi ** 2) * (corr_nodes ** 2) * k2)
    return np.fft.irfftn(F, s=shape, axes=tuple(range(len(shape))))


def random_field(n: int = 152, n_pml: int = 12, nsrc: int = 8, nrec_side: int = 64,
                 ppw: float = 6.0, seed: int = SEED_BASE + 4,
                 blob_amp: float = 0.05) -> Workload:
    """Gaussian random field (correlation 10h) mapped to [1.5, 3.0], sources on a
    plane near the top and a nrec_side^2 receiver plane near the bottom.
    ``c_true`` carries the perturbed model m_true = m0 (1 + 0.05 blob)."""
    rng = np.random.default_rng(seed)
    g = _smooth_noise_fft((n + 1,) * 3, 10.0, rng)
    g = (g - g.min()) / (g.max() - g.min())
    c = 1.5 + 1.5 * g
    h, omega = grid_params(n, n_pml, float(c.min()), ppw)
    X, Y, Z = _mesh(n, n_pml)
    blob = np.exp(-((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) / (2 * 0.12 ** 2))
    m0 = 1.0 / c ** 2
    m_true = m0 * (1.0 + blob_amp * blob)
    c_true = 1.0 / np.sqrt(m_true)
    zs = n_pml + 4
    lo, hi = n_pml + 4, n - n_pml - 4
    xs = np.linspace(lo, hi, nsrc // 2 if nsrc > 1 else 1).round().astype(int)
    src = []
    for s in range(nsrc):
        ix = int(xs[s % len(xs)])
        iy = int(lo + (hi - lo) * (0.3 if s < len(xs) else 0.7))
        src.append((ix, iy, zs, 1.0 + 0.0j))
    zr = n - n_pml - 4
    phys = n - 2 * n_pml
    step = max(1, phys // nrec_side)
    r0 = n_pml + (phys - step * (nrec_side - 1)) // 2
    rx = r0 + step * np.arange(nrec_side)
    RY, RX = np.meshgrid(rx, rx, indexing="ij")
    rec = np.stack([RX.ravel(), RY.ravel(), np.full(RX.size, zr)], axis=1).astype(np.int64)
    return Workload("random_field", n, n_pml, h, omega, c, src, receivers=rec,
                    seed=seed, c_true=c_true)


def geophysical(n: int = 960, n_pml: int = 24, nsrc: int = 4, ppw: float = 6.0,
                seed: int = SEED_BASE + 5, dtype=np.float32) -> Workload:
    """Depth gradient 1.5 -> 4.5, a salt-like body at 4.5 (union of three
    random ellipsoids), +-3% small-scale perturbations (correlation ~3h),
    clipped to [1.5, 4.5].  Built plane by plane to bound host memory."""
    rng = np.random.default_rng(seed)
    N1 = n + 1
    xb = xbar(n, n_pml)
    ell = [(rng.uniform(0.3, 0.7, 3), rng.uniform(0.08, 0.2, 3)) for _ in range(3)]
    coarse_n = N1 // 3 + 2
    coarse = rng.uniform(-1.0, 1.0, size=(coarse_n,) * 3)
    t = np.arange(N1) / 3.0
    i0 = np.floor(t).astype(int)
    fr = t - i0
    c = np.empty((N1,) * 3, dtype=dtype)
    Y, X = np.meshgrid(xb, xb, indexing="ij")
    # trilinear upsampling of the coarse noise, one z plane at a time
    cy0 = coarse[:, i0, :] * (1 - fr)[None, :, None] + coarse[:, i0 + 1, :] * fr[None, :, None]
    cyx = cy0[:, :, i0] * (1 - fr)[None, None, :] + cy0[:, :, i0 + 1] * fr[None, None, :]
    for iz in range(N1):
        zb = xb[iz]
        plane = 1.5 + 3.0 * np.clip(zb, 0.0, 1.0) + np.zeros_like(X)
        inside = np.zeros_like(X, dtype=bool)
        for (cen, rad) in ell:
            q = ((X - cen[0]) / rad[0]) ** 2 + ((Y - cen[1]) / rad[1]) ** 2 + ((zb - cen[2]) / rad[2]) ** 2
            inside |= q <= 1.0
        plane = np.where(inside, 4.5, plane)
        noise = cyx[i0[iz]] * (1 - fr[iz]) + cyx[i0[iz] + 1] * fr[iz]
        plane = plane * (1.0 + 0.03 * noise)
        c[iz] = np.clip(plane, 1.5, 4.5)
    h, omega = grid_params(n, n_pml, 1.5, ppw)
    lo, hi = n_pml + 8, n - n_pml - 8
    src = [(int(lo + (hi - lo) * f), n // 2, n_pml + 8, 1.0 + 0.0j)
           for f in np.linspace(0.2, 0.8, nsrc)]
    return Workload("geophysical", n, n_pml, h, omega, c, src, seed=seed)


PAPER_MEDIA = ("homogeneous", "lens", "wedge", "barrier")


def paper_medium(kind: str, n: int = 512, n_pml: int = 8, ppw: float = 6.0) -> Workload:
    """The benchmark media of the paper's performance study (Sec. 6, "Benchmark
    Media"; Table 5 uses n = 512, n_pml = 8, ppw_min = 6): unit speed; the
    converging lens c = 4/3 (1 - exp(-32 |xbar - 1/2|^2) / 2); the three-layer
    wedge whose interfaces are the planes zbar = 0.4 + 0.1 ybar and
    zbar = 0.8 - 0.2 ybar (speeds 2, 1.5, 3 from the bottom); the barrier of
    speed 1e10 on [0,1] x [0.25,0.3] x [0,0.75] in unit speed.  Coordinates are
    normalised to the physical box; omega puts ppw points in the shortest
    wavelength; one unit point source at the centre node (reading of "a grid
    point near the center")."""
    X, Y, Z = _mesh(n, n_pml)
    if kind == "homogeneous":
        c = np.ones_like(X)
        c_min = 1.0
    elif kind == "lens":
        r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
        c = (4.0 / 3.0) * (1.0 - 0.5 * np.exp(-32.0 * r2))
        c_min = 2.0 / 3.0
    elif kind == "wedge":
        c = np.where(Z <= 0.4 + 0.1 * Y, 2.0, np.where(Z <= 0.8 - 0.2 * Y, 1.5, 3.0))
        c_min = 1.5
    elif kind == "barrier":
        inside = (X >= 0.0) & (X <= 1.0) & (Y >= 0.25) & (Y <= 0.3) & (Z >= 0.0) & (Z <= 0.75)
        c = np.where(inside, 1e10, 1.0)
        c_min = 1.0
    else:
        raise ValueError(f"unknown medium {kind!r}")
    h, omega = grid_params(n, n_pml, c_min, ppw)
    src = [(n // 2, n // 2, n // 2, 1.0 + 0.0j)]
    return Workload(f"paper_{kind}", n, n_pml, h, omega, np.ascontiguousarray(c, dtype=np.float64), src, seed=0)


def scaled(kind: str, n: int, n_pml: int, **kw) -> Workload:
    """Same medium recipe at another size (tests use small versions)."""
    f = {"homogeneous": homogeneous, "gaussian_lens": gaussian_lens,
         "layered_inclusion": layered_inclusion, "random_field": random_field,
         "geophysical": geophysical}[kind]
    return f(n=n, n_pml=n_pml, **kw)


# The full-size workloads, named by medium, grid intervals and source count.
WORKLOADS = {
    "homogeneous_48": homogeneous,
    "gaussian_lens_288": gaussian_lens,
    "layered_inclusion_224x16": layered_inclusion,
    "random_field_152x8": random_field,
    "geophysical_960x4": geophysical,
}


def by_name(name: str) -> Workload:
    """One of the full-size workloads at its default size and seed."""
    return WORKLOADS[name]()


def random_complex(shape, seed, dtype=np.complex128):
    """Seeded complex Gaussian test vector."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return v.astype(dtype)
