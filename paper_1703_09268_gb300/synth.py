"""Seeded synthetic inputs for the Helmholtz misfit/gradient workloads.

This module only builds inputs: velocity models, acquisition geometry
(source and receiver node indices) and observed data containers.  It holds
none of the method's arithmetic (no damping layer, no stencil, no solve), so
both the CUDA path and the CPU checker may consume what it produces.

Workload shapes follow the paper's regimes (Sec. 5: 2D FWI on a 10 m grid,
3D Overthrust-like models at 25-50 m and a few Hz, 5-15 points per
wavelength).  The paper's own velocity models (BG Compass, SEG/EAGE
Overthrust) are not used; every model here is a seeded synthetic stand-in.

Conventions shared with the C ABI:
  * a physical model is a real array of shape (nz, ny, nx), x fastest;
    2D problems use ny == 1;
  * node indices are physical-grid linear indices ix + nx*(iy + ny*iz);
  * m = 1/v**2 (s^2/m^2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


@dataclass
class Workload:
    """One misfit+gradient problem: geometry, models, acquisition, frequencies."""
    name: str
    dim: int
    n: tuple            # (nx, ny, nz) physical nodes
    h: float            # grid spacing [m]
    npml: tuple         # (px, py, pz) damping-layer cells per side
    v_ref: float        # reference velocity for the damping strength [m/s]
    freqs_hz: np.ndarray
    m_true: np.ndarray  # (nz, ny, nx) float64, 1/v^2
    m0: np.ndarray      # (nz, ny, nx) float64, model at which f, g are evaluated
    src_idx: np.ndarray  # (n_srcloc,) int32 physical linear indices
    Q: np.ndarray       # (n_srcloc, nsrc) complex128 source weights
    rec_idx: np.ndarray  # (nrec,) int32 physical linear indices
    wavelet: Optional[np.ndarray] = None  # (nfreq,) complex128 or None (= 1)
    meta: dict = field(default_factory=dict)

    @property
    def nsrc(self) -> int:
        return int(self.Q.shape[1])

    @property
    def nrec(self) -> int:
        return int(self.rec_idx.shape[0])

    @property
    def nfreq(self) -> int:
        return int(len(self.freqs_hz))

    @property
    def n_phys(self) -> int:
        return int(self.n[0] * self.n[1] * self.n[2])


def lin_index(n, ix, iy, iz):
    """Physical linear node index, x fastest."""
    nx, ny, _ = n
    return np.asarray(ix) + nx * (np.asarray(iy) + ny * np.asarray(iz))


def point_sources(n, nodes):
    """One unit point source per listed node: Q = identity over the nodes."""
    idx = np.array([lin_index(n, *p) for p in nodes], dtype=np.int32)
    Q = np.eye(len(nodes), dtype=np.complex128)
    return idx, Q


def surface_receivers(n, iz):
    """Receivers at every node of the horizontal plane iz."""
    nx, ny, _ = n
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    return lin_index(n, ix.ravel(), iy.ravel(), np.full(ix.size, iz)).astype(np.int32)


def _gaussian_smooth(a, sigma):
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(a, sigma=sigma, mode="nearest")


def layered_velocity(rng, n, nlayers=8, vmin=1500.0, vmax=4500.0, smooth=2.0):
    """Horizontal layers with velocity increasing with depth, Gaussian-smoothed.

    Interface depths are sorted uniform draws over the depth axis; layer
    velocities are sorted uniform draws in [vmin, vmax]."""
    nx, ny, nz = n
    depths = np.sort(rng.uniform(0, nz, size=nlayers - 1))
    vel = np.sort(rng.uniform(vmin, vmax, size=nlayers))
    z = np.arange(nz) + 0.5
    layer = np.searchsorted(depths, z)
    v = np.broadcast_to(vel[layer][:, None, None], (nz, ny, nx)).copy()
    if smooth > 0:
        v = _gaussian_smooth(v, smooth) if ny > 1 else _gaussian_smooth(v[:, 0, :], smooth)[:, None, :]
    return v


def add_gaussian_inclusions(rng, v, count, amp=400.0, rmin=3.0, rmax=10.0):
    """Add `count` Gaussian blobs of amplitude +-amp with radii in [rmin, rmax] cells."""
    nz, ny, nx = v.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = v.copy()
    for _ in range(count):
        c = rng.uniform([0, 0, 0], [nz, ny, nx])
        r = rng.uniform(rmin, rmax)
        s = rng.choice([-1.0, 1.0])
        d2 = (zz - c[0]) ** 2 + (yy - c[1]) ** 2 + (xx - c[2]) ** 2
        out += s * amp * np.exp(-d2 / (2 * r * r))
    return out


def smooth_random_velocity(rng, n, sigma=8.0, vmin=1500.0, vmax=4500.0):
    """White noise smoothed by a Gaussian of `sigma` cells, rescaled to [vmin, vmax]."""
    nx, ny, nz = n
    w = rng.standard_normal((nz, ny, nx))
    s = _gaussian_smooth(w, sigma)
    s = (s - s.min()) / max(s.max() - s.min(), 1e-30)
    return vmin + (vmax - vmin) * s


def slowness2(v):
    return 1.0 / (np.asarray(v, dtype=np.float64) ** 2)


# --------------------------------------------------------------------------
# The workloads (sizes in nodes; h in metres; frequencies in Hz)
# --------------------------------------------------------------------------

def workload_2d(seed: int = 1, n: int = 101, h: float = 10.0, npml: int = 20) -> Workload:
    """2D 101x101, h=10 m, 20-cell layer, Gaussian +300 m/s anomaly (sigma 100 m)
    on 2000 m/s, 5 Hz, one unit point source at (500 m, 20 m), 101 receivers
    along z = 20 m.  f and g are evaluated at the 2000 m/s background."""
    nx = nz = n
    x = np.arange(nx) * h
    z = np.arange(nz) * h
    cx = cz = 0.5 * (n - 1) * h
    zz, xx = np.meshgrid(z, x, indexing="ij")
    v = 2000.0 + 300.0 * np.exp(-((xx - cx) ** 2 + (zz - cz) ** 2) / (2 * 100.0 ** 2))
    dims = (nx, 1, nz)
    iz_src = int(round(20.0 / h))
    src_idx, Q = point_sources(dims, [((n - 1) // 2, 0, iz_src)])
    rec_idx = surface_receivers(dims, iz_src)
    return Workload(
        name=f"2d-{n}x{n}-h{h:g}-pml{npml}-5Hz", dim=2, n=dims, h=h, npml=(npml, 0, npml),
        v_ref=2000.0, freqs_hz=np.array([5.0]), m_true=slowness2(v)[:, None, :],
        m0=np.full((nz, 1, nx), 1.0 / 2000.0 ** 2), src_idx=src_idx, Q=Q, rec_idx=rec_idx,
        meta={"seed": seed})


def workload_25d(seed: int = 6, nx: int = 401, nz: int = 201, h: float = 10.0, npml: int = 20,
                 nsrc: int = 32, freq: float = 8.0) -> Workload:
    """2.5D (a y-invariant model on the x-z plane): 401 x 201, h = 10 m, 20-cell
    layers, 8 seeded layers (1500-4500 m/s, smoothed sigma = 2 cells) plus one
    Gaussian inclusion as the true model, evaluated at the sigma = 6 smoothed
    model; nsrc sources spread along z = 2 cells, receivers at every x of that
    row (in the sources' plane), one frequency."""
    rng = np.random.default_rng(seed)
    dims = (nx, 1, nz)
    v = layered_velocity(rng, dims, nlayers=8, smooth=2.0)
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    vt = v + 300.0 * np.exp(-((xx - nx / 2.0) ** 2 + (zz - nz / 2.0) ** 2) / (2 * (nz / 8.0) ** 2))[:, None, :]
    v0 = _gaussian_smooth(v[:, 0, :], 6.0)[:, None, :]
    xs = np.linspace(nx / (2 * nsrc), nx - nx / (2 * nsrc), nsrc).round().astype(int)
    src_idx, Q = point_sources(dims, [(int(x), 0, 2) for x in xs])
    rec_idx = surface_receivers(dims, 2)
    return Workload(
        name=f"2.5d-{nx}x{nz}-h{h:g}-pml{npml}-{freq:g}Hz-{nsrc}src", dim=2, n=dims, h=h, npml=(npml, 0, npml),
        v_ref=3000.0, freqs_hz=np.array([freq]), m_true=slowness2(vt), m0=slowness2(v0), src_idx=src_idx, Q=Q,
        rec_idx=rec_idx, meta={"seed": seed, "vmin": float(v0.min())})


def workload_3d_layered(seed: int = 2, n: int = 64, h: float = 25.0, npml: int = 10,
                        nsrc_side: int = 4, freq: float = 4.0) -> Workload:
    """3D n^3 layered model (8 seeded layers, 1500-4500 m/s, smoothed sigma=2 cells)
    plus one Gaussian inclusion as the true model; f, g at the sigma=6 smoothed
    model; nsrc_side^2 point sources at z = 2 cells; receivers at every z = 0 node."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    v = layered_velocity(rng, dims, nlayers=8, smooth=2.0)
    c = n / 2.0
    zz, yy, xx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    v_true = v + 300.0 * np.exp(-((zz - c) ** 2 + (yy - c) ** 2 + (xx - c) ** 2) / (2 * (n / 8.0) ** 2))
    v0 = _gaussian_smooth(v, 6.0)
    pos = [int((i + 0.5) * n / nsrc_side) for i in range(nsrc_side)]
    nodes = [(ix, iy, 2) for iy in pos for ix in pos]
    src_idx, Q = point_sources(dims, nodes)
    rec_idx = surface_receivers(dims, 0)
    return Workload(
        name=f"3d-layered-{n}^3-h{h:g}-pml{npml}-{freq:g}Hz-{len(nodes)}src", dim=3, n=dims, h=h,
        npml=(npml,) * 3, v_ref=4500.0, freqs_hz=np.array([freq]), m_true=slowness2(v_true),
        m0=slowness2(v0), src_idx=src_idx, Q=Q, rec_idx=rec_idx, meta={"seed": seed})


def workload_3d_inclusions(seed: int = 4, n: int = 256, h: float = 20.0, npml: int = 12,
                           nsrc: int = 32, freq: float = 6.0, ninc: int = 20) -> Workload:
    """Layered model plus `ninc` Gaussian inclusions of +-400 m/s (radius 3-10 cells)."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    v = layered_velocity(rng, dims, nlayers=8, smooth=2.0)
    v_true = add_gaussian_inclusions(rng, v, ninc)
    v_true = np.clip(v_true, 1200.0, 5000.0)
    v0 = _gaussian_smooth(v, 6.0)
    ny_s = 4
    nx_s = nsrc // ny_s
    nodes = [(int((i + 0.5) * n / nx_s), int((j + 0.5) * n / ny_s), 2)
             for j in range(ny_s) for i in range(nx_s)]
    src_idx, Q = point_sources(dims, nodes)
    rec_idx = surface_receivers(dims, 0)
    return Workload(
        name=f"3d-inclusions-{n}^3-h{h:g}-pml{npml}-{freq:g}Hz-{nsrc}src", dim=3, n=dims, h=h,
        npml=(npml,) * 3, v_ref=4500.0, freqs_hz=np.array([freq]), m_true=slowness2(v_true),
        m0=slowness2(v0), src_idx=src_idx, Q=Q, rec_idx=rec_idx, meta={"seed": seed})


def workload_3d_multifreq(seed: int = 5, n: int = 192, h: float = 25.0, npml: int = 10,
                          nsx: int = 8, nsy: int = 16, nfreq: int = 8,
                          fmin: float = 2.0, fmax: float = 8.0) -> Workload:
    """Layered + inclusions true model, smoothed starting model, nsx*nsy sources
    at z = 2 cells, receivers at every surface node, nfreq frequencies."""
    rng = np.random.default_rng(seed)
    dims = (n, n, n)
    v = layered_velocity(rng, dims, nlayers=8, smooth=2.0)
    v_true = np.clip(add_gaussian_inclusions(rng, v, 20), 1200.0, 5000.0)
    v0 = _gaussian_smooth(v, 6.0)
    nodes = [(int((i + 0.5) * n / nsx), int((j + 0.5) * n / nsy), 2)
             for j in range(nsy) for i in range(nsx)]
    src_idx, Q = point_sources(dims, nodes)
    rec_idx = surface_receivers(dims, 0)
    return Workload(
        name=f"3d-multifreq-{n}^3-h{h:g}-{nsx*nsy}src-{nfreq}f", dim=3, n=dims, h=h,
        npml=(npml,) * 3, v_ref=4500.0, freqs_hz=np.linspace(fmin, fmax, nfreq),
        m_true=slowness2(v_true), m0=slowness2(v0), src_idx=src_idx, Q=Q, rec_idx=rec_idx,
        meta={"seed": seed})


def centre_source(wl: Workload) -> int:
    """Index of the source column whose node lies nearest the centre of the surface."""
    nx, ny, _ = wl.n
    loc = wl.src_idx[np.argmax(np.abs(wl.Q), axis=0)]
    ix, iy = loc % nx, (loc // nx) % ny
    return int(np.argmin((ix - (nx - 1) / 2.0) ** 2 + (iy - (ny - 1) / 2.0) ** 2))


def source_subset(wl: Workload, cols) -> tuple:
    """(src_idx, Q) of the listed source columns only (point sources)."""
    cols = list(cols)
    rows = np.nonzero(np.any(wl.Q[:, cols] != 0, axis=1))[0]
    return wl.src_idx[rows].astype(np.int32), np.ascontiguousarray(wl.Q[np.ix_(rows, cols)])


def batch_models(seed: int = 3, sizes=(48, 64, 80, 96, 112, 128, 144, 160), h: float = 25.0,
                 npml: int = 10) -> List[Workload]:
    """Eight models of uneven size, smooth random velocity in [1500, 4500] m/s,
    32 sources (4x8 surface grid at z = 2 cells), 3/4/5 Hz."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        dims = (n, n, n)
        v = smooth_random_velocity(rng, dims, sigma=8.0)
        nodes = [(int((i + 0.5) * n / 8), int((j + 0.5) * n / 4), 2) for j in range(4) for i in range(8)]
        src_idx, Q = point_sources(dims, nodes)
        rec_idx = surface_receivers(dims, 0)
        m = slowness2(v)
        out.append(Workload(
            name=f"batch-{n}^3", dim=3, n=dims, h=h, npml=(npml,) * 3, v_ref=4500.0,
            freqs_hz=np.array([3.0, 4.0, 5.0]), m_true=m, m0=slowness2(_gaussian_smooth(v, 4.0)),
            src_idx=src_idx, Q=Q, rec_idx=rec_idx, meta={"seed": seed}))
    return out


def random_complex(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
