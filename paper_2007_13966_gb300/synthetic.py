"""Seeded synthetic reservoirs: grids, rock fields, wells and the EOS constants.

This module only draws and lays out inputs. It holds none of the method's
arithmetic (no transmissibility, no EOS root, no residual): both the CUDA path
and the CPU oracle consume what it returns.

Stand-ins for the paper's fields (the Case-1 H-shaped zone, the MRST random
field of Case-2 and the SPE10 model of Case-3 are not available):

* ``lognormal``: ln k = ln(k_ref) + sigma * g, where g is i.i.d. N(0, 1) noise
  filtered by a Gaussian kernel (correlation length in cells, reflecting
  boundaries) and renormalised to zero mean and unit variance. Porosity is
  uniform in [0.15, 0.25].
* ``channelised``: per layer, a few sinuous high-permeability channels
  (1000 mD) in a 1 mD matrix, in the SPE10 geometry (Section 4, Case-3).

Physical constants follow Section 4 (phi, mu, R, W, T); the fluid is methane.
Wells: an injector at 10 atm and a producer at 1 atm in opposite corners (2D),
or in opposite corner columns through all layers (3D); the initial pressure is
1 atm, as in the paper's cases.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

ATM = 101325.0           # Pa
MILLIDARCY = 9.869233e-16  # m^2
DAY = 86400.0            # s


@dataclasses.dataclass
class Grid:
    """Cell-centred box grid; cell n = i + nx*(j + ny*k) (x fastest)."""
    nx: int
    ny: int
    nz: int
    hx: float
    hy: float
    hz: float

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def dim(self) -> int:
        return 2 if self.nz == 1 else 3

    @property
    def shape_zyx(self):
        return (self.nz, self.ny, self.nx)


@dataclasses.dataclass
class Fluid:
    """Single-component gas described by the Peng-Robinson EOS (Section 2).

    Units: K, Pa, J/(mol K), kg/mol, Pa s.
    """
    Tc: float = 190.6
    pc: float = 4.599e6
    omega: float = 0.011
    Tb: float = 111.67
    omega_from_Tb: bool = False
    T: float = 298.0
    R: float = 8.3147295
    W: float = 16e-3
    mu: float = 11.067e-3 * 1e-3

    @classmethod
    def paper_methane(cls) -> "Fluid":
        """The constants printed in Section 4 (omega derived from T_b)."""
        return cls(Tc=190.58, pc=4.604e6, omega=float("nan"), Tb=111.67,
                   omega_from_Tb=True)


@dataclasses.dataclass
class Connections:
    """Fixed-pressure connections (wells and Dirichlet faces).

    Each entry joins cell ``cell[q]`` to a fixed pressure ``p[q]`` through a
    geometric transmissibility ``T[q]`` (m^3); entries are sorted by cell.
    """
    cell: np.ndarray  # int32
    p: np.ndarray     # float64, Pa
    T: np.ndarray     # float64, m^3

    def __post_init__(self):
        order = np.argsort(self.cell, kind="stable")
        self.cell = np.ascontiguousarray(self.cell[order], dtype=np.int32)
        self.p = np.ascontiguousarray(self.p[order], dtype=np.float64)
        self.T = np.ascontiguousarray(self.T[order], dtype=np.float64)

    def __len__(self) -> int:
        return int(self.cell.size)


@dataclasses.dataclass
class Reservoir:
    grid: Grid
    fluid: Fluid
    kx: np.ndarray   # [N] m^2
    ky: np.ndarray
    kz: np.ndarray
    phi: np.ndarray  # [N]
    conns: Connections
    p0: float = ATM
    dt: float = 0.1 * DAY
    name: str = ""
    gravity: float = 0.0   # m/s^2 along the z axis, depth increasing with the z index
    upwind: bool = False   # face mobility of the upstream cell instead of the mean
    rate_Q: np.ndarray | None = None   # [N] m^3/s of Darcy inflow through boundary faces per cell
    conservative: bool = False          # accumulation as phi D_t(p/Z) instead of phi c(p) D_t p


def _gauss_kernel(corr: float) -> np.ndarray:
    half = int(math.ceil(3.0 * corr))
    x = np.arange(-half, half + 1, dtype=np.float64)
    w = np.exp(-0.5 * (x / corr) ** 2)
    return w / w.sum()


def _reflect_filter_axis(f: np.ndarray, axis: int, w: np.ndarray) -> np.ndarray:
    half = (w.size - 1) // 2
    n = f.shape[axis]
    pad = [(0, 0)] * f.ndim
    pad[axis] = (half, half)
    g = np.pad(f, pad, mode="symmetric") if half <= n else np.pad(f, pad, mode="reflect")
    out = np.zeros_like(f)
    for t in range(w.size):
        sl = [slice(None)] * f.ndim
        sl[axis] = slice(t, t + n)
        out += w[t] * g[tuple(sl)]
    return out


def correlated_gaussian(shape_zyx, corr_cells: float, seed: int) -> np.ndarray:
    """Zero-mean unit-variance Gaussian field with Gaussian correlation."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(shape_zyx)
    w = _gauss_kernel(corr_cells)
    for ax in range(g.ndim):
        if g.shape[ax] > 1:
            g = _reflect_filter_axis(g, ax, w)
    g -= g.mean()
    s = g.std()
    if s > 0:
        g /= s
    return g


def corner_wells(grid: Grid, k: np.ndarray, p_inj: float = 10 * ATM,
                 p_prod: float = 1 * ATM) -> Connections:
    """Injector in the (0,0) corner column, producer in the opposite one.

    The well index is a half-cell connection through the x face,
    WI = 2 k A_x / h_x (same form as a Dirichlet face).
    """
    cells, ps, Ts = [], [], []
    ax = grid.hy * grid.hz
    for kk in range(grid.nz):
        c_inj = 0 + grid.nx * (0 + grid.ny * kk)
        c_prd = (grid.nx - 1) + grid.nx * ((grid.ny - 1) + grid.ny * kk)
        for c, pw in ((c_inj, p_inj), (c_prd, p_prod)):
            cells.append(c)
            ps.append(pw)
            Ts.append(2.0 * k[c] * ax / grid.hx)
    return Connections(np.array(cells), np.array(ps), np.array(Ts))


def dirichlet_faces(grid: Grid, kx: np.ndarray, ky: np.ndarray, kz: np.ndarray,
                    faces) -> Connections:
    """Dirichlet boundary faces: ``faces`` is a list of (cell, axis, p_D).

    Half-cell transmissibility T_D = 2 k A_f / h (axis 0=x, 1=y, 2=z).
    """
    cells, ps, Ts = [], [], []
    for c, axis, pd in faces:
        if axis == 0:
            T = 2.0 * kx[c] * grid.hy * grid.hz / grid.hx
        elif axis == 1:
            T = 2.0 * ky[c] * grid.hx * grid.hz / grid.hy
        else:
            T = 2.0 * kz[c] * grid.hx * grid.hy / grid.hz
        cells.append(c)
        ps.append(pd)
        Ts.append(T)
    return Connections(np.array(cells, dtype=np.int64), np.array(ps), np.array(Ts))


def lognormal_reservoir(nx, ny, nz, lx, ly, lz, sigma=1.0, corr=8.0,
                        k_ref_md=100.0, seed_k=1, seed_phi=2, name="") -> Reservoir:
    grid = Grid(nx, ny, nz, lx / nx, ly / ny, lz / nz)
    g = correlated_gaussian(grid.shape_zyx, corr, seed_k).reshape(-1)
    k = k_ref_md * MILLIDARCY * np.exp(sigma * g)
    rng = np.random.default_rng(seed_phi)
    phi = rng.uniform(0.15, 0.25, size=grid.n)
    return Reservoir(grid, Fluid(), k.copy(), k.copy(), k.copy(), phi,
                     corner_wells(grid, k), name=name)


def channelised_reservoir(nx=60, ny=220, nz=85, seed_k=5, seed_phi=6,
                          name="channelised 60x220x85") -> Reservoir:
    """SPE10-geometry stand-in: sinuous channels along y in every layer."""
    ft = 0.3048
    grid = Grid(nx, ny, nz, 1200 * ft / nx, 2200 * ft / ny, 170 * ft / nz)
    rng = np.random.default_rng(seed_k)
    kmd = np.full(grid.shape_zyx, 1.0)
    y = np.arange(ny)
    xs = np.arange(nx)
    for kk in range(nz):
        for _ in range(int(rng.integers(3, 7))):
            x0 = rng.uniform(0, nx)
            amp = rng.uniform(5, 15)
            lam = rng.uniform(60, 200)
            psi = rng.uniform(0, 2 * math.pi)
            width = rng.uniform(4, 8)
            xc = x0 + amp * np.sin(2 * math.pi * y / lam + psi)
            inside = np.abs(xs[None, :] - xc[:, None]) <= 0.5 * width
            kmd[kk][inside] = 1000.0
    k = (kmd * MILLIDARCY).reshape(-1)
    rng2 = np.random.default_rng(seed_phi)
    phi = rng2.uniform(0.15, 0.25, size=grid.n)
    return Reservoir(grid, Fluid(), k.copy(), k.copy(), k.copy(), phi,
                     corner_wells(grid, k), name=name)


def config_small_2d() -> Reservoir:
    """2D 64x64 on 100 m x 100 m, thickness 1 m, ln k ~ N(0,1) correlated 8 cells."""
    return lognormal_reservoir(64, 64, 1, 100.0, 100.0, 1.0, sigma=1.0, corr=8.0,
                               seed_k=1, seed_phi=2, name="2d 64x64 lognormal")


def config_3d_1m() -> Reservoir:
    """3D 128x128x64 (1.05M cells) on 100 m x 100 m x 50 m, sigma_lnk = 1.5."""
    return lognormal_reservoir(128, 128, 64, 100.0, 100.0, 50.0, sigma=1.5, corr=8.0,
                               seed_k=3, seed_phi=4, name="3d 128x128x64 lognormal")


def small_3d(nx=24, ny=20, nz=12, sigma=1.5, seed=11) -> Reservoir:
    """Small 3D case (same recipe as the 1M-cell case) for parity tests."""
    return lognormal_reservoir(nx, ny, nz, 100.0 * nx / 128, 100.0 * ny / 128,
                               50.0 * nz / 64, sigma=sigma, corr=4.0,
                               seed_k=seed, seed_phi=seed + 1,
                               name=f"3d {nx}x{ny}x{nz} lognormal")


def random_pressure(res: Reservoir, seed: int, lo=1.0, hi=10.0) -> np.ndarray:
    """A smooth-ish pressure field in [lo, hi] atm for kernel-level tests."""
    g = correlated_gaussian(res.grid.shape_zyx, 3.0, seed).reshape(-1)
    u = 0.5 * (1 + np.tanh(g))
    return (lo + (hi - lo) * u) * ATM


def random_vector(n: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(n)
