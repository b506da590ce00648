"""Seeded synthetic inputs for the PFLBM workloads.

This module builds initial fields (phi0, u0, p0) and parameter sets only; it
holds none of the method's arithmetic (no equilibria, collisions or forces).
Both the CUDA path and the CPU oracle take its arrays as inputs.

Geometry follows the paper's setups: the diffuse interface is initialised with
the tanh profile phi = 1/2 +- 1/2 tanh(d / (xi/2)) across the interface
(section "Numerical experiments", initialisation of the PFLBM), heavy phase at
phi = 1.  Cell i sits at coordinate i; walls (halfway bounce-back) sit at -1/2
and n - 1/2.  Arrays are x-fastest: shape (nz, ny, nx); vectors (3, nz, ny, nx).
"""
from dataclasses import dataclass, field, asdict
import math

import numpy as np

PERIODIC, NOSLIP = 0, 1


@dataclass
class Params:
    nx: int
    ny: int
    nz: int
    bc: tuple = (PERIODIC,) * 6          # -x,+x,-y,+y,-z,+z
    rho_h: float = 1.0
    rho_l: float = 1e-3
    nu_h: float = 1.0 / 60.0
    nu_l: float = 1.0 / 60.0
    sigma: float = 1e-4
    mobility: float = 0.02
    xi: float = 5.0
    gravity: tuple = (0.0, 0.0, 0.0)
    collision: int = 0                    # 0 weighted-orthogonal MRT, 1 BGK
    engine: int = 0                       # 0 auto (fused two-array step), 1 in-place AA + phi pass
    h_lattice: int = 15                   # phase-field lattice: 15 (D3Q15), 27 (D3Q27) or 9 (D2Q9 h and g, 2-D)
    solid: object = None                  # optional solid-cell mask (nz, ny, nx), nonzero = solid
    hydrostatic: int = 0                  # 1: with p0 None the library starts from the hydrostatic p*
    p_level: float = 0.0                  # ... with zero pressure at this coordinate along the gravity axis

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def oracle_kwargs(self):
        d = asdict(self)
        return d


def coords(p):
    z, y, x = np.meshgrid(np.arange(p.nz, dtype=np.float64), np.arange(p.ny, dtype=np.float64),
                          np.arange(p.nx, dtype=np.float64), indexing="ij")
    return x, y, z


def tanh_profile(signed_distance, xi):
    """phi across an interface; positive distance -> light phase (phi -> 0)."""
    return 0.5 - 0.5 * np.tanh(signed_distance / (xi / 2.0))


def sphere(p, center, radius, heavy_inside=True):
    x, y, z = coords(p)
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    d = r - radius
    return tanh_profile(d if heavy_inside else -d, p.xi)


def cylinder_z(p, center, radius, heavy_inside=True):
    x, y, _ = coords(p)
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2)
    d = r - radius
    return tanh_profile(d if heavy_inside else -d, p.xi)


def wave(p, depth, amplitude, wavelength):
    """Heavy phase below y = depth + amplitude cos(2 pi x / wavelength)."""
    x, y, _ = coords(p)
    ys = depth + amplitude * np.cos(2.0 * math.pi * x / wavelength)
    return tanh_profile(y - ys, p.xi)


def flat(p, y0):
    _, y, _ = coords(p)
    return tanh_profile(y - y0, p.xi)


def noise(shape, seed, amplitude):
    """Seeded uniform noise in [-amplitude, amplitude] (PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return amplitude * (2.0 * rng.random(shape) - 1.0)


# ------------------------------------------------------------ workloads ----

def static_drop(n=32, R=10.0, xi=5.0, sigma=1e-4, mobility=0.02, nu=1.0 / 60.0, rho_ratio=1000.0,
                u_noise=0.0, seed=1234, collision=0):
    """Static heavy drop of radius R centred in a periodic n^3 box."""
    p = Params(n, n, n, (PERIODIC,) * 6, 1.0, 1.0 / rho_ratio, nu, nu, sigma, mobility, xi,
               (0.0, 0.0, 0.0), collision)
    c = (n - 1) / 2.0
    phi0 = sphere(p, (c, c, c), R, heavy_inside=True)
    u0 = noise((3,) + p.shape, seed, u_noise) if u_noise > 0 else None
    return p, phi0, u0, None


def static_cylinder(n=64, R=16.0, xi=5.0, sigma=1e-4, mobility=0.02, nu=1.0 / 60.0, rho_ratio=1000.0,
                    collision=0):
    """Quasi-2D static heavy column (n x n x 1, periodic); Laplace jump sigma/R."""
    p = Params(n, n, 1, (PERIODIC,) * 6, 1.0, 1.0 / rho_ratio, nu, nu, sigma, mobility, xi,
               (0.0, 0.0, 0.0), collision)
    c = (n - 1) / 2.0
    return p, cylinder_z(p, (c, c), R, heavy_inside=True), None, None


def capillary_wave(L=200, ny=None, a0=None, xi=5.0, M=0.02, sigma=1e-4, nu=0.01, rho_ratio=1000.0,
                   depth=None, collision=0):
    """Standing capillary wave: L x ny x 1, periodic x and z, no-slip walls in y."""
    ny = 2 * L if ny is None else ny
    a0 = 0.01 * L if a0 is None else a0
    depth = (ny - 1) / 2.0 if depth is None else depth
    bc = (PERIODIC, PERIODIC, NOSLIP, NOSLIP, PERIODIC, PERIODIC)
    p = Params(L, ny, 1, bc, 1.0, 1.0 / rho_ratio, nu, nu, sigma, M, xi, (0.0, 0.0, 0.0), collision)
    return p, wave(p, depth, a0, float(L)), None, None


def flat_interface(ny=64, xi=5.0, M=0.02, sigma=1e-4, nu=1.0 / 60.0, rho_ratio=1000.0, y0=None,
                   collision=0):
    """1 x ny x 1 column, walls in y, heavy phase below y0."""
    y0 = (ny - 1) / 2.0 if y0 is None else y0
    bc = (PERIODIC, PERIODIC, NOSLIP, NOSLIP, PERIODIC, PERIODIC)
    p = Params(1, ny, 1, bc, 1.0, 1.0 / rho_ratio, nu, nu, sigma, M, xi, (0.0, 0.0, 0.0), collision)
    return p, flat(p, y0), None, None


def poiseuille(H=16, nx=1, g=1e-6, nu=1.0 / 8.0, collision=0):
    """Single-phase channel (phi = 1), walls in y, body force along x."""
    bc = (PERIODIC, PERIODIC, NOSLIP, NOSLIP, PERIODIC, PERIODIC)
    p = Params(nx, H, 1, bc, 1.0, 1e-3, nu, nu, 1e-4, 0.02, 5.0, (g, 0.0, 0.0), collision)
    return p, np.ones(p.shape), None, None


def hydrostatic_pstar(p, phi0, level, inclusions=()):
    """Initial normalised pressure p* = p / (rho(phi) c_s^2) of a liquid at rest
    under gravity along -y (the paper initialises hydrostatic pressure in its
    gravity cases): p = rho_h |g| (level - y) in the liquid, zero reference at
    y = level; each inclusion (weight field, pressure) adds a region of uniform
    pressure (a bubble at the liquid pressure of its centre plus its Laplace
    jump, or a falling drop at its Laplace jump), blended by its weight."""
    _, y, _ = coords(p)
    g = abs(p.gravity[1])
    p_liq = p.rho_h * g * (level - y)
    pres = p_liq
    for weight, value in inclusions:
        pres = (1.0 - weight) * pres + weight * value
    rho = p.rho_l + phi0 * (p.rho_h - p.rho_l)
    return 3.0 * pres / rho


def column_hydrostatic_pstar(p, phi0, level):
    """p* = p / (rho(phi) c_s^2) of fluid at rest under gravity along -y, with
    dp/dy = -rho(phi) |g| integrated up each (x, z) column by the trapezoid
    rule between cell centres and p = 0 at height `level` (linear
    interpolation between the two cells around it)."""
    g = abs(p.gravity[1])
    rho = p.rho_l + phi0 * (p.rho_h - p.rho_l)                     # (nz, ny, nx)
    steps = 0.5 * (rho[:, 1:, :] + rho[:, :-1, :])
    P = np.concatenate([np.zeros_like(rho[:, :1, :]), -g * np.cumsum(steps, axis=1)], axis=1)
    j = min(max(int(math.floor(level)), 0), p.ny - 2)
    t = level - j
    P -= (1.0 - t) * P[:, j:j + 1, :] + t * P[:, j + 1:j + 2, :]
    return 3.0 * P / rho


def gravity_wave(L=100, Re=10.0, omega_h=1.99, rho_ratio=1000.0, xi=5.0, M=0.02, sigma=0.0, collision=0):
    """Standing gravity wave (section "Gravity wave"): L x L x 1, periodic x and
    z, no-slip walls in y, heavy phase below y = d + a0 cos(k x) with d = L / 2
    above the bottom wall, a0 = 0.01 L, k = 2 pi / L; nu_h from omega_h and
    nu_l = nu_h (kinematic ratio 1); g from Re = a0 omega0 L / nu and
    omega0^2 = g k tanh(k d); surface tension off; hydrostatic start with zero
    pressure at the mean level."""
    nu = (1.0 / omega_h - 0.5) / 3.0
    a0 = 0.01 * L
    d = 0.5 * L
    k = 2.0 * math.pi / L
    omega0 = Re * nu / (a0 * L)
    g = omega0 ** 2 / (k * math.tanh(k * d))
    bc = (PERIODIC, PERIODIC, NOSLIP, NOSLIP, PERIODIC, PERIODIC)
    p = Params(L, L, 1, bc, 1.0, 1.0 / rho_ratio, nu, nu, sigma, M, xi, (0.0, -g, 0.0), collision)
    # the halfway wall sits half a cell below y = 0: the mean level is y = d - 1/2
    phi0 = wave(p, d - 0.5, a0, float(L))
    return p, phi0, None, column_hydrostatic_pstar(p, phi0, d - 0.5)


def rising_bubble(nx=128, ny=384, nz=128, D=32.0, xi=4.0, M=0.02, rho_ratio=1000.0, mu_ratio=100.0,
                  Eo=10.0, Mo=1e-3, nu_h=1.0 / 60.0, collision=0, hydrostatic=True, level=None):
    """Gas bubble of diameter D at 1.5 D above the bottom (y up), walls on all sides.

    Gravity and sigma from the Eotvos and Morton numbers with the heavy-phase
    viscosity fixed: g = nu_h^2 Eo^{3/2} / (D^3 sqrt(Mo)), sigma = g D^2 / Eo
    (rho_h = 1); nu_l = nu_h rho_ratio / mu_ratio (dynamic viscosity ratio).
    """
    g = nu_h ** 2 * Eo ** 1.5 / (D ** 3 * math.sqrt(Mo))
    sigma = g * D * D / Eo
    nu_l = nu_h * rho_ratio / mu_ratio
    p = Params(nx, ny, nz, (NOSLIP,) * 6, 1.0, 1.0 / rho_ratio, nu_h, nu_l, sigma, M, xi,
               (0.0, -g, 0.0), collision)
    c = ((nx - 1) / 2.0, 1.5 * D, (nz - 1) / 2.0)
    phi0 = sphere(p, c, D / 2.0, heavy_inside=False)
    p0 = None
    if hydrostatic:
        # zero pressure at the bubble's height keeps p* = 3 p / rho small in the gas
        level = c[1] if level is None else level
        p_bubble = p.rho_h * g * (level - c[1]) + 2.0 * sigma / (D / 2.0)
        p0 = hydrostatic_pstar(p, phi0, level, [(1.0 - phi0, p_bubble)])
    return p, phi0, None, p0


def drop_impact(nx=512, ny=384, nz=512, D=64.0, depth=128.0, gap=8.0, We=200.0, Fr=200.0, U=0.05,
                omega_h=1.988, rho_ratio=1000.0, mu_ratio=50.0, xi=5.0, M=0.02, collision=0, hydrostatic=True):
    """Vertical drop impact into a pool (y up), no-slip walls on all sides.

    sigma = rho_h U^2 D / We, g = U^2 / (Fr D), nu_h from omega_h,
    nu_l = nu_h rho_ratio / mu_ratio; the drop moves down with speed U.
    """
    sigma = U * U * D / We
    g = U * U / (Fr * D)
    nu_h = (1.0 / omega_h - 0.5) / 3.0
    nu_l = nu_h * rho_ratio / mu_ratio
    p = Params(nx, ny, nz, (NOSLIP,) * 6, 1.0, 1.0 / rho_ratio, nu_h, nu_l, sigma, M, xi,
               (0.0, -g, 0.0), collision)
    x, y, z = coords(p)
    cy = depth + gap + D / 2.0
    c = ((nx - 1) / 2.0, cy, (nz - 1) / 2.0)
    drop = sphere(p, c, D / 2.0, heavy_inside=True)
    pool = tanh_profile(y - depth, xi)
    phi0 = np.maximum(drop, pool)
    u0 = np.zeros((3,) + p.shape)
    u0[1] = -U * drop * (y > depth + gap / 2.0)
    p0 = None
    if hydrostatic:
        # liquid below the pool surface at its hydrostatic pressure, gas at the
        # surface pressure, the drop at its Laplace jump
        _, yy, _ = coords(p)
        p_pool = p.rho_h * g * np.maximum(depth - yy, 0.0) * pool
        pres = p_pool + drop * 2.0 * sigma / (D / 2.0)
        rho = p.rho_l + phi0 * (p.rho_h - p.rho_l)
        p0 = 3.0 * pres / rho
    return p, phi0, u0, p0


def pipe_mask(p, diameter):
    """Solid cells outside a tube of the given diameter along y, centred in x and z."""
    x, y, z = coords(p)
    r = np.sqrt((x - (p.nx - 1) / 2.0) ** 2 + (z - (p.nz - 1) / 2.0) ** 2)
    return (r > diameter / 2.0).astype(np.uint8)


def hagen_poiseuille(D=16, L=4, g=1e-6, nu=1.0 / 6.0):
    """Single-phase flow driven by a body force along y in a voxelised tube of
    diameter D (solid cells outside), periodic along y."""
    n = D + 2
    p = Params(n, L, n, (PERIODIC,) * 6, 1.0, 1e-3, nu, nu, 1e-4, 0.02, 5.0, (0.0, g, 0.0))
    p.solid = pipe_mask(p, D)
    return p, np.ones(p.shape), None, None


def taylor_bubble(D=64, Bo=100.0, Mo=0.015, rho_ratio=744.0, mu_ratio=4236.0, omega_h=1.76, xi=3.0, M=0.08,
                  collision=0, p_level=None):
    """Taylor bubble (section "Taylor bubble"): a vertical tube of diameter D
    along y (solid cells outside it, one solid ring at least: the lattice is
    (D + 2) x 10D x (D + 2)), no-slip top and bottom; a gas cylinder of
    diameter 0.75 D and length 3 D with its bottom at D; nu_H from omega_H,
    nu_L = nu_H rho_ratio / mu_ratio; with rho_H = 1 the Bond number
    Bo = g D^2 / sigma and the Morton number Mo = g mu_H^4 (1 - rho_L) / sigma^3
    give sigma = mu_H^2 sqrt(Bo (1 - rho_L) / Mo) / D and g.  Hydrostatic start
    with zero pressure at height p_level: by default the bubble's top, so that
    the gas starts near zero pressure (the pressure force -p* c_s^2 grad rho
    makes the model sensitive to the gas pressure level); the paper's
    reference height is 5 D."""
    nu_h = (1.0 / omega_h - 0.5) / 3.0
    rho_l = 1.0 / rho_ratio
    sigma = nu_h ** 2 * math.sqrt(Bo * (1.0 - rho_l) / Mo) / D
    g = Bo * sigma / (D * D)
    bc = (PERIODIC, PERIODIC, NOSLIP, NOSLIP, PERIODIC, PERIODIC)
    n = D + 2
    p = Params(n, 10 * D, n, bc, 1.0, rho_l, nu_h, nu_h * rho_ratio / mu_ratio, sigma, M, xi, (0.0, -g, 0.0),
               collision)
    p.solid = pipe_mask(p, D)
    x, y, z = coords(p)
    r = np.sqrt((x - (n - 1) / 2.0) ** 2 + (z - (n - 1) / 2.0) ** 2)
    yb, yt = D - 0.5, 4 * D - 0.5            # the bottom wall sits half a cell below y = 0
    d = np.maximum(r - 0.375 * D, np.maximum(yb - y, y - yt))   # < 0 inside the gas cylinder
    phi0 = tanh_profile(-d, xi)
    level = yt if p_level is None else p_level
    return p, phi0, None, column_hydrostatic_pstar(p, phi0, level)


def gas_centroid_y(phi, solid):
    """Height of the gas centroid, sum (1 - phi) y / sum (1 - phi) over fluid cells."""
    fluid = np.asarray(solid).reshape(phi.shape) == 0
    gas = np.where(fluid, 1.0 - phi, 0.0)
    y = np.arange(phi.shape[1], dtype=np.float64)[None, :, None]
    return float((gas * y).sum() / gas.sum())


def batched_sweep(count=512, seed=20240601, small=False):
    """Seeded mix of static drops (cubes n^3) and capillary waves (nx x 2nx x 1).

    Half the instances are cubes with n ~ U{24..96}, half quasi-2D waves with
    nx ~ U{64..256}; M ~ U[0.005, 0.1], xi ~ U[3, 8], sigma ~ logU[1e-5, 1e-3],
    rho ratio 1000, nu = 1/60.  Drops have R = n/4, waves a0 = 0.01 nx.
    small=True shrinks the sizes (cubes 12..24, waves 32..64) for tests.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        M = float(rng.uniform(0.005, 0.1))
        xi = float(rng.uniform(3.0, 8.0))
        sigma = float(10.0 ** rng.uniform(-5.0, -3.0))
        if i % 2 == 0:
            n = int(rng.integers(12, 25)) if small else int(rng.integers(24, 97))
            p, phi0, u0, p0 = static_drop(n, n / 4.0, xi=xi, sigma=sigma, mobility=M)
        else:
            nx = int(rng.integers(32, 65)) if small else int(rng.integers(64, 257))
            p, phi0, u0, p0 = capillary_wave(nx, ny=2 * nx, a0=0.01 * nx, xi=xi, M=M, sigma=sigma, nu=1.0 / 60.0)
        out.append((p, phi0, u0, p0))
    return out
