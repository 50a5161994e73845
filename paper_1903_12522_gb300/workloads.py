"""Seeded synthetic Helmholtz workloads shared by the tests, the benchmark and smoke().

This module only builds problem DATA (wave speed c(x), interior source f, boundary datum g_S,
Dirichlet obstacle mask, frequency, time-step target).  It holds none of the method's
arithmetic: no discrete operator, no time step, no weights.  Both the CUDA path and the CPU
oracle receive the arrays it returns.

Array conventions (shared with the C ABI): nodes x_j = j*h, j in {0..n}^d, x fastest.  A
numpy array of a 3D field has shape (nz+1, ny+1, nx+1); a 2D field (ny+1, nx+1).
Boundary faces are ordered (-x, +x, -y, +y, -z, +z) with codes ABC=0, NEUMANN=1,
DIRICHLET=2.

The problem statement these workloads instantiate is the Helmholtz boundary-value problem
of Sec. 2.1 (Eq. HE): -Lap u - k^2 u = f, du/dn - i k u = g_S on the absorbing part, with
k = omega/c and time convention exp(-i omega t).  The synthetic inputs stand in for the
paper's Marmousi model and obstacle meshes (Sec. 4.3), which are not available here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

ABC, NEUMANN, DIRICHLET = 0, 1, 2


@dataclasses.dataclass
class Workload:
    name: str
    n: tuple                      # intervals per axis, (nx, ny[, nz])
    h: float
    c: np.ndarray                 # float64, numpy shape of the grid
    omega: float
    faces: tuple                  # 6 codes (-x,+x,-y,+y,-z,+z); unused z entries ignored in 2D
    dt_target: float              # target time step; the solver rounds to T/N
    order: int = 2
    mask: Optional[np.ndarray] = None   # uint8, 1 = Dirichlet obstacle node
    f: Optional[np.ndarray] = None      # complex128 interior source amplitude
    g: Optional[np.ndarray] = None      # complex128 boundary datum g_S at ABC nodes

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        return tuple(m + 1 for m in reversed(self.n))

    @property
    def num_nodes(self) -> int:
        return int(np.prod(self.shape))


def coords(n: Sequence[int], h: float):
    """Node coordinates as broadcastable arrays in numpy order: returns (x, y[, z])."""
    d = len(n)
    axes = []
    for a in range(d):
        shp = [1] * d
        shp[d - 1 - a] = n[a] + 1
        axes.append((np.arange(n[a] + 1, dtype=np.float64) * h).reshape(shp))
    return axes


def gaussian_source(n, h, center, sigma, amplitude=1.0) -> np.ndarray:
    """Real Gaussian f(x) = A exp(-|x - x_s|^2 / (2 sigma^2)) as a complex field."""
    xs = coords(n, h)
    r2 = sum((xa - ca) ** 2 for xa, ca in zip(xs, center))
    return (amplitude * np.exp(-r2 / (2.0 * sigma * sigma))).astype(np.complex128)


def sphere_mask(n, h, center, radius) -> np.ndarray:
    """Staircase obstacle: nodes with |x - x_c| <= r."""
    xs = coords(n, h)
    r2 = sum((xa - ca) ** 2 for xa, ca in zip(xs, center))
    return (r2 <= radius * radius + 1e-12).astype(np.uint8)


def plane_wave_boundary_datum(n, h, omega, c_boundary, direction, faces) -> np.ndarray:
    """g_S = (d/dn - i k) u_in on the absorbing faces, u_in = exp(i k x.d), k = omega/c.

    With this datum and no obstacle the total field u = u_in solves the Helmholtz problem
    exactly.  A node on several absorbing faces (edge, corner) gets the plain mean of the
    faces' values; every face through such a node has the same lumped area there, so the
    mean is the area-weighted mean.  Nodes on no absorbing face get 0.
    """
    d = len(n)
    xs = coords(n, h)
    k = omega / c_boundary
    phase = sum(xa * da for xa, da in zip(xs, direction))
    uin = np.exp(1j * k * phase) * np.ones(tuple(m + 1 for m in reversed(n)))
    acc = np.zeros_like(uin)
    cnt = np.zeros(uin.shape, dtype=np.float64)
    for a in range(d):
        for side in (0, 1):
            if faces[2 * a + side] != ABC:
                continue
            normal = -1.0 if side == 0 else 1.0
            sl = [slice(None)] * d
            sl[d - 1 - a] = 0 if side == 0 else n[a]
            sl = tuple(sl)
            val = 1j * k * (normal * direction[a] - 1.0) * uin[sl]
            acc[sl] += val
            cnt[sl] += 1.0
    out = np.where(cnt > 0, acc / np.maximum(cnt, 1.0), 0.0)
    return out.astype(np.complex128)


def smooth_random_field(n, seed, corr_len=0.1, lo=1.0, hi=2.0) -> np.ndarray:
    """Smooth Gaussian random field: white noise, Gaussian filter (via FFT), affine map to [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = tuple(m + 1 for m in reversed(n))
    noise = rng.standard_normal(shape)
    h = 1.0 / max(n)
    sig = corr_len / h
    spec = np.fft.fftn(noise)
    filt = np.ones(shape)
    for ax, m in enumerate(shape):
        fr = np.fft.fftfreq(m)
        g = np.exp(-2.0 * (math.pi * sig * fr) ** 2)
        sh = [1] * len(shape)
        sh[ax] = m
        filt = filt * g.reshape(sh)
    field = np.real(np.fft.ifftn(spec * filt))
    fmin, fmax = field.min(), field.max()
    if fmax - fmin < 1e-300:
        return np.full(shape, 0.5 * (lo + hi))
    return lo + (hi - lo) * (field - fmin) / (fmax - fmin)


# ----------------------------------------------------------------------------------------
# The five synthetic workloads.  Sizes are parameters so that tests can run the same
# recipe on small grids; the defaults are the full sizes.
# ----------------------------------------------------------------------------------------

def gaussian_2d(n: int = 128, ppw_freq: float = 8.0, dt_frac: float = 0.5) -> Workload:
    """2D unit square, c = 1, omega = 2 pi * 8 (16 points per wavelength at n = 128),
    Gaussian source sigma = 0.05 at (0.5, 0.5), absorbing on all four sides, dt = h/2."""
    h = 1.0 / n
    shape = (n + 1, n + 1)
    omega = 2.0 * math.pi * ppw_freq * (n / 128.0)
    return Workload(
        name=f"2d_gaussian_n{n}", n=(n, n), h=h, c=np.ones(shape), omega=omega,
        faces=(ABC,) * 4 + (NEUMANN, NEUMANN), dt_target=dt_frac * h,
        f=gaussian_source((n, n), h, (0.5, 0.5), 0.05),
    )


def sphere_3d(n: int = 256, ppw: float = 10.0, dt_frac: float = 0.4, obstacle: bool = True,
              heterogeneous: bool = True) -> Workload:
    """3D unit cube, c(x) = 1 + 0.3 sin(2 pi x) sin(2 pi y) sin(2 pi z) in [0.7, 1.3],
    omega = 2 pi c_min / (ppw h) (10 points per wavelength at the slowest speed), sound-soft
    sphere r = 0.1 at the centre, plane wave with direction d = (1/2, 0, sqrt(3)/2) entering
    through absorbing faces (c = 1 on the faces), dt = 0.4 h."""
    h = 1.0 / n
    x, y, z = coords((n, n, n), h)
    if heterogeneous:
        c = 1.0 + 0.3 * np.sin(2 * math.pi * x) * np.sin(2 * math.pi * y) * np.sin(2 * math.pi * z)
        c_min = 0.7
    else:
        c = np.ones((n + 1,) * 3) + 0.0 * x
        c_min = 1.0
    c = np.ascontiguousarray(np.broadcast_to(c, (n + 1,) * 3), dtype=np.float64)
    omega = 2.0 * math.pi * c_min / (ppw * h)
    faces = (ABC,) * 6
    g = plane_wave_boundary_datum((n, n, n), h, omega, 1.0, (0.5, 0.0, math.sqrt(3.0) / 2.0), faces)
    mask = sphere_mask((n, n, n), h, (0.5, 0.5, 0.5), 0.1) if obstacle else None
    return Workload(name=f"3d_sphere_n{n}", n=(n, n, n), h=h, c=c, omega=omega, faces=faces,
                    dt_target=dt_frac * h, mask=mask, g=g)


def layered_3d(n: int = 512, seed: int = 3, freq: float = 40.0, order: int = 4) -> Workload:
    """3D cube, 3-layer medium c = 1.0 / 1.5 / 2.0 along z, omega = 2 pi * 40 at n = 512
    (scaled with n), 4 seeded Gaussian point sources sigma = 0.01 * 512/n, absorbing faces,
    dt = T / ceil(T / (0.9 h / (2 c_max)))."""
    h = 1.0 / n
    x, y, z = coords((n, n, n), h)
    c = np.where(z < 1.0 / 3.0, 1.0, np.where(z < 2.0 / 3.0, 1.5, 2.0))
    c = np.ascontiguousarray(np.broadcast_to(c, (n + 1,) * 3), dtype=np.float64)
    omega = 2.0 * math.pi * freq * (n / 512.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(0.2, 0.8, size=(4, 3))
    sigma = 0.01 * 512.0 / n
    f = np.zeros((n + 1,) * 3, dtype=np.complex128)
    for p in pos:
        f += gaussian_source((n, n, n), h, tuple(p), sigma)
    return Workload(name=f"3d_layered_n{n}", n=(n, n, n), h=h, c=c, omega=omega,
                    faces=(ABC,) * 6, dt_target=0.9 * h / (2.0 * 2.0), order=order, f=f)


def random_2d_instance(i: int, n: Optional[int] = None) -> Workload:
    """One instance of the uneven 2D batch: seed 1000+i, n ~ U{96..1024}, p ~ U[8, 20]
    points per wavelength, c = smooth random field in [1, 2], omega = 2 pi c_min/(p h),
    one Gaussian source sigma = 0.4 p h at U[0.2, 0.8]^2, absorbing on all sides,
    dt target 0.9 h / (sqrt(2) c_max)."""
    rng = np.random.Generator(np.random.PCG64(1000 + i))
    n_i = int(rng.integers(96, 1025)) if n is None else int(n)
    p = float(rng.uniform(8.0, 20.0))
    src = rng.uniform(0.2, 0.8, size=2)
    h = 1.0 / n_i
    c = smooth_random_field((n_i, n_i), seed=1000 + i)
    omega = 2.0 * math.pi * 1.0 / (p * h)
    f = gaussian_source((n_i, n_i), h, tuple(src), 0.4 * p * h)
    return Workload(name=f"2d_random_{i}_n{n_i}", n=(n_i, n_i), h=h, c=c, omega=omega,
                    faces=(ABC,) * 4 + (NEUMANN, NEUMANN), dt_target=0.9 * h / (math.sqrt(2.0) * 2.0), f=f)


def square_obstacle_2d(n: int = 128, cavity: bool = False, wavelengths: float = 10.0) -> Workload:
    """Plane-wave scattering off a sound-soft square obstacle (Sec. 4.2): the paper's domain of
    10 x 10 wavelengths rescaled to the unit square, c = 1, omega = 2 pi * wavelengths, total
    field with g_S = (d/dn - i k) u_in for u_in incident at 135 degrees, absorbing on all four
    sides, dt = 0.4 h.  Convex case: the square |x - 1/2|, |y - 1/2| <= 0.15 (3 wavelengths).
    Cavity case: the same square with its interior |.| < 0.12 removed (walls 0.03 thick) and a
    mouth |y - 1/2| < 0.05 cut into its +x wall, which faces the incoming wave: a semi-open
    cavity that traps waves."""
    h = 1.0 / n
    omega = 2.0 * math.pi * wavelengths
    x, y = coords((n, n), h)
    solid = (np.abs(x - 0.5) <= 0.15 + 1e-12) & (np.abs(y - 0.5) <= 0.15 + 1e-12)
    if cavity:
        hollow = (np.abs(x - 0.5) < 0.12 - 1e-12) & (np.abs(y - 0.5) < 0.12 - 1e-12)
        mouth = (x > 0.5) & (np.abs(y - 0.5) < 0.05 - 1e-12)
        solid = solid & ~hollow & ~mouth
    faces = (ABC,) * 4 + (NEUMANN, NEUMANN)
    theta = math.radians(135.0)
    g = plane_wave_boundary_datum((n, n), h, omega, 1.0, (math.cos(theta), math.sin(theta)), faces)
    return Workload(name=f"2d_{'cavity' if cavity else 'square'}_n{n}", n=(n, n), h=h,
                    c=np.ones((n + 1, n + 1)), omega=omega, faces=faces, dt_target=0.4 * h,
                    mask=solid.astype(np.uint8), g=g)


def neumann_box_2d(n: int = 64, dt_frac: float = 0.5) -> Workload:
    """The physically bounded domain of Sec. 3.5 lifted to the unit square: homogeneous Neumann
    on all four sides, c = 1, k = omega = pi/4, and the source f = -u'' - k^2 u of the exact
    solution u(x, y) = 16 x^2 (x - 1)^2 (constant in y, zero normal derivative on every side).
    (4k)^2 = pi^2 is a Neumann eigenvalue: the wave equation has a mode of period T/4."""
    h = 1.0 / n
    k = math.pi / 4.0
    x, y = coords((n, n), h)
    u = 16.0 * x ** 2 * (x - 1.0) ** 2 + 0.0 * y
    f = -(192.0 * x ** 2 - 192.0 * x + 32.0) - k * k * u + 0.0 * y
    return Workload(name=f"2d_neumann_box_n{n}", n=(n, n), h=h, c=np.ones((n + 1, n + 1)), omega=k,
                    faces=(NEUMANN,) * 6, dt_target=dt_frac * h, f=f.astype(np.complex128))


def neumann_box_exact(n: int) -> np.ndarray:
    """u(x, y) = 16 x^2 (x - 1)^2 on the nodes of neumann_box_2d(n)."""
    x, y = coords((n, n), 1.0 / n)
    return (16.0 * x ** 2 * (x - 1.0) ** 2 + 0.0 * y).astype(np.complex128)


def manufactured_plane_wave_field(n, h, k_axis: float) -> np.ndarray:
    """u(x) = exp(i k x_1): a plane wave along x used by the manufactured-solution checks."""
    x = coords(n, h)[0]
    shape = tuple(m + 1 for m in reversed(n))
    return (np.exp(1j * k_axis * x) * np.ones(shape)).astype(np.complex128)


def random_fields(shape, count: int, seed: int):
    """Seeded standard-normal float64 fields (for adjoint dot-product and parity tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [rng.standard_normal(shape) for _ in range(count)]
