"""Seeded synthetic initial fields (rho, u) for the lattice Boltzmann workloads.

These generators hold none of the method's arithmetic: they only produce the
macroscopic initial conditions (density and velocity on the lattice nodes) that
both the CUDA library and the CPU oracle start from.  Nodes sit at integer
coordinates, cell index ``x + nx*(y + ny*z)``; ``u`` is ``[D, C]`` (SoA).

Random inputs use ``numpy.random.Generator(PCG64(20020250 + config_index))``.
"""
import numpy as np

SEED_BASE = 20020250


def rng(config_index: int = 0, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(config_index) + 1000 * int(salt)))


def _grid(dims):
    nx, ny, nz = (list(dims) + [1, 1, 1])[:3]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64), (nx, ny, nz)


def shear_wave(dims, amp, D, flow_axis, grad_axis, background=None, rho0=1.0):
    """u[flow_axis] = amp * sin(2 pi x_grad / n_grad) (+ a uniform background velocity)."""
    x, y, z, n = _grid(dims)
    coords = (x, y, z)
    C = int(np.prod(n))
    u = np.zeros((D, C))
    u[flow_axis] = amp * np.sin(2.0 * np.pi * coords[grad_axis].reshape(C) / n[grad_axis])
    if background is not None:
        for a, U in enumerate(background):
            u[a] += U
    rho = np.full(C, float(rho0))
    return rho, u


def taylor_green_3d(dims, u0, cs2, rho0=1.0):
    """3-D Taylor-Green vortex with k = 2 pi / n per axis (cubic box assumed per axis).

    u = u0 ( sin kx cos ky cos kz, -cos kx sin ky cos kz, 0 ),
    p = rho0 u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2),  rho = rho0 + p / cs2."""
    nx, ny, nz = (list(dims) + [1, 1, 1])[:3]
    x = np.arange(nx) * (2 * np.pi / nx)
    y = (np.arange(ny) * (2 * np.pi / ny))[:, None]
    z = (np.arange(nz) * (2 * np.pi / nz))[:, None, None]
    C = nx * ny * nz
    u = np.zeros((3, C))
    u[0] = (u0 * np.sin(x) * np.cos(y) * np.cos(z)).reshape(C)
    u[1] = (-u0 * np.cos(x) * np.sin(y) * np.cos(z)).reshape(C)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = (rho0 + p / cs2).reshape(C)
    return rho, u


def taylor_green_2d(dims, u0, cs2, D=2, rho0=1.0):
    """2-D Taylor-Green vortex (z-invariant when D=3).

    u = u0 ( -cos kx sin ky, sin kx cos ky ),  p = -rho0 u0^2 / 4 (cos 2kx + cos 2ky)."""
    x, y, z, (nx, ny, nz) = _grid(dims)
    kx, ky = 2 * np.pi / nx, 2 * np.pi / ny
    C = nx * ny * nz
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * np.sin(kx * x) * np.cos(ky * y)
    p = -rho0 * u0 * u0 / 4.0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    u = np.zeros((D, C))
    u[0] = ux.reshape(C)
    u[1] = uy.reshape(C)
    return (rho0 + p / cs2).reshape(C), u


def random_fields(dims, D, config_index=0, salt=0, drho=0.01, umax=0.05):
    """rho = 1 + drho * N(0,1), u ~ U(-umax, umax) per component and cell."""
    g = rng(config_index, salt)
    C = int(np.prod((list(dims) + [1, 1, 1])[:3]))
    rho = 1.0 + drho * g.standard_normal(C)
    u = g.uniform(-umax, umax, size=(D, C))
    return rho, u


def random_smooth_fields(dims, D, config_index=0, salt=0, u0=0.05, drho=0.01, kmax=1):
    """Seeded smooth fields: a sum of Fourier modes with |k_a| <= kmax per axis, random amplitudes
    and phases, scaled so that max|u| = u0 and max|rho - 1| = drho."""
    g = rng(config_index, 100 + salt)
    x, y, z, n = _grid(dims)
    C = int(np.prod(n))
    pos = (x.reshape(C), y.reshape(C), z.reshape(C))

    def field():
        out = np.zeros(C)
        for _ in range(6):
            k = [int(g.integers(-kmax, kmax + 1)) if n[a] > 1 else 0 for a in range(3)]
            ph = 2 * np.pi * sum(k[a] * pos[a] / n[a] for a in range(3)) + g.uniform(0, 2 * np.pi)
            out += g.standard_normal() * np.cos(ph)
        m = np.max(np.abs(out))
        return out / m if m > 0 else out

    rho = 1.0 + drho * field()
    u = np.stack([u0 * field() for _ in range(D)])
    return rho, u


def random_distributions(Q, C, config_index=0, salt=0, scale=0.02):
    """Strictly positive random distributions around 1/Q, with arbitrary non-equilibrium content."""
    g = rng(config_index, salt)
    return (1.0 / Q) * (1.0 + scale * g.standard_normal((Q, C)))
