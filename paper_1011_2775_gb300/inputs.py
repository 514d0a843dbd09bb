"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the solver: it only draws random gauge
fields, gauge transformations and sources.  Everything is FP64/complex128 on
the host (numpy), in the library's layout:

* gauge field ``U``: shape ``(Lt, Lz, Ly, Lx, 4, 3, 3)`` -- ``[t][z][y][x][mu][a][b]``,
  x fastest, ``mu`` = 0..3 for x, y, z, t;
* spinor: shape ``(Lt, Lz, Ly, Lx, 4, 3)`` -- ``[t][z][y][x][spin][colour]``.

Gauge ensemble (a stand-in for the paper's production lattices, which are not
available): ``U = exp(i eps H)`` with ``H = sum_a h_a lambda_a / 2``,
``h_a ~ N(0, 1)``, followed by ``n`` steps of 4D APE smearing
``U' = Proj_SU3[(1 - alpha) U + alpha/6 * sum of the 6 staples]`` where
``Proj_SU3`` is the polar projection ``W (W^dag W)^{-1/2}`` divided by the
principal cube root of its determinant.  Random numbers come from
``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gell_mann",
    "lattice_shape",
    "unit_gauge",
    "random_gauge",
    "ape_smear",
    "make_gauge",
    "gaussian_source",
    "point_source",
    "random_gauge_transform",
    "config_seeds",
]


def config_seeds(k: int) -> dict:
    """Seeds of workload ``k``: gauge 1000k+1, source 1000k+2, null vectors 1000k+3."""
    return {"gauge": 1000 * k + 1, "source": 1000 * k + 2, "nullvec": 1000 * k + 3}


def lattice_shape(dims) -> tuple:
    """``dims = (Lx, Ly, Lz, Lt)`` -> array shape ``(Lt, Lz, Ly, Lx)``."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1] = -1j
    l[1, 1, 0] = 1j
    l[2, 0, 0], l[2, 1, 1] = 1, -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2] = -1j
    l[4, 2, 0] = 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2] = -1j
    l[6, 2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def _shift(f, mu, sign):
    """Periodic shift on the site axes: ``f(x + sign*mu_hat)``."""
    return np.roll(f, -sign, axis=3 - mu)


def _project_su3(w: np.ndarray) -> np.ndarray:
    """Polar projection ``w (w^dag w)^{-1/2}`` then division by ``det^{1/3}``."""
    h = _dag(w) @ w
    e, q = np.linalg.eigh(h)
    inv_sqrt = (q * (1.0 / np.sqrt(e))[..., None, :]) @ _dag(q)
    u = w @ inv_sqrt
    det = np.linalg.det(u)
    root = np.exp(1j * np.angle(det) / 3.0)
    return u / root[..., None, None]


def unit_gauge(dims) -> np.ndarray:
    shp = lattice_shape(dims)
    u = np.zeros(shp + (4, 3, 3), dtype=np.complex128)
    u[..., :, :, :] = np.eye(3)
    return u


def gauge_normals(dims, seed: int) -> np.ndarray:
    """The Gaussian coefficients ``h[t][z][y][x][mu][a]`` of ``random_gauge``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(lattice_shape(dims) + (4, 8))


def links_from_normals(h: np.ndarray, eps: float) -> np.ndarray:
    """``exp(i eps H)`` with ``H = sum_a h_a lambda_a/2`` per link (site-local,
    so any block of sites can be done on its own)."""
    H = np.einsum("...a,aij->...ij", h, gell_mann() / 2.0)
    e, q = np.linalg.eigh(H)
    u = (q * np.exp(1j * eps * e)[..., None, :]) @ _dag(q)
    return _project_su3(u)


def random_gauge(dims, eps: float, seed: int) -> np.ndarray:
    """``U = exp(i eps H)``, ``H = sum_a h_a lambda_a/2``, by eigendecomposition of ``H``."""
    return links_from_normals(gauge_normals(dims, seed), eps)


def ape_step(u: np.ndarray, alpha: float) -> np.ndarray:
    """One 4D APE step with all six staples per link, periodic on the array's
    own site axes.  A site's new links read only sites one step away, so for a
    block of time slices with one slice of halo on each side the interior
    slices of the result are those of the step on the whole lattice."""
    new = np.empty_like(u)
    for mu in range(4):
        umu = u[..., mu, :, :]
        staple = np.zeros_like(umu)
        for nu in range(4):
            if nu == mu:
                continue
            unu = u[..., nu, :, :]
            # upper: U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
            staple += unu @ _shift(umu, nu, +1) @ _dag(_shift(unu, mu, +1))
            # lower: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu)
            unu_m = _shift(unu, nu, -1)
            staple += _dag(unu_m) @ _shift(umu, nu, -1) @ _shift(unu_m, mu, +1)
        new[..., mu, :, :] = _project_su3((1.0 - alpha) * umu + (alpha / 6.0) * staple)
    return new


def ape_smear(u: np.ndarray, steps: int, alpha: float) -> np.ndarray:
    """4D APE smearing with all six staples per link, ``steps`` times."""
    for _ in range(int(steps)):
        u = ape_step(u, alpha)
    return u


def make_gauge(dims, eps: float, ape_steps: int = 0, alpha: float = 0.5, seed: int = 1) -> np.ndarray:
    """The synthetic ensemble: ``exp(i eps H)`` then ``ape_steps`` APE steps."""
    u = random_gauge(dims, eps, seed)
    if ape_steps:
        u = ape_smear(u, ape_steps, alpha)
    return np.ascontiguousarray(u)


def gaussian_source(dims, seed: int, nrhs: int | None = None) -> np.ndarray:
    """Complex Gaussian noise, Re and Im ~ N(0, 1/2) per spin-colour component."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = lattice_shape(dims) + (4, 3)
    if nrhs is not None:
        shp = (int(nrhs),) + shp
    z = rng.standard_normal(shp + (2,)) * np.sqrt(0.5)
    return np.ascontiguousarray(z[..., 0] + 1j * z[..., 1])


def point_source(dims, alpha0: int, site=(0, 0, 0, 0)) -> np.ndarray:
    """``delta_{x,site} delta_{(spin,colour), alpha0}``; ``site = (x, y, z, t)``."""
    s = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    s[t, z, y, x, alpha0 // 3, alpha0 % 3] = 1.0
    return s


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Haar-random SU(3) matrix per site: QR of a complex Gaussian, phase-fixed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shp = lattice_shape(dims)
    z = (rng.standard_normal(shp + (3, 3)) + 1j * rng.standard_normal(shp + (3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / np.exp(1j * np.angle(det) / 3.0)[..., None, None]
