"""Scattering problems: body, discretisation sizes, materials and excitation.

Conventions: time dependence e^{-i omega t}, c = 1, so kappa_s = omega
sqrt(eps_s mu_s) (Sec. II, the Maxwell systems for the interior and exterior
media).  Wavelengths are exterior wavelengths lambda_e = 2 pi / kappa_e.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .geometry import Body, cubed_sphere, open_cheb_nodes, sample_body

__all__ = ["Problem", "sphere_problem", "CONFIG_SPHERE_SMALL", "CONFIG_SPHERE_MEDIUM",
           "random_densities", "plane_wave"]


@dataclass
class Problem:
    body: Body
    nc: int                      # Chebyshev nodes per patch direction
    ng: int                      # oversampled geometry grid per patch direction
    eps_ext: float
    eps_int: float
    mu_ext: float = 1.0
    mu_int: float = 1.0
    omega: float = 2 * np.pi
    name: str = ""
    _cache: dict = field(default_factory=dict, repr=False)

    @property
    def k_ext(self) -> float:
        return self.omega * np.sqrt(self.eps_ext * self.mu_ext)

    @property
    def k_int(self) -> float:
        return self.omega * np.sqrt(self.eps_int * self.mu_int)

    @property
    def num_patches(self) -> int:
        return self.body.num_patches

    @property
    def n(self) -> int:
        return self.num_patches * self.nc * self.nc

    def nodes(self):
        """(x, x_u, x_v) flattened to [N, 3] in node order l = j + Nc i + p Nc^2."""
        if "nodes" not in self._cache:
            x, xu, xv = sample_body(self.body, open_cheb_nodes(self.nc))
            self._cache["nodes"] = tuple(a.reshape(-1, 3).copy() for a in (x, xu, xv))
        return self._cache["nodes"]

    def fine(self):
        """Oversampled geometry [P, Ng, Ng, 9] = (x, x_u, x_v) on the Ng open Chebyshev grid."""
        if "fine" not in self._cache:
            x, xu, xv = sample_body(self.body, open_cheb_nodes(self.ng))
            self._cache["fine"] = np.ascontiguousarray(np.concatenate([x, xu, xv], axis=-1))
        return self._cache["fine"]


def sphere_problem(radius: float, split: int, nc: int, eps_int: float, ng: int | None = None,
                   eps_ext: float = 1.0, wavelength: float = 1.0, name: str = "") -> Problem:
    omega = 2 * np.pi / (wavelength * np.sqrt(eps_ext))
    return Problem(body=cubed_sphere(radius, split), nc=nc, ng=ng or max(2 * nc, 24),
                   eps_ext=eps_ext, eps_int=eps_int, omega=omega, name=name)


def CONFIG_SPHERE_SMALL(nc: int = 8, ng: int | None = None) -> Problem:
    """Sphere of radius lambda_e/2 (kappa_e a = pi), eps_r = 2.25, 6 patches x Nc^2 nodes."""
    return sphere_problem(0.5, 1, nc, 2.25, ng=ng, name="sphere_r0.5_eps2.25_P6")


def CONFIG_SPHERE_MEDIUM(nc: int = 10, ng: int | None = None) -> Problem:
    """Sphere of radius 2 lambda_e, eps_r = 4, 96 patches (4x4 per cube face) x Nc^2 nodes."""
    return sphere_problem(2.0, 4, nc, 4.0, ng=ng, name="sphere_r2_eps4_P96")


def random_densities(n: int, seed: int, batch: int | None = None) -> np.ndarray:
    """Complex Gaussian CN(0,1) densities y = [m1, m2, j1, j2], shape [4, N] (or [B, 4, N])."""
    rng = np.random.default_rng(seed)
    shape = (4, n) if batch is None else (batch, 4, n)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def plane_wave(x: np.ndarray, k_ext: float, omega: float, mu_ext: float = 1.0,
               direction=(0.0, 0.0, 1.0), polarization=(1.0, 0.0, 0.0)):
    """Incident plane wave E = p e^{i k d.x}, H = (k/(omega mu)) (d x p) e^{i k d.x}.

    Returns an array [6, N] complex: (Ex, Ey, Ez, Hx, Hy, Hz) at the points x [N, 3].
    """
    d = np.asarray(direction, dtype=np.float64)
    p = np.asarray(polarization, dtype=np.float64)
    ph = np.exp(1j * k_ext * (x @ d))
    E = p[:, None] * ph[None, :]
    H = (k_ext / (omega * mu_ext)) * np.cross(d, p)[:, None] * ph[None, :]
    return np.concatenate([E, H], axis=0)


def fibonacci_directions(n_dirs: int = 32):
    """Directions d_k on a Fibonacci sphere, z_k = 1 - (2k+1)/n_dirs, phi_k = k pi (3 - sqrt 5), and
    their polarisations e1 = z x d / |z x d| (x when d is along z), e2 = d x e1: three [n_dirs, 3]."""
    D, E1, E2 = [], [], []
    for k in range(n_dirs):
        z = 1.0 - (2 * k + 1) / n_dirs
        r = np.sqrt(max(0.0, 1.0 - z * z))
        ph = k * np.pi * (3.0 - np.sqrt(5.0))
        d = np.array([r * np.cos(ph), r * np.sin(ph), z])
        e1 = np.cross([0.0, 0.0, 1.0], d)
        e1 = e1 / np.linalg.norm(e1) if np.linalg.norm(e1) > 1e-12 else np.array([1.0, 0.0, 0.0])
        D.append(d)
        E1.append(e1)
        E2.append(np.cross(d, e1))
    return np.array(D), np.array(E1), np.array(E2)


def fibonacci_incidences(x: np.ndarray, k_ext: float, omega: float, n_dirs: int = 32, mu_ext: float = 1.0):
    """2 n_dirs plane waves: the directions of fibonacci_directions, each with its two
    polarisations e1, e2 (incidence 2k + i has direction d_k and polarisation e_{i+1}).
    Returns [2 n_dirs, 6, N] complex (see plane_wave)."""
    D, E1, E2 = fibonacci_directions(n_dirs)
    out = []
    for d, e1, e2 in zip(D, E1, E2):
        for p in (e1, e2):
            out.append(plane_wave(x, k_ext, omega, mu_ext, direction=d, polarization=p))
    return np.stack(out)


def ellipsoid_batch(count: int = 16, seed: int = 3, nc: int = 10, wavelength: float = 1.0):
    """The uneven batch of dielectric ellipsoids: semi-axes uniform in [0.5, 3] wavelengths,
    eps_r uniform in [2, 12], ambient eps = 1; each cube face split s x s with s the smallest
    number giving 8 nodes per interior wavelength along the longest quarter-ellipse, clipped
    to [2, 6].  Returns a list of Problems."""
    from .geometry import ellipsoid
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        axes = rng.uniform(0.5, 3.0, size=3) * wavelength
        eps = float(rng.uniform(2.0, 12.0))
        lam_i = wavelength / np.sqrt(eps)
        s = int(np.clip(np.ceil(8.0 * (0.5 * np.pi * axes.max()) / (nc * lam_i)), 2, 6))
        out.append(Problem(body=ellipsoid(tuple(axes), s), nc=nc, ng=max(2 * nc, 24), eps_ext=1.0,
                           eps_int=eps, omega=2 * np.pi / wavelength, name=f"ellipsoid{i}"))
    return out


def dipole_field(x: np.ndarray, k_ext: float, omega: float, r0, j, mu_ext: float = 1.0):
    """Incident field of a point current j delta(x - r0) in the exterior medium (e^{-i omega t}):
    E = i omega mu [g j + k^-2 (grad grad g) j], H = grad g x j, g = e^{i k R} / (4 pi R),
    R = |x - r0|.  Returns [6, N] complex (Ex, Ey, Ez, Hx, Hy, Hz) at the points x [N, 3]."""
    j = np.asarray(j, dtype=np.complex128)
    d = np.asarray(x, dtype=np.float64) - np.asarray(r0, dtype=np.float64)[None, :]
    R = np.linalg.norm(d, axis=1)
    n = d / R[:, None]
    k = k_ext
    g = np.exp(1j * k * R) / (4 * np.pi * R)
    nj = n @ j
    ggj = g[:, None] * ((3 / R**2 - 3j * k / R - k * k)[:, None] * nj[:, None] * n +
                        (1j * k / R - 1 / R**2)[:, None] * j[None, :])
    E = 1j * omega * mu_ext * (g[:, None] * j[None, :] + ggj / (k * k))
    H = (g * (1j * k - 1 / R))[:, None] * np.cross(n, j[None, :])
    return np.concatenate([E.T, H.T], axis=0)


def star_batch(count: int, seed: int, radius: float = 0.75, split: int = 4, nc: int = 8,
               eps_range=(2.0, 12.0), wavelength: float = 1.0):
    """Random star-shaped dielectric bodies r(w) = a (1 + sum_{1<=l<=4} c_lm Y_lm(w)) with
    c_lm ~ N(0, 0.03^2) and eps_r uniform in eps_range, ambient eps = 1, cube faces split
    split x split.  Returns a list of Problems."""
    from .geometry import star_body
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        coeffs = {(l, m): 0.03 * rng.standard_normal() for l in range(1, 5) for m in range(-l, l + 1)}
        eps = float(rng.uniform(*eps_range))
        out.append(Problem(body=star_body(radius * wavelength, coeffs, split), nc=nc, ng=max(2 * nc, 24),
                           eps_ext=1.0, eps_int=eps, omega=2 * np.pi / wavelength, name=f"star{seed}_{i}"))
    return out


def gaussian_beam(x: np.ndarray, k_ext: float, omega: float, focus, waist: float, mu_ext: float = 1.0,
                  direction=(1.0, 0.0, 0.0), polarization=(0.0, 1.0, 0.0)):
    """Paraxial Gaussian beam (e^{-i omega t}) with waist w0 at `focus`, travelling along d:
    xi = d.(x - f), rho^2 = |x - f|^2 - xi^2, z_R = k w0^2 / 2, q = xi - i z_R,
    E = p (-i z_R / q) exp(i k xi + i k rho^2 / (2 q)),  H = (k / (omega mu)) d x E.
    |E| = (w0 / w(xi)) exp(-rho^2 / w(xi)^2) with w(xi) = w0 sqrt(1 + (xi/z_R)^2), and the phase
    carries the Gouy term -atan(xi / z_R).  Only paraxially a Maxwell field: it serves as a
    right-hand side.  Returns [6, N] complex (Ex, Ey, Ez, Hx, Hy, Hz) at the points x [N, 3]."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    p = np.asarray(polarization, dtype=np.float64)
    p = p - (p @ d) * d
    p = p / np.linalg.norm(p)
    r = np.asarray(x, dtype=np.float64) - np.asarray(focus, dtype=np.float64)[None, :]
    xi = r @ d
    rho2 = np.maximum(np.sum(r * r, axis=1) - xi * xi, 0.0)
    k = k_ext
    zr = 0.5 * k * waist * waist
    q = xi - 1j * zr
    u = (-1j * zr / q) * np.exp(1j * k * xi + 1j * k * rho2 / (2.0 * q))
    E = p[:, None] * u[None, :]
    H = (k / (omega * mu_ext)) * np.cross(d, p)[:, None] * u[None, :]
    return np.concatenate([E, H], axis=0)


def waveguide_bar(patch_size: float = 0.035, nc: int = 10, wavelength: float = 1.0,
                  half_lengths=(10.0, 0.15, 0.07), end_length: float = 0.15, eps_ext: float = 2.1,
                  eps_int: float = 12.1, center=(0.0, 0.0, 0.0), exponent: int = 8):
    """The elongated waveguide bar: a straight bar 2A = 20 vacuum wavelengths long with the
    rounded-rectangle cross-section |y/B|^8 + |z/C|^8 = 1 (B = 0.15, C = 0.07: 0.3 x 0.14),
    closed by superellipsoidal ends 0.15 long (``rounded_bar``); silicon-like eps_int = 12.1
    in an oxide-like eps_ext = 2.1, omega = 2 pi / lambda_0.  Patches of side about
    `patch_size` wavelengths: 0.035 gives about 1.5M nodes at nc = 10."""
    from .geometry import rounded_bar
    hl = tuple(float(h) * wavelength for h in half_lengths)
    body = rounded_bar(hl, end_length * wavelength, patch_size * wavelength, center=center, exponent=exponent)
    return Problem(body=body, nc=nc, ng=max(2 * nc, 24), eps_ext=eps_ext, eps_int=eps_int,
                   omega=2 * np.pi / wavelength, name=f"bar_h{patch_size:g}_P{body.num_patches}")
