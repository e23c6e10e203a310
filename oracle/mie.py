"""Mie series for a dielectric sphere under a plane wave (accuracy reference, Sec. IV-B).

TEST INFRASTRUCTURE ONLY (see oracle/cbie.py).  The paper checks its solver
against the Mie series but does not print it; this is the textbook
vector-spherical-wave solution (Bohren & Huffman, "Absorption and Scattering
of Light by Small Particles", Ch. 4), written here from the formulas:
e^{-i omega t}, incident E = exp(i k z) x_hat, H = (k/(omega mu)) exp(i k z) y_hat,
sphere of radius a centred at the origin, relative index m = k_int/k_ext,
equal permeabilities.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _psi(n, x):
    return x * spherical_jn(n, x)


def _dpsi(n, x):
    return spherical_jn(n, x) + x * spherical_jn(n, x, derivative=True)


def _xi(n, x):
    return x * (spherical_jn(n, x) + 1j * spherical_yn(n, x))


def _dxi(n, x):
    h = spherical_jn(n, x) + 1j * spherical_yn(n, x)
    dh = spherical_jn(n, x, derivative=True) + 1j * spherical_yn(n, x, derivative=True)
    return h + x * dh


def n_terms(k_ext: float, a: float, m: float) -> int:
    x = k_ext * a * max(1.0, abs(m))
    return int(np.ceil(x + 4.0 * x ** (1.0 / 3.0) + 10))


def coefficients(k_ext: float, k_int: float, a: float, nmax: int | None = None):
    """Scattering (a_n, b_n) and internal (c_n, d_n) coefficients, n = 1..nmax (mu_int = mu_ext)."""
    m = k_int / k_ext
    x = k_ext * a
    nmax = nmax or n_terms(k_ext, a, m)
    n = np.arange(1, nmax + 1)
    px, dpx = _psi(n, x), _dpsi(n, x)
    pmx, dpmx = _psi(n, m * x), _dpsi(n, m * x)
    xx, dxx = _xi(n, x), _dxi(n, x)
    an = (m * pmx * dpx - px * dpmx) / (m * pmx * dxx - xx * dpmx)
    bn = (pmx * dpx - m * px * dpmx) / (pmx * dxx - m * xx * dpmx)
    cn = (m * px * dxx - m * xx * dpx) / (pmx * dxx - m * xx * dpmx)
    dn = (m * px * dxx - m * xx * dpx) / (m * pmx * dxx - xx * dpmx)
    return an, bn, cn, dn


def _angular(nmax, ct):
    """pi_n(cos theta), tau_n(cos theta) for n = 1..nmax; shapes [nmax, npts]."""
    pi = np.zeros((nmax + 1, ct.size))
    tau = np.zeros((nmax + 1, ct.size))
    pi[1] = 1.0
    tau[1] = ct
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) / (n - 1)) * ct * pi[n - 1] - (n / (n - 1)) * pi[n - 2]
        tau[n] = n * ct * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def _vsh(nmax, kind, rho, ct, st, cp, sp):
    """M_o1n, M_e1n, N_o1n, N_e1n in spherical components (r, theta, phi); shape [4, nmax, 3, npts]."""
    n = np.arange(1, nmax + 1)[:, None]
    if kind == 1:
        z = np.array([spherical_jn(k, rho) for k in range(1, nmax + 1)])
        dz = np.array([spherical_jn(k, rho, derivative=True) for k in range(1, nmax + 1)])
    else:
        z = np.array([spherical_jn(k, rho) + 1j * spherical_yn(k, rho) for k in range(1, nmax + 1)])
        dz = np.array([spherical_jn(k, rho, derivative=True) + 1j * spherical_yn(k, rho, derivative=True)
                       for k in range(1, nmax + 1)])
    drz = (z + rho * dz) / rho                  # [rho z_n]' / rho
    pi, tau = _angular(nmax, ct)
    zero = np.zeros_like(z)
    Mo = np.stack([zero, cp * pi * z, -sp * tau * z], axis=1)
    Me = np.stack([zero, -sp * pi * z, -cp * tau * z], axis=1)
    No = np.stack([sp * n * (n + 1) * st * pi * z / rho, sp * tau * drz, cp * pi * drz], axis=1)
    Ne = np.stack([cp * n * (n + 1) * st * pi * z / rho, cp * tau * drz, -sp * pi * drz], axis=1)
    return Mo, Me, No, Ne


def _to_cartesian(v, ct, st, cp, sp):
    er = np.stack([st * cp, st * sp, ct])
    et = np.stack([ct * cp, ct * sp, -st])
    ep = np.stack([-sp, cp, np.zeros_like(cp)])
    return (v[0][None] * er + v[1][None] * et + v[2][None] * ep).T


def _sph(pts):
    pts = np.asarray(pts, dtype=np.float64)
    r = np.linalg.norm(pts, axis=1)
    ct = pts[:, 2] / r
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = np.arctan2(pts[:, 1], pts[:, 0])
    return r, ct, st, np.cos(ph), np.sin(ph)


def fields(pts, which: str, k_ext: float, k_int: float, a: float, omega: float, mu: float = 1.0,
           nmax: int | None = None):
    """E and H [npts, 3] at the points: which = 'inc' | 'sca' | 'int' (internal total field)."""
    an, bn, cn, dn = coefficients(k_ext, k_int, a, nmax)
    nmax = an.size
    r, ct, st, cp, sp = _sph(pts)
    n = np.arange(1, nmax + 1)
    En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
    if which == "int":
        k = k_int
        Mo, Me, No, Ne = _vsh(nmax, 1, k * r, ct, st, cp, sp)
        E = np.einsum("n,nkp->kp", En * cn, Mo) - 1j * np.einsum("n,nkp->kp", En * dn, Ne)
        H = (-k / (omega * mu)) * (np.einsum("n,nkp->kp", En * dn, Me) + 1j * np.einsum("n,nkp->kp", En * cn, No))
    elif which == "sca":
        k = k_ext
        Mo, Me, No, Ne = _vsh(nmax, 3, k * r, ct, st, cp, sp)
        E = 1j * np.einsum("n,nkp->kp", En * an, Ne) - np.einsum("n,nkp->kp", En * bn, Mo)
        H = (k / (omega * mu)) * (1j * np.einsum("n,nkp->kp", En * bn, No) + np.einsum("n,nkp->kp", En * an, Me))
    elif which == "inc":
        k = k_ext
        Mo, Me, No, Ne = _vsh(nmax, 1, k * r, ct, st, cp, sp)
        E = np.einsum("n,nkp->kp", En, Mo) - 1j * np.einsum("n,nkp->kp", En, Ne)
        H = (-k / (omega * mu)) * (np.einsum("n,nkp->kp", En, Me) + 1j * np.einsum("n,nkp->kp", En, No))
    else:
        raise ValueError(which)
    return _to_cartesian(E, ct, st, cp, sp), _to_cartesian(H, ct, st, cp, sp)


def efficiencies(k_ext: float, k_int: float, a: float):
    """(Q_ext, Q_sca) from the scattering coefficients."""
    an, bn, _, _ = coefficients(k_ext, k_int, a)
    n = np.arange(1, an.size + 1)
    x = k_ext * a
    qext = (2.0 / x ** 2) * np.sum((2 * n + 1) * np.real(an + bn))
    qsca = (2.0 / x ** 2) * np.sum((2 * n + 1) * (np.abs(an) ** 2 + np.abs(bn) ** 2))
    return qext, qsca


def fibonacci_sphere(n: int, radius: float):
    """n quasi-uniform points on a sphere (test points of Sec. IV-B, reading R13)."""
    k = np.arange(n)
    z = 1 - (2 * k + 1) / n
    phi = k * np.pi * (3 - np.sqrt(5))
    s = np.sqrt(1 - z * z)
    return radius * np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
