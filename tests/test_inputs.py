"""Pins of the synthetic incident fields: they satisfy Maxwell's equations in
the exterior medium (checked by centred differences), independently of the
solver."""
import numpy as np

from inputs import dipole_field, plane_wave


def _curl(f, x, h):
    """curl of f(points [M,3]) -> [3, M] complex by centred differences."""
    def d(a, b):   # d f_a / d x_b
        e = np.zeros(3)
        e[b] = h
        return (f(x + e)[a] - f(x - e)[a]) / (2 * h)
    return np.stack([d(2, 1) - d(1, 2), d(0, 2) - d(2, 0), d(1, 0) - d(0, 1)])


def _check_maxwell(field, k, omega, mu, eps, pts):
    h = 1e-4
    E = lambda p: field(p)[:3]
    H = lambda p: field(p)[3:]
    cE, cH = _curl(E, pts, h), _curl(H, pts, h)
    f = field(pts)
    r1 = np.abs(cE - 1j * omega * mu * f[3:]).max() / np.abs(omega * mu * f[3:]).max()
    r2 = np.abs(cH + 1j * omega * eps * f[:3]).max() / np.abs(omega * eps * f[:3]).max()
    return r1, r2


def test_dipole_field_satisfies_maxwell():
    rng = np.random.default_rng(3)
    omega, eps, mu = 2 * np.pi, 1.0, 1.0
    k = omega * np.sqrt(eps * mu)
    r0, j = np.array([0.3, -0.2, 1.5]), np.array([0.4, 1.0 - 0.5j, 0.2j])
    pts = rng.uniform(-1.0, 1.0, size=(20, 3))          # at least ~0.4 wavelengths from the source
    r1, r2 = _check_maxwell(lambda p: dipole_field(p, k, omega, r0, j, mu), k, omega, mu, eps, pts)
    assert r1 < 1e-6 and r2 < 1e-6
    # far from the source the field is transverse and |E| = (omega mu / k) |H| = |H| here
    far = np.array([[0.3, -0.2, 1.5 + 40.0]])
    f = dipole_field(far, k, omega, r0, np.array([1.0, 0.0, 0.0]), mu)
    assert abs(np.linalg.norm(f[:3]) / np.linalg.norm(f[3:]) - 1.0) < 1e-2


def test_plane_wave_satisfies_maxwell():
    rng = np.random.default_rng(4)
    omega, eps, mu = 2 * np.pi, 2.0, 1.0
    k = omega * np.sqrt(eps * mu)
    d = np.array([1.0, 2.0, -0.5]) / np.linalg.norm([1.0, 2.0, -0.5])
    p = np.cross(d, [0.0, 0.0, 1.0])
    p /= np.linalg.norm(p)
    pts = rng.uniform(-1.0, 1.0, size=(10, 3))
    r1, r2 = _check_maxwell(lambda q: plane_wave(q, k, omega, mu, direction=d, polarization=p), k, omega, mu,
                            eps, pts)
    assert r1 < 1e-6 and r2 < 1e-6
