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


def test_gaussian_beam_closed_forms():
    """Paraxial Gaussian beam: amplitude exp(-rho^2/w0^2) with zero phase in the focal plane,
    on-axis modulus 1/sqrt(1 + (xi/z_R)^2) and phase k xi - atan(xi/z_R) (Gouy), power
    conserved across planes (|E|^2 integrated over rho is pi w0^2 / 2), H = (k/(omega mu)) d x E."""
    from inputs import gaussian_beam
    omega, eps = 2 * np.pi, 2.1
    k = omega * np.sqrt(eps)
    w0, f = 0.2, np.array([-10.5, 0.0, 0.0])
    zr = 0.5 * k * w0 * w0
    rho = np.linspace(0.0, 0.5, 11)
    pts = f + np.stack([np.zeros_like(rho), rho / np.sqrt(2), rho / np.sqrt(2)], axis=1)
    F = gaussian_beam(pts, k, omega, focus=f, waist=w0)
    assert np.allclose(F[1], np.exp(-rho ** 2 / w0 ** 2), rtol=0, atol=1e-14)
    assert np.abs(F[[0, 2, 3, 4]]).max() == 0.0
    assert np.allclose(F[5], (k / omega) * F[1], rtol=0, atol=1e-14)
    xi = np.array([-3.0, -0.4, 0.1, 0.7, 5.0])
    F = gaussian_beam(f + xi[:, None] * np.array([1.0, 0.0, 0.0]), k, omega, focus=f, waist=w0)
    assert np.allclose(np.abs(F[1]), 1.0 / np.sqrt(1.0 + (xi / zr) ** 2), rtol=1e-13)
    ph = np.angle(F[1] * np.exp(-1j * (k * xi - np.arctan(xi / zr))))
    assert np.abs(ph).max() < 1e-12
    # transverse power at two planes (radial quadrature over 0 <= rho <= 8 w(xi))
    for x0 in (0.0, 1.3):
        w = w0 * np.sqrt(1 + (x0 / zr) ** 2)
        r, wr = np.polynomial.legendre.leggauss(200)
        r = 4.0 * w * (r + 1.0)
        wr = 4.0 * w * wr
        P = gaussian_beam(f + np.stack([np.full_like(r, x0), r, 0 * r], axis=1), k, omega, focus=f, waist=w0)
        power = np.sum(wr * 2 * np.pi * r * np.abs(P[1]) ** 2)
        assert abs(power / (np.pi * w0 ** 2 / 2) - 1.0) < 1e-10


def test_gaussian_beam_satisfies_paraxial_equation():
    """The envelope u = E_y e^{-i k xi} solves 2 i k du/dxi + d2u/dy2 + d2u/dz2 = 0."""
    from inputs import gaussian_beam
    omega = 2 * np.pi
    k = omega * np.sqrt(2.1)
    f = np.array([-10.5, 0.0, 0.0])
    rng = np.random.default_rng(4)
    pts = f + rng.uniform([-1.0, -0.2, -0.2], [1.0, 0.2, 0.2], size=(16, 3))
    u = lambda p: gaussian_beam(p, k, omega, focus=f, waist=0.2)[1] * np.exp(-1j * k * (p[:, 0] - f[0]))
    h = 1e-4
    e = np.eye(3) * h
    dxi = (u(pts + e[0]) - u(pts - e[0])) / (2 * h)
    lap = sum((u(pts + e[i]) - 2 * u(pts) + u(pts - e[i])) / h ** 2 for i in (1, 2))
    res = 2j * k * dxi + lap
    assert np.abs(res).max() / np.abs(lap).max() < 1e-5


def test_rounded_bar_closed_surface_volume_and_orientation():
    """The waveguide bar closes (sum of n dA = 0), encloses the analytic volume
    2(A - L) * 4BC G(9/8)^2/G(5/4) + 8LBC G(9/8)^3/G(11/8) of a rounded-rectangle prism with
    two superellipsoidal half ends, has outward normals, and its complex-step derivatives
    agree with centred differences."""
    from math import gamma
    from inputs.geometry import rounded_bar
    A, B, C, L = 10.0, 0.15, 0.07, 0.15
    body = rounded_bar((A, B, C), L, 0.12)
    t, w = np.polynomial.legendre.leggauss(16)
    U, V = np.meshgrid(t, t, indexing="ij")
    W = w[:, None] * w[None, :]
    vol, ntot = 0.0, np.zeros(3)
    for p in range(body.num_patches):
        x, xu, xv = body.eval(p, U, V)
        n = np.cross(xu, xv)
        vol += np.sum(W * np.sum(x * n, -1)) / 3
        ntot += np.sum(W[..., None] * n, axis=(0, 1))
        r = x.copy()
        r[..., 0] = x[..., 0] - np.clip(x[..., 0], -(A - L), A - L)
        assert (np.sum(r * n, -1) > 0).all(), p
        if p % 97 == 0:
            h = 1e-6
            xp, _, _ = body.eval(p, U + h, V)
            xm, _, _ = body.eval(p, U - h, V)
            assert np.abs((xp - xm) / (2 * h) - xu).max() < 1e-7 * np.abs(xu).max()
    exact = 2 * (A - L) * 4 * B * C * gamma(1.125) ** 2 / gamma(1.25) + 8 * L * B * C * gamma(1.125) ** 3 / gamma(1.375)
    assert abs(vol / exact - 1.0) < 1e-10
    assert np.abs(ntot).max() < 1e-13


def test_waveguide_bar_sizes():
    from inputs import waveguide_bar
    prob = waveguide_bar(0.2)
    assert prob.k_int / prob.k_ext == np.sqrt(12.1 / 2.1)
    assert abs(prob.k_ext - 2 * np.pi * np.sqrt(2.1)) < 1e-14
    x, _, _ = prob.nodes()
    assert np.allclose(x.min(0), -x.max(0), atol=1e-12)
    ext = x.max(0)
    assert 9.99 < ext[0] <= 10.0 + 1e-12 and 0.149 < ext[1] <= 0.15 + 1e-12 and 0.069 < ext[2] <= 0.07 + 1e-12
    w = x / np.array([1.0, 0.15, 0.07])
    straight = np.abs(x[:, 0]) <= 9.85
    assert np.abs(w[straight, 1] ** 8 + w[straight, 2] ** 8 - 1.0).max() < 1e-12
    xe = (np.abs(x[~straight, 0]) - 9.85) / 0.15
    assert np.abs(xe ** 8 + w[~straight, 1] ** 8 + w[~straight, 2] ** 8 - 1.0).max() < 1e-12


def test_rounded_bar_arguments_and_exponent():
    """The bar's cross-section follows the chosen even exponent, and invalid shapes are
    refused."""
    import pytest
    from inputs import waveguide_bar
    from inputs.geometry import rounded_bar
    with pytest.raises(ValueError):
        rounded_bar((1.0, 0.15, 0.07), 0.15, 0.2, exponent=3)
    with pytest.raises(ValueError):
        rounded_bar((0.1, 0.15, 0.07), 0.15, 0.2)
    for e in (2, 4):
        prob = waveguide_bar(0.2, half_lengths=(1.0, 0.15, 0.07), exponent=e)
        x, _, _ = prob.nodes()
        straight = np.abs(x[:, 0]) <= 0.85
        w = x[straight] / np.array([1.0, 0.15, 0.07])
        assert np.abs(np.abs(w[:, 1]) ** e + np.abs(w[:, 2]) ** e - 1.0).max() < 1e-12
