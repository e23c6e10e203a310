"""Pins for the oracle's surface discretisation: areas, normals, surface
calculus on the sphere against closed forms."""
import numpy as np
import pytest

from inputs import cubed_sphere, ellipsoid, sphere_problem
from oracle import cbie


@pytest.fixture(scope="module")
def sphere():
    prob = sphere_problem(1.3, 2, 12, 4.0)
    return prob, cbie.geometry_of(prob)


def test_sphere_area_volume_and_closure(sphere):
    prob, g = sphere
    a = 1.3
    assert abs(g.omega.sum() - 4 * np.pi * a * a) < 1e-9 * 4 * np.pi * a * a
    assert np.abs(g.n.T @ g.omega).max() < 1e-10           # int n = 0 on a closed surface
    vol = (np.sum(g.x * g.n, 1) @ g.omega) / 3.0             # divergence theorem
    assert abs(vol - 4 / 3 * np.pi * a ** 3) < 1e-9
    assert np.allclose(g.n, g.x / a, atol=1e-12)             # outward unit normals


def test_ellipsoid_volume():
    from inputs.problems import Problem
    prob = Problem(body=ellipsoid((1.0, 0.7, 0.4), 2), nc=12, ng=24, eps_ext=1, eps_int=2)
    g = cbie.geometry_of(prob)
    vol = (np.sum(g.x * g.n, 1) @ g.omega) / 3.0
    assert abs(vol - 4 / 3 * np.pi * 1.0 * 0.7 * 0.4) < 1e-8


def test_frame_is_orthonormal_and_tangent(sphere):
    _, g = sphere
    assert np.allclose(np.sum(g.t1 * g.t2, 1), 0, atol=1e-14)
    assert np.allclose(np.sum(g.t1 * g.n, 1), 0, atol=1e-13)
    assert np.allclose(np.linalg.norm(g.t2, axis=1), 1, atol=1e-14)


def test_surface_gradient_of_linear_function(sphere):
    _, g = sphere
    c = np.array([0.3, -1.1, 0.7])
    grad = cbie.surface_grad(g.x @ c, g)
    PTc = c - (g.n @ c)[:, None] * g.n
    assert np.abs(grad - PTc).max() < 1e-7


def test_surface_divergence_closed_forms(sphere):
    _, g = sphere
    a = 1.3
    c = np.array([0.3, -1.1, 0.7])
    # div_G (P_T c) = -2 (c.n)/a on a sphere of radius a (Laplace-Beltrami of a degree-1 harmonic)
    PTc = c - (g.n @ c)[:, None] * g.n
    assert np.abs(cbie.surface_div(PTc, g) + 2 * (g.n @ c) / a).max() < 1e-6
    # rotational fields n x c are divergence free
    assert np.abs(cbie.surface_div(np.cross(g.n, c), g)).max() < 1e-6
    # Laplace-Beltrami of the l = 2 harmonic x y: -6 x y / a^2
    f = g.x[:, 0] * g.x[:, 1]
    lap = cbie.surface_div(cbie.surface_grad(f, g), g)
    assert np.abs(lap + 6 * f / a ** 2).max() < 1e-5


def test_node_layout_contract():
    # node l = j + Nc i + p Nc^2 sits at (u_i, u_j) of patch p (Eq. mesh_pts_l)
    prob = sphere_problem(1.0, 1, 6, 2.0)
    x, xu, xv = prob.nodes()
    u = cbie.cheb_nodes(6)
    body = cubed_sphere(1.0, 1)
    p, i, j = 4, 2, 5
    xe, _, _ = body.eval(p, np.array(u[i]), np.array(u[j]))
    assert np.allclose(x[j + 6 * i + 36 * p], xe)
