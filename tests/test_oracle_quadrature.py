"""Pins for the oracle's 1D building blocks: Chebyshev grid, Fejer rule,
values-to-coefficients map, differentiation, the clustering change of variables.

Each pin is a closed form or an exactness property, not a re-typed formula.
"""
import os

import numpy as np
import pytest

from oracle import cbie

NS = [2, 3, 5, 8, 10, 16, 24]


@pytest.mark.parametrize("n", NS)
def test_fejer_integrates_chebyshev_exactly(n):
    # int_{-1}^{1} T_k = 2/(1-k^2) for even k, 0 for odd k; exact for k < n (Eq. fejer_weighs)
    x = cbie.cheb_nodes(n)
    w = cbie.fejer_weights(n)
    T = cbie.cheb_T(x, n)
    for k in range(n):
        exact = 0.0 if k % 2 else 2.0 / (1.0 - k * k)
        assert abs(w @ T[:, k] - exact) < 1e-13
    assert np.all(w > 0)


def test_fejer_monomials_and_sum():
    w = cbie.fejer_weights(12)
    x = cbie.cheb_nodes(12)
    assert abs(w.sum() - 2.0) < 1e-14
    assert abs(w @ x ** 10 - 2.0 / 11.0) < 1e-13
    # a non-polynomial integrand converges spectrally
    w40, x40 = cbie.fejer_weights(40), cbie.cheb_nodes(40)
    assert abs(w40 @ np.exp(x40) - (np.e - 1 / np.e)) < 1e-14


@pytest.mark.parametrize("n", NS)
def test_values_to_coefficients_exact_on_polynomials(n):
    rng = np.random.default_rng(n)
    c = rng.standard_normal(n)
    x = cbie.cheb_nodes(n)
    f = cbie.cheb_T(x, n) @ c
    assert np.allclose(cbie.vals_to_coefs(n) @ f, c, atol=1e-13)
    # evaluation off the grid reproduces the polynomial
    xs = np.linspace(-1, 1, 7)
    assert np.allclose(cbie.cheb_T(xs, n) @ (cbie.vals_to_coefs(n) @ f),
                       np.polynomial.chebyshev.chebval(xs, c), atol=1e-12)


@pytest.mark.parametrize("n", [3, 6, 10, 16])
def test_differentiation_exact_on_polynomials(n):
    x = cbie.cheb_nodes(n)
    p = np.polynomial.Polynomial(np.arange(1.0, n + 1.0) / n)   # degree n-1
    assert np.allclose(cbie.cheb_diff(n) @ p(x), p.deriv()(x), atol=1e-10)


def test_cov_endpoints_monotone_and_mass():
    tau = cbie.cheb_nodes(64)
    wt = cbie.fejer_weights(64)
    for alpha in [-1.0, -0.73, 0.0, 0.31, 0.999, 1.0]:
        xi, mu = cbie.change_of_variables(alpha, np.array([-1.0, 0.0, 1.0]), 4.0)
        assert abs(xi[0] + 1) < 1e-14 and abs(xi[2] - 1) < 1e-14
        if abs(alpha) < 1:
            assert abs(xi[1] - alpha) < 1e-15 and mu[1] == 0.0
        xs, ms = cbie.change_of_variables(alpha, np.linspace(-1, 1, 401), 4.0)
        assert np.all(np.diff(xs) >= -1e-15)
        assert np.all(ms >= 0)
        # the Fejer rule on dxi/dtau integrates 1 over [-1, 1] (Eqs. cov, int_moments_1)
        _, m64 = cbie.change_of_variables(alpha, tau, 4.0)
        assert abs(wt @ m64 - 2.0) < 1e-6
        # and a smooth function of xi
        x64, _ = cbie.change_of_variables(alpha, tau, 4.0)
        assert abs(wt @ (np.cos(x64) * m64) - 2 * np.sin(1.0)) < 1e-6


@pytest.mark.parametrize("d", [2.0, 3.0, 4.0, 6.0])
def test_cov_clusters_to_order_d(d):
    # w has vanishing derivatives up to order d-1 at the end points (Eq. mk_cov_1):
    # xi(tau) - alpha ~ C |tau|^d near tau = 0
    t = np.array([1e-3, 2e-3])
    xi, _ = cbie.change_of_variables(0.0, t, d)
    ratio = xi[1] / xi[0]
    assert abs(np.log2(ratio) - d) < 0.05


def _materials():
    path = os.path.join(os.path.dirname(__file__), "golden", "materials_sec4.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows.append((name, *map(float, vals)))
    return rows


@pytest.mark.parametrize("row", _materials(), ids=lambda r: r[0])
def test_wavenumber_convention_matches_printed_examples(row):
    # kappa_s = omega sqrt(eps_s mu_s): the printed interior wavenumbers follow
    # from the printed exterior ones to the printed digits (reading R3).
    _, ee, me, ke, ei, mi, ki_printed = row
    omega = ke / np.sqrt(ee * me)
    assert abs(omega * np.sqrt(ei * mi) - ki_printed) < 0.015
