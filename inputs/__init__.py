"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package only describes the scattering problem: surface
parametrisations (and their exact parametric derivatives) sampled at
caller-chosen parameter points, the incident field, material constants and
random densities.  It contains none of the solver's arithmetic (no
quadrature weights, kernels, interpolation or operator algebra), so both the
CPU oracle and the GPU library can consume it without sharing code.
"""
from .geometry import (Body, cubed_sphere, ellipsoid, star_body, superellipsoid_bar, rounded_bar,
                       open_cheb_nodes, sample_body)
from .problems import (Problem, sphere_problem, CONFIG_SPHERE_SMALL, CONFIG_SPHERE_MEDIUM,
                       random_densities, plane_wave, fibonacci_directions, fibonacci_incidences, ellipsoid_batch,
                       dipole_field, star_batch, gaussian_beam, waveguide_bar)

__all__ = ["fibonacci_directions", "gaussian_beam", "waveguide_bar", "star_batch", "dipole_field", "ellipsoid_batch", "fibonacci_incidences", "Body", "cubed_sphere", "ellipsoid", "star_body", "superellipsoid_bar", "rounded_bar",
           "open_cheb_nodes", "sample_body", "Problem", "sphere_problem",
           "CONFIG_SPHERE_SMALL", "CONFIG_SPHERE_MEDIUM", "random_densities", "plane_wave"]
