"""Full-size parity on the 153,600-node sphere (radius 4 wavelengths, eps_r
2.25, 600 patches x 16 x 16 nodes; 614,400 unknowns): the plain FP64 path
against the oracle on whole sampled patches, and the FP32 IFGF forward map
against the FP32 direct far sum.

Bar of the FP64 comparison: 5e-12.  This body uses a 32 x 32 oversampled
geometry grid per patch; the self-patch dG/dn weights depend on the
curvature of that interpolant, whose second derivatives next to a patch edge
carry ~Ng^4 times the rounding of its Chebyshev coefficients (GPU and oracle
form the coefficients in different summation orders).  Measured 2.0e-12;
the 24 x 24 grids of the other parity bodies stay below 1e-12."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import random_densities, sphere_problem  # noqa: E402
from oracle import cbie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def big():
    prob = sphere_problem(4.0, 10, 16, 2.25)
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0)
    return prob, qp


def apply(plan, y):
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = torch.empty_like(yd)
    plan.apply(yd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_full_size_fp64_direct_matches_oracle_on_sampled_patches(big):
    prob, qp = big
    g = cbie.geometry_of(prob)
    y = random_densities(prob.n, 71)
    plan = lib.Plan.from_problem(prob, delta=qp.delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                                 precision=lib.IFGF_FP64, max_krylov=10)
    out = apply(plan, y)
    plan.close()
    npp = prob.nc ** 2
    phi = cbie.densities(y, g)
    for p in (0, 417):
        rows = np.arange(p * npp, (p + 1) * npp)
        K, _ = cbie.kernel_rows(prob, g, rows, qp)
        S = np.zeros((2, 8, prob.n), dtype=complex)
        D = np.zeros((2, 6, prob.n), dtype=complex)
        S[:, :, rows], D[:, :, rows] = cbie.scalar_fields(K, phi)
        assert rel(out[:, rows], cbie.combine(prob, g, y, S, D)[:, rows]) < 5e-12, p


def test_full_size_ifgf_fp32_matches_direct_fp32(big):
    prob, qp = big
    y = random_densities(prob.n, 72)
    outs = []
    for far in (lib.IFGF_FAR_IFGF, lib.IFGF_FAR_DIRECT):
        plan = lib.Plan.from_problem(prob, delta=qp.delta, n_beta=48, cov_d=4.0, far_mode=far,
                                     precision=lib.IFGF_FP32, ns0=2, na0=3, max_krylov=10)
        outs.append(apply(plan, y))
        plan.close()
    assert rel(outs[0], outs[1]) < 1e-4
