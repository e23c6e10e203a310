"""Far-field pattern of the scattered field (ifgf_far_field) through the C ABI: against the
oracle's far_field on the same solution (same Nystrom moments, FP64), against the Mie series'
far field for the GMRES solution, and reciprocity of the far-field patterns over the 64
plane-wave incidences of the batched configuration (32 Fibonacci directions x 2 polarisations):
p_b . E_inf^a(-d_b) = p_a . E_inf^b(-d_a)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_SMALL, fibonacci_directions, fibonacci_incidences, plane_wave  # noqa: E402
from inputs import random_densities  # noqa: E402
from oracle import cbie, mie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small():
    prob = CONFIG_SPHERE_SMALL(8)
    return prob, cbie.default_delta(prob)


def test_far_field_matches_oracle_and_mie(small):
    prob, delta = small
    plan = lib.Plan.from_problem(prob, delta=delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                                 precision=lib.IFGF_FP64, max_krylov=100)
    dirs = mie.fibonacci_sphere(40, 1.0)
    dd = torch.from_numpy(np.ascontiguousarray(dirs)).cuda()
    y = random_densities(prob.n, 41)
    out = torch.empty((40, 3), dtype=torch.complex128, device="cuda")
    plan.far_field(torch.from_numpy(y).cuda(), dd, out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), cbie.far_field(prob, y, dirs)) < 1e-12
    # the GMRES solution's far field against the Mie series (large-r limit, Richardson)
    x, _, _ = prob.nodes()
    inc = torch.from_numpy(np.ascontiguousarray(plane_wave(x, prob.k_ext, prob.omega))).cuda()
    ys = torch.empty((4, prob.n), dtype=torch.complex128, device="cuda")
    plan.solve(inc, ys, tol=1e-10, max_iter=100)
    plan.far_field(ys, dd, out)
    torch.cuda.synchronize()
    k = prob.k_ext
    lim = [mie.fields(R * dirs, "sca", k, prob.k_int, 0.5, prob.omega)[0] * R * np.exp(-1j * k * R)
           for R in (1600.0, 3200.0)]
    e = rel(out.cpu().numpy(), 2 * lim[1] - lim[0])
    print(f"far field vs Mie: {e:.2e}")
    assert e < 3e-3
    plan.close()


def test_far_field_reciprocity_of_the_64_incidences(small):
    prob, delta = small
    plan = lib.Plan.from_problem(prob, delta=delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                                 precision=lib.IFGF_FP64, max_krylov=100, batch=64)
    x, _, _ = prob.nodes()
    inc = torch.from_numpy(np.ascontiguousarray(fibonacci_incidences(x, prob.k_ext, prob.omega))).cuda()
    y = torch.empty((64, 4, prob.n), dtype=torch.complex128, device="cuda")
    its, rrs, st = plan.solve_batch(inc, y, tol=1e-10, max_iter=100)
    assert st == lib.IFGF_OK
    D, E1, E2 = fibonacci_directions(32)
    d = np.repeat(D, 2, axis=0)                                   # incidence 2k + i: direction d_k
    p = np.stack([E1, E2], axis=1).reshape(64, 3)                 # polarisation e_{i+1}
    ff = torch.empty((64, 64, 3), dtype=torch.complex128, device="cuda")
    plan.far_field(y, torch.from_numpy(np.ascontiguousarray(-d)).cuda(), ff)
    torch.cuda.synchronize()
    F = ff.cpu().numpy()                                          # F[a, b] = E_inf^a(-d_b)
    A = np.einsum("abk,bk->ab", F, p)                             # p_b . E_inf^a(-d_b)
    defect = np.abs(A - A.T).max() / np.abs(A).max()
    print(f"reciprocity defect over 64 x 64 incidence pairs: {defect:.2e}")
    assert defect < 3e-3
    plan.close()
