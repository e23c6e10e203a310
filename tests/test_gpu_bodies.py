"""GPU parity on non-spherical bodies (ellipsoid, star-shaped body): the
plain FP64 path against the oracle's CBIE forward map on whole sampled
patches, and the IFGF forward map against the plain FP64 path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import ellipsoid, random_densities, star_body  # noqa: E402
from inputs.problems import Problem  # noqa: E402
from oracle import cbie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rowmax(a, b):
    """Largest per-node relative difference over a node's 4 outputs ([4, rows] arrays)."""
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


def bodies():
    rng = np.random.default_rng(42)
    coeffs = {(l, m): 0.03 * rng.standard_normal() for l in range(1, 5) for m in range(-l, l + 1)}
    return {
        "ellipsoid": Problem(body=ellipsoid((1.1, 0.8, 0.55), 2), nc=8, ng=24, eps_ext=1.0, eps_int=3.0,
                             omega=2 * np.pi),
        "star": Problem(body=star_body(0.9, coeffs, 2), nc=8, ng=24, eps_ext=1.0, eps_int=6.0, omega=2 * np.pi),
    }


def gpu_apply(plan, y):
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = torch.empty_like(yd)
    plan.apply(yd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("name", ["ellipsoid", "star"])
def test_body_fp64_plain_path_matches_oracle(name):
    prob = bodies()[name]
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0)
    g = cbie.geometry_of(prob)
    plan = lib.Plan.from_problem(prob, delta=qp.delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                                 precision=lib.IFGF_FP64)
    y = random_densities(prob.n, 8)
    out = gpu_apply(plan, y)
    phi = cbie.densities(y, g)
    npp = prob.nc ** 2
    for p in (0, 9, 17):
        rows = np.arange(p * npp, (p + 1) * npp)
        K, _ = cbie.kernel_rows(prob, g, rows, qp)
        S = np.zeros((2, 8, prob.n), dtype=complex)
        D = np.zeros((2, 6, prob.n), dtype=complex)
        Sr, Dr = cbie.scalar_fields(K, phi)
        S[:, :, rows] = Sr
        D[:, :, rows] = Dr
        ref = cbie.combine(prob, g, y, S, D)[:, rows]
        print(f"{name} patch {p}: rel l2 {rel(out[:, rows], ref):.2e}, worst row {rowmax(out[:, rows], ref):.2e}")
        assert rel(out[:, rows], ref) < 1e-12, (name, p)
        assert rowmax(out[:, rows], ref) < 2e-11, (name, p)
    # FP32 plain path: same operator in single precision
    plan32 = lib.Plan.from_problem(prob, delta=qp.delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                                   precision=lib.IFGF_FP32)
    assert rel(gpu_apply(plan32, y), out) < 1e-5
    plan.close()
    plan32.close()


@pytest.mark.parametrize("name", ["ellipsoid", "star"])
def test_body_ifgf_vs_plain(name):
    prob = bodies()[name]
    delta = cbie.default_delta(prob)
    y = random_densities(prob.n, 9)
    pd = lib.Plan.from_problem(prob, delta=delta, far_mode=lib.IFGF_FAR_DIRECT, precision=lib.IFGF_FP64)
    ref = gpu_apply(pd, y)
    pd.close()
    for prec in (lib.IFGF_FP64, lib.IFGF_FP32):
        pi = lib.Plan.from_problem(prob, delta=delta, far_mode=lib.IFGF_FAR_IFGF, precision=prec, ns0=2, na0=3,
                                   leaf_size=0.15)
        assert pi.stats()["levels"] >= 4
        e = rel(gpu_apply(pi, y), ref)
        assert e < 1e-4, (name, prec, e)
        pi.close()
