"""The waveguide bar: a 20 x 0.3 x 0.14 (vacuum wavelengths) silicon-like bar,
eps 12.1 in eps 2.1, at patch side 0.2 (610 patches x 10 x 10 nodes, N = 61,000),
planned with the point-count leaf rule (at most 64 points per leaf box).

The plain FP64 path is compared with the oracle on whole sampled patches (a
straight-side patch and an end patch); the FP32 IFGF forward map with the
FP64 direct far sum on sampled patches (ifgf_apply_direct_patches), which is
itself checked against the full FP64 direct forward map (bit for bit); and a
GMRES solve for a Gaussian-beam excitation on a shorter bar by its true
residual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import gaussian_beam, random_densities, waveguide_bar  # noqa: E402
from oracle import cbie  # noqa: E402

LEAF_PTS = 64


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def bar():
    prob = waveguide_bar(0.2)
    x, _, _ = prob.nodes()
    xp = x.reshape(prob.num_patches, prob.nc ** 2, 3)
    diam = [np.linalg.norm(xp[p][:, None] - xp[p][None], axis=-1).max() for p in range(prob.num_patches)]
    return prob, 0.6 * float(np.median(diam))


def make(prob, delta, precision, far, **kw):
    return lib.Plan.from_problem(prob, delta=delta, n_beta=48, cov_d=4.0, precision=precision, far_mode=far,
                                 ns0=2, na0=3, max_leaf_pts=LEAF_PTS, **kw)


def oracle_rows(prob, delta, y, rows):
    qp = cbie.QuadParams(delta=delta, n_beta=48, cov_d=4.0)
    g = cbie.geometry_of(prob)
    K, _ = cbie.kernel_rows(prob, g, rows, qp)
    S = np.zeros((2, 8, prob.n), dtype=complex)
    D = np.zeros((2, 6, prob.n), dtype=complex)
    S[:, :, rows], D[:, :, rows] = cbie.scalar_fields(K, cbie.densities(y, g))
    return cbie.combine(prob, g, y, S, D)[:, rows]


def test_bar_fp64_direct_matches_oracle_on_sampled_patches(bar):
    """A straight-side patch to 1e-12.  On the end patches the normal-derivative weights
    lose digits to the body's coordinates (|x| ~ 10 against near distances ~1e-3, where
    n.(x - y) is second order in |x - y|): the oracle itself moves by ~2e-11 when the same
    bar is translated by 9.85 along x (an exact symmetry of the operator), so there the bar
    is four times that measured translation change."""
    prob, delta = bar
    y = random_densities(prob.n, 81)
    plan = make(prob, delta, lib.IFGF_FP64, lib.IFGF_FAR_DIRECT, max_krylov=10)
    yd = torch.from_numpy(y).cuda()
    out = torch.empty_like(yd)
    plan.apply(yd, out)
    out = out.cpu().numpy()
    plan.close()
    npp = prob.nc ** 2
    end_patch = [k for k, p in enumerate(prob.body.patches) if p[0] == 1][0]
    rows = np.arange(3 * npp, 4 * npp)
    assert rel(out[:, rows], oracle_rows(prob, delta, y, rows)) < 1e-12
    rows = np.arange(end_patch * npp, (end_patch + 1) * npp)
    ref = oracle_rows(prob, delta, y, rows)
    moved = waveguide_bar(0.2, center=(-9.85, 0.0, 0.0))
    floor = rel(oracle_rows(moved, delta, y, rows), ref)
    assert 1e-13 < floor < 1e-10
    assert rel(out[:, rows], ref) < max(1e-12, 4 * floor), (rel(out[:, rows], ref), floor)


def nodes_of(prob, pats):
    npp = prob.nc ** 2
    return torch.from_numpy((np.asarray(pats)[:, None] * npp + np.arange(npp)[None]).ravel().astype(np.int64)).cuda()


def test_direct_patches_equal_the_full_direct_map(bar):
    prob, delta = bar
    plan = make(prob, delta, lib.IFGF_FP64, lib.IFGF_FAR_DIRECT, max_krylov=10)
    y = torch.from_numpy(random_densities(prob.n, 82)).cuda()
    full = torch.empty_like(y)
    part = torch.empty_like(y)
    plan.apply(y, full)
    pats = np.sort(np.random.default_rng(83).choice(prob.num_patches, size=37, replace=False))
    plan.apply_direct_patches(y, part, pats)
    r = nodes_of(prob, pats)
    # same block origins and summation order as the full FP64 map: equal to the bit
    assert torch.equal(full[:, r], part[:, r])
    plan.close()


def test_direct_patches_rejects_invalid_lists(bar):
    prob, delta = bar
    plan = make(prob, delta, lib.IFGF_FP32, lib.IFGF_FAR_IFGF, max_krylov=10)
    y = torch.from_numpy(random_densities(prob.n, 84)).cuda()
    out = torch.empty_like(y)
    for pats in ([1, 2, 2], [0, prob.num_patches], [-1], []):
        with pytest.raises(lib.IfgfError) as e:
            plan.apply_direct_patches(y, out, pats)
        assert e.value.status == lib.IFGF_EINVAL
    plan.apply(y, out)           # the plan stays usable
    torch.cuda.synchronize()
    plan.close()


def test_bar_ifgf_fp32_matches_direct_on_sampled_patches(bar):
    """The FP32 IFGF forward map against the same plan with an FP64 direct far sum on
    40 sampled patches (4,000 rows)."""
    prob, delta = bar
    plan = make(prob, delta, lib.IFGF_FP32, lib.IFGF_FAR_IFGF, max_krylov=10)
    st = plan.stats()
    assert st["levels"] >= 9      # the point-count rule deepens the tree past the wavelength rule (8)
    y = torch.from_numpy(random_densities(prob.n, 85)).cuda()
    out = torch.empty_like(y)
    ref = torch.empty_like(y)
    plan.apply(y, out)
    pats = np.sort(np.random.default_rng(86).choice(prob.num_patches, size=40, replace=False))
    plan.apply_direct_patches(y, ref, pats)
    r = nodes_of(prob, pats)
    err = float(torch.linalg.norm(out[:, r] - ref[:, r]) / torch.linalg.norm(ref[:, r]))
    plan.close()
    assert err < 1e-4, err


def test_short_bar_gaussian_beam_solve_true_residual():
    """GMRES on a 2.5-long bar (eps 12.1 in 2.1, patch side 0.2, 8,800 nodes) with the
    right scaling, tolerance 1e-5.  GMRES alone stops on its Arnoldi estimate, which the FP32
    map's rounding (amplified by the Krylov combination) undercuts: the residual the FP32 map
    itself gives stays a few times higher.  Refinement against the FP32 map reports the residual
    it forms and stops where that map's rounding floor is (about 3e-5 here: ENOCONV, honestly).
    Mixed-precision refinement, residuals formed by the FP64 IFGF map of the same body and
    corrections solved with the FP32 map, reaches the tolerance against the FP64 map.  (The
    iteration count grows about linearly with the bar's length: 83 at length 2.5, 148 at 5,
    about 300 at 10.)"""
    prob = waveguide_bar(0.2, half_lengths=(1.25, 0.15, 0.07))
    x, _, _ = prob.nodes()
    xp = x.reshape(prob.num_patches, prob.nc ** 2, 3)
    delta = 0.6 * float(np.median([np.linalg.norm(xp[p][:, None] - xp[p][None], axis=-1).max()
                                   for p in range(prob.num_patches)]))
    inc = torch.from_numpy(np.ascontiguousarray(
        gaussian_beam(x, prob.k_ext, prob.omega, focus=(-1.75, 0.0, 0.0), waist=0.2)[None])).cuda()
    p64 = make(prob, delta, lib.IFGF_FP64, lib.IFGF_FAR_IFGF, max_krylov=10)
    b = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
    p64.rhs(inc, b)

    def resid(plan, y):
        Ay = torch.empty_like(y)
        plan.apply_batch(y, Ay)
        return float(torch.linalg.norm(b - Ay) / torch.linalg.norm(b))

    res = {}
    for name, refine, other in (("gmres", 0, None), ("own", 3, None), ("fp64", 3, p64)):
        plan = make(prob, delta, lib.IFGF_FP32, lib.IFGF_FAR_IFGF, max_krylov=200, gmres_scaling=1,
                    refine=refine)
        if other is not None:
            plan.set_residual(other)
        y = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
        its, rrs, st = plan.solve_batch(inc, y, tol=1e-5, max_iter=200)
        res[name] = (int(its[0]), float(rrs[0]), int(st), resid(plan, y), resid(p64, y))
        plan.close()
        print(f"short bar, {name}: {its[0]} iterations, reported {rrs[0]:.2e}, status {st}, "
              f"residual of the FP32 map {res[name][3]:.2e}, of the FP64 map {res[name][4]:.2e}")
    p64.close()
    its0, est0, st0, own0, _ = res["gmres"]
    assert st0 == lib.IFGF_OK and est0 <= 1e-5 and its0 <= 150 and own0 < 1e-4, res
    # refinement reports what it formed: the FP32 map's residual, OK exactly when it is <= tol
    its1, rep1, st1, own1, _ = res["own"]
    assert abs(rep1 - own1) <= 1e-9 * own1 and own1 <= own0, res
    assert (st1 == lib.IFGF_OK) == (rep1 <= 1e-5), res
    # mixed-precision refinement reaches the tolerance against the FP64 map
    its2, rep2, st2, _, r64 = res["fp64"]
    assert st2 == lib.IFGF_OK and abs(rep2 - r64) <= 1e-9 * r64 and r64 <= 1e-5, res
    assert its2 <= its0 + 150, res

