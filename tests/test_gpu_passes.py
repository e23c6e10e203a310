"""IFGF with fewer fields per octree traversal (plan field fields_per_pass; Sec. III, "IFGF for
Multiple Densities: Speed-vs-Memory Trade-off", and the Remark "On selection of IFGF approach"):
8 fields (one kernel per traversal) and 1 field (IFGF_Seq, one (density, kernel) sum per
traversal) compute the same approximation as the all-fields traversal (IFGF_Vec).

* far fields against the oracle's own IFGF (oracle/ifgf.py) at the FP32 bar of the all-fields
  kernels, 5e-5;
* the whole forward map against the all-fields FP32 plan: two FP32 evaluations of one
  approximation, which differ by rounding only; the bar 1e-5 is a fifth of the FP32 IFGF bar
  and ~100 times the unit roundoff;
* the mixed plan (FP32 IFGF kernels, FP64 fields) the same way;
* batched right-hand sides equal separate applies bit for bit;
* the plan's device bytes shrink by exactly the coefficient bytes the estimate predicts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_MEDIUM, CONFIG_SPHERE_SMALL, random_densities, sphere_problem  # noqa: E402
from oracle import cbie  # noqa: E402
from oracle import ifgf as oifgf  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def plan_of(prob, **kw):
    return lib.Plan.from_problem(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0, **kw)


def gpu_apply(plan, y):
    yd = torch.from_numpy(np.ascontiguousarray(y)).cuda()
    out = torch.empty_like(yd)
    plan.apply(yd, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("fpp", [8, 1])
def test_pass_far_fields_match_the_oracle_ifgf(fpp):
    """S and dS/dn far fields of both wavenumbers and all 8 densities against the oracle's IFGF
    (the same configuration as the all-fields FP32 check)."""
    prob = sphere_problem(0.5, 1, 6, 2.25)
    g = cbie.geometry_of(prob)
    rng = np.random.default_rng(23)
    phi = rng.standard_normal((8, prob.n)) + 1j * rng.standard_normal((8, prob.n))
    plan = plan_of(prob, far_mode=lib.IFGF_FAR_IFGF, precision=lib.IFGF_FP32, ns0=2, na0=3, leaf_size=0.11,
                   fields_per_pass=fpp)
    pd = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()
    f = torch.empty((prob.n, 28), dtype=torch.complex128, device="cuda")
    plan.fields(pd, f, lib.IFGF_PART_FAR)
    torch.cuda.synchronize()
    got = f.cpu().numpy().T
    plan.close()
    tree = oifgf.build_tree(g.x, 0.11, max(prob.k_ext, prob.k_int), 2, 3)
    ref = oifgf.ifgf_far(tree, g.x, g.n, phi.T * g.omega[:, None], prob.k_ext, prob.k_int).T
    e_s, e_d = rel(got[:16], ref[:16]), rel(got[16:], ref[16:])
    print(f"fields_per_pass {fpp}: S {e_s:.2e}, dS/dn {e_d:.2e} from the oracle's IFGF")
    assert e_s < 5e-5 and e_d < 5e-5


@pytest.mark.parametrize("prec", [lib.IFGF_FP32, lib.IFGF_MIXED])
def test_pass_forward_maps_equal_the_all_fields_map(prec):
    """The forward map of the 9,600-node sphere with 8 and 1 fields per traversal against the
    all-fields traversal of the same precision."""
    prob = CONFIG_SPHERE_MEDIUM()
    y = random_densities(prob.n, 5)
    base = dict(far_mode=lib.IFGF_FAR_IFGF, precision=prec, ns0=2, na0=3, max_krylov=10)
    pv = plan_of(prob, **base)
    ref = gpu_apply(pv, y)
    pv.close()
    for fpp in (8, 1):
        p = plan_of(prob, fields_per_pass=fpp, **base)
        out = gpu_apply(p, y)
        p.close()
        e = rel(out, ref)
        print(f"precision {prec}, fields_per_pass {fpp}: {e:.2e} from the all-fields map")
        assert e < 1e-5


def test_pass_batched_apply_equals_separate_applies():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, batch=3,
                   fields_per_pass=1)
    ys = torch.from_numpy(np.stack([random_densities(prob.n, 40 + r) for r in range(3)])).cuda()
    out = torch.empty_like(ys)
    plan.apply_batch(ys, out)
    for r in range(3):
        single = torch.empty_like(ys[r])
        plan.apply(ys[r].contiguous(), single)
        torch.cuda.synchronize()
        assert torch.equal(out[r], single), r
    plan.close()


def test_pass_plan_memory_matches_the_estimate():
    prob = CONFIG_SPHERE_SMALL(8)
    base = dict(precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, max_krylov=10)
    bytes_of = {}
    for fpp in (0, 8, 1):
        p = plan_of(prob, fields_per_pass=fpp, **base)
        bytes_of[fpp] = p.stats()["device_bytes"]
        p.close()
    est = {fpp: lib.Plan.estimate(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0, fields_per_pass=fpp,
                                  **base)["bytes_coefs"] for fpp in (0, 8, 1)}
    assert est[0] == 2 * est[8] == 16 * est[1]
    for fpp in (8, 1):
        assert bytes_of[0] - bytes_of[fpp] == est[0] - est[fpp]
