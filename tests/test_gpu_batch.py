"""Batched right-hand sides through the C ABI: one batched forward map equals
separate applies bit for bit, batched GMRES equals separate solves, and batch
limits are enforced."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_SMALL, plane_wave, random_densities  # noqa: E402
from oracle import cbie  # noqa: E402


def plan_of(prob, **kw):
    return lib.Plan.from_problem(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0, **kw)


@pytest.mark.parametrize("prec,far", [(lib.IFGF_FP32, lib.IFGF_FAR_IFGF), (lib.IFGF_FP64, lib.IFGF_FAR_DIRECT),
                                      (lib.IFGF_FP64, lib.IFGF_FAR_IFGF)])
def test_batched_apply_equals_separate_applies(prec, far):
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=prec, far_mode=far, ns0=2, na0=3, batch=4)
    ys = torch.from_numpy(np.stack([random_densities(prob.n, 30 + r) for r in range(3)])).cuda()   # [3, 4, N]
    out = torch.empty_like(ys)
    plan.apply_batch(ys, out)
    for r in range(3):
        single = torch.empty_like(ys[r])
        plan.apply(ys[r].contiguous(), single)
        torch.cuda.synchronize()
        assert torch.equal(out[r], single), r
    plan.close()


def test_batched_solve_equals_separate_solves():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, batch=3,
                   max_krylov=120)
    x, _, _ = prob.nodes()
    incs = [plane_wave(x, prob.k_ext, prob.omega, direction=d) for d in ((0, 0, 1), (1, 0, 0))]
    incs.append(np.zeros_like(incs[0]))                     # a zero right-hand side: y = 0 at once
    inc = torch.from_numpy(np.ascontiguousarray(np.stack(incs))).cuda()
    y = torch.empty((3, 4, prob.n), dtype=torch.complex128, device="cuda")
    its, rrs, st = plan.solve_batch(inc, y, tol=1e-8, max_iter=120)
    assert st == lib.IFGF_OK
    assert its[2] == 0 and rrs[2] == 0.0 and torch.count_nonzero(y[2]) == 0
    for r in range(2):
        yr = torch.empty((4, prob.n), dtype=torch.complex128, device="cuda")
        it, rr, st1 = plan.solve(inc[r].contiguous(), yr, tol=1e-8, max_iter=120)
        assert st1 == lib.IFGF_OK and it == its[r] and rr == rrs[r]
        assert torch.equal(yr, y[r])
    # the two incidences converge in different iteration counts only by chance; both reach tol
    assert max(rrs[:2]) <= 1e-8
    plan.close()


def test_batch_limits():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, batch=2, max_krylov=10)
    y = torch.zeros((3, 4, prob.n), dtype=torch.complex128, device="cuda")
    out = torch.empty_like(y)
    with pytest.raises(lib.IfgfError):
        plan.apply_batch(y, out)                            # 3 > batch
    with pytest.raises(lib.IfgfError):
        plan.apply_batch(y[:0], out[:0])                    # nrhs = 0
    plan.apply_batch(y[:2].contiguous(), out[:2])           # within the limit
    torch.cuda.synchronize()
    plan.close()


def test_uneven_batch_of_bodies_equals_separate_solves():
    from inputs import ellipsoid
    from inputs.problems import Problem
    bodies = [Problem(body=ellipsoid((0.6, 0.45, 0.35), 1), nc=8, ng=24, eps_ext=1.0, eps_int=3.0, omega=2 * np.pi),
              Problem(body=ellipsoid((0.8, 0.5, 0.5), 1), nc=8, ng=24, eps_ext=1.0, eps_int=6.0, omega=2 * np.pi),
              CONFIG_SPHERE_SMALL(8)]
    plans = [plan_of(b, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, max_krylov=150)
             for b in bodies]
    incs, ys = [], []
    for b in bodies:
        x, _, _ = b.nodes()
        incs.append(torch.from_numpy(np.ascontiguousarray(plane_wave(x, b.k_ext, b.omega)[None])).cuda())
        ys.append(torch.empty((1, 4, b.n), dtype=torch.complex128, device="cuda"))
    its, rrs, sts, st = lib.bie_solve_many(plans, incs, ys, tol=1e-5, max_iter=150)
    assert all(s in (lib.IFGF_OK, lib.IFGF_ENOCONV) for s in sts)
    assert sts[2] == lib.IFGF_OK                             # the sphere converges well inside the cap
    for i, (p, b) in enumerate(zip(plans, bodies)):
        y1 = torch.empty((4, b.n), dtype=torch.complex128, device="cuda")
        it, rr, s1 = p.solve(incs[i][0].contiguous(), y1, tol=1e-5, max_iter=150)
        assert s1 == sts[i] and it == its[i][0] and rr == rrs[i][0]   # same solve, run concurrently
        assert torch.equal(y1, ys[i][0])
    with pytest.raises(lib.IfgfError):
        lib.bie_solve_many([plans[0], plans[0]], incs[:1] * 2, ys[:1] * 2, tol=1e-6, max_iter=10)
    for p in plans:
        p.close()


def test_dipole_reciprocity_on_the_gpu():
    # point-current excitation, two right-hand sides in one batched solve on the plain FP64
    # path: the reciprocity products equal the oracle's and meet the same bound
    from test_oracle_solve import _reciprocity, oracle_solve, reciprocity_body
    prob = reciprocity_body(10)
    plan = plan_of(prob, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, batch=2, max_krylov=400)

    def gpu_solve(incs):
        inc = torch.from_numpy(np.ascontiguousarray(np.stack(incs))).cuda()
        y = torch.empty((2, 4, prob.n), dtype=torch.complex128, device="cuda")
        its, rrs, st = plan.solve_batch(inc, y, tol=1e-10, max_iter=400)
        assert st == lib.IFGF_OK
        return list(y.cpu().numpy())

    a, b = _reciprocity(prob, gpu_solve)
    ao, bo = _reciprocity(prob, oracle_solve(prob))
    assert abs(a - ao) / abs(ao) < 1e-8 and abs(b - bo) / abs(bo) < 1e-8
    assert abs(a - b) / abs(a) < 1e-2
    plan.close()
