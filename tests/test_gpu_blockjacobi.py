"""The block-Jacobi right preconditioner through the C ABI: its blocks are the inverses of the
oracle's diagonal blocks (the operator restricted to one patch's unknowns), flexible GMRES with
it reaches the unpreconditioned solution in fewer iterations on a high-contrast body, and a
network with zero output weights on top of it changes nothing while its training targets become
the error the block-Jacobi product leaves."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import plane_wave, random_densities, sphere_problem  # noqa: E402
from oracle import cbie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sphere_e8():
    # radius lambda/2, eps_r 8, 6 patches x 6 x 6 nodes: 864 unknowns, 6 blocks of 144
    prob = sphere_problem(0.5, 1, 6, 8.0)
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0)
    A = cbie.assemble(cbie.build_operator(prob, qp))
    return prob, qp, A


def plan_of(prob, qp, **kw):
    return lib.Plan.from_problem(prob, delta=qp.delta, n_beta=qp.n_beta, cov_d=qp.cov_d, gs_iters=qp.gs_iters,
                                 **kw)


def patch_index(prob):
    N, npp = prob.n, prob.nc ** 2
    return [np.concatenate([k * N + np.arange(p * npp, (p + 1) * npp) for k in range(4)])
            for p in range(prob.num_patches)]


def test_block_jacobi_inverts_the_oracle_diagonal_blocks(sphere_e8):
    prob, qp, A = sphere_e8
    plan = plan_of(prob, qp, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, max_krylov=10, batch=4)
    plan.block_jacobi()
    rng = np.random.default_rng(5)
    u = rng.standard_normal(A.shape[0]) + 1j * rng.standard_normal(A.shape[0])
    v = np.zeros_like(u)
    for ix in patch_index(prob):
        v[ix] = A[np.ix_(ix, ix)] @ u[ix]
    vd = torch.from_numpy(v.reshape(1, 4, prob.n)).cuda()
    zd = torch.empty_like(vd)
    plan.precond_apply(vd, zd)
    torch.cuda.synchronize()
    z = zd.cpu().numpy().reshape(-1)
    plan.close()
    err = rel(z, u)
    print(f"block-Jacobi inverse vs the oracle's diagonal blocks: {err:.2e}")
    # the plain FP64 operator equals the oracle's to ~1e-12; the blocks' condition numbers (~1e2)
    assert err < 1e-9, err


def test_block_jacobi_solve_matches_plain_gmres_in_fewer_iterations(sphere_e8):
    prob, qp, _ = sphere_e8
    x, _, _ = prob.nodes()
    inc = torch.from_numpy(np.ascontiguousarray(plane_wave(x, prob.k_ext, prob.omega)[None])).cuda()
    plain = plan_of(prob, qp, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, max_krylov=400, gmres_scaling=1)
    y0 = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
    it0, rr0, st0 = plain.solve_batch(inc, y0, tol=1e-8, max_iter=400)
    plain.close()
    bj = plan_of(prob, qp, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, max_krylov=400)
    bj.block_jacobi()
    y1 = torch.empty_like(y0)
    it1, rr1, st1 = bj.solve_precond(inc, y1, tol=1e-8, max_iter=400)
    b = torch.empty_like(y1)
    bj.rhs(inc, b)
    Ay = torch.empty_like(y1)
    bj.apply_batch(y1, Ay)
    true = float(torch.linalg.norm(b - Ay) / torch.linalg.norm(b))
    bj.close()
    e = rel(y1.cpu().numpy(), y0.cpu().numpy())
    print(f"eps 8 sphere: right-scaled GMRES {it0[0]} iterations, block Jacobi {it1[0]}; solutions {e:.2e}, "
          f"true residual {true:.2e}")
    assert st0 == lib.IFGF_OK and st1 == lib.IFGF_OK
    assert it1[0] < it0[0], (it0, it1)
    # both solves stop at 1e-8 in residual; their solutions differ by the conditioning times that
    assert e < 1e-5 and true < 1e-7, (e, true)


def test_network_on_block_jacobi_corrects_its_product(sphere_e8):
    prob, qp, _ = sphere_e8
    plan = plan_of(prob, qp, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, max_krylov=10, batch=2)
    plan.block_jacobi()
    v = torch.from_numpy(random_densities(prob.n, 6, batch=2)).cuda()
    zb = torch.empty_like(v)
    plan.precond_apply(v, zb)                  # block Jacobi alone
    net = lib.Preconditioner(plan, hidden=16)  # zero output layer: no correction
    zn = torch.empty_like(v)
    net.apply(v, zn)
    e = torch.from_numpy(random_densities(prob.n, 7, batch=2)).cuda()
    P, n_in = prob.num_patches, 8 * prob.nc ** 2
    X = torch.empty((2 * P, n_in), dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    net.features(v, e, X, T)
    torch.cuda.synchronize()
    assert torch.equal(zn, zb)
    # targets: (e_p - (A_pp^-1 v)_p) / s_p, with the features' own layout (component, node, re/im)
    npp = prob.nc ** 2
    vv, ee, bb = v.cpu().numpy(), e.cpu().numpy(), zb.cpu().numpy()
    for r in range(2):
        for p in range(P):
            sl = slice(p * npp, (p + 1) * npp)
            x = np.stack([vv[r][:, sl].real, vv[r][:, sl].imag], -1).reshape(-1)
            t = np.stack([(ee[r] - bb[r])[:, sl].real, (ee[r] - bb[r])[:, sl].imag], -1).reshape(-1)
            s = np.linalg.norm(x)
            np.testing.assert_allclose(T[r * P + p].cpu().numpy(), (t / s).astype(np.float32), rtol=1e-5, atol=1e-6)
    plan.close()
