"""Learned right preconditioner and flexible GMRES through the C ABI: the
network apply and feature kernels against numpy, training on a learnable
target, zero output weights reducing flexible GMRES to plain GMRES exactly,
and a preconditioned solve reaching the tolerance in true residual."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_SMALL, plane_wave, random_densities  # noqa: E402
from oracle import cbie  # noqa: E402


def plan_of(prob, **kw):
    return lib.Plan.from_problem(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0, **kw)


def bf16(a):
    """Round float32 to bfloat16 (nearest, ties to even) and back, for the numpy reference."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def patch_features(v, P, npp):
    """[nrhs, 4, N] complex -> [nrhs, P, 8 npp] reals in the library's feature order."""
    nr = v.shape[0]
    x = v.reshape(nr, 4, P, npp).transpose(0, 2, 1, 3)          # [nrhs, P, 4, npp]
    return np.stack([x.real, x.imag], axis=-1).reshape(nr, P, 8 * npp)


def test_apply_and_features_match_numpy():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, batch=2, max_krylov=10)
    rng = np.random.default_rng(1)
    n_in, H = 8 * 64, 32
    W1 = rng.standard_normal((n_in, H)) * 0.05
    b1 = rng.standard_normal(H) * 0.1
    W2 = rng.standard_normal((H, n_in)) * 0.05
    b2 = rng.standard_normal(n_in) * 0.01
    pc = lib.Preconditioner(plan, hidden=H, weights=(W1, b1, W2, b2))
    v = np.stack([random_densities(prob.n, 41), random_densities(prob.n, 42)])
    vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    z = torch.empty_like(vd)
    pc.apply(vd, z)
    # numpy reference with the same BF16 weights, FP32 biases
    P = prob.num_patches
    x = patch_features(v, P, 64)
    s = np.linalg.norm(x, axis=-1, keepdims=True)
    h = np.maximum((x / s) @ bf16(W1).astype(np.float64) + b1.astype(np.float32), 0.0)
    o = h @ bf16(W2).astype(np.float64) + b2.astype(np.float32)
    zf = x + s * o
    got = patch_features(z.cpu().numpy(), P, 64)
    assert np.abs(got - zf).max() / np.abs(zf).max() < 2e-5
    # features: X = v_p / s_p, T = (e_p - v_p) / s_p
    e = np.stack([random_densities(prob.n, 43), random_densities(prob.n, 44)])
    X = torch.empty((2 * P, n_in), dtype=torch.float32, device="cuda")
    T = torch.empty_like(X)
    pc.features(vd, torch.from_numpy(np.ascontiguousarray(e)).cuda(), X, T)
    xe = patch_features(e, P, 64)
    assert np.allclose(X.cpu().numpy(), (x / s).reshape(2 * P, n_in), rtol=1e-5, atol=1e-6)
    assert np.allclose(T.cpu().numpy(), ((xe - x) / s).reshape(2 * P, n_in), rtol=1e-4, atol=1e-5)
    plan.close()


def test_training_fits_a_learnable_target():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, max_krylov=10)
    pc = lib.Preconditioner(plan, hidden=64, seed=3)
    rng = np.random.default_rng(5)
    n, n_in = 4096, 8 * 64
    X = rng.standard_normal((n, n_in)).astype(np.float32)
    K = (rng.standard_normal((n_in, 8)) @ rng.standard_normal((8, n_in)) / n_in).astype(np.float32)   # rank 8
    T = np.maximum(X @ K, 0.0) - 0.5 * (X @ K)
    loss = pc.train(torch.from_numpy(X).cuda(), torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).cuda(),
                    steps=1500, batch=256, lr=3e-3)
    assert np.all(np.isfinite(loss))
    assert loss[-100:].mean() < 0.1 * loss[:20].mean()
    plan.close()


def test_zero_output_weights_reduce_fgmres_to_gmres():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, max_krylov=80)
    lib.Preconditioner(plan, hidden=16, seed=7)            # W2 = 0, b2 = 0: z = v exactly
    x, _, _ = prob.nodes()
    inc = torch.from_numpy(np.ascontiguousarray(plane_wave(x, prob.k_ext, prob.omega)[None])).cuda()
    y0 = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
    y1 = torch.empty_like(y0)
    it0, rr0, s0 = plan.solve_batch(inc, y0, tol=1e-8, max_iter=80)
    it1, rr1, s1 = plan.solve_precond(inc, y1, tol=1e-8, max_iter=80)
    assert s0 == s1 == lib.IFGF_OK and it0 == it1 and rr0 == rr1
    assert torch.equal(y0, y1)
    plan.close()


def test_preconditioned_solve_reaches_the_tolerance_in_true_residual():
    prob = CONFIG_SPHERE_SMALL(8)
    plan = plan_of(prob, precision=lib.IFGF_FP64, far_mode=lib.IFGF_FAR_DIRECT, max_krylov=120)
    rng = np.random.default_rng(11)
    n_in, H = 8 * 64, 32
    # a fixed, non-trivial network (the method does not require it to be trained)
    lib.Preconditioner(plan, hidden=H, weights=(rng.standard_normal((n_in, H)) * 0.05, np.zeros(H),
                                                rng.standard_normal((H, n_in)) * 0.01, np.zeros(n_in)))
    x, _, _ = prob.nodes()
    inc_np = plane_wave(x, prob.k_ext, prob.omega)
    inc = torch.from_numpy(np.ascontiguousarray(inc_np[None])).cuda()
    y = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
    its, rrs, st = plan.solve_precond(inc, y, tol=1e-8, max_iter=120)
    assert st == lib.IFGF_OK
    # true residual |b - A y| / |b| with the plan's own forward map and the oracle's right-hand side
    g = cbie.geometry_of(prob)
    b = cbie.rhs(prob, g, inc_np)
    Ay = torch.empty_like(y[0])
    plan.apply(y[0].contiguous(), Ay)
    r = np.linalg.norm(b - Ay.cpu().numpy()) / np.linalg.norm(b)
    assert r < 1e-7
    plan.close()
