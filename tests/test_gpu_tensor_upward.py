"""The upward step (b) on the tensor cores (plan option upward_tc = 1: tcgen05 TF32 contractions
with a three-term hi/lo split, FP32 accumulation in tensor memory) against the FP32 SIMT upward
step of the same plan settings, through the C ABI: the far fields agree to FP32 rounding, the
forward map stays within the IFGF bar of the plain FP64 path, and a batched apply equals the
separate ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_MEDIUM, plane_wave, random_densities  # noqa: E402
from oracle import cbie  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def medium():
    prob = CONFIG_SPHERE_MEDIUM(10)
    return prob, cbie.default_delta(prob)


def plan(prob, delta, **kw):
    return lib.Plan.from_problem(prob, delta=delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3,
                                 max_krylov=10, **kw)


@pytest.mark.parametrize("prec", [lib.IFGF_FP32, lib.IFGF_MIXED])
def test_tensor_core_upward_step_matches_simt(medium, prec):
    prob, delta = medium
    rng = np.random.default_rng(31)
    phi = torch.from_numpy(np.ascontiguousarray(
        rng.standard_normal((prob.n, 8)) + 1j * rng.standard_normal((prob.n, 8)))).cuda()
    far = {}
    for tc in (0, 1):
        p = plan(prob, delta, precision=prec, upward_tc=tc)
        f = torch.empty((prob.n, 28), dtype=torch.complex128, device="cuda")
        p.fields(phi, f, lib.IFGF_PART_FAR)
        torch.cuda.synchronize()
        far[tc] = f.cpu().numpy()
        p.close()
    e = rel(far[1], far[0])
    print(f"tensor-core vs SIMT upward step, far fields: {e:.2e}")
    # both are FP32 evaluations of the same sums (measured 2.4e-6: the IFGF chain's FP32 rounding)
    assert e < 5e-6


def test_tensor_core_forward_map_and_batch(medium):
    prob, delta = medium
    y = torch.from_numpy(random_densities(prob.n, 32, batch=2)).cuda()
    pd = lib.Plan.from_problem(prob, delta=delta, n_beta=48, cov_d=4.0, far_mode=lib.IFGF_FAR_DIRECT,
                               precision=lib.IFGF_FP64)
    ref = torch.empty_like(y[0])
    pd.apply(y[0].contiguous(), ref)
    pd.close()
    p = plan(prob, delta, precision=lib.IFGF_FP32, upward_tc=1, batch=2)
    out = torch.empty_like(y)
    p.apply_batch(y, out)
    one = torch.empty_like(ref)
    p.apply(y[0].contiguous(), one)
    torch.cuda.synchronize()
    p.close()
    assert torch.equal(out[0], one)
    e = rel(one.cpu().numpy(), ref.cpu().numpy())
    print(f"tensor-core IFGF forward map vs plain FP64: {e:.2e}")
    assert e < 1e-4


def test_tensor_core_wait_timeout_is_reported_and_the_plan_stays_usable(medium):
    """The one device-side wait (the MMAs of the tensor-core upward step) is bounded: with fault
    injection the first MMAs of every block are not issued, so the wait expires (1 ms), the step
    records IFGF_ETIMEOUT in the plan's status word, frees its tensor memory and returns.  The
    host reads the status (ifgf_plan_check, and the solves before returning), the context stays
    usable, and the next apply equals the one before the injection."""
    prob, delta = medium
    y = torch.from_numpy(random_densities(prob.n, 33)).cuda()
    p = plan(prob, delta, precision=lib.IFGF_FP32, upward_tc=1)
    ref = torch.empty_like(y)
    p.apply(y, ref)
    p.check()                                     # nothing pending
    p.inject(1)
    bad = torch.empty_like(y)
    p.apply(y, bad)
    with pytest.raises(lib.IfgfError) as e:
        p.check()
    assert e.value.status == lib.IFGF_ETIMEOUT and "tensor-core" in str(e.value)
    p.check()                                     # the check cleared the word
    x, _, _ = prob.nodes()
    inc = torch.from_numpy(np.ascontiguousarray(plane_wave(x, prob.k_ext, prob.omega)[None])).cuda()
    ys = torch.empty((1, 4, prob.n), dtype=torch.complex128, device="cuda")
    with pytest.raises(lib.IfgfError) as e:
        p.solve_batch(inc, ys, tol=1e-3, max_iter=5)
    assert e.value.status == lib.IFGF_ETIMEOUT
    p.inject(0)
    again = torch.empty_like(y)
    p.apply(y, again)
    p.check()
    torch.cuda.synchronize()
    p.close()
    assert torch.equal(again, ref)
