"""The allocation-free entry point, through the C ABI.

ifgf_far_direct_noalloc serves callers that cannot allocate device memory
where they need the far-field sums: an application that owns all device
memory through its own pool, or a latency-critical loop that cannot afford
cudaMalloc's implicit synchronisation.  It keeps its working arrays in one
fixed device array of the library.  Its results are checked against the
oracle's plain far sum (same leaf boxes) and against the plan-based entry
point, on two calls in a row, and device free memory must not change across
a call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_SMALL  # noqa: E402
from oracle import cbie, ifgf  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [(lib.IFGF_FP64, 1e-12), (lib.IFGF_FP32, 1e-5)])
def test_noalloc_far_sums_match_oracle_and_plan_entry_point(precision, tol):
    prob = CONFIG_SPHERE_SMALL(8)
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0)
    plan = lib.Plan.from_problem(prob, delta=qp.delta, n_beta=qp.n_beta, cov_d=qp.cov_d,
                                 far_mode=lib.IFGF_FAR_DIRECT, precision=precision)
    n = prob.n
    g = cbie.geometry_of(prob)
    # leaf boxes by the oracle's own octree under the plan's leaf rule (0.25 exterior wavelengths)
    tree = ifgf.build_tree(g.x, 0.25 * 2 * np.pi / prob.k_ext, max(prob.k_ext, prob.k_int), 2, 3)
    leafc = tree.leafc.astype(np.int32)
    _, plan_leafc = lib.Tree.of_plan(plan.handle, n).perm()
    assert np.array_equal(leafc, plan_leafc)
    rng = np.random.default_rng(11)
    phi_h = rng.standard_normal((n, 8)) + 1j * rng.standard_normal((n, 8))
    oracle_far = ifgf.direct_far(g.x, g.n, phi_h * g.omega[:, None], prob.k_ext, prob.k_int, leafc)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    x, nrm, w, lc = dev(g.x, np.float64), dev(g.n, np.float64), dev(g.omega, np.float64), dev(leafc, np.int32)
    phi = dev(phi_h, np.complex128)
    ref = torch.empty((n, 28), dtype=torch.complex128, device="cuda")
    plan.fields(phi, ref, lib.IFGF_PART_FAR)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    assert rel(ref, oracle_far) < tol
    outs = [torch.full((n, 28), np.nan + 0j, dtype=torch.complex128, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for k, out in enumerate(outs):        # two calls in a row share the fixed array
        free0 = torch.cuda.mem_get_info()[0]
        lib.ifgf_far_direct_noalloc(x, nrm, w, lc, phi, prob.k_ext, prob.k_int, out, precision=precision)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if k == 1:
            # after the first call (symbol lookup, kernel loading) a call takes no device memory
            assert free1 == free0, (free0, free1)
        got = out.cpu().numpy()
        assert rel(got, oracle_far) < tol
        assert rel(got, ref) < tol
    plan.close()


def test_noalloc_rejects_sizes_beyond_the_fixed_array():
    # n above the fixed array's capacity is refused before any GPU work, with its own message
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    st = lib.load().ifgf_far_direct_noalloc(100001, p, p, p, p, p, 1.0, 1.0, lib.IFGF_FP64, p, None)
    assert st == lib.IFGF_EUNSUPPORTED
    assert b"100000" in lib.load().ifgf_status_string(lib.IFGF_EUNSUPPORTED)
    with pytest.raises(lib.IfgfError, match="100000"):
        n = 100001
        big = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        lib.ifgf_far_direct_noalloc(big, big, torch.zeros(n, dtype=torch.float64, device="cuda"),
                                    torch.zeros((n, 3), dtype=torch.int32, device="cuda"),
                                    torch.zeros((n, 8), dtype=torch.complex128, device="cuda"), 1.0, 1.0,
                                    torch.zeros((n, 28), dtype=torch.complex128, device="cuda"))
