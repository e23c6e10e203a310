"""The IFGF far fields of the library against the oracle's own IFGF (oracle/ifgf.py): the
same algorithm and readings written independently, so the approximation itself is compared (to
rounding in FP64), not only its distance to the exact far sum.  The octree and cone tables the
comparison relies on are checked equal on the host by tests/test_oracle_ifgf.py."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import sphere_problem  # noqa: E402
from oracle import cbie  # noqa: E402
from oracle import ifgf as oifgf  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_fields(plan, phi, which):
    pd = torch.from_numpy(np.ascontiguousarray(phi.T)).cuda()          # [N, 8]
    f = torch.empty((phi.shape[1], 28), dtype=torch.complex128, device="cuda")
    plan.fields(pd, f, which)
    torch.cuda.synchronize()
    return f.cpu().numpy().T                                            # [28, N]


@pytest.mark.parametrize("prec,tol", [(lib.IFGF_FP64, 1e-10), (lib.IFGF_FP32, 5e-5)])
def test_ifgf_far_fields_match_the_oracle_ifgf(prec, tol):
    """The IFGF far fields (S and dS/dn, both wavenumbers, 8 densities) against the oracle's
    own IFGF (oracle/ifgf.py: the same algorithm and readings, written independently): equal
    up to rounding in FP64 -- the approximation itself is compared, not only its distance to
    the exact sum -- and to FP32 rounding in FP32."""
    prob = sphere_problem(0.5, 1, 6, 2.25)
    g = cbie.geometry_of(prob)
    rng = np.random.default_rng(23)
    phi = rng.standard_normal((8, prob.n)) + 1j * rng.standard_normal((8, prob.n))
    plan = lib.Plan.from_problem(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0,
                                 far_mode=lib.IFGF_FAR_IFGF, precision=prec, ns0=2, na0=3, leaf_size=0.11)
    got = gpu_fields(plan, phi, lib.IFGF_PART_FAR)          # [28, N]
    plan.close()
    tree = oifgf.build_tree(g.x, 0.11, max(prob.k_ext, prob.k_int), 2, 3)
    ref = oifgf.ifgf_far(tree, g.x, g.n, phi.T * g.omega[:, None], prob.k_ext, prob.k_int).T
    assert rel(got[:16], ref[:16]) < tol
    assert rel(got[16:], ref[16:]) < tol
