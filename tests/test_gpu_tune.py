"""The autotuner (ifgf_plan_tune) through the C ABI: it times both target-step shapes and both
upward-step shapes per level and both near-matvec block sizes, keeps the faster, and the forward
map after tuning agrees with the one before to FP32 rounding (only summation orders change)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2408_02274_gb300 as lib  # noqa: E402
from inputs import CONFIG_SPHERE_MEDIUM, random_densities  # noqa: E402
from oracle import cbie  # noqa: E402


def test_tune_keeps_the_faster_shape_and_the_result():
    prob = CONFIG_SPHERE_MEDIUM(10)
    plan = lib.Plan.from_problem(prob, delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0,
                                 precision=lib.IFGF_FP32, far_mode=lib.IFGF_FAR_IFGF, ns0=2, na0=3, max_krylov=10)
    y = torch.from_numpy(random_densities(prob.n, 51)).cuda()
    before, after = torch.empty_like(y), torch.empty_like(y)
    plan.apply(y, before)
    choices, times = plan.tune(reps=3)
    plan.apply(y, after)
    torch.cuda.synchronize()
    levels = plan.stats()["levels"]
    for d in range(3, levels + 1):
        assert choices[d] in (0, 1)
        t0, t1 = times[2 * d], times[2 * d + 1]
        assert t0 > 0 and t1 > 0
        assert choices[d] == (1 if t1 < t0 else 0)
    assert choices[25] in (128, 256) and times[50] > 0 and times[51] > 0
    for d in range(3, levels):   # upward step into parent level d: runs per slot, warp per slot, runs per item
        assert choices[32 + d] in (0, 1, 2)
        t = [times[64 + 2 * d], times[65 + 2 * d], times[100 + d]]
        assert min(t) > 0
        assert choices[32 + d] == int(np.argmin(t))
    assert choices[30] in (0, 1) and times[60] > 0 and times[61] > 0   # leaf: SIMT or tensor-pipe products
    assert choices[30] == (1 if times[61] < times[60] else 0)
    print("leaf products (SIMT, tensor pipe) ms:", times[60:62], "choice", choices[30])
    print("target shape per level:", choices[3:levels + 1], "ms:", times[6:2 * levels + 2], "near threads:", choices[25],
          "upward shape per level:", choices[35:32 + levels], "ms:", times[70:64 + 2 * levels],
          times[103:100 + levels])
    e = float(torch.linalg.norm(after - before) / torch.linalg.norm(before))
    assert e < 1e-5, e
    plan.close()
