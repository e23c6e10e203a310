"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
rejects bad descriptors without touching a GPU, and its host-only octree /
cone-segment setup (Sec. III-F) satisfies the invariants the IFGF relies on."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2408_02274_gb300 as lib
from inputs import CONFIG_SPHERE_SMALL, sphere_problem
from paper_2408_02274_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    libbuild.build()
    lib.load()


def test_every_declared_symbol_is_exported():
    header = open(os.path.join(ROOT, "include", "ifgf.h")).read()
    declared = set(re.findall(r"^(?:ifgf_status|const char\*)\s+(\w+)\s*\(", header, flags=re.M))
    assert {"ifgf_plan_create", "ifgf_apply", "bie_solve", "ifgf_plan_destroy"} <= declared
    L = lib.load()
    for name in declared:
        assert hasattr(L, name), name
    assert set(lib.EXPORTS) == declared


def test_status_strings():
    L = lib.load()
    for s in range(8):
        assert len(L.ifgf_status_string(s)) > 0


def test_invalid_descriptors_rejected_before_any_gpu_work():
    prob = CONFIG_SPHERE_SMALL(4, ng=8)
    x, xu, xv = prob.nodes()
    base = dict(nodes=x, dxdu=xu, dxdv=xv, fine=prob.fine(), num_patches=prob.num_patches, nc=prob.nc,
                k_ext=prob.k_ext, k_int=prob.k_int, eps_ext=1.0, eps_int=2.25, delta=0.3)
    for bad, status in [({"delta": 0.0}, lib.IFGF_EINVAL), ({"k_ext": -1.0}, lib.IFGF_EINVAL),
                        ({"n_beta": 2}, lib.IFGF_EINVAL), ({"cov_d": 1.0}, lib.IFGF_EINVAL),
                        ({"precision": 7}, lib.IFGF_EINVAL), ({"ps": 4}, lib.IFGF_EUNSUPPORTED),
                        ({"nc": 1}, lib.IFGF_EINVAL), ({"max_krylov": 5000}, lib.IFGF_EINVAL),
                        ({"batch": -1}, lib.IFGF_EINVAL), ({"batch": 5000}, lib.IFGF_EINVAL),
                        ({"max_leaf_pts": -3}, lib.IFGF_EINVAL)]:
        kw = dict(base)
        kw.update(bad)
        with pytest.raises(lib.IfgfError) as e:
            lib.ifgf_plan_create(**kw)
        assert e.value.status == status


def test_null_plan_arguments_rejected():
    L = lib.load()
    patches = (ctypes.c_int32 * 2)(0, 1)
    assert L.ifgf_apply_direct_patches(None, None, None, patches, 2, None) == lib.IFGF_EINVAL
    assert L.ifgf_apply(None, None, None, None) == lib.IFGF_EINVAL


def _coverage(tree, x, k_max):
    """Count, for every (target, source) pair, the levels at which the source's
    box is evaluated at the target (step 3 of the algorithm summary)."""
    n = x.shape[0]
    perm, leafc = tree.perm()
    D = tree.levels
    iperm = np.empty(n, dtype=np.int64)
    iperm[perm] = np.arange(n)
    cover = np.zeros((n, n), dtype=np.int32)
    max_s = 0.0
    for d in range(3, D + 1):
        coords, ptr, cones, ns, na = tree.level(d)
        tp, ts, sb = tree.targets(d)
        key = {tuple(c): b for b, c in enumerate(coords)}
        src_box = np.array([key[tuple(c >> (D - d))] for c in leafc])           # original order
        E = np.zeros((n, coords.shape[0]), dtype=np.int32)                      # original target order
        H = tree.h1 / 2 ** (d - 1)
        for s in range(n):
            l = perm[s]
            boxes = sb[ts[tp[s]:tp[s + 1]]]
            assert len(set(boxes.tolist())) == boxes.size                      # one cone per source box
            E[l, boxes] += 1
            cen = tree.corner + H * (coords[boxes] + 0.5)
            r = np.linalg.norm(x[l] - cen, axis=1)
            if r.size:
                max_s = max(max_s, (np.sqrt(3) / 2 * H / r).max())
        cover += E[:, src_box]
    near = np.all(np.abs(leafc[:, None, :] - leafc[None, :, :]) <= 1, axis=-1)
    return cover, near, max_s


@pytest.mark.parametrize("split,leaf", [(1, 0.25), (2, 0.11), (2, 0.06)])
def test_ifgf_exactly_once_coverage(split, leaf):
    prob = sphere_problem(0.5, split, 6, 2.25)
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=leaf, k_max=prob.k_int)
    cover, near, max_s = _coverage(tree, x, prob.k_int)
    assert tree.levels >= 3
    assert np.all(cover[near] == 0)
    assert np.all(cover[~near] == 1)
    # every evaluated target is at least one box away: s = h/r <= sqrt(3)/3 (Sec. III-E)
    assert max_s <= np.sqrt(3) / 3 + 1e-12


def test_cone_counts_follow_the_doubling_rule():
    prob = sphere_problem(2.0, 2, 6, 4.0)
    x, _, _ = prob.nodes()
    k = prob.k_int
    tree = lib.Tree(x, leaf_size=0.25, k_max=k, ns0=1, na0=2)
    D = tree.levels
    ns_prev, na_prev = 1, 2
    for d in range(D, 2, -1):
        _, _, _, ns, na = tree.level(d)
        H = tree.h1 / 2 ** (d - 1)
        a = 2 if k * H > 0.5 else 1
        assert (ns, na) == (max(a * ns_prev, 2), a * na_prev)   # radial floor 2 n_{s;D+1}
        ns_prev, na_prev = a * ns_prev, na


def test_relevant_cones_contain_their_targets():
    # every (target, slot) pair of step 3 refers to the cone segment that holds the target
    prob = sphere_problem(0.5, 2, 6, 2.25)
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=0.11, k_max=prob.k_int)
    perm, _ = tree.perm()
    D = tree.levels
    for d in range(3, D + 1):
        coords, ptr, cones, ns, na = tree.level(d)
        tp, ts, sb = tree.targets(d)
        H = tree.h1 / 2 ** (d - 1)
        h = np.sqrt(3) / 2 * H
        for s in range(0, x.shape[0], 7):
            for slot in ts[tp[s]:tp[s + 1]]:
                b, cone = sb[slot], cones[slot]
                rel = x[perm[s]] - (tree.corner + H * (coords[b] + 0.5))
                r = np.linalg.norm(rel)
                sv, th = h / r, np.arctan2(np.hypot(rel[0], rel[1]), rel[2])
                ph = np.arctan2(rel[1], rel[0]) % (2 * np.pi)
                g3 = int(cone) & ((1 << 21) - 1)
                g2 = (int(cone) >> 21) & ((1 << 21) - 1)
                g1 = int(cone) >> 42
                assert min(int(sv / (np.sqrt(3) / 3 / ns)), ns - 1) == g1
                assert min(int(th / (np.pi / na)), na - 1) == g2
                assert min(int(ph / (np.pi / na)), 2 * na - 1) == g3


def test_point_count_leaf_rule_on_a_thin_bar():
    """The point-count rule deepens the octree until no leaf box holds more than
    max_leaf_pts nodes, and no further (one level less would exceed it)."""
    from inputs import waveguide_bar
    prob = waveguide_bar(0.2, nc=6)
    x, _, _ = prob.nodes()
    base = lib.Tree(x, leaf_size=0.25 * 2 * np.pi / prob.k_ext, k_max=prob.k_int, ns0=2, na0=3)
    for cap in (64, 16):
        tree = lib.Tree(x, leaf_size=0.25 * 2 * np.pi / prob.k_ext, k_max=prob.k_int, ns0=2, na0=3,
                        max_leaf_pts=cap)
        _, leafc = tree.perm()
        counts = np.unique(leafc, axis=0, return_counts=True)[1]
        assert counts.max() <= cap < 0 + np.unique(leafc >> 1, axis=0, return_counts=True)[1].max()
        assert tree.levels > base.levels
        tree.close()
    base.close()


def test_bar_tree_exact_once_coverage_sorted_keys_and_radial_floor():
    """On a deep point-count tree of the bar: every far pair is evaluated exactly once,
    each box's relevant cone keys are sorted and distinct, every (target, slot) pair refers
    to the cell holding the target, and the leaf keeps at least 2 n_s;D+1 radial cells."""
    from inputs import waveguide_bar
    prob = waveguide_bar(0.5, nc=4, half_lengths=(2.5, 0.15, 0.07))
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=0.25 * 2 * np.pi / prob.k_ext, k_max=prob.k_int, ns0=2, na0=3, max_leaf_pts=8)
    cover, near, max_s = _coverage(tree, x, prob.k_int)
    assert np.all(cover[near] == 0) and np.all(cover[~near] == 1)
    assert max_s <= np.sqrt(3) / 3 + 1e-12
    D = tree.levels
    perm, _ = tree.perm()
    for d in range(3, D + 1):
        coords, ptr, cones, ns, na = tree.level(d)
        for b in range(coords.shape[0]):
            kb = cones[ptr[b]:ptr[b + 1]]
            assert np.all(np.diff(kb) > 0)
        tp, ts, sb = tree.targets(d)
        H = tree.h1 / 2 ** (d - 1)
        h = np.sqrt(3) / 2 * H
        for s in range(0, x.shape[0], 5):
            for slot in ts[tp[s]:tp[s + 1]]:
                b, cone = sb[slot], int(cones[slot])
                rel = x[perm[s]] - (tree.corner + H * (coords[b] + 0.5))
                r = np.linalg.norm(rel)
                g1, g2, g3 = cone >> 42, (cone >> 21) & ((1 << 21) - 1), cone & ((1 << 21) - 1)
                assert min(int(h / r / (np.sqrt(3) / 3 / ns)), ns - 1) == g1
                th = np.arctan2(np.hypot(rel[0], rel[1]), rel[2])
                assert min(int(th / (np.pi / na)), na - 1) == g2
                ph = np.arctan2(rel[1], rel[0]) % (2 * np.pi)
                assert min(int(ph / (np.pi / na)), 2 * na - 1) == g3
    _, _, _, ns_leaf, _ = tree.level(D)
    assert ns_leaf >= 4
    tree.close()


def test_plan_estimate_host_only():
    """ifgf_plan_estimate runs on the host (no GPU here) and its parts add up; the GMRES
    workspace grows by 16 * 4N bytes per Krylov vector (plus the Hessenberg matrix), the
    per-apply and coefficient buffers scale with the batch, and FP64 near values take twice
    the FP32 bytes per nonzero."""
    prob = CONFIG_SPHERE_SMALL(6, ng=12)
    base = dict(delta=0.3, ns0=2, na0=3, precision=lib.IFGF_FP32)
    e = lib.Plan.estimate(prob, max_krylov=50, **base)
    parts = ("bytes_geometry", "bytes_near_max", "bytes_tables", "bytes_coefs", "bytes_apply", "bytes_gmres")
    assert e["bytes_plan_max"] == sum(e[k] for k in parts)
    assert all(e[k] > 0 for k in parts)
    assert e["bytes_setup_peak_max"] >= e["bytes_plan_max"]
    assert e["levels"] >= 3 and e["near_nnz_max"] > 0 and e["candidate_pairs"] > 0
    n4 = 4 * prob.n
    e2 = lib.Plan.estimate(prob, max_krylov=60, **base)
    dv = e2["bytes_gmres"] - e["bytes_gmres"]
    basis_and_h = 10 * 16 * n4 + 16 * (61 ** 2 - 51 ** 2)   # 10 more basis vectors, Hessenberg 61^2 vs 51^2
    assert basis_and_h <= dv < basis_and_h + 2000           # + rotations, projections, partial sums
    e3 = lib.Plan.estimate(prob, max_krylov=50, batch=3, **base)
    assert e3["bytes_apply"] == 3 * e["bytes_apply"] and e3["bytes_coefs"] == 3 * e["bytes_coefs"]
    e4 = lib.Plan.estimate(prob, max_krylov=50, **dict(base, precision=lib.IFGF_FP64))
    nnz = e["near_nnz_max"]
    assert e4["bytes_near_max"] - e["bytes_near_max"] == 32 * nnz
    assert e4["near_nnz_max"] == nnz and e4["cones"] == e["cones"]
    e5 = lib.Plan.estimate(prob, max_krylov=50, far_mode=lib.IFGF_FAR_DIRECT, **base)
    assert e5["bytes_coefs"] == 0
    with pytest.raises(lib.IfgfError) as err:
        lib.Plan.estimate(prob, **dict(base, delta=0.0))
    assert err.value.status == lib.IFGF_EINVAL


def test_fields_per_pass_memory_and_options():
    """The speed-vs-memory trade-off of Sec. III ("IFGF for Multiple Densities") as the estimate
    sees it: one kernel per traversal (8 fields) halves the interpolation coefficients' bytes,
    one (density, kernel) sum per traversal (IFGF_Seq) takes 1/16 of them; nothing else
    changes.  The option needs FP32 IFGF kernels, the IFGF far field and the SIMT upward step."""
    prob = CONFIG_SPHERE_SMALL(6, ng=12)
    base = dict(delta=0.3, ns0=2, na0=3, precision=lib.IFGF_FP32, max_krylov=20)
    vec = lib.Plan.estimate(prob, **base)
    assert lib.Plan.estimate(prob, fields_per_pass=16, **base) == vec
    for f, div in ((8, 2), (1, 16)):
        e = lib.Plan.estimate(prob, fields_per_pass=f, **base)
        assert e["bytes_coefs"] * div == vec["bytes_coefs"]
        for k in ("bytes_geometry", "bytes_near_max", "bytes_tables", "bytes_apply", "bytes_gmres"):
            assert e[k] == vec[k]
        assert e["bytes_plan_max"] == vec["bytes_plan_max"] - vec["bytes_coefs"] + e["bytes_coefs"]
    mixed = lib.Plan.estimate(prob, fields_per_pass=1, **dict(base, precision=lib.IFGF_MIXED))
    assert mixed["bytes_coefs"] * 16 == vec["bytes_coefs"]
    for bad in (2, 4, -1, 17):
        with pytest.raises(lib.IfgfError) as err:
            lib.Plan.estimate(prob, fields_per_pass=bad, **base)
        assert err.value.status == lib.IFGF_EINVAL
    for opts in (dict(precision=lib.IFGF_FP64), dict(far_mode=lib.IFGF_FAR_DIRECT), dict(upward_tc=1)):
        with pytest.raises(lib.IfgfError) as err:
            lib.Plan.estimate(prob, fields_per_pass=8, **dict(base, **opts))
        assert err.value.status == lib.IFGF_EUNSUPPORTED


def test_upward_items_group_slots_of_one_cone_and_child_set():
    """The upward step's items (the FP32 step per item, the tensor-core step): every slot of the
    parent level lies in exactly one item; an item's slots share their cone key, on which the
    item's one prologue depends, and come in the order (set of child octants, slot); -1 only
    after an item's last slot; items in the order of their first slot."""
    prob = sphere_problem(2.0, 2, 6, 4.0)
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=0.25, k_max=prob.k_int, ns0=2, na0=3)
    assert tree.levels >= 5
    for d in range(3, tree.levels):
        coords, ptr, cones, _, _ = tree.level(d)
        present = set(map(tuple, tree.level(d + 1)[0].tolist()))
        box_of_slot = np.repeat(np.arange(ptr.size - 1), np.diff(ptr))
        mask = [sum(1 << o for o in range(8)
                    if (2 * c[0] + (o & 1), 2 * c[1] + ((o >> 1) & 1), 2 * c[2] + (o >> 2)) in present)
                for c in coords.tolist()]
        it = tree.items(d)
        assert it.shape[1] == 4 and it.shape[0] >= (cones.size + 3) // 4
        assert sorted(it[it >= 0].tolist()) == list(range(cones.size))
        for row in it:
            k = int(np.sum(row >= 0))
            assert k >= 1 and np.all(row[:k] >= 0) and np.all(row[k:] == -1)
            assert len(set(cones[row[:k]].tolist())) == 1
            ks = [(mask[box_of_slot[j]], int(j)) for j in row[:k]]
            assert ks == sorted(ks) and len(set(ks)) == k
        assert np.all(np.diff(it[:, 0]) > 0)
    with pytest.raises(lib.IfgfError):
        tree.items(tree.levels)
    tree.close()


def test_upward_run_tables_partition_every_parent_point():
    """The upward tables of each parent level: per (compact cone, octant) the ranking is a
    permutation of the 75 points; the runs of a (compact cone, warp group) cover each
    (octant, point) of that group exactly once, are at most 32 long, longest first, and the
    points of a run share their warp group and child cone."""
    prob = sphere_problem(2.0, 2, 6, 4.0)
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=0.25, k_max=prob.k_int, ns0=2, na0=3)

    def group(q):   # ranks by snake-ordered angular position, radial index within; 19/19/19/18
        a = q % 25
        it, ip = a // 5, a % 5
        rank = (it * 5 + (4 - ip if it & 1 else ip)) * 3 + q // 25
        return 0 if rank < 19 else (1 if rank < 38 else (2 if rank < 57 else 3))

    for d in range(3, tree.levels):
        cc, order, task, ptr = tree.upward(d)
        assert np.all(np.diff(ptr) >= 0) and ptr[-1] == task.size
        for ci in range(cc.shape[0]):
            for o in range(8):
                assert sorted(order[ci, o].tolist()) == list(range(75))
            for w in range(4):
                seen = np.zeros((8, 75), dtype=np.int32)
                lens = []
                for tk in task[ptr[ci * 4 + w]:ptr[ci * 4 + w + 1]]:
                    r0, ln, o = tk & 255, (tk >> 8) & 255, (tk >> 16) & 7
                    assert 1 <= ln <= 32
                    lens.append(ln)
                    qs = order[ci, o, r0:r0 + ln]
                    assert all(group(q) == w for q in qs)
                    assert len(set(cc[ci, o, qs].tolist())) == 1
                    seen[o, qs] += 1
                assert lens == sorted(lens, reverse=True)
                mine = np.array([group(q) == w for q in range(75)])
                assert np.all(seen[:, mine] == 1) and np.all(seen[:, ~mine] == 0)
    tree.close()


def test_plan_estimate_uses_the_plan_tree():
    """The estimate's levels and relevant-cone counts are those of the host tree the plan
    builds (same leaf rules, wavenumber and cone base)."""
    from inputs import waveguide_bar
    prob = waveguide_bar(0.5, nc=4, half_lengths=(2.5, 0.15, 0.07))
    leaf = 0.25 * 2 * np.pi / prob.k_ext
    e = lib.Plan.estimate(prob, delta=0.3, ns0=2, na0=3, max_leaf_pts=8, precision=lib.IFGF_FP32, max_krylov=10)
    x, _, _ = prob.nodes()
    tree = lib.Tree(x, leaf_size=leaf, k_max=max(prob.k_ext, prob.k_int), ns0=2, na0=3, max_leaf_pts=8)
    assert e["levels"] == tree.levels
    for d in range(3, tree.levels + 1):
        _, _, cones, _, _ = tree.level(d)
        assert e["cones"][d] == cones.size
    tree.close()


def _all_tables(tree):
    perm, leafc = tree.perm()
    out = [perm, leafc]
    for d in range(3, tree.levels + 1):
        coords, ptr, cones, ns, na = tree.level(d)
        out += [coords, ptr, cones, np.array([ns, na])]
        out += list(tree.targets(d))
        if d < tree.levels:
            out += list(tree.upward(d))
    return out


@pytest.mark.parametrize("case", ["bar", "fine_cones"])
def test_host_tables_do_not_depend_on_the_thread_count(case, monkeypatch):
    """The host setup splits its work over IFGF_HOST_THREADS threads (default: all cores); the
    octree, relevant-cone, target and upward tables are the same for 1, 3 and all threads.
    'bar': a deep point-count tree (many boxes, small cone counts, bit-per-cone de-duplication);
    'fine_cones': ns0 = na0 = 64, so that the top levels have more than 2^24 cones and the
    relevant cones are de-duplicated by sorting."""
    from inputs import waveguide_bar
    if case == "bar":
        prob = waveguide_bar(0.5, nc=4, half_lengths=(2.5, 0.15, 0.07))
        kw = dict(leaf_size=0.25 * 2 * np.pi / prob.k_ext, k_max=prob.k_int, ns0=2, na0=3, max_leaf_pts=8)
    else:
        prob = sphere_problem(0.5, 1, 6, 2.25)
        kw = dict(leaf_size=0.11, k_max=max(prob.k_ext, prob.k_int), ns0=64, na0=64)
    x, _, _ = prob.nodes()
    ref = None
    for nth in ("", "1", "3"):
        monkeypatch.setenv("IFGF_HOST_THREADS", nth)
        tree = lib.Tree(x, **kw)
        tabs = _all_tables(tree)
        if case == "fine_cones":
            _, _, _, ns, na = tree.level(3)
            assert ns * na * 2 * na > 1 << 24
        tree.close()
        if ref is None:
            ref = tabs
        else:
            assert len(tabs) == len(ref)
            for a, b in zip(tabs, ref):
                assert np.array_equal(a, b)


def test_degenerate_and_unsupported_point_sets_are_rejected_on_the_host():
    """Non-finite coordinates, fewer than two distinct points, more than 21 octree levels and
    cone counts beyond the 21-bit cone-key fields are refused with IFGF_EINVAL before any table
    is built; the plan estimate (host only) refuses non-finite nodes the same way."""
    rng = np.random.default_rng(3)
    good = rng.standard_normal((40, 3))
    for bad in (np.nan, np.inf, -np.inf):
        x = good.copy()
        x[7, 1] = bad
        with pytest.raises(lib.IfgfError) as e:
            lib.Tree(x, leaf_size=0.3, k_max=5.0, ns0=2, na0=3)
        assert e.value.status == lib.IFGF_EINVAL
    for x in (np.zeros((1, 3)), np.zeros((5, 3))):
        with pytest.raises(lib.IfgfError):
            lib.Tree(x, leaf_size=0.3, k_max=5.0, ns0=2, na0=3)
    with pytest.raises(lib.IfgfError):
        lib.Tree(good, leaf_size=0.3, k_max=5.0, ns0=2, na0=3, min_levels=22)
    t = lib.Tree(good, leaf_size=0.3, k_max=5.0, ns0=2, na0=3, min_levels=21)   # the largest depth
    assert t.levels == 21
    t.close()
    # every level doubles the cones (k_max H > 1/2 down to the leaves): 64 * 2^15 angular cells
    with pytest.raises(lib.IfgfError) as e:
        lib.Tree(good, leaf_size=1e-5, k_max=1e7, ns0=64, na0=64)
    assert e.value.status == lib.IFGF_EINVAL
    prob = CONFIG_SPHERE_SMALL(8)
    x, xu, xv = prob.nodes()
    x = x.copy()
    x[5, 0] = np.nan
    with pytest.raises(lib.IfgfError) as e:
        lib.ifgf_plan_estimate(x, xu, xv, prob.fine(), prob.num_patches, prob.nc, prob.k_ext, prob.k_int,
                               prob.eps_ext, prob.eps_int, delta=0.1)
    assert e.value.status == lib.IFGF_EINVAL


def test_host_thread_cap_ignores_values_that_are_not_positive(monkeypatch):
    """IFGF_HOST_THREADS values that are not a positive number (0, -3, text, empty) fall back to
    all cores; the tables stay the same."""
    prob = sphere_problem(0.5, 1, 6, 2.25)
    x, _, _ = prob.nodes()
    kw = dict(leaf_size=0.11, k_max=max(prob.k_ext, prob.k_int), ns0=2, na0=3)
    monkeypatch.delenv("IFGF_HOST_THREADS", raising=False)
    t = lib.Tree(x, **kw)
    ref = _all_tables(t)
    t.close()
    for v in ("0", "-3", "many", ""):
        monkeypatch.setenv("IFGF_HOST_THREADS", v)
        t = lib.Tree(x, **kw)
        got = _all_tables(t)
        t.close()
        assert all(np.array_equal(a, b) for a, b in zip(got, ref))
