"""Pins of the oracle's IFGF (oracle/ifgf.py): the interpolation pieces against their
definitions, the decomposition against the plain far sum (exact box sums), the interpolation
error against cone refinement, and its octree / relevant cones / cousin records against the
library's host tables built independently from the same readings."""
import numpy as np
import pytest

from inputs import sphere_problem, waveguide_bar
from oracle import cbie, ifgf


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_chebyshev_transform_is_exact_on_the_tensor_polynomials():
    """Values of any polynomial of degree (2, 4, 4) at the 3 x 5 x 5 open nodes give back the
    polynomial everywhere, and the derivative bases differentiate it."""
    rng = np.random.default_rng(0)
    c = rng.standard_normal((3, 5, 5))
    poly = lambda s, t, p: np.einsum("ijk,mi,mj,mk->m", c, ifgf.cheb_T(s, 3), ifgf.cheb_T(t, 5), ifgf.cheb_T(p, 5))
    xs, xa = ifgf.cheb_nodes(3), ifgf.cheb_nodes(5)
    S, T, P = np.meshgrid(xs, xa, xa, indexing="ij")
    vals = poly(S.ravel(), T.ravel(), P.ravel())
    coef = ifgf._coefs(vals.reshape(1, 75, 1))[0]
    m = rng.uniform(-1, 1, size=(50, 3))
    B = ifgf._basis(m[:, 0], m[:, 1], m[:, 2])
    assert np.abs(B @ coef[:, 0] - poly(m[:, 0], m[:, 1], m[:, 2])).max() < 1e-12
    h = 1e-6
    Bs = ifgf._basis(m[:, 0], m[:, 1], m[:, 2], (1, 0, 0))
    fd = (poly(m[:, 0] + h, m[:, 1], m[:, 2]) - poly(m[:, 0] - h, m[:, 1], m[:, 2])) / (2 * h)
    assert np.abs(Bs @ coef[:, 0] - fd).max() < 1e-6


def test_interpolation_points_lie_in_their_cone_at_the_nodes():
    lv = ifgf.Level(d=4, H=0.3, ns=4, na=6)
    cones = np.array([[0, 0, 0], [3, 5, 11], [1, 2, 7], [2, 5, 0]])
    X = ifgf.interp_points(lv, cones)
    for i, g in enumerate(cones):
        got = ifgf.cone_of(lv, X[i])
        assert np.all(got == g)
        ts, tt, tp, _, _, _ = ifgf.local_coords(lv, np.repeat(g[None], 75, axis=0), X[i])
        q = np.arange(75)
        assert np.allclose(ts, ifgf.cheb_nodes(3)[q // 25], atol=1e-12)
        assert np.allclose(tt, ifgf.cheb_nodes(5)[(q // 5) % 5], atol=1e-12)
        assert np.allclose(tp, ifgf.cheb_nodes(5)[q % 5], atol=1e-12)


def _densities(prob, seed):
    g = cbie.geometry_of(prob)
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((prob.n, 8)) + 1j * rng.standard_normal((prob.n, 8))
    return g, phi * g.omega[:, None]


@pytest.mark.parametrize("case", ["sphere", "bar"])
def test_exact_box_sums_reproduce_the_plain_far_sum(case):
    """With every interpolation replaced by the exact box sum, the decomposition (cousin
    records of every level) gives the plain far sum: each far pair counted once."""
    if case == "sphere":
        prob = sphere_problem(0.5, 1, 6, 2.25)
        tree_kw = dict(leaf_size=0.11, ns0=2, na0=3)
    else:
        prob = waveguide_bar(0.5, nc=4, half_lengths=(1.5, 0.15, 0.07))
        tree_kw = dict(leaf_size=0.25 * 2 * np.pi / prob.k_ext, ns0=2, na0=3, max_leaf_pts=8)
    g, a = _densities(prob, 1)
    tree = ifgf.build_tree(g.x, k_max=max(prob.k_ext, prob.k_int), **tree_kw)
    ref = ifgf.direct_far(g.x, g.n, a, prob.k_ext, prob.k_int, tree.leafc)
    ex = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int, exact=True)
    assert rel(ex, ref) < 1e-13


def test_interpolation_error_falls_with_cone_refinement():
    """The IFGF approximation of the far sums (S and dS/dn fields, 6-patch sphere, D = 5)
    improves as the cone segments are refined: cones (1,2), (2,3), (4,6) at level D+1."""
    prob = sphere_problem(0.5, 1, 6, 2.25)
    g, a = _densities(prob, 2)
    errs = []
    for cones in ((1, 2), (2, 3), (4, 6)):
        tree = ifgf.build_tree(g.x, 0.11, max(prob.k_ext, prob.k_int), *cones)
        ref = ifgf.direct_far(g.x, g.n, a, prob.k_ext, prob.k_int, tree.leafc)
        ap = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int)
        errs.append((rel(ap[:, :16], ref[:, :16]), rel(ap[:, 16:], ref[:, 16:])))
    for k in range(2):
        assert errs[0][k] > 3 * errs[1][k] > 9 * errs[2][k], errs
    assert errs[2][0] < 2e-6 and errs[2][1] < 5e-5, errs


@pytest.mark.parametrize("case", ["sphere", "sphere6", "bar", "fine_cones"])
def test_oracle_tree_matches_the_library_host_tables(case):
    """Levels, cone counts, relevant cone segments per box and every (target, box, cone)
    record of the oracle's tree equal the library's host tables (ifgf_tree_*).  'fine_cones'
    (ns0 = na0 = 64) gives levels with more than 2^24 cones, where the library de-duplicates a
    box's cones by sorting instead of one bit per cone."""
    lib = pytest.importorskip("paper_2408_02274_gb300")
    if case == "sphere":
        prob = sphere_problem(0.5, 2, 6, 2.25)
        kw = dict(leaf_size=0.11, ns0=2, na0=3)
    elif case == "sphere6":     # the body of the GPU comparison of the IFGF fields
        prob = sphere_problem(0.5, 1, 6, 2.25)
        kw = dict(leaf_size=0.11, ns0=2, na0=3)
    elif case == "fine_cones":
        prob = sphere_problem(0.5, 1, 6, 2.25)
        kw = dict(leaf_size=0.11, ns0=64, na0=64)
    else:
        prob = waveguide_bar(0.5, nc=4, half_lengths=(1.5, 0.15, 0.07))
        kw = dict(leaf_size=0.25 * 2 * np.pi / prob.k_ext, ns0=2, na0=3, max_leaf_pts=8)
    x, _, _ = prob.nodes()
    kmax = max(prob.k_ext, prob.k_int)
    ot = ifgf.build_tree(x, k_max=kmax, **kw)
    ht = lib.Tree(x, k_max=kmax, **kw)
    assert ht.levels == ot.D
    perm, leafc = ht.perm()
    assert np.array_equal(leafc, ot.leafc)
    mask = (1 << 21) - 1
    for d in range(3, ot.D + 1):
        lv = ot.levels[d]
        coords, ptr, cones, ns, na = ht.level(d)
        assert (ns, na) == (lv.ns, lv.na)
        where = {tuple(c): b for b, c in enumerate(lv.boxes.tolist())}
        trip = np.stack([cones >> 42, (cones >> 21) & mask, cones & mask], axis=1)
        for hb, c in enumerate(coords.tolist()):
            ob = where[tuple(c)]
            assert np.array_equal(lv.key(trip[ptr[hb]:ptr[hb + 1]]), lv.cones[ob])
        tp, ts, sb = ht.targets(d)
        host = set()
        for s in range(x.shape[0]):
            for slot in ts[tp[s]:tp[s + 1]]:
                host.add((int(perm[s]), tuple(coords[sb[slot]].tolist()), int(lv.key(trip[slot][None])[0])))
        mine = {(int(n), tuple(lv.boxes[b].tolist()), int(k)) for n, b, k in zip(lv.tgt_node, lv.tgt_box, lv.tgt_key)}
        assert host == mine
    ht.close()


def test_radial_floor_on_a_low_frequency_leaf():
    """Reading R25 on the oracle: a deep point-count tree whose leaf level has k_max H_D <= 1/2
    keeps the base radial count 2 without the floor; the floor's 4 cells cut the error about
    four-fold (measured S 8.5e-5 -> 2.2e-5, dS/dn 6.4e-4 -> 1.6e-4)."""
    prob = waveguide_bar(0.5, nc=4, half_lengths=(1.5, 0.15, 0.07), eps_ext=1.0, eps_int=2.25)
    g, a = _densities(prob, 1)
    leaf = 0.25 * 2 * np.pi / prob.k_ext
    kmax = max(prob.k_ext, prob.k_int)
    errs = {}
    for floor in (False, True):
        tree = ifgf.build_tree(g.x, leaf, kmax, 2, 3, max_leaf_pts=8, radial_floor=floor)
        assert kmax * tree.levels[tree.D].H <= 0.5
        assert tree.levels[tree.D].ns == (4 if floor else 2)
        ref = ifgf.direct_far(g.x, g.n, a, prob.k_ext, prob.k_int, tree.leafc)
        ap = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int)
        errs[floor] = (rel(ap[:, :16], ref[:, :16]), rel(ap[:, 16:], ref[:, 16:]))
    assert errs[True][0] < 0.4 * errs[False][0] and errs[True][1] < 0.4 * errs[False][1], errs


DIRECT_FAR_MUTANTS = [
    ("dG = nd * (1j * kap - 1.0 / dist) * G", "dG = nd * (1j * kap + 1.0 / dist) * G"),   # sign of 1/r
    ("G = np.exp(1j * kap * dist) / (4 * np.pi * dist)",
     "G = np.exp(1j * kap * dist) / (2 * np.pi * dist)"),                                # 1/(4 pi)
    ("nd = (R @ nrm[l]) / dist", "nd = -(R @ nrm[l]) / dist"),                           # x - y reversed
    ("G = np.exp(1j * kap * dist)", "G = np.exp(-1j * kap * dist)"),                     # outgoing wave
]


def test_direct_far_equals_the_cores_regular_patch_entries():
    """The plain far sum (direct_far, the reference of every IFGF pin) against the C core's
    kernel rows, which the sphere eigen-relations pin independently: for a target l and a
    source m on a patch regular for l, the core's entries are the Fejer terms G_s(x_l, x_m)
    omega_m and dG_s/dn(x_l) omega_m (Eq. non_sing).  Sources on patches that may be singular
    for a tested row (node distance <= delta + the patch's node gap, the core's own safe
    prefilter) get zero density, so both sides sum the same pairs: the far pairs of the leaf
    rule on regular patches.  Planted mistakes in direct_far (sign of the 1/r term of dG/dn,
    the 1/(4 pi), the direction of x - y, an incoming wave) fail the same comparison."""
    import inspect
    import textwrap

    prob = sphere_problem(1.0, 3, 6, 2.25)          # 54 patches x 36 nodes
    g = cbie.geometry_of(prob)
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=24, cov_d=4.0)
    P, npp = prob.num_patches, prob.nc ** 2
    rows = np.arange(7 * npp, 8 * npp)
    gap = cbie.node_gap(g.x, P, prob.nc)
    xp = g.x.reshape(P, npp, 3)
    maybe_sing = np.zeros(P, dtype=bool)
    for l in rows:
        dmin = np.linalg.norm(xp - g.x[l], axis=-1).min(axis=1)
        maybe_sing |= dmin <= qp.delta + gap
    assert 0 < maybe_sing.sum() < 0.5 * P
    tree = ifgf.build_tree(g.x, 0.2, max(prob.k_ext, prob.k_int), 2, 3)
    rng = np.random.default_rng(21)
    phi = rng.standard_normal((prob.n, 8)) + 1j * rng.standard_normal((prob.n, 8))
    phi[np.repeat(maybe_sing, npp)] = 0.0
    K, _ = cbie.kernel_rows(prob, g, rows, qp)
    far = np.array([np.any(np.abs(tree.leafc - tree.leafc[l]) > 1, axis=1) for l in rows])   # [rows, N]
    assert far.sum() > 0.5 * rows.size * prob.n * (1 - maybe_sing.mean())
    ref = np.empty((rows.size, 28), dtype=complex)
    for s in range(2):
        ref[:, 8 * s:8 * s + 8] = (K[s] * far) @ phi
        ref[:, 16 + 6 * s:22 + 6 * s] = (K[2 + s] * far) @ phi[:, :6]

    def worst(fn):
        got = fn(g.x, g.n, phi * g.omega[:, None], prob.k_ext, prob.k_int, tree.leafc)[rows]
        return max(rel(got[:, :16], ref[:, :16]), rel(got[:, 16:], ref[:, 16:]))

    assert worst(ifgf.direct_far) < 1e-13
    src = textwrap.dedent(inspect.getsource(ifgf.direct_far))
    for old, new in DIRECT_FAR_MUTANTS:
        assert src.count(old) == 1, old
        ns = dict(vars(ifgf))
        exec(compile(src.replace(old, new), "<mutant of direct_far>", "exec"), ns)
        assert worst(ns["direct_far"]) > 1e-3, (old, new)
