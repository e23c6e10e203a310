"""Planted mistakes in the oracle fail its pins (CPU only).

Each mutant rewrites one expression of an oracle function's source (a flipped sign, a dropped
term, a wrong wavenumber or index, a transposed operand), compiles it beside the original, and
runs the pin that must catch it against the mutated oracle: the Mie comparison for the N-Mueller
combination and the right-hand side, the distance to the plain far sum for the IFGF steps, and the
sphere eigenvalues of S and dS/dn for the C core (kernel rows, singular quadrature).  The
unmutated oracle passes the same check in the same test, so a pin that cannot tell them apart
fails here."""
import inspect
import textwrap

import numpy as np
import pytest

from inputs import CONFIG_SPHERE_SMALL, plane_wave, sphere_problem
from oracle import cbie, ifgf, mie


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def mutant(module, name, old, new):
    """module.name with the single occurrence of `old` in its source replaced by `new`."""
    src = textwrap.dedent(inspect.getsource(getattr(module, name)))
    assert src.count(old) == 1, (name, old)
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant of {module.__name__}.{name}>", "exec"), ns)
    return ns[name]


# ------------------------------------------------------------------ N-Mueller operator vs Mie
@pytest.fixture(scope="module")
def mie_case():
    prob = CONFIG_SPHERE_SMALL(8)
    op = cbie.build_operator(prob, cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48))
    inc = plane_wave(op.g.x, prob.k_ext, prob.omega)
    a = 0.5
    pin, pout = mie.fibonacci_sphere(100, 0.7 * a), mie.fibonacci_sphere(100, 1.5 * a)
    refs = (mie.fields(pin, "int", prob.k_ext, prob.k_int, a, prob.omega)
            + mie.fields(pout, "sca", prob.k_ext, prob.k_int, a, prob.omega))
    return prob, op, inc, pin, pout, refs


def mie_error(case):
    """Largest relative error of (E, H) inside and scattered outside against the Mie series for
    the oracle's GMRES solution (the pin's bar is 3e-3)."""
    prob, op, inc, pin, pout, refs = case
    b = cbie.rhs(prob, op.g, inc)
    y, _, _ = cbie.gmres(lambda v: cbie.apply(op, v.reshape(4, -1)).reshape(-1), b.reshape(-1),
                         tol=1e-10, maxiter=200)
    y = y.reshape(4, -1)
    got = cbie.fields_off_surface(prob, y, pin, "int") + cbie.fields_off_surface(prob, y, pout, "ext")
    return max(rel(g, r) for g, r in zip(got, refs))


MIE_MUTANTS = [
    ("combine", "(Tj_e - Tj_i)", "(Tj_e + Tj_i)"),                              # sign of T on j
    ("combine", " + (mue * Km_e - mui * Km_i)", ""),                            # K term dropped
    ("combine", "ki ** 2 * Rj_i", "ke ** 2 * Rj_i"),                            # wrong wavenumber
    ("combine", "m = y[0][:, None] * g.t1 + y[1][:, None] * g.t2",
                "m = y[0][:, None] * g.t2 + y[1][:, None] * g.t1"),             # tangents transposed
    ("combine", "out[3] = np.sum(row2 * g.t2, 1)", "out[3] = np.sum(row2 * g.t1, 1)"),   # wrong index
    ("rhs", "nH = np.cross(g.n, H)", "nH = np.cross(H, g.n)"),                  # sign of n x H
]


def test_mie_pin_catches_planted_operator_mistakes(mie_case, monkeypatch):
    assert mie_error(mie_case) < 3e-3
    for name, old, new in MIE_MUTANTS:
        with monkeypatch.context() as m:
            m.setattr(cbie, name, mutant(cbie, name, old, new))
            err = mie_error(mie_case)
        assert err > 3e-3, (name, old, new, err)


# ------------------------------------------------------------------ IFGF steps vs the plain far sum
IFGF_MUTANTS = [
    ("ifgf_far", "fac = (rp / rc) * np.exp", "fac = (rc / rp) * np.exp"),          # re-centring inverted
    ("ifgf_far", "nph = -n[:, 0] * sp + n[:, 1] * cp", "nph = n[:, 0] * sp + n[:, 1] * cp"),   # d/dn sign
    ("ifgf_far", "dG = nr * (1j * kap - 1.0 / r) * G", "dG = nr * (1j * kap + 1.0 / r) * G"),  # dG sign
    ("_analytic_factor", "np.exp(1j * kap * (d - r))", "np.exp(1j * kap * (r - d))"),     # factor sign
    ("local_coords", "tt = 2.0 * (th / lv.dth - cones[:, 1]) - 1.0",
                     "tt = 2.0 * (th / lv.dth - cones[:, 1]) + 1.0"),                  # shifted cell
]


def test_far_sum_pin_catches_planted_ifgf_mistakes(monkeypatch):
    """Cones (1, 2) on a 96-node sphere: the oracle IFGF is within 1e-4 (S) and 5e-4 (dS/dn)
    of the plain far sum; every mutant is off by more than 1e-2 in one of the two."""
    prob = sphere_problem(0.5, 1, 4, 2.25)
    g = cbie.geometry_of(prob)
    rng = np.random.default_rng(2)
    a = (rng.standard_normal((prob.n, 8)) + 1j * rng.standard_normal((prob.n, 8))) * g.omega[:, None]
    tree = ifgf.build_tree(g.x, 0.11, max(prob.k_ext, prob.k_int), 1, 2)
    assert tree.D >= 4                                     # an upward step is exercised
    ref = ifgf.direct_far(g.x, g.n, a, prob.k_ext, prob.k_int, tree.leafc)

    def errs():
        ap = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int)
        return rel(ap[:, :16], ref[:, :16]), rel(ap[:, 16:], ref[:, 16:])

    e_s, e_d = errs()
    assert e_s < 1e-4 and e_d < 5e-4
    for name, old, new in IFGF_MUTANTS:
        with monkeypatch.context() as m:
            m.setattr(ifgf, name, mutant(ifgf, name, old, new))
            e = errs()
        assert max(e) > 1e-2, (name, old, new, e)


# ------------------------------------------------------------------ C core (kernel rows) vs sphere eigenvalues
C_MUTANTS = [
    ("K[2 + s] = nd * (I * kk[s] * r - 1.0) * g / (r * r);",
     "K[2 + s] = nd * (I * kk[s] * r + 1.0) * g / (r * r);"),                       # dG/dn sign
    ("if (n > 1) Dk[1] = delta;", "if (n > 1) Dk[1] = -delta;"),                  # first difference
    ("double wt = J * ub[2 * i + 1] * vb[2 * j + 1] * w_beta[i] * w_beta[j];",
     "double wt = J * ub[2 * i + 1] * w_beta[i] * w_beta[j];"),                     # Jacobian in v dropped
    ("kernels4n(dneg, -ne, ke, ki, k4);", "kernels4n(dneg, ne, ke, ki, k4);"),    # own-patch normal sign
    ("acc += A[m * nc + ip] * tmp2", "acc += A[ip * nc + m] * tmp2"),              # transposed map
    ("*dw = 2.0 * M_PI * (da * b - a * db)", "*dw = 2.0 * M_PI * (da * b + a * db)"),   # cov derivative
]


def eigen_case():
    """Sphere of radius 1, k_e = 2, k_i = 4, N_c = 10; every 37th node is a tested row."""
    prob = sphere_problem(1.0, 2, 10, 4.0)
    prob.omega = 2.0
    g = cbie.geometry_of(prob)
    qp = cbie.QuadParams(delta=cbie.default_delta(prob), n_beta=48, cov_d=4.0)
    rows = np.arange(0, g.x.shape[0], 37)
    return prob, g, qp, rows


def eigen_errors(prob, g, rows, K):
    """Largest relative error of the kernel rows K [4, rows, N] against the eigenvalues of S and
    p.v. dS/dn on the real Y_lm (l <= 4), separately for S and dS/dn."""
    from scipy.special import sph_harm_y, spherical_jn, spherical_yn

    r = np.linalg.norm(g.x, axis=1)
    th, ph = np.arccos(np.clip(g.x[:, 2] / r, -1, 1)), np.arctan2(g.x[:, 1], g.x[:, 0])
    e = [0.0, 0.0]
    for l, m in ((0, 0), (1, 1), (2, -1), (3, 2), (4, 0)):
        Yc = sph_harm_y(l, abs(m), th, ph)
        Y = np.real(Yc) if m >= 0 else np.imag(Yc)
        for s, k in enumerate((prob.k_ext, prob.k_int)):
            j, dj = spherical_jn(l, k), spherical_jn(l, k, derivative=True)
            h, dh = j + 1j * spherical_yn(l, k), dj + 1j * spherical_yn(l, k, derivative=True)
            lam = (1j * k * j * h, 0.5j * k * k * (dj * h + j * dh))
            for q in range(2):
                err = np.abs(K[2 * q + s] @ Y - lam[q] * Y[rows]).max() / (abs(lam[q]) * np.abs(Y).max())
                e[q] = max(e[q], float(err))
    return e


def core_variant(tmp_path, name, old, new):
    """Path of a library compiled from the oracle's C core with `old` replaced by `new`."""
    import os
    import subprocess

    src = open(os.path.join(os.path.dirname(cbie.__file__), "cbie_core.c")).read()
    assert src.count(old) == 1, old
    c, so = tmp_path / f"core_{name}.c", tmp_path / f"libcore_{name}.so"
    c.write_text(src.replace(old, new))
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", str(c), "-o", str(so), "-lm"])
    return str(so)


def test_eigenvalue_pin_catches_planted_core_mistakes(tmp_path, monkeypatch):
    """Every 37th kernel row against the eigenvalues of S and p.v. dS/dn on Y_lm (l <= 4; the
    pin's bar is 1e-4).  Each mutant of the C core is compiled into its own library and loaded
    in place of the oracle's."""
    prob, g, qp, rows = eigen_case()

    def worst():
        K, _ = cbie.kernel_rows(prob, g, rows, qp)
        return max(eigen_errors(prob, g, rows, K))

    assert worst() < 1e-4
    for i, (old, new) in enumerate(C_MUTANTS):
        so = core_variant(tmp_path, f"mutant{i}", old, new)
        with monkeypatch.context() as m:
            m.setattr(cbie, "_LIB", None)
            m.setattr(cbie, "build_core", lambda force=False, so=so: so)
            e = worst()
        assert e > 1e-4, (old, new, e)


def test_first_order_normal_term_is_below_the_quadrature_error(tmp_path, monkeypatch):
    """Reading R21: on the target's own patch the core forms n.(x - y) from the second-order
    remainder of the patch interpolant and leaves out its first-order part du n.eta_u +
    dv n.eta_v, which vanishes on the exact surface.  A core that keeps it (the plain
    n.(x - y) of the interpolant's displacement) changes the dS/dn rows by ~3e-11 relative
    (measured), six orders of magnitude below the eigen-relation pin's own quadrature error
    (~7e-5 at N_beta = 48), and leaves that error unchanged to 1e-12: the reading changes no
    result at the oracle's accuracy."""
    prob, g, qp, rows = eigen_case()
    K0, _ = cbie.kernel_rows(prob, g, rows, qp)
    so = core_variant(tmp_path, "plain_normal", "*ne = nrm[0] * R[0] + nrm[1] * R[1] + nrm[2] * R[2];",
                      "*ne = nrm[0] * e[0] + nrm[1] * e[1] + nrm[2] * e[2];")
    with monkeypatch.context() as m:
        m.setattr(cbie, "_LIB", None)
        m.setattr(cbie, "build_core", lambda force=False: so)
        K1, _ = cbie.kernel_rows(prob, g, rows, qp)
    e0, e1 = eigen_errors(prob, g, rows, K0), eigen_errors(prob, g, rows, K1)
    assert max(e0) < 1e-4 and max(e1) < 1e-4
    assert np.array_equal(K0[:2], K1[:2])                 # single-layer rows do not use n.(x - y)
    for q in (2, 3):
        d = rel(K1[q], K0[q])
        assert 0 < d < 1e-3 * e0[1], (q, d, e0)
    assert abs(e1[1] - e0[1]) < 1e-12


# ------------------------------------------------------------------ octree and cone tables
TREE_MUTANTS = [
    ("if c not in mine)", "if True)"),                                            # cousins keep neighbours
    ("for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]",
     "for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1) if abs(dx) + abs(dy) + abs(dz) <= 1]"),
    ("a = 2 if k_max * H > 0.5 else 1", "a = 1"),                                 # cones never refined
    ("keys.append(lv.key(cone_of(lv, X)))", "pass"),                              # parent points dropped
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")   # a mutant that pairs a box with itself divides by 0
def test_tree_pins_catch_planted_mistakes(monkeypatch):
    """Mistakes in the octree step (neighbours, cousins, cone counts, relevant cones) fail the
    exact-decomposition pin (exact box sums = plain far sum to 1e-13) or the accuracy pin
    (IFGF within 1e-4 / 5e-4 of the plain far sum), on the 216-node sphere whose cone counts double
    on the upper levels; an exception in the mutated oracle also counts as caught."""
    prob = sphere_problem(0.5, 1, 6, 2.25)
    g = cbie.geometry_of(prob)
    rng = np.random.default_rng(4)
    a = (rng.standard_normal((prob.n, 8)) + 1j * rng.standard_normal((prob.n, 8))) * g.omega[:, None]
    kmax = max(prob.k_ext, prob.k_int)

    def pins_hold():
        tree = ifgf.build_tree(g.x, 0.11, kmax, 1, 2)
        ref = ifgf.direct_far(g.x, g.n, a, prob.k_ext, prob.k_int, tree.leafc)
        ex = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int, exact=True)
        if rel(ex, ref) >= 1e-13:
            return False
        ap = ifgf.ifgf_far(tree, g.x, g.n, a, prob.k_ext, prob.k_int)
        return rel(ap[:, :16], ref[:, :16]) < 1e-4 and rel(ap[:, 16:], ref[:, 16:]) < 5e-4

    assert pins_hold()
    for old, new in TREE_MUTANTS:
        with monkeypatch.context() as m:
            m.setattr(ifgf, "build_tree", mutant(ifgf, "build_tree", old, new))
            try:
                held = pins_hold()
            except Exception:
                held = False
        assert not held, (old, new)
