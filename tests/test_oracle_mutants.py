"""Planted mistakes in the oracle fail its pins (CPU only).

Each mutant rewrites one expression of an oracle function's source (a flipped sign, a dropped
term, a wrong wavenumber or index, a transposed operand), compiles it beside the original, and
runs the pin that must catch it against the mutated oracle: the Mie comparison for the N-Mueller
combination and the right-hand side, the distance to the plain far sum for the IFGF steps.  The
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
