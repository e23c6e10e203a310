"""Plain CPU FP64 oracle of the CBIE N-Mueller forward map, RHS, solve and fields.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library and never runs on its product path.

What it computes is the unaccelerated discrete operator of Paul & Sideris
(the "CBIE" forward map of Sec. IV-A), written step by step:

* discretisation: open Chebyshev grid (Eq. cheby_nodes), node order
  l = j + Nc i + p Nc^2 (Eq. mesh_pts_l), Fejer weights (Eq. fejer_weighs);
* scalar operators S (Eq. sl_scalar) and D = dS/dn (Eq. dl_scalar) at the
  nodes: Fejer rule for regular patches (Eq. non_sing), precomputed
  moments for singular patches (Eqs. rp_exp, int_moments, int_moments_cov)
  -- both in the C core ``cbie_core.c``;
* the vector operators R, K, T (Eqs. potential_r/k/t) rebuilt from S and D
  with Chebyshev surface derivatives (Sec. III, first paragraph), and the
  N-Mueller block operator (Eqs. n_muller, k_delta, r_delta, t_delta);
* the right-hand side omega^{-1}(n x E^inc, n x H^inc) and GMRES on A y = b
  (Eq. lin_system).

Where the paper leaves a point open, the reading taken is noted at the
function that uses it (readings R1..R16).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build_core(force: bool = False) -> str:
    """Compile the C core with gcc (test infrastructure)."""
    so = os.path.join(_HERE, "libcbie_oracle.so")
    src = os.path.join(_HERE, "cbie_core.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", src, "-o", so, "-lm"])
    return so


def _lib():
    global _LIB
    if _LIB is None:
        _LIB = ctypes.CDLL(build_core())
        d = ctypes.POINTER(ctypes.c_double)
        i = ctypes.POINTER(ctypes.c_int)
        _LIB.ora_kernel_rows.restype = ctypes.c_int
        _LIB.ora_kernel_rows.argtypes = [ctypes.c_int] * 3 + [d] * 7 + [ctypes.c_double] * 3 + \
            [ctypes.c_int, d, d, ctypes.c_double, ctypes.c_int, ctypes.c_int, i, d, i]
        _LIB.ora_closest_point.restype = ctypes.c_double
        _LIB.ora_closest_point.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, d, ctypes.c_int, d]
        _LIB.ora_cov.restype = None
        _LIB.ora_cov.argtypes = [ctypes.c_double, ctypes.c_int, d, ctypes.c_double, d, d]
    return _LIB


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ----------------------------------------------------------------------------- 1D Chebyshev
def cheb_nodes(n: int) -> np.ndarray:
    """Open Chebyshev nodes u_k = cos((k + 0.5) pi / n) (Eq. cheby_nodes)."""
    return np.cos((np.arange(n) + 0.5) * np.pi / n)


def fejer_weights(n: int) -> np.ndarray:
    """Fejer's first-rule weights on the open Chebyshev nodes (Eq. fejer_weighs)."""
    w = np.empty(n)
    for k in range(n):
        s = 0.0
        for m in range(1, n // 2 + 1):
            s += np.cos(m * np.pi * (2 * k + 1) / n) / (4.0 * m * m - 1.0)
        w[k] = (2.0 / n) * (1.0 - 2.0 * s)
    return w


def cheb_T(x, n: int) -> np.ndarray:
    """Matrix [len(x), n] of T_k(x) by the three-term recurrence."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    T = np.empty((x.size, n))
    T[:, 0] = 1.0
    if n > 1:
        T[:, 1] = x
    for k in range(2, n):
        T[:, k] = 2 * x * T[:, k - 1] - T[:, k - 2]
    return T


def cheb_dT(x, n: int) -> np.ndarray:
    """Matrix [len(x), n] of T_k'(x) = k U_{k-1}(x)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    U = np.empty((x.size, max(n, 1)))
    U[:, 0] = 1.0
    if n > 1:
        U[:, 1] = 2 * x
    for k in range(2, n):
        U[:, k] = 2 * x * U[:, k - 1] - U[:, k - 2]
    dT = np.zeros((x.size, n))
    for k in range(1, n):
        dT[:, k] = k * U[:, k - 1]
    return dT


def vals_to_coefs(n: int) -> np.ndarray:
    """Map A with a = A f: coefficients of the degree n-1 interpolant on the open grid.

    Sec. III-E (1D Chebyshev interpolation).  The paper attaches the factor
    c_0 = 1/2 to the sample index; the discrete orthogonality of T_k on these
    nodes puts it on the coefficient index (reading R7): a_0 = (1/n) sum f_j,
    a_i = (2/n) sum_j f_j T_i(x_j).
    """
    x = cheb_nodes(n)
    T = cheb_T(x, n)                 # [j, i]
    A = (2.0 / n) * T.T.copy()       # [i, j]
    A[0, :] *= 0.5
    return A


def cheb_diff(n: int) -> np.ndarray:
    """Differentiation matrix at the open nodes: derivative of the interpolant (Sec. III, recurrences)."""
    x = cheb_nodes(n)
    return cheb_dT(x, n) @ vals_to_coefs(n)


# ----------------------------------------------------------------------------- geometry
@dataclass
class Geometry:
    P: int
    nc: int
    x: np.ndarray        # [N,3]
    xu: np.ndarray       # [N,3]
    xv: np.ndarray       # [N,3]
    n: np.ndarray        # [N,3] unit normal (eta_u x eta_v)/J
    J: np.ndarray        # [N]   |eta_u x eta_v|
    omega: np.ndarray    # [N]   J w_i w_j (Sec. III-C)
    t1: np.ndarray       # [N,3] eta_u/|eta_u|
    t2: np.ndarray       # [N,3] n x t1
    guu: np.ndarray      # inverse metric components [N]
    guv: np.ndarray
    gvv: np.ndarray


def make_geometry(P: int, nc: int, x, xu, xv) -> Geometry:
    """Normals, Jacobians and quadrature weights at the nodes (Eqs. sl_p, non_sing, reading R5)."""
    cr = np.cross(xu, xv)
    J = np.linalg.norm(cr, axis=1)
    n = cr / J[:, None]
    w = fejer_weights(nc)
    ww = np.outer(w, w).reshape(-1)
    omega = J * np.tile(ww, P)
    t1 = xu / np.linalg.norm(xu, axis=1)[:, None]
    t2 = np.cross(n, t1)
    E = np.sum(xu * xu, 1)
    F = np.sum(xu * xv, 1)
    G = np.sum(xv * xv, 1)
    det = E * G - F * F
    return Geometry(P, nc, x, xu, xv, n, J, omega, t1, t2, G / det, -F / det, E / det)


def geometry_of(problem) -> Geometry:
    x, xu, xv = problem.nodes()
    return make_geometry(problem.num_patches, problem.nc, x, xu, xv)


def _patch_derivs(f, g: Geometry):
    """Parametric derivatives (f_u, f_v) of node values f [..., N] by per-patch Chebyshev differentiation."""
    Dm = cheb_diff(g.nc)
    sh = f.shape[:-1]
    fp = f.reshape(sh + (g.P, g.nc, g.nc))
    fu = np.einsum("ik,...pkj->...pij", Dm, fp).reshape(f.shape)
    fv = np.einsum("jk,...pik->...pij", Dm, fp).reshape(f.shape)
    return fu, fv


def surface_grad(f, g: Geometry):
    """Surface gradient of node values f [..., N] -> [..., N, 3] (sum g^{ab} f_a eta_b)."""
    fu, fv = _patch_derivs(f, g)
    cu = g.guu * fu + g.guv * fv
    cv = g.guv * fu + g.gvv * fv
    return cu[..., None] * g.xu + cv[..., None] * g.xv


def surface_div(V, g: Geometry):
    """Surface divergence of tangential node vectors V [N,3]: (1/J)[(J V^u)_u + (J V^v)_v]."""
    a = np.sum(V * g.xu, 1)
    b = np.sum(V * g.xv, 1)
    Vu = g.guu * a + g.guv * b
    Vv = g.guv * a + g.gvv * b
    du, _ = _patch_derivs(g.J * Vu, g)
    _, dv = _patch_derivs(g.J * Vv, g)
    return (du + dv) / g.J


# ----------------------------------------------------------------------------- densities
def densities(y, g: Geometry):
    """The eight scalar densities of Sec. III (first paragraph): m_xyz, j_xyz, div m, div j.

    y = [m1, m2, j1, j2] are the components on the orthonormal frame (t1, t2)
    (reading R4).  Returns phi [8, N] complex.
    """
    y = np.asarray(y)
    m = y[0][:, None] * g.t1 + y[1][:, None] * g.t2
    j = y[2][:, None] * g.t1 + y[3][:, None] * g.t2
    phi = np.empty((8, g.x.shape[0]), dtype=np.complex128)
    phi[0:3] = m.T
    phi[3:6] = j.T
    phi[6] = surface_div(m, g)
    phi[7] = surface_div(j, g)
    return phi


# ----------------------------------------------------------------------------- kernel rows
def fine_coefficients(fine, ng: int) -> np.ndarray:
    """2D Chebyshev coefficients of the oversampled patch geometry [P, ng, ng, 9]."""
    A = vals_to_coefs(ng)
    return np.ascontiguousarray(np.einsum("mi,nj,pijc->pmnc", A, A, fine))


def node_gap(x, P: int, nc: int) -> np.ndarray:
    """Per-patch margin: twice the largest node-cell diagonal (reading R15)."""
    xp = x.reshape(P, nc, nc, 3)
    d1 = np.linalg.norm(xp[:, 1:, 1:] - xp[:, :-1, :-1], axis=-1)
    d2 = np.linalg.norm(xp[:, 1:, :-1] - xp[:, :-1, 1:], axis=-1)
    return 2.0 * np.maximum(d1.max(axis=(1, 2)), d2.max(axis=(1, 2)))


@dataclass
class QuadParams:
    delta: float            # singular-set distance threshold (Eq. patch_sing)
    n_beta: int = 24        # Fejer points per direction for the moments (Eq. int_moments_cov)
    cov_d: float = 4.0      # change-of-variables order d >= 2 (Eq. mk_cov_1)
    gs_iters: int = 60      # golden-section iterations per level (Eq. dist_min)


def default_delta(problem) -> float:
    """Reading R14: delta = 0.6 x the largest patch diameter (max node distance within a patch)."""
    x, _, _ = problem.nodes()
    P, nc = problem.num_patches, problem.nc
    xp = x.reshape(P, nc * nc, 3)
    diam = 0.0
    for p in range(P):
        d = np.linalg.norm(xp[p][:, None, :] - xp[p][None, :, :], axis=-1)
        diam = max(diam, d.max())
    return 0.6 * diam


def kernel_rows(problem, g: Geometry, rows, qp: QuadParams):
    """Four dense kernel rows [4, len(rows), N] (S_e, S_i, D_e, D_i) acting on phi, plus |S_l|."""
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    P, nc, ng = problem.num_patches, problem.nc, problem.ng
    N = P * nc * nc
    coef = fine_coefficients(problem.fine(), ng)
    gap = node_gap(g.x, P, nc)
    u = cheb_nodes(nc)
    A = np.ascontiguousarray(vals_to_coefs(nc))
    tb = cheb_nodes(qp.n_beta)
    wb = fejer_weights(qp.n_beta)
    K = np.zeros((4, rows.size, N), dtype=np.complex128)
    sing = np.zeros(rows.size, dtype=np.int32)
    x = np.ascontiguousarray(g.x)
    nrm = np.ascontiguousarray(g.n)
    om = np.ascontiguousarray(g.omega)
    rc = _lib().ora_kernel_rows(
        P, nc, ng, _dp(x), _dp(nrm), _dp(om), _dp(coef), _dp(gap), _dp(u), _dp(A),
        problem.k_ext, problem.k_int, qp.delta, qp.n_beta, _dp(tb), _dp(wb), qp.cov_d,
        qp.gs_iters, rows.size, rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        K.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        sing.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != 0:
        raise RuntimeError("ora_kernel_rows failed")
    return K, sing


def closest_point(problem, p: int, x, gs_iters: int = 60):
    nc, ng = problem.nc, problem.ng
    coef = np.ascontiguousarray(fine_coefficients(problem.fine(), ng)[p])
    xs, _, _ = problem.nodes()
    pn = np.ascontiguousarray(xs.reshape(problem.num_patches, nc * nc, 3)[p])
    u = cheb_nodes(nc)
    uv = np.zeros(2)
    xx = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    d = _lib().ora_closest_point(nc, ng, _dp(pn), _dp(coef), _dp(u), _dp(xx), gs_iters, _dp(uv))
    return d, uv


def change_of_variables(alpha: float, tau, d: float = 4.0):
    tau = np.ascontiguousarray(np.asarray(tau, dtype=np.float64))
    xi = np.zeros_like(tau)
    mu = np.zeros_like(tau)
    _lib().ora_cov(alpha, tau.size, _dp(tau), d, _dp(xi), _dp(mu))
    return xi, mu


# ----------------------------------------------------------------------------- operator
@dataclass
class Operator:
    """The discrete CBIE N-Mueller operator for one problem (dense kernel matrices)."""
    problem: object
    g: Geometry
    K: np.ndarray            # [4, N, N]  S_e, S_i, D_e, D_i acting on phi
    qp: QuadParams

    @property
    def N(self):
        return self.g.x.shape[0]


def build_operator(problem, qp: QuadParams | None = None) -> Operator:
    g = geometry_of(problem)
    qp = qp or QuadParams(delta=default_delta(problem))
    K, _ = kernel_rows(problem, g, np.arange(g.x.shape[0]), qp)
    return Operator(problem, g, K, qp)


def scalar_fields(K, phi):
    """S fields [2, 8, rows] and D fields [2, 6, rows] from the kernel rows and densities."""
    S = np.stack([K[0] @ phi.T, K[1] @ phi.T]).transpose(0, 2, 1)
    D = np.stack([K[2] @ phi[:6].T, K[3] @ phi[:6].T]).transpose(0, 2, 1)
    return S, D


def combine(problem, g: Geometry, y, S, D):
    """N-Mueller combination (Eqs. n_muller, k_delta, r_delta, t_delta) from S and D at all nodes.

    Readings (R6): with frozen n = n(x),
      K_s[Phi] = sum_c n_c grad_G S_s[Phi_c] - P_T D_s[Phi],
      R_s[Phi] = n x S_s[Phi],   T_s[Phi] = n x grad_G S_s[div_G Phi],
    where D_s is the direct (principal) value of dS/dn on Gamma.
    Returns out [4, N] = (row1.t1, row1.t2, row2.t1, row2.t2).
    """
    y = np.asarray(y)
    m = y[0][:, None] * g.t1 + y[1][:, None] * g.t2
    j = y[2][:, None] * g.t1 + y[3][:, None] * g.t2
    n = g.n
    ke, ki = problem.k_ext, problem.k_int
    om = problem.omega

    def PT(v):
        return v - np.sum(v * n, 1)[:, None] * n

    ops = {}
    for s in range(2):
        grads = surface_grad(S[s], g)            # [8, N, 3]
        Km = sum(n[:, c][:, None] * grads[c] for c in range(3)) - PT(D[s][0:3].T)
        Kj = sum(n[:, c][:, None] * grads[3 + c] for c in range(3)) - PT(D[s][3:6].T)
        Rm = np.cross(n, S[s][0:3].T)
        Rj = np.cross(n, S[s][3:6].T)
        Tm = np.cross(n, grads[6])
        Tj = np.cross(n, grads[7])
        ops[s] = (Km, Kj, Rm, Rj, Tm, Tj)
    Km_e, Kj_e, Rm_e, Rj_e, Tm_e, Tj_e = ops[0]
    Km_i, Kj_i, Rm_i, Rj_i, Tm_i, Tj_i = ops[1]
    mue, mui = problem.mu_ext, problem.mu_int
    epe, epi = problem.eps_ext, problem.eps_int
    RT_j = (ke ** 2 * Rj_e - ki ** 2 * Rj_i) + (Tj_e - Tj_i)      # omega/(-i) (R^D + T^D) j
    RT_m = (ke ** 2 * Rm_e - ki ** 2 * Rm_i) + (Tm_e - Tm_i)
    row1 = 0.5 * (mue + mui) * m + (mue * Km_e - mui * Km_i) + (1j / om) * RT_j
    row2 = (-1j / om) * RT_m + 0.5 * (epe + epi) * j + (epe * Kj_e - epi * Kj_i)
    out = np.empty((4, g.x.shape[0]), dtype=np.complex128)
    out[0] = np.sum(row1 * g.t1, 1)
    out[1] = np.sum(row1 * g.t2, 1)
    out[2] = np.sum(row2 * g.t1, 1)
    out[3] = np.sum(row2 * g.t2, 1)
    return out


def apply(op: Operator, y):
    """Forward map A y (the left-hand side of Eq. n_muller), y [4, N] -> [4, N]."""
    phi = densities(y, op.g)
    S, D = scalar_fields(op.K, phi)
    return combine(op.problem, op.g, y, S, D)


def assemble(op: Operator) -> np.ndarray:
    """Dense 4N x 4N matrix of the forward map (columns = A e_k), for small N."""
    N = op.N
    A = np.empty((4 * N, 4 * N), dtype=np.complex128)
    for k in range(4 * N):
        e = np.zeros(4 * N, dtype=np.complex128)
        e[k] = 1.0
        A[:, k] = apply(op, e.reshape(4, N)).reshape(-1)
    return A


def rhs(problem, g: Geometry, inc):
    """b = omega^{-1} (n x E^inc, n x H^inc) projected on (t1, t2) (Eq. n_muller right side)."""
    E = np.asarray(inc[0:3]).T
    H = np.asarray(inc[3:6]).T
    nE = np.cross(g.n, E) / problem.omega
    nH = np.cross(g.n, H) / problem.omega
    b = np.empty((4, g.x.shape[0]), dtype=np.complex128)
    b[0] = np.sum(nE * g.t1, 1)
    b[1] = np.sum(nE * g.t2, 1)
    b[2] = np.sum(nH * g.t1, 1)
    b[3] = np.sum(nH * g.t2, 1)
    return b


# ----------------------------------------------------------------------------- GMRES
def gmres(matvec, b, tol: float = 1e-6, maxiter: int = 500):
    """Unrestarted GMRES from y0 = 0 with classical Gram-Schmidt applied twice (reading R16).

    Stops when the Arnoldi residual estimate |g_{k+1}| / |b| <= tol.  Returns
    (y, iterations, relative residual estimate).
    """
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    nb = np.linalg.norm(b)
    if nb == 0:
        return np.zeros_like(b), 0, 0.0
    V = np.zeros((maxiter + 1, b.size), dtype=np.complex128)
    H = np.zeros((maxiter + 1, maxiter), dtype=np.complex128)
    cs = np.zeros(maxiter, dtype=np.complex128)
    sn = np.zeros(maxiter, dtype=np.complex128)
    gvec = np.zeros(maxiter + 1, dtype=np.complex128)
    V[0] = b / nb
    gvec[0] = nb
    k = 0
    res = 1.0
    for k in range(maxiter):
        w = np.asarray(matvec(V[k]), dtype=np.complex128).reshape(-1)
        h = V[: k + 1].conj() @ w
        w = w - V[: k + 1].T @ h
        h2 = V[: k + 1].conj() @ w
        w = w - V[: k + 1].T @ h2
        h = h + h2
        hn = np.linalg.norm(w)
        H[: k + 1, k] = h
        H[k + 1, k] = hn
        for i in range(k):                       # previous rotations
            t = np.conj(cs[i]) * H[i, k] + np.conj(sn[i]) * H[i + 1, k]
            H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
            H[i, k] = t
        a, c = H[k, k], H[k + 1, k]
        den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
        cs[k] = a / den if den else 1.0
        sn[k] = c / den if den else 0.0
        H[k, k] = np.conj(cs[k]) * a + np.conj(sn[k]) * c
        H[k + 1, k] = 0.0
        gvec[k + 1] = -sn[k] * gvec[k]
        gvec[k] = np.conj(cs[k]) * gvec[k]
        res = abs(gvec[k + 1]) / nb
        if hn != 0:
            V[k + 1] = w / hn
        if res <= tol or hn == 0:
            k += 1
            break
    else:
        k = maxiter
    z = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        z[i] = (gvec[i] - H[i, i + 1:k] @ z[i + 1:k]) / H[i, i]
    y = V[:k].T @ z
    return y, k, res


# ----------------------------------------------------------------------------- fields off Gamma
def upsampled_quadrature(problem, y, nq: int):
    """Densities and geometry on an nq x nq open Chebyshev grid per patch (for off-surface points).

    Densities (Cartesian m, j and their surface divergences) are interpolated
    with their degree Nc-1 Chebyshev interpolants; geometry is sampled
    exactly.  Returns (points [Q,3], weights [Q], m [Q,3], j [Q,3], dm [Q], dj [Q]).
    """
    from inputs.geometry import sample_body
    g = geometry_of(problem)
    phi = densities(y, g)
    P, nc = problem.num_patches, problem.nc
    A = vals_to_coefs(nc)
    uq = cheb_nodes(nq)
    Tq = cheb_T(uq, nc)
    M = Tq @ A                                    # [nq, nc] interpolation matrix
    fq = np.einsum("ai,bj,kpij->kpab", M, M, phi.reshape(8, P, nc, nc)).reshape(8, -1)
    xq, xuq, xvq = sample_body(problem.body, uq)
    Jq = np.linalg.norm(np.cross(xuq, xvq), axis=-1).reshape(-1)
    wq = fejer_weights(nq)
    W = Jq * np.tile(np.outer(wq, wq).reshape(-1), P)
    return xq.reshape(-1, 3), W, fq[0:3].T, fq[3:6].T, fq[6], fq[7]


def far_field(problem, y, dirs, nq: int | None = None):
    """Far-field pattern of the scattered electric field, E^sc(r d) = e^{i k r}/r E_inf(d) + O(1/r^2)
    for r -> infinity along the unit directions dirs [Q, 3]; returns E_inf [Q, 3].

    From the exterior representation of reading R2, E^sc = -omega mu_e curl S_e[m] - i (k^2 S_e[j]
    + grad S_e[div j]) with k = kappa_e: along d, G(x, y) = e^{i k r}/(4 pi r) e^{-i k d.y} (1 +
    O(1/r)) and grad_x -> i k d, so with the far-field moments F[f] = (1/4 pi) int f(y)
    e^{-i k d.y} dy:
        E_inf = -i k omega mu_e (d x F[m]) - i k^2 F[j] + k d F[div j].
    The moments use the Nystrom nodes and weights omega (nq None), or the densities' Chebyshev
    interpolants on an nq x nq grid per patch (the quadrature of fields_off_surface).
    """
    k, mu, om = problem.k_ext, problem.mu_ext, problem.omega
    d = np.asarray(dirs, dtype=np.float64).reshape(-1, 3)
    if nq is None:
        g = geometry_of(problem)
        phi = densities(y, g)
        ys, W, m, j, dj = g.x, g.omega, phi[0:3].T, phi[3:6].T, phi[7]
    else:
        ys, W, m, j, _, dj = upsampled_quadrature(problem, y, nq)
    E = np.exp(-1j * k * (d @ ys.T)) * W[None, :] / (4 * np.pi)            # [Q, nodes]
    Fm, Fj, Fq = E @ m, E @ j, E @ dj
    return -1j * k * om * mu * np.cross(d, Fm) - 1j * k * k * Fj + k * d * Fq[:, None]


def fields_off_surface(problem, y, pts, medium: str, nq: int = 40, chunk: int = 256):
    """E and H of the representation (reading R2) at points off Gamma.

    medium 'int': E_i, H_i with kappa_i (total field inside);
    medium 'ext': E^sc, H^sc with kappa_e (scattered field outside).
      E_s = -omega mu_s curl S_s[m] - i (kappa_s^2 S_s[j] + grad S_s[div j])
      H_s = -omega eps_s curl S_s[j] + i (kappa_s^2 S_s[m] + grad S_s[div m])
    """
    ys, W, m, j, dm, dj = upsampled_quadrature(problem, y, nq)
    if medium == "int":
        k, mu, eps = problem.k_int, problem.mu_int, problem.eps_int
    else:
        k, mu, eps = problem.k_ext, problem.mu_ext, problem.eps_ext
    om = problem.omega
    pts = np.asarray(pts, dtype=np.float64)
    E = np.zeros((pts.shape[0], 3), dtype=np.complex128)
    H = np.zeros_like(E)
    for a in range(0, pts.shape[0], chunk):
        X = pts[a:a + chunk]
        d = X[:, None, :] - ys[None, :, :]                       # x - y
        r = np.linalg.norm(d, axis=-1)
        G = np.exp(1j * k * r) / (4 * np.pi * r) * W[None, :]
        dG = (d * ((1j * k * r - 1) / (r * r) * G)[..., None])  # grad_x G * W
        Sm = G @ m
        Sj = G @ j
        curlSm = np.einsum("qyk,yk->qk", np.roll(dG, -1, axis=2), np.roll(m, -2, axis=1)) - \
            np.einsum("qyk,yk->qk", np.roll(dG, -2, axis=2), np.roll(m, -1, axis=1))
        curlSj = np.einsum("qyk,yk->qk", np.roll(dG, -1, axis=2), np.roll(j, -2, axis=1)) - \
            np.einsum("qyk,yk->qk", np.roll(dG, -2, axis=2), np.roll(j, -1, axis=1))
        gradSdj = np.einsum("qyk,y->qk", dG, dj)
        gradSdm = np.einsum("qyk,y->qk", dG, dm)
        E[a:a + chunk] = -om * mu * curlSm - 1j * (k * k * Sj + gradSdj)
        H[a:a + chunk] = -om * eps * curlSj + 1j * (k * k * Sm + gradSdm)
    return E, H
