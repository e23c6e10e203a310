"""Synthetic closed surfaces made of curvilinear quadrilateral patches.

Every body is a list of patches eta_p : [-1,1]^2 -> R^3 with
eta_u x eta_v pointing out of the enclosed volume (Sec. III-A, the patch
decomposition Gamma = U_p Gamma_p).  ``Body.eval(p, u, v)`` returns the
exact point and both exact parametric tangents at arbitrary parameter
points; nothing here depends on how the solver discretises the patches.

Node layout contract (Sec. III-A, the node index l = j + Nc*i + p*Nc^2):
``sample_body(body, u)`` returns arrays shaped [P, n, n, 3] whose entry
[p, i, j] is eta_p(u[i], u[j]); ``open_cheb_nodes(n)`` gives the open
Chebyshev parameter points cos((k + 1/2) pi / n) that the surface grids use.
"""
from __future__ import annotations

import numpy as np

__all__ = ["Body", "cubed_sphere", "ellipsoid", "star_body", "superellipsoid_bar", "rounded_bar",
           "open_cheb_nodes", "sample_body"]


def open_cheb_nodes(n: int) -> np.ndarray:
    """Parameter points of the open Chebyshev grid, cos((k+1/2)pi/n), k = 0..n-1."""
    k = np.arange(n, dtype=np.float64)
    return np.cos((k + 0.5) * np.pi / n)


# Proper rotations (det = +1) taking the +z cube face to the six faces, so
# that the outward orientation of the +z face map is preserved.
_FACE_ROT = [
    np.eye(3),
    np.array([[1.0, 0, 0], [0, -1, 0], [0, 0, -1]]),      # -z
    np.array([[0.0, 0, 1], [0, 1, 0], [-1, 0, 0]]),       # +x
    np.array([[0.0, 0, -1], [0, 1, 0], [1, 0, 0]]),       # -x
    np.array([[1.0, 0, 0], [0, 0, 1], [0, -1, 0]]),       # +y
    np.array([[1.0, 0, 0], [0, 0, -1], [0, 1, 0]]),       # -y
]


class Body:
    """A closed surface given by patch maps.

    Each patch is a tuple (face, I, J, split): the cube face index, the
    sub-square (I along u, J along v) and the number of sub-squares per face
    edge.  ``radial`` maps unit directions w (shape [..., 3]) to surface
    points and returns (x, dx/dw as a [..., 3, 3] Jacobian); the cube-face
    direction map is q/|q|_norm with q = (tan(pi U/4), tan(pi V/4), 1) for
    spheres, or the generalised q/|q|_p for superellipsoids.
    """

    def __init__(self, patches, surf, name: str):
        self.patches = list(patches)
        self._surf = surf
        self.name = name
        self.sample = None   # optional: all patches at once, same values as eval per patch

    @property
    def num_patches(self) -> int:
        return len(self.patches)

    def eval(self, p: int, u, v):
        """Exact eta_p(u, v), d eta_p/du and d eta_p/dv for arrays u, v of equal shape."""
        face, I, J, split = self.patches[p]
        u = np.asarray(u, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        U = -1.0 + (2.0 * I + (u + 1.0)) / split
        V = -1.0 + (2.0 * J + (v + 1.0)) / split
        tu = np.tan(np.pi * U / 4.0)
        tv = np.tan(np.pi * V / 4.0)
        q = np.stack([tu, tv, np.ones_like(tu)], axis=-1)
        dq_du = np.zeros_like(q)
        dq_dv = np.zeros_like(q)
        dq_du[..., 0] = (np.pi / 4.0) * (1.0 + tu * tu) / split
        dq_dv[..., 1] = (np.pi / 4.0) * (1.0 + tv * tv) / split
        R = _FACE_ROT[face]
        q = q @ R.T
        dq_du = dq_du @ R.T
        dq_dv = dq_dv @ R.T
        x, jac = self._surf(q)                       # x [...,3], jac [...,3,3] = dx/dq
        xu = np.einsum("...ij,...j->...i", jac, dq_du)
        xv = np.einsum("...ij,...j->...i", jac, dq_dv)
        return x, xu, xv


def _face_patches(split: int):
    return [(f, I, J, split) for f in range(6) for I in range(split) for J in range(split)]


def _sphere_surf(radius, axes, center):
    A = np.diag(np.asarray(axes, dtype=np.float64)) * radius
    c = np.asarray(center, dtype=np.float64)

    def surf(q):
        nq = np.sqrt(np.sum(q * q, axis=-1))
        w = q / nq[..., None]
        # d(q/|q|)/dq = (I - w w^T)/|q|
        eye = np.eye(3)
        dw = (eye - w[..., :, None] * w[..., None, :]) / nq[..., None, None]
        x = w @ A.T + c
        jac = np.einsum("ij,...jk->...ik", A, dw)
        return x, jac

    return surf


def cubed_sphere(radius: float, split: int, center=(0.0, 0.0, 0.0)) -> Body:
    """Equiangular cubed sphere: 6 * split^2 patches."""
    return Body(_face_patches(split), _sphere_surf(radius, (1.0, 1.0, 1.0), center),
                f"sphere(r={radius},split={split})")


def ellipsoid(semi_axes, split: int, center=(0.0, 0.0, 0.0)) -> Body:
    """Cubed-sphere map stretched along the axes: x = diag(a,b,c) q/|q|."""
    return Body(_face_patches(split), _sphere_surf(1.0, semi_axes, center),
                f"ellipsoid({tuple(semi_axes)},split={split})")


def superellipsoid_bar(half_lengths, exponent: int, split_per_face, center=(0.0, 0.0, 0.0)) -> Body:
    """|x/A|^e + |y/B|^e + |z/C|^e = 1 (e even): x = diag(A,B,C) q/|q|_e.

    ``split_per_face`` is an int (same split on every face) or a list of six
    (nu, nv) pairs; faces are listed in the order +z, -z, +x, -x, +y, -y.
    """
    e = int(exponent)
    if e % 2:
        raise ValueError("exponent must be even")
    A = np.diag(np.asarray(half_lengths, dtype=np.float64))
    c = np.asarray(center, dtype=np.float64)

    def surf(q):
        s = np.sum(q ** e, axis=-1)
        nrm = s ** (1.0 / e)
        w = q / nrm[..., None]
        # d(q/|q|_e)/dq = I/|q|_e - q (q^{e-1})^T / |q|_e^{e+1}
        g = q ** (e - 1)
        eye = np.eye(3)
        dw = eye / nrm[..., None, None] - q[..., :, None] * g[..., None, :] / (nrm ** (e + 1))[..., None, None]
        x = w @ A.T + c
        jac = np.einsum("ij,...jk->...ik", A, dw)
        return x, jac

    if isinstance(split_per_face, int):
        patches = _face_patches(split_per_face)
        return Body(patches, surf, f"superellipsoid({tuple(half_lengths)},e={e})")
    patches = []
    for f, (nu, nv) in enumerate(split_per_face):
        for I in range(nu):
            for J in range(nv):
                patches.append((f, I, J, (nu, nv)))
    body = Body(patches, surf, f"superellipsoid({tuple(half_lengths)},e={e})")
    body.eval = _anisotropic_eval(body, surf)
    return body


def rounded_bar(half_lengths, end_length: float, patch_size: float, center=(0.0, 0.0, 0.0),
                exponent: int = 8) -> Body:
    """A straight bar of length 2A along x with rounded-rectangle cross-section
    |y/B|^e + |z/C|^e = 1 (e = `exponent`, even; 8 by default), closed at each end by half of the
    superellipsoid |x'/L|^e + |y/B|^e + |z/C|^e = 1 (x' the distance past the end of the straight
    part, L = `end_length`), so the total length stays 2A.  The surface is C^(e-1) where the
    straight part meets the ends and analytic on every patch.

    Parts (each split into patches of side about `patch_size`):
      - four straight sides (normals +z, -z, +y, -y): x = (A - L) U linear in U, and across the
        side the 2-D cube map (t, 1)/(1 + t^e)^(1/e), t = tan(pi V/4), scaled by (B, C);
      - at each end, the end face of the small superellipsoid (L, B, C) under the cube-face map
        w = q/|q|_e, q = (tan(pi U/4), tan(pi V/4), 1) rotated, and the halves of its four side
        faces that lie beyond the straight part; at the junction these take the same
        cross-section parametrisation as the straight sides.
    Patch tuples are (kind, face, I, J, (nu, nv), (U0, U1)) with kind 0 = straight side,
    1 = end face, 2 = end half face, face the cube face of the rotation table, and U in
    [U0, U1] split nu ways.  Derivatives come from complex-step differentiation of the
    analytic maps (exact to rounding)."""
    A, B, C = (float(v) for v in half_lengths)
    L = float(end_length)
    e = int(exponent)
    if e < 2 or e % 2:
        raise ValueError("exponent must be even and >= 2")
    if not (0.0 < L < A):
        raise ValueError("need 0 < end_length < A")
    scale = np.array([1.0, B, C])
    cen = np.asarray(center, dtype=np.float64)
    a0 = A - L

    def point(kind, face, side, uu, vv):
        R = _FACE_ROT[face]
        tv = np.tan(np.pi * vv / 4.0)
        if kind == 0:
            s = 1.0 / (1.0 + tv ** e) ** (1.0 / e)
            w = np.stack([np.zeros_like(tv), s * tv, s * np.ones_like(tv)], axis=-1) @ R.T
            return w * scale + np.stack([a0 * uu + 0.0 * tv, 0.0 * tv, 0.0 * tv], axis=-1) + cen
        tu = np.tan(np.pi * uu / 4.0)
        q = np.stack([tu, tv, np.ones_like(tu)], axis=-1) @ R.T
        w = q / np.sum(q ** e, axis=-1)[..., None] ** (1.0 / e)
        return w * np.array([L, B, C]) + np.array([side * a0, 0.0, 0.0]) + cen

    # parts: (kind, face, U0, U1)
    parts = [(0, f, -1.0, 1.0) for f in (0, 1, 4, 5)]
    parts += [(1, 2, -1.0, 1.0), (1, 3, -1.0, 1.0)]
    parts += [(2, f, 0.0, 1.0) for f in (0, 1, 4, 5)] + [(2, f, -1.0, 0.0) for f in (0, 1, 4, 5)]
    g = np.linspace(0.0, 1.0, 801)
    t, wq = np.polynomial.legendre.leggauss(60)
    tq = 0.5 * (t + 1.0)
    patches = []
    for kind, face, U0, U1 in parts:
        side = 1.0 if (face == 2 or (kind == 2 and U0 >= 0.0)) else -1.0
        uu = U0 + (U1 - U0) * g
        xa = point(kind, face, side, uu, np.zeros_like(g))
        xb = point(kind, face, side, np.full_like(g, 0.5 * (U0 + U1)), -1.0 + 2.0 * g)
        au = float(np.sum(np.linalg.norm(np.diff(xa, axis=0), axis=1)))
        av = float(np.sum(np.linalg.norm(np.diff(xb, axis=0), axis=1)))
        Uq, Vq = np.meshgrid(U0 + (U1 - U0) * tq, -1.0 + 2.0 * tq, indexing="ij")
        h = 1e-30
        xu = np.imag(point(kind, face, side, Uq + 1j * h, Vq.astype(np.complex128))) / h
        xv = np.imag(point(kind, face, side, Uq.astype(np.complex128), Vq + 1j * h)) / h
        area = float(np.sum(np.outer(wq, wq) * np.linalg.norm(np.cross(xu, xv), axis=-1))) * 0.5 * (U1 - U0)
        sc = np.sqrt(area / (au * av))
        nu = max(1, int(np.ceil(au * sc / patch_size)))
        nv = max(1, int(np.ceil(av * sc / patch_size)))
        for I in range(nu):
            for J in range(nv):
                patches.append((kind, face, I, J, (nu, nv), (U0, U1)))
    body = Body(patches, None, f"rounded_bar({A},{B},{C},L={L},h={patch_size})")

    def ev(p, u, v):
        kind, face, I, J, (nu, nv), (U0, U1) = body.patches[p]
        side = 1.0 if (face == 2 or (kind == 2 and U0 >= 0.0)) else -1.0
        u = np.asarray(u, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        du = (U1 - U0) / nu
        U = U0 + du * (I + 0.5 * (u + 1.0))
        V = -1.0 + (2.0 * J + (v + 1.0)) / nv
        h = 1e-30
        x = point(kind, face, side, U, V)
        xu = np.imag(point(kind, face, side, U + 1j * (0.5 * du * h), V.astype(np.complex128))) / h
        xv = np.imag(point(kind, face, side, U.astype(np.complex128), V + 1j * (h / nv))) / h
        return x, xu, xv

    def sample(u):
        # every patch of one part at once (the same elementwise arithmetic as ev)
        u = np.asarray(u, dtype=np.float64)
        Ug, Vg = np.meshgrid(u, u, indexing="ij")
        n = u.size
        out = [np.empty((body.num_patches, n, n, 3)) for _ in range(3)]
        p0 = 0
        while p0 < body.num_patches:
            kind, face, _, _, (nu, nv), (U0, U1) = body.patches[p0]
            npart = nu * nv
            side = 1.0 if (face == 2 or (kind == 2 and U0 >= 0.0)) else -1.0
            I = np.repeat(np.arange(nu), nv)[:, None, None]
            J = np.tile(np.arange(nv), nu)[:, None, None]
            du = (U1 - U0) / nu
            U = U0 + du * (I + 0.5 * (Ug[None] + 1.0))
            V = -1.0 + (2.0 * J + (Vg[None] + 1.0)) / nv
            h = 1e-30
            sl = slice(p0, p0 + npart)
            out[0][sl] = point(kind, face, side, U, V)
            out[1][sl] = np.imag(point(kind, face, side, U + 1j * (0.5 * du * h), V.astype(np.complex128))) / h
            out[2][sl] = np.imag(point(kind, face, side, U.astype(np.complex128), V + 1j * (h / nv))) / h
            p0 += npart
        return tuple(out)

    body.eval = ev
    body.sample = sample
    return body


def _anisotropic_eval(body, surf):
    def ev(p, u, v):
        face, I, J, (nu, nv) = body.patches[p]
        u = np.asarray(u, dtype=np.float64)
        v = np.asarray(v, dtype=np.float64)
        U = -1.0 + (2.0 * I + (u + 1.0)) / nu
        V = -1.0 + (2.0 * J + (v + 1.0)) / nv
        tu = np.tan(np.pi * U / 4.0)
        tv = np.tan(np.pi * V / 4.0)
        q = np.stack([tu, tv, np.ones_like(tu)], axis=-1)
        dq_du = np.zeros_like(q)
        dq_dv = np.zeros_like(q)
        dq_du[..., 0] = (np.pi / 4.0) * (1.0 + tu * tu) / nu
        dq_dv[..., 1] = (np.pi / 4.0) * (1.0 + tv * tv) / nv
        R = _FACE_ROT[face]
        x, jac = surf(q @ R.T)
        xu = np.einsum("...ij,...j->...i", jac, dq_du @ R.T)
        xv = np.einsum("...ij,...j->...i", jac, dq_dv @ R.T)
        return x, xu, xv
    return ev


def _real_ylm_cartesian(l, m, w):
    """Unnormalised real solid-harmonic-like smooth functions of the unit vector w.

    Only used to perturb star-shaped bodies; any smooth function works, so a
    simple polynomial family in (x, y, z) of degree l is used.
    """
    x, y, z = w[..., 0], w[..., 1], w[..., 2]
    terms = {
        (1, -1): y, (1, 0): z, (1, 1): x,
        (2, -2): x * y, (2, -1): y * z, (2, 0): 3 * z * z - 1, (2, 1): x * z, (2, 2): x * x - y * y,
        (3, -3): y * (3 * x * x - y * y), (3, -2): x * y * z, (3, -1): y * (5 * z * z - 1),
        (3, 0): z * (5 * z * z - 3), (3, 1): x * (5 * z * z - 1), (3, 2): z * (x * x - y * y),
        (3, 3): x * (x * x - 3 * y * y),
        (4, -4): x * y * (x * x - y * y), (4, -3): y * z * (3 * x * x - y * y), (4, -2): x * y * (7 * z * z - 1),
        (4, -1): y * z * (7 * z * z - 3), (4, 0): 35 * z ** 4 - 30 * z * z + 3, (4, 1): x * z * (7 * z * z - 3),
        (4, 2): (x * x - y * y) * (7 * z * z - 1), (4, 3): x * z * (x * x - 3 * y * y),
        (4, 4): x ** 4 - 6 * x * x * y * y + y ** 4,
    }
    return terms[(l, m)]


def star_body(radius: float, coeffs: dict, split: int, center=(0.0, 0.0, 0.0)) -> Body:
    """r(w) = radius (1 + sum c_lm Y_lm(w)) along the cubed-sphere direction w."""
    c = np.asarray(center, dtype=np.float64)
    items = sorted(coeffs.items())
    h = 1e-6

    def rad(w):
        r = np.ones(w.shape[:-1])
        for (l, m), cl in items:
            r = r + cl * _real_ylm_cartesian(l, m, w)
        return radius * r

    def surf(q):
        nq = np.sqrt(np.sum(q * q, axis=-1))
        w = q / nq[..., None]
        eye = np.eye(3)
        dw = (eye - w[..., :, None] * w[..., None, :]) / nq[..., None, None]
        r = rad(w)
        # gradient of r(w) along w by central differences on the polynomial (exact to ~1e-10)
        grad = np.zeros(w.shape)
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            grad[..., k] = (rad(w + e) - rad(w - e)) / (2 * h)
        x = r[..., None] * w + c
        # dx/dw = r I + w grad^T ; dx/dq = dx/dw dw/dq
        dxdw = r[..., None, None] * eye + w[..., :, None] * grad[..., None, :]
        jac = np.einsum("...ij,...jk->...ik", dxdw, dw)
        return x, jac

    return Body(_face_patches(split), surf, f"star(r={radius})")


def sample_body(body: Body, u: np.ndarray):
    """Sample every patch on the tensor grid u x u.

    Returns (x, xu, xv), each shaped [P, n, n, 3] with entry [p, i, j] at
    (u[i], u[j]).
    """
    if getattr(body, "sample", None) is not None:
        return body.sample(u)
    u = np.asarray(u, dtype=np.float64)
    U, V = np.meshgrid(u, u, indexing="ij")
    P = body.num_patches
    n = u.size
    x = np.empty((P, n, n, 3))
    xu = np.empty_like(x)
    xv = np.empty_like(x)
    for p in range(P):
        x[p], xu[p], xv[p] = body.eval(p, U, V)
    return x, xu, xv
