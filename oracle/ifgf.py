"""Plain CPU FP64 oracle of the IFGF approximation of the far-field sums.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library and never runs on its product path.

The unaccelerated far sum is an exact definition (``direct_far``); the IFGF
value is an approximation of it, so ``ifgf_far`` takes the algorithm's steps
in the paper's order (Sec. III-G "summary of the algorithm"), for the vector
of Eq. ifgf_sum_em (8 densities x 2 wavenumbers) and the normal derivatives
of the same sums at the targets (Sec. III-I):

1. the box hierarchy (level-1 box, children, relevant boxes Eq. rele_boxes,
   neighbours Eq. box_neighbor, cousins Eq. box_cousin), the cone counts of
   Remark "Choosing cone-structure sizes" and the relevant cone segments
   (Eq. rele_cone_d), recursively from level 3 down to D;
2. on level D, the analytic factor F of every relevant box (Eq.
   bkd_contr_ana_fac) at the interpolation points of its relevant cone
   segments, by direct summation;
3. for d = D, ..., 3: every cousin point is evaluated by interpolating F and
   multiplying by the centred factor (Eq. bkd_contr); every parent's F is
   obtained at its own interpolation points by interpolating each child's F,
   re-centring by G(x, x_child)/G(x, x_parent) and summing over the children.

Interpolation inside a cone segment is the tensor Chebyshev interpolant of
Sec. III-E: P_s = 3 points in s = h/r, P_a = 5 in theta and in phi, the
open Chebyshev nodes of Eq. cheby_nodes mapped to the segment, coefficients
from the values by the 1D transform with c_0 = 1/2 on the coefficient index
(reading R7).  The readings the CUDA library documents for the same steps
are taken here too, each written out where it is used: the level-1 box and
D (R11), neighbours by the infinity norm (R10), half-open cells clamped at
the top with phi = atan2 in [0, 2 pi) (R8), cone counts from
(n_s, n_a)_{D+1} with a_d = 2 iff k_max H_d > 1/2 and k_max the larger
wavenumber (R9), the radial floor n_s >= 2 n_{s;D+1} (R25), an optional
point-count leaf rule, and the analytic normal derivative of the
interpolant (R1).

With ``exact=True`` every interpolation is replaced by the exact box sum, so
the result must be the direct far sum: a check of the decomposition (each
far pair counted once) separate from the interpolation error.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ETA = 0.57735026918962576451   # sqrt(3)/3: the largest s of a cousin point (Sec. III-E)
PS, PA = 3, 5                  # interpolation points per cone segment: radial, angular
NQ = PS * PA * PA


def cheb_nodes(n: int) -> np.ndarray:
    """Open Chebyshev nodes cos((k + 1/2) pi / n), k = 0..n-1 (Eq. cheby_nodes)."""
    return np.cos((np.arange(n) + 0.5) * np.pi / n)


def cheb_T(t, n: int) -> np.ndarray:
    """T_0..T_{n-1} at t (any shape) -> [..., n]."""
    t = np.asarray(t)
    out = np.empty(t.shape + (n,), dtype=np.result_type(t, 1.0))
    out[..., 0] = 1.0
    if n > 1:
        out[..., 1] = t
    for k in range(2, n):
        out[..., k] = 2 * t * out[..., k - 1] - out[..., k - 2]
    return out


def cheb_dT(t, n: int) -> np.ndarray:
    """T_k'(t), k = 0..n-1 -> [..., n] (T_k' = k U_{k-1})."""
    t = np.asarray(t)
    U = np.empty(t.shape + (max(n - 1, 1),), dtype=np.result_type(t, 1.0))
    U[..., 0] = 1.0
    if n > 2:
        U[..., 1] = 2 * t
    for k in range(2, n - 1):
        U[..., k] = 2 * t * U[..., k - 1] - U[..., k - 2]
    out = np.zeros(t.shape + (n,), dtype=U.dtype)
    for k in range(1, n):
        out[..., k] = k * U[..., k - 1]
    return out


def vals_to_coefs(n: int) -> np.ndarray:
    """Values at the n open nodes -> Chebyshev coefficients: a_0 = (1/n) sum f_j,
    a_i = (2/n) sum f_j T_i(x_j) (reading R7)."""
    T = cheb_T(cheb_nodes(n), n)            # [j, i]
    A = (2.0 / n) * T.T
    A[0] *= 0.5
    return A


@dataclass
class Level:
    d: int
    H: float
    ns: int
    na: int
    boxes: np.ndarray = None       # [nb, 3] integer coordinates
    points: list = field(default_factory=list)         # per box: node indices
    nbr: list = field(default_factory=list)
    cousin: list = field(default_factory=list)
    parent: np.ndarray = None
    children: list = field(default_factory=list)       # per box: {octant: child box}
    cones: list = field(default_factory=list)          # per box: sorted relevant cone keys
    slot_ptr: np.ndarray = None    # per box: first slot (slots = relevant cones, box-major)
    tgt_node: np.ndarray = None    # cousin-point records: (node, box, cone key)
    tgt_box: np.ndarray = None
    tgt_key: np.ndarray = None

    @property
    def h(self) -> float:
        return 0.5 * np.sqrt(3.0) * self.H

    @property
    def ds(self) -> float:
        return ETA / self.ns

    @property
    def dth(self) -> float:
        return np.pi / self.na

    def key(self, g):
        """Cone triples [M, 3] -> keys (g1 n_a + g2) 2 n_a + g3."""
        return (g[:, 0] * self.na + g[:, 1]) * (2 * self.na) + g[:, 2]

    def triple(self, k):
        k = np.asarray(k, dtype=np.int64)
        return np.stack([k // (2 * self.na * self.na), (k // (2 * self.na)) % self.na, k % (2 * self.na)], axis=-1)

    def slot(self, box, key):
        """Slots of (box, cone key) pairs (each must be relevant)."""
        box = np.asarray(box)
        key = np.asarray(key)
        out = np.empty(box.shape, dtype=np.int64)
        for b in np.unique(box):
            m = box == b
            ks = self.cones[b]
            i = np.searchsorted(ks, key[m])
            if np.any(i >= ks.size) or np.any(ks[np.minimum(i, ks.size - 1)] != key[m]):
                raise AssertionError("cone not relevant")
            out[m] = self.slot_ptr[b] + i
        return out


@dataclass
class Tree:
    D: int
    H1: float
    corner: np.ndarray
    leafc: np.ndarray          # [N, 3] integer leaf coordinates
    levels: dict               # d -> Level (d = 1..D)

    def center(self, d: int, b) -> np.ndarray:
        """x^d_k = corner + H_d (k + 1/2) for box b (0-based integer coordinates k)."""
        lv = self.levels[d]
        return self.corner + lv.H * (lv.boxes[b].astype(np.float64) + 0.5)


def cone_of(lv: Level, rel: np.ndarray):
    """Cone triples (g1, g2, g3) of points rel [M, 3] relative to a box centre: half-open
    cells of s = h/r, theta and phi in [0, 2 pi), clamped at the top (reading R8)."""
    x, y, z = rel[:, 0], rel[:, 1], rel[:, 2]
    rho = np.sqrt(x * x + y * y)
    r = np.sqrt(rho * rho + z * z)
    s = lv.h / r
    th = np.arctan2(rho, z)
    ph = np.arctan2(y, x)
    ph = np.where(ph < 0, ph + 2 * np.pi, ph)
    g1 = np.clip(np.floor(s / lv.ds).astype(np.int64), 0, lv.ns - 1)
    g2 = np.clip(np.floor(th / lv.dth).astype(np.int64), 0, lv.na - 1)
    g3 = np.clip(np.floor(ph / lv.dth).astype(np.int64), 0, 2 * lv.na - 1)
    return np.stack([g1, g2, g3], axis=1)


def interp_points(lv: Level, cones: np.ndarray) -> np.ndarray:
    """The 75 interpolation points of each cone segment (g1, g2, g3) [M, 3], relative to the
    box centre -> [M, 75, 3], point order q = (i_s * 5 + i_theta) * 5 + i_phi."""
    cones = np.asarray(cones, dtype=np.int64).reshape(-1, 3)
    xs, xa = cheb_nodes(PS), cheb_nodes(PA)
    i_s, i_t, i_p = np.meshgrid(np.arange(PS), np.arange(PA), np.arange(PA), indexing="ij")
    s = (cones[:, 0:1] + 0.5 * (1.0 + xs[i_s.ravel()][None])) * lv.ds
    th = (cones[:, 1:2] + 0.5 * (1.0 + xa[i_t.ravel()][None])) * lv.dth
    ph = (cones[:, 2:3] + 0.5 * (1.0 + xa[i_p.ravel()][None])) * lv.dth
    r = lv.h / s
    return np.stack([r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)], axis=-1)


def local_coords(lv: Level, cones: np.ndarray, rel: np.ndarray):
    """Coordinates in [-1, 1]^3 of points rel [M, 3] inside their cones [M, 3], plus the
    spherical quantities the normal derivative needs."""
    x, y, z = rel[:, 0], rel[:, 1], rel[:, 2]
    rho = np.sqrt(x * x + y * y)
    r = np.sqrt(rho * rho + z * z)
    s = lv.h / r
    th = np.arctan2(rho, z)
    ph = np.arctan2(y, x)
    php = ph - cones[:, 2] * lv.dth            # phi measured from the cell start, wrapped
    php = np.where(php < -np.pi, php + 2 * np.pi, php)
    php = np.where(php > np.pi, php - 2 * np.pi, php)
    ts = 2.0 * (s / lv.ds - cones[:, 0]) - 1.0
    tt = 2.0 * (th / lv.dth - cones[:, 1]) - 1.0
    tp = 2.0 * php / lv.dth - 1.0
    return ts, tt, tp, r, th, ph


def build_tree(x: np.ndarray, leaf_size: float, k_max: float, ns0: int, na0: int, max_leaf_pts: int = 0,
               min_levels: int = 3, radial_floor: bool = True) -> Tree:
    """Step 1 of the algorithm: boxes, neighbours, cousins, cone counts, relevant cones.
    `radial_floor` False drops reading R25 (the paper's recursion alone)."""
    x = np.asarray(x, dtype=np.float64)
    lo, hi = x.min(axis=0), x.max(axis=0)
    H1 = float(np.max(hi - lo)) * (1.0 + 1e-9)        # level-1 box: the bounding box's largest side (R11)
    corner = 0.5 * (lo + hi) - 0.5 * H1
    D = max(3, min_levels)
    while H1 / 2.0 ** (D - 1) > leaf_size and D < 21:
        D += 1

    def leaf_coords(Dv):
        HD = H1 / 2.0 ** (Dv - 1)
        return np.clip(np.floor((x - corner) / HD).astype(np.int64), 0, 2 ** (Dv - 1) - 1)

    if max_leaf_pts > 0:
        while D < 21:
            _, counts = np.unique(leaf_coords(D), axis=0, return_counts=True)
            if counts.max() <= max_leaf_pts:
                break
            D += 1
    leafc = leaf_coords(D)
    # cone counts (Remark on cone-structure sizes; R9) with the radial floor (R25)
    levels = {}
    ns, na = ns0, na0
    for d in range(D, 0, -1):
        H = H1 / 2.0 ** (d - 1)
        a = 2 if k_max * H > 0.5 else 1
        if d >= 3:
            ns, na = ns * a, na * a
        levels[d] = Level(d=d, H=H, ns=(max(ns, 2 * ns0) if radial_floor else ns) if d >= 3 else 0,
                          na=na if d >= 3 else 0)
    # relevant boxes per level, with their points (Eq. rele_boxes)
    box_of = {}
    for d in range(1, D + 1):
        lv = levels[d]
        keys, inv = np.unique(leafc >> (D - d), axis=0, return_inverse=True)
        inv = inv.ravel()
        lv.boxes = keys
        order = np.argsort(inv, kind="stable")
        bounds = np.searchsorted(inv[order], np.arange(len(keys) + 1))
        lv.points = [order[bounds[b]:bounds[b + 1]] for b in range(len(keys))]
        box_of[d] = inv
    index = {d: {tuple(int(v) for v in k): b for b, k in enumerate(levels[d].boxes)} for d in levels}
    # parents and children
    for d in range(1, D + 1):
        lv = levels[d]
        lv.parent = np.full(len(lv.boxes), -1)
        lv.children = [dict() for _ in range(len(lv.boxes))]
        if d > 1:
            up = levels[d - 1]
            for b, k in enumerate(lv.boxes):
                p = index[d - 1][(int(k[0]) >> 1, int(k[1]) >> 1, int(k[2]) >> 1)]
                lv.parent[b] = p
                up.children[p][int((k[0] & 1) | ((k[1] & 1) << 1) | ((k[2] & 1) << 2))] = b
    # neighbours (infinity norm, R10; relevant boxes only) and cousins (Eq. box_cousin)
    for d in range(1, D + 1):
        lv = levels[d]
        lv.nbr = []
        for k in lv.boxes:
            nb = [index[d].get((int(k[0]) + dx, int(k[1]) + dy, int(k[2]) + dz))
                  for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
            lv.nbr.append(sorted(j for j in nb if j is not None))
        lv.cousin = [[] for _ in range(len(lv.boxes))]
        if d >= 2:
            up = levels[d - 1]
            for b in range(len(lv.boxes)):
                mine = set(lv.nbr[b])
                lv.cousin[b] = sorted(c for pn in up.nbr[lv.parent[b]] for c in up.children[pn].values()
                                      if c not in mine)
    # relevant cone segments, recursively from level 3 (Eq. rele_cone_d)
    for d in range(3, D + 1):
        lv = levels[d]
        rel = []
        tn, tb, tk = [], [], []
        for B in range(len(lv.boxes)):
            keys = []
            # (1) cones holding a cousin point of B; every such point is a target of B
            if lv.cousin[B]:
                src = np.concatenate([lv.points[A] for A in lv.cousin[B]])
                k1 = lv.key(cone_of(lv, x[src] - (corner + lv.H * (lv.boxes[B] + 0.5))))
                keys.append(k1)
                tn.append(src)
                tb.append(np.full(src.size, B))
                tk.append(k1)
            # (2) cones holding an interpolation point of a relevant cone of the parent
            if d >= 4:
                up = levels[d - 1]
                p = lv.parent[B]
                if up.cones[p].size:
                    off = (corner + lv.H * (lv.boxes[B] + 0.5)) - (corner + up.H * (up.boxes[p] + 0.5))
                    X = interp_points(up, up.triple(up.cones[p])).reshape(-1, 3) - off
                    keys.append(lv.key(cone_of(lv, X)))
            rel.append(np.unique(np.concatenate(keys)) if keys else np.zeros(0, dtype=np.int64))
        lv.cones = rel
        lv.slot_ptr = np.concatenate([[0], np.cumsum([r.size for r in rel])])
        lv.tgt_node = np.concatenate(tn) if tn else np.zeros(0, dtype=np.int64)
        lv.tgt_box = np.concatenate(tb) if tb else np.zeros(0, dtype=np.int64)
        lv.tgt_key = np.concatenate(tk) if tk else np.zeros(0, dtype=np.int64)
    return Tree(D=D, H1=H1, corner=corner, leafc=leafc, levels=levels)


def _analytic_factor(X, Yrel, kap):
    """g_S(x, y) = (r/|x - y|) e^{i kap (|x - y| - r)} with x, y relative to the box centre,
    r = |x| (Eq. ifgf_ana_factor)."""
    r = np.linalg.norm(X, axis=1)[:, None]
    d = np.linalg.norm(X[:, None, :] - Yrel[None, :, :], axis=-1)
    return (r / d) * np.exp(1j * kap * (d - r))


def _coefs(vals: np.ndarray) -> np.ndarray:
    """[M, 75, F] values on the 3 x 5 x 5 grid -> [M, 75, F] Chebyshev coefficients in the same
    (i_s, i_theta, i_phi) order, by the 1D transform along each direction."""
    A3, A5 = vals_to_coefs(PS), vals_to_coefs(PA)
    v = vals.reshape(vals.shape[0], PS, PA, PA, vals.shape[-1])
    v = np.einsum("ai,mijkf->majkf", A3, v)
    v = np.einsum("bj,majkf->mabkf", A5, v)
    v = np.einsum("ck,mabkf->mabcf", A5, v)
    return v.reshape(vals.shape)


def _basis(ts, tt, tp, which=(0, 0, 0)):
    """[M, 75] products T_i(ts) T_j(tt) T_k(tp) (or their derivatives where `which` is 1)."""
    Ts = cheb_dT(ts, PS) if which[0] else cheb_T(ts, PS)
    Tt = cheb_dT(tt, PA) if which[1] else cheb_T(tt, PA)
    Tp = cheb_dT(tp, PA) if which[2] else cheb_T(tp, PA)
    return (Ts[:, :, None, None] * Tt[:, None, :, None] * Tp[:, None, None, :]).reshape(ts.size, NQ)


def _eval(coef, slots, bases):
    """Interpolants at M points: bases [M, nb, 75] (basis products per point), slots [M] the
    cone segment of each point -> [M, nb, F] = bases @ coef[slot], one product per segment."""
    out = np.empty(bases.shape[:2] + (coef.shape[-1],), dtype=np.complex128)
    order = np.argsort(slots, kind="stable")
    ss = slots[order]
    bounds = np.flatnonzero(np.diff(ss)) + 1
    for idx in np.split(order, bounds):
        out[idx] = bases[idx] @ coef[slots[idx[0]]]
    return out


def _scatter(out, nodes, c0, vals):
    """out[nodes, c0:c0+k] += vals (repeated nodes accumulate)."""
    for j in range(vals.shape[1]):
        np.add.at(out[:, c0 + j], nodes, vals[:, j])


def ifgf_far(tree: Tree, x: np.ndarray, nrm: np.ndarray, a: np.ndarray, k_ext: float, k_int: float,
             exact: bool = False, chunk: int = 4096) -> np.ndarray:
    """Far fields [N, 28] complex: S_e[phi_k] (k < 8), S_i[phi_k], dS_e/dn[phi_k] (k < 6),
    dS_i/dn[phi_k], summed over the sources outside each target's neighbour boxes, with
    weighted densities a [N, 8] (a = phi * quadrature weight).  Steps 2 and 3 of the
    algorithm; `exact` replaces every interpolation by the exact box sum."""
    x = np.asarray(x, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    a = np.asarray(a, dtype=np.complex128)
    N = x.shape[0]
    D = tree.D
    kaps = (k_ext, k_int)
    out = np.zeros((N, 28), dtype=np.complex128)
    if exact:
        return _exact_far(tree, x, nrm, a, kaps, out)
    # step 2: level-D analytic factors at the interpolation points, by direct summation
    lv = tree.levels[D]
    coef = np.zeros((lv.slot_ptr[-1], NQ, 16), dtype=np.complex128)
    for b, keys in enumerate(lv.cones):
        if not keys.size:
            continue
        X = interp_points(lv, lv.triple(keys)).reshape(-1, 3)
        Y = x[lv.points[b]] - tree.center(D, b)
        vals = np.concatenate([_analytic_factor(X, Y, k) @ a[lv.points[b]] for k in kaps], axis=1)
        coef[lv.slot_ptr[b]:lv.slot_ptr[b + 1]] = _coefs(vals.reshape(keys.size, NQ, 16))
    for d in range(D, 2, -1):
        lv = tree.levels[d]
        # step 3, first item: the cousin points of every box, from its interpolant
        for e0 in range(0, lv.tgt_node.size, chunk):
            nodes = lv.tgt_node[e0:e0 + chunk]
            boxes = lv.tgt_box[e0:e0 + chunk]
            keys = lv.tgt_key[e0:e0 + chunk]
            cones = lv.triple(keys)
            rel = x[nodes] - (tree.corner + lv.H * (lv.boxes[boxes] + 0.5))
            n = nrm[nodes]
            ts, tt, tp, r, th, ph = local_coords(lv, cones, rel)
            bases = np.stack([_basis(ts, tt, tp, w) for w in ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))], axis=1)
            vals = _eval(coef, lv.slot(boxes, keys), bases)
            F, Fs, Ft, Fp = vals[:, 0], vals[:, 1], vals[:, 2], vals[:, 3]
            # n . grad of (s, theta, phi) (R1): grad s = -(h/r^2) r_hat,
            # grad theta = theta_hat / r, grad phi = phi_hat / (r sin theta)
            st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
            nr = np.sum(n * rel, axis=1) / r
            nth = n[:, 0] * ct * cp + n[:, 1] * ct * sp - n[:, 2] * st
            nph = -n[:, 0] * sp + n[:, 1] * cp
            a_s = -(lv.h / r ** 2) * nr * (2.0 / lv.ds)
            a_t = nth / r * (2.0 / lv.dth)
            a_p = nph / (r * np.maximum(st, 1e-7)) * (2.0 / lv.dth)
            dF = a_s[:, None] * Fs + a_t[:, None] * Ft + a_p[:, None] * Fp
            for ks, kap in enumerate(kaps):
                # centred factor G(x, x_B) = e^{i kap r}/(4 pi r) and its normal derivative
                G = np.exp(1j * kap * r) / (4 * np.pi * r)
                dG = nr * (1j * kap - 1.0 / r) * G
                Fk = F[:, 8 * ks:8 * ks + 8]
                dFk = dF[:, 8 * ks:8 * ks + 8]
                _scatter(out, nodes, 8 * ks, G[:, None] * Fk)
                _scatter(out, nodes, 16 + 6 * ks, dG[:, None] * Fk[:, :6] + G[:, None] * dFk[:, :6])
        if d == 3:
            break
        # step 3, second item: the parent's analytic factor at its interpolation points,
        # from every child by interpolation and re-centring
        up = tree.levels[d - 1]
        pcoef = np.zeros((up.slot_ptr[-1], NQ, 16), dtype=np.complex128)
        for p, pkeys in enumerate(up.cones):
            if not pkeys.size:
                continue
            XP = interp_points(up, up.triple(pkeys)).reshape(-1, 3)     # relative to the parent
            rp = np.linalg.norm(XP, axis=1)
            vals = np.zeros((XP.shape[0], 16), dtype=np.complex128)
            for o, b in up.children[p].items():
                Xc = XP - (tree.center(d, b) - tree.center(d - 1, p))
                rc = np.linalg.norm(Xc, axis=1)
                cones = cone_of(lv, Xc)
                ts, tt, tp, _, _, _ = local_coords(lv, cones, Xc)
                Fc = _eval(coef, lv.slot(np.full(Xc.shape[0], b), lv.key(cones)), _basis(ts, tt, tp)[:, None])[:, 0]
                for ks, kap in enumerate(kaps):
                    fac = (rp / rc) * np.exp(1j * kap * (rc - rp))        # G(x, x_child) / G(x, x_parent)
                    vals[:, 8 * ks:8 * ks + 8] += fac[:, None] * Fc[:, 8 * ks:8 * ks + 8]
            pcoef[up.slot_ptr[p]:up.slot_ptr[p + 1]] = _coefs(vals.reshape(pkeys.size, NQ, 16))
        coef = pcoef
    return out


def _exact_far(tree, x, nrm, a, kaps, out):
    """The decomposition with exact box sums: every (target, box) record of every level
    adds the box's sources' G and dG/dn at the target directly."""
    for d in range(tree.D, 2, -1):
        lv = tree.levels[d]
        for B in np.unique(lv.tgt_box):
            nodes = lv.tgt_node[lv.tgt_box == B]
            src = lv.points[B]
            R = x[nodes][:, None, :] - x[src][None, :, :]
            dist = np.linalg.norm(R, axis=-1)
            nd = np.einsum("tsk,tk->ts", R, nrm[nodes]) / dist
            for ks, kap in enumerate(kaps):
                G = np.exp(1j * kap * dist) / (4 * np.pi * dist)
                dG = nd * (1j * kap - 1.0 / dist) * G
                _scatter(out, nodes, 8 * ks, G @ a[src])
                _scatter(out, nodes, 16 + 6 * ks, dG @ a[src][:, :6])
    return out


def direct_far(x: np.ndarray, nrm: np.ndarray, a: np.ndarray, k_ext: float, k_int: float,
               leafc: np.ndarray) -> np.ndarray:
    """The same far fields [N, 28] by the plain double sum over every (target, source) pair
    whose leaf boxes are not neighbours (infinity-norm distance of leaf coordinates > 1)."""
    x = np.asarray(x, dtype=np.float64)
    N = x.shape[0]
    out = np.zeros((N, 28), dtype=np.complex128)
    for l in range(N):
        far = np.any(np.abs(leafc - leafc[l]) > 1, axis=1)
        R = x[l] - x[far]
        dist = np.linalg.norm(R, axis=1)
        nd = (R @ nrm[l]) / dist
        for ks, kap in enumerate((k_ext, k_int)):
            G = np.exp(1j * kap * dist) / (4 * np.pi * dist)
            dG = nd * (1j * kap - 1.0 / dist) * G
            out[l, 8 * ks:8 * ks + 8] = G @ a[far]
            out[l, 16 + 6 * ks:22 + 6 * ks] = dG @ a[far][:, :6]
    return out
