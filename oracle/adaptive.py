"""Plain CPU FP64 heterogeneous FMM on an adaptive quadtree (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this module; the product path never does.

Tree (Sec. 3.1): the root is the smallest bounding square of the points; a
box is split into its four children while it holds more than ``leaf_size``
points (and is above ``max_level``); empty children are pruned.  Leaves
therefore sit at different levels.

Free-space lists, the usual ones for an adaptive tree (the paper names only
"the interaction list" and "neighbouring boxes"; reading taken):
  colleagues(B)  existing boxes of B's level adjacent to B (B included);
  V(B)           children of the colleagues of B's parent that are not
                 adjacent to B (same level; M2L, Sec. 3.3);
  U(B)           for a leaf B: every leaf adjacent to B, of any level
                 (direct H0 sum, Algorithm 1 step 5);
  W(B)           for a leaf B: boxes D below B's colleagues that are not
                 adjacent to B while their parent is (multipole of D
                 evaluated at B's points: M2P);
  X(B)           the leaves C with B in W(C) (C's points into B's local
                 expansion: P2L).
With multipole and local expansions as in oracle.fmm, M2P is the M2L into a
local expansion of radius zero at the point and P2L the M2L from the
multipole of a single point:
  M2P:  u(x) = (i/4) sum_m alpha_m C_m(x - c),
  P2L:  beta_p += q_j C_{-p}(l - x_j).

Reaction part: the pair recursion of oracle.fmm.reaction_lists on boxes of
one level, starting at (root, root).  An admissible pair (image box one box
below the target box) is translated by the reaction M2L at that level; an
inadmissible pair is split into its children's pairs while both boxes have
children; when either box is a leaf, the pair is summed directly over all
points of both boxes (G^s by quadrature).  On a uniform tree this is exactly
oracle.fmm's rule.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import hankel1, jv

from . import fmm, green


class Box:
    __slots__ = ("level", "ix", "iy", "idx", "children", "parent")

    def __init__(self, level, ix, iy, idx, parent):
        self.level = level
        self.ix = ix
        self.iy = iy
        self.idx = idx              # point indices (caller order)
        self.children = []
        self.parent = parent

    @property
    def leaf(self):
        return not self.children

    @property
    def key(self):
        return (self.level, self.ix, self.iy)


class AdaptiveTree:
    """Boxes keyed (level, ix, iy); h(l), centre(l, ix, iy) as in oracle.fmm.Tree."""

    def __init__(self, xy, leaf_size=32, max_level=16):
        xy = np.asarray(xy, dtype=float)
        self.xy = xy
        n = xy.shape[0]
        self.x0 = float(np.min(xy[:, 0]))
        self.y0 = float(np.min(xy[:, 1]))
        S = max(float(np.max(xy[:, 0])) - self.x0, float(np.max(xy[:, 1])) - self.y0)
        self.S = S if S > 0 else 1.0
        D = max_level
        m = 1 << D
        scale = float(m) / self.S
        qx = np.minimum(np.floor((xy[:, 0] - self.x0) * scale), m - 1).astype(np.int64)
        qy = np.minimum(np.floor((xy[:, 1] - self.y0) * scale), m - 1).astype(np.int64)
        self.boxes = {}
        root = Box(0, 0, 0, np.arange(n, dtype=np.int64), None)
        self.boxes[root.key] = root
        self.root = root
        stack = [root]
        while stack:
            b = stack.pop()
            if b.idx.size <= leaf_size or b.level >= D:
                continue
            sh = D - b.level - 1
            cx = (qx[b.idx] >> sh) & 1
            cy = (qy[b.idx] >> sh) & 1
            for c in range(4):
                sel = b.idx[(cx == (c & 1)) & (cy == (c >> 1))]
                if sel.size == 0:
                    continue
                ch = Box(b.level + 1, 2 * b.ix + (c & 1), 2 * b.iy + (c >> 1), sel, b)
                b.children.append(ch)
                self.boxes[ch.key] = ch
                stack.append(ch)
        self.L = max(k[0] for k in self.boxes)

    def h(self, l):
        return self.S / (1 << l)

    def centre(self, l, ix, iy):
        h = self.h(l)
        return self.x0 + (ix + 0.5) * h, self.y0 + (iy + 0.5) * h

    def level_boxes(self, l):
        return [b for k, b in self.boxes.items() if k[0] == l]

    def leaves(self):
        return [b for b in self.boxes.values() if b.leaf]


def adjacent(A, B):
    """Closed boxes A, B touch or overlap (corners included)."""
    l = max(A.level, B.level)
    sa, sb = l - A.level, l - B.level
    ax0, ax1 = A.ix << sa, (A.ix + 1) << sa
    ay0, ay1 = A.iy << sa, (A.iy + 1) << sa
    bx0, bx1 = B.ix << sb, (B.ix + 1) << sb
    by0, by1 = B.iy << sb, (B.iy + 1) << sb
    return ax0 <= bx1 and bx0 <= ax1 and ay0 <= by1 and by0 <= ay1


def colleagues(tree, B):
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            C = tree.boxes.get((B.level, B.ix + dx, B.iy + dy))
            if C is not None:
                out.append(C)
    return out


def v_list(tree, B):
    if B.parent is None:
        return []
    return [D for C in colleagues(tree, B.parent) for D in C.children if not adjacent(D, B)]


def u_list(tree, B):
    """Leaves adjacent to leaf B (B included)."""
    out = []
    stack = [tree.root]
    while stack:
        C = stack.pop()
        if not adjacent(C, B):
            continue
        if C.leaf:
            out.append(C)
        else:
            stack.extend(C.children)
    return out


def w_list(tree, B):
    """Boxes below B's colleagues, not adjacent to leaf B, whose parent is."""
    out = []
    stack = [D for C in colleagues(tree, B) if C is not B for D in C.children]
    while stack:
        D = stack.pop()
        if adjacent(D, B):
            stack.extend(D.children)
        else:
            out.append(D)
    return out


def reaction_pairs(tree):
    """(R, direct): R[l] = same-level box pairs (T, S) through the reaction
    M2L; direct = box pairs summed directly (at least one is a leaf)."""
    R = {l: [] for l in range(tree.L + 1)}
    direct = []
    stack = [(tree.root, tree.root)]
    while stack:
        T, S = stack.pop()
        l = T.level
        if fmm.reaction_admissible(tree, l, T.iy, S.iy):
            R[l].append((T, S))
        elif T.leaf or S.leaf:
            direct.append((T, S))
        else:
            for a in T.children:
                for b in S.children:
                    stack.append((a, b))
    return R, direct


class AdaptiveCpuFmm:
    """y = G q with G_ij = g(x_i, x_j) (i != j) + G^s(x_i - x_j, y_i + y_j)
    on an adaptive tree; ``parts`` as in oracle.fmm.CpuFmm.apply (W and X
    belong to the free far field)."""

    NEAR_FREE, FAR_FREE, FAR_REACT, NEAR_REACT = 1, 2, 4, 8

    def __init__(self, xy, medium, tol=1e-6, leaf_size=32, p=0, max_level=16):
        self.medium = medium
        self.k = medium.k1
        self.tree = AdaptiveTree(xy, leaf_size, max_level)
        self.p = fmm.p_schedule(self.k, self.tree, tol, p)
        self.R, self.direct_pairs = reaction_pairs(self.tree)
        t = self.tree
        self.V = {b.key: v_list(t, b) for b in t.boxes.values() if b.level >= 2}
        self.U = {b.key: u_list(t, b) for b in t.leaves()}
        self.W = {b.key: w_list(t, b) for b in t.leaves()}
        self.X = {}
        for b in t.leaves():
            for D in self.W[b.key]:
                self.X.setdefault(D.key, []).append(b)
        # coarsest level with translation work
        self.lmin = next(l for l in range(t.L + 1) if self.R[l] or l >= 2 or l == t.L)
        self._A = {}

    def A(self, l, dx, ysum):
        key = (l, dx, ysum)
        if key not in self._A:
            t = self.tree
            h = t.h(l)
            self._A[key] = green.hetero_m2l_kernel(self.medium, dx * h, 2.0 * t.y0 + (ysum + 1) * h, 2 * self.p[l])
        return self._A[key]

    def apply(self, q, parts=15):
        q = np.asarray(q, dtype=complex)
        squeeze = q.ndim == 1
        if squeeze:
            q = q[None, :]
        nrhs = q.shape[0]
        t = self.tree
        k = self.k
        p = self.p
        xy = t.xy
        lmin = self.lmin
        far = parts & (self.FAR_FREE | self.FAR_REACT)

        # Step 2: P2M at every leaf of level >= lmin, M2M for the boxes above
        mult = {}
        for l in range(t.L, lmin - 1, -1):
            for B in t.level_boxes(l):
                if B.leaf:
                    cx, cy = t.centre(l, B.ix, B.iy)
                    dx = xy[B.idx, 0] - cx
                    dy = xy[B.idx, 1] - cy
                    rho = np.hypot(dx, dy)
                    th = np.arctan2(dy, dx)
                    m = np.arange(-p[l], p[l] + 1)
                    basis = jv(m[:, None], k * rho[None, :]) * np.exp(-1j * m[:, None] * th[None, :])
                    mult[B.key] = basis @ q[:, B.idx].T
                else:
                    hc = t.h(l + 1)
                    acc = np.zeros((2 * p[l] + 1, nrhs), dtype=complex)
                    for C in B.children:
                        a = (C.ix & 1) + 2 * (C.iy & 1)
                        v = ((0.5 - (a & 1)) * hc, (0.5 - (a >> 1)) * hc)   # P - c
                        acc += fmm.m2m_matrix(p[l + 1], p[l], v, k) @ mult[C.key]
                    mult[B.key] = acc

        # Step 3: downward pass: L2L, V-list M2L, X-list P2L, reaction M2L
        loc = {}
        y = np.zeros((nrhs, xy.shape[0]), dtype=complex)
        if far:
            for l in range(lmin, t.L + 1):
                h = t.h(l)
                for B in t.level_boxes(l):
                    acc = np.zeros((2 * p[l] + 1, nrhs), dtype=complex)
                    if l > lmin:
                        a = (B.ix & 1) + 2 * (B.iy & 1)
                        v = (((a & 1) - 0.5) * h, ((a >> 1) - 0.5) * h)     # c - P
                        acc += fmm.l2l_matrix(p[l - 1], p[l], v, k) @ loc[B.parent.key]
                    if parts & self.FAR_FREE:
                        for S in self.V.get(B.key, []):
                            D = ((B.ix - S.ix) * h, (B.iy - S.iy) * h)
                            acc += fmm.m2l_free_matrix(p[l], D, k) @ mult[S.key]
                        cx, cy = t.centre(l, B.ix, B.iy)
                        for C in self.X.get(B.key, []):
                            # P2L: beta_p += q_j C_{-p}(l - x_j)
                            dx = cx - xy[C.idx, 0]
                            dy = cy - xy[C.idx, 1]
                            r = np.hypot(dx, dy)
                            th = np.arctan2(dy, dx)
                            pp = np.arange(-p[l], p[l] + 1)
                            Cm = hankel1(-pp[:, None], k * r[None, :]) * np.exp(-1j * pp[:, None] * th[None, :])
                            acc += Cm @ q[:, C.idx].T
                    loc[B.key] = acc
                if parts & self.FAR_REACT:
                    for T, S in self.R[l]:
                        An = self.A(l, T.ix - S.ix, T.iy + S.iy)
                        loc[T.key] += fmm.m2l_reaction_matrix(p[l], An) @ mult[S.key]

            # Step 4: L2P at every leaf, M2P from its W list
            for B in t.leaves():
                l = B.level
                cx, cy = t.centre(l, B.ix, B.iy)
                if l >= lmin:
                    dx = xy[B.idx, 0] - cx
                    dy = xy[B.idx, 1] - cy
                    rho = np.hypot(dx, dy)
                    th = np.arctan2(dy, dx)
                    m = np.arange(-p[l], p[l] + 1)
                    basis = jv(m[None, :], k * rho[:, None]) * np.exp(1j * m[None, :] * th[:, None])
                    y[:, B.idx] += 0.25j * (basis @ loc[B.key]).T
                if parts & self.FAR_FREE:
                    for D in self.W[B.key]:
                        ld = D.level
                        dcx, dcy = t.centre(ld, D.ix, D.iy)
                        dx = xy[B.idx, 0] - dcx
                        dy = xy[B.idx, 1] - dcy
                        r = np.hypot(dx, dy)
                        th = np.arctan2(dy, dx)
                        m = np.arange(-p[ld], p[ld] + 1)
                        Cm = hankel1(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])
                        y[:, B.idx] += 0.25j * (Cm @ mult[D.key]).T

        # Step 5: direct interactions
        if parts & self.NEAR_FREE:
            for B in t.leaves():
                idx = B.idx
                for S in self.U[B.key]:
                    jdx = S.idx
                    r = np.hypot(xy[idx, 0][:, None] - xy[jdx, 0][None, :],
                                 xy[idx, 1][:, None] - xy[jdx, 1][None, :])
                    same = idx[:, None] == jdx[None, :]
                    Gm = np.where(same, 0.0, 0.25j * hankel1(0, k * np.where(same, 1.0, r)))
                    y[:, idx] += (Gm @ q[:, jdx].T).T
        if parts & self.NEAR_REACT:
            for T, S in self.direct_pairs:
                X = xy[T.idx, 0][:, None] - xy[S.idx, 0][None, :]
                Y = xy[T.idx, 1][:, None] + xy[S.idx, 1][None, :]
                Gm = green.green_reaction(self.medium, X, Y)
                y[:, T.idx] += (Gm @ q[:, S.idx].T).T
        return y[0] if squeeze else y
