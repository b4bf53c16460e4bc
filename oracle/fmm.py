"""Plain CPU FP64 heterogeneous FMM (test infrastructure, see oracle/green.py).

Follows Algorithm 1 of the paper step by step on a uniform-depth quadtree:
  Step 1  tree over the smallest bounding square, leaf level L; tables;
  Step 2  upward pass: P2M at the leaves (Eq. (multi_coeff)), free-space M2M;
  Step 3  downward pass: free-space L2L, then M2L over the interaction lists:
          free part (Graf, Sec. 3.3) and heterogeneous (reaction) part with
          A_n of Eq. (eq:m2loperator) applied to the image coefficients;
  Step 4  L2P at every target (Eq. (multipole_free) / local expansion);
  Step 5  direct interactions: free-space H0 over neighbouring leaves, and
          the reaction G^s by quadrature for leaf pairs whose images are not
          well separated from the target leaf.

Conventions (all checked by tests against SciPy / the direct sum):
  C_n(D) = H_n(k|D|) e^{i n angle D},  J_n(D) = J_n(k|D|) e^{i n angle D}
  multipole about c:  u(x) = (i/4) sum_m alpha_m C_m(x - c),
                      alpha_m = sum_j q_j e^{-i m theta_j} J_m(k rho_j)
  local about l:      u(x) = (i/4) sum_p beta_p J_p(x - l)
  M2M c -> P:  alpha^P_j = sum_m alpha^c_m J_{m-j}(P - c)
  M2L c -> l:  beta_p   = sum_m alpha_m C_{m-p}(l - c)
  L2L P -> c:  beta^c_m = sum_n beta^P_n J_{n-m}(c - P)
  image coefficients (linear, not conjugated):  alpha^im_m = (-1)^m alpha_{-m}
  reaction M2L S -> T: beta_p += sum_m A_{m-p}(x_T - x_S, y_T + y_S) alpha^im_m

Interaction lists.  Free part: the usual V list (children of the parent's
neighbours that are not neighbours), levels 2..L, and U list (neighbouring
leaves, self included) for the direct part.  Reaction part: the paper's error
analysis (Remark 3) only needs the target box and the image box to be well
separated; a pair (T, S) at level l is taken through the reaction M2L when the
image box lies at least one box below the target box, i.e.
    y_T + y_S >= 2 h_l          (box centres, h_l the box side),
otherwise the pair is split into its children; pairs still not admissible at
the leaf level are summed directly.  For the points of the paper's own test
(far above y = 0) this puts the whole reaction field into one root-level M2L;
the paper's "at least one box size away from the interface" rule for leaves
is the leaf-level case of the same test.

Expansion order per level (shared written rule, see p_schedule).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import hankel1, jv

from . import green


# ---------------------------------------------------------------------------
# tree
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    xy: np.ndarray
    x0: float
    y0: float
    S: float
    L: int
    leaf_ix: np.ndarray
    leaf_iy: np.ndarray
    leaves: dict          # (ix, iy) -> array of point indices

    def h(self, l):
        return self.S / (1 << l)

    def centre(self, l, ix, iy):
        h = self.h(l)
        return self.x0 + (ix + 0.5) * h, self.y0 + (iy + 0.5) * h

    def nonempty(self, l):
        """set of (ix, iy) boxes at level l holding at least one point."""
        sh = self.L - l
        return {(ix >> sh, iy >> sh) for (ix, iy) in self.leaves}


def choose_levels(n, leaf_size):
    """Leaf level: smallest L >= 2 with n <= leaf_size * 4^L."""
    L = 2
    while n > leaf_size * (4 ** L):
        L += 1
    return L


def build_tree(xy, leaf_size=32, L=None):
    """Uniform-depth quadtree over the smallest bounding square.
    Leaf index of a point: ix = min(floor((x - x0) * (2^L / S)), 2^L - 1)."""
    xy = np.asarray(xy, dtype=float)
    n = xy.shape[0]
    x0 = float(np.min(xy[:, 0]))
    y0 = float(np.min(xy[:, 1]))
    S = max(float(np.max(xy[:, 0])) - x0, float(np.max(xy[:, 1])) - y0)
    if not S > 0:
        S = 1.0
    if L is None:
        L = choose_levels(n, leaf_size)
    m = 1 << L
    scale = float(m) / S
    ix = np.minimum(np.floor((xy[:, 0] - x0) * scale), m - 1).astype(np.int64)
    iy = np.minimum(np.floor((xy[:, 1] - y0) * scale), m - 1).astype(np.int64)
    leaves = {}
    order = np.lexsort((np.arange(n), iy, ix))
    for j in order:
        leaves.setdefault((int(ix[j]), int(iy[j])), []).append(int(j))
    leaves = {key: np.array(v, dtype=np.int64) for key, v in leaves.items()}
    return Tree(xy, x0, y0, S, L, ix, iy, leaves)


# ---------------------------------------------------------------------------
# interaction lists
# ---------------------------------------------------------------------------

def u_list(tree, T):
    ix, iy = T
    out = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            S = (ix + dx, iy + dy)
            if S in tree.leaves:
                out.append(S)
    return out


def v_list(tree, l, T, nonempty):
    ix, iy = T
    px, py = ix >> 1, iy >> 1
    out = []
    for qx in range(px - 1, px + 2):
        for qy in range(py - 1, py + 2):
            for cx in (0, 1):
                for cy in (0, 1):
                    S = (2 * qx + cx, 2 * qy + cy)
                    if S not in nonempty:
                        continue
                    if max(abs(S[0] - ix), abs(S[1] - iy)) >= 2:
                        out.append(S)
    return out


def reaction_admissible(tree, l, iyT, iyS):
    """Image box at least one box below the target box:
    y_T + y_S >= 2 h_l  <=>  iyT + iyS >= 1  or  2 y0 >= h_l."""
    return (iyT + iyS >= 1) or (2.0 * tree.y0 >= tree.h(l))


def reaction_lists(tree):
    """Returns (R, direct): R[l] = list of (T, S) pairs translated by the
    reaction M2L at level l; direct = leaf pairs (T, S) summed directly."""
    R = {l: [] for l in range(tree.L + 1)}
    direct = []
    cand = [((0, 0), (0, 0))]
    for l in range(tree.L + 1):
        ne = tree.nonempty(l)
        nxt = []
        for T, S in cand:
            if T not in ne or S not in ne:
                continue
            if reaction_admissible(tree, l, T[1], S[1]):
                R[l].append((T, S))
            elif l == tree.L:
                direct.append((T, S))
            else:
                for a in range(4):
                    for b in range(4):
                        nxt.append(((2 * T[0] + (a & 1), 2 * T[1] + (a >> 1)),
                                    (2 * S[0] + (b & 1), 2 * S[1] + (b >> 1))))
        cand = nxt
    return R, direct


# ---------------------------------------------------------------------------
# expansion orders
# ---------------------------------------------------------------------------

def p_low(tol):
    """Order for boxes small against the wavelength: the error of this FMM
    falls about 2.5x per added order (calibrated on the impedance
    workloads against the direct sum)."""
    d = max(1.0, -math.log10(tol))
    return max(4, int(math.ceil(2.5 * d - 6.5)))


def p_schedule(k, tree, tol, p_fixed=0):
    """p_l = base + ceil(k R_l + 1.8 d^(2/3) max(k R_l - 1, 0)^(1/3)),
    R_l = h_l / sqrt(2), d = -log10(tol), base = p_fixed if given, else
    p_low(tol).  The second term is the excess bandwidth of wide-band FMMs
    for boxes larger than the wavelength.

    Range cap: the translations use unscaled H_n(k r), n <= 2 p_l, whose size
    near the closest translated distance r = min(2 h_l, 2 y0 + h_l) is about
    (n-1)! (2/(k r))^n / pi for k r << n; p_l is lowered until
    lgamma(2p) + 2p log(2/(k r)) <= 680, so every entry stays inside the
    double range (e^709).  This only binds at low frequency on deep trees
    with a large fixed p (e.g. k = 0.1 and p = 39 below h = 1/32).
    Returns p per level 0..L."""
    base = p_fixed if p_fixed > 0 else p_low(tol)
    d = max(1.0, -math.log10(tol))
    out = []
    for l in range(tree.L + 1):
        h = tree.h(l)
        kR = k * h / math.sqrt(2.0)
        p = base + int(math.ceil(kR + 1.8 * d ** (2.0 / 3.0) * max(kR - 1.0, 0.0) ** (1.0 / 3.0)))
        lx = math.log(2.0 / (k * min(2.0 * h, 2.0 * tree.y0 + h)))
        while p > 1 and math.lgamma(2.0 * p) + 2.0 * p * lx > 680.0:
            p -= 1
        out.append(p)
    return out


# ---------------------------------------------------------------------------
# translation helpers (SciPy Bessel functions)
# ---------------------------------------------------------------------------

def _cyl_h(nlo, nhi, D, k):
    n = np.arange(nlo, nhi + 1)
    r = math.hypot(D[0], D[1])
    th = math.atan2(D[1], D[0])
    return hankel1(n, k * r) * np.exp(1j * n * th)


def _cyl_j(nlo, nhi, D, k):
    n = np.arange(nlo, nhi + 1)
    r = math.hypot(D[0], D[1])
    th = math.atan2(D[1], D[0])
    return jv(n, k * r) * np.exp(1j * n * th)


def m2m_matrix(pc, pp, v, k):
    """alpha^P_j = sum_m alpha^c_m J_{m-j}(v),  v = P - c; [2pp+1, 2pc+1]."""
    Jn = _cyl_j(-(pc + pp), pc + pp, v, k)
    j = np.arange(-pp, pp + 1)[:, None]
    m = np.arange(-pc, pc + 1)[None, :]
    return Jn[(m - j) + pc + pp]


def l2l_matrix(pp, pc, v, k):
    """beta^c_m = sum_n beta^P_n J_{n-m}(v),  v = c - P; [2pc+1, 2pp+1]."""
    Jn = _cyl_j(-(pc + pp), pc + pp, v, k)
    m = np.arange(-pc, pc + 1)[:, None]
    n = np.arange(-pp, pp + 1)[None, :]
    return Jn[(n - m) + pc + pp]


def m2l_free_matrix(p, D, k):
    """beta_p = sum_m alpha_m C_{m-p}(D),  D = l - c; [2p+1, 2p+1]."""
    Cn = _cyl_h(-2 * p, 2 * p, D, k)
    pp = np.arange(-p, p + 1)[:, None]
    m = np.arange(-p, p + 1)[None, :]
    return Cn[(m - pp) + 2 * p]


def m2l_reaction_matrix(p, An):
    """Matrix acting on alpha (not alpha^im):
    beta_p = sum_m A_{m-p} alpha^im_m = sum_m A_{-m-p} (-1)^m alpha_m."""
    pp = np.arange(-p, p + 1)[:, None]
    m = np.arange(-p, p + 1)[None, :]
    sign = np.where(m % 2 == 0, 1.0, -1.0)
    return An[(-m - pp) + 2 * p] * sign


# ---------------------------------------------------------------------------
# the FMM
# ---------------------------------------------------------------------------

class CpuFmm:
    """y = G q with G_ij = g(x_i, x_j) (i != j) + G^s(x_i - x_j, y_i + y_j)."""

    def __init__(self, xy, medium, tol=1e-6, leaf_size=32, p=0, L=None, plevels=None):
        self.medium = medium
        self.k = medium.k1
        self.tree = build_tree(xy, leaf_size, L)
        self.p = list(plevels) if plevels is not None else p_schedule(self.k, self.tree, tol, p)
        self.R, self.direct_pairs = reaction_lists(self.tree)
        self._A = {}
        self._direct_cache = {}

    # -- tables -----------------------------------------------------------
    def A(self, l, dx, ysum):
        key = (l, dx, ysum)
        if key not in self._A:
            t = self.tree
            h = t.h(l)
            X = dx * h
            Y = 2.0 * t.y0 + (ysum + 1) * h
            self._A[key] = green.hetero_m2l_kernel(self.medium, X, Y, 2 * self.p[l])
        return self._A[key]

    # -- apply --------------------------------------------------------------
    NEAR_FREE, FAR_FREE, FAR_REACT, NEAR_REACT = 1, 2, 4, 8

    def apply(self, q, parts=15):
        """y = G q; ``parts`` selects terms: 1 free direct (step 5), 2 free
        far field, 4 reaction far field (steps 2-4), 8 directly summed
        reaction (step 5)."""
        q = np.asarray(q, dtype=complex)
        squeeze = q.ndim == 1
        if squeeze:
            q = q[None, :]
        nrhs = q.shape[0]
        t = self.tree
        k = self.k
        L = t.L
        p = self.p
        ne = [t.nonempty(l) for l in range(L + 1)]
        # lowest level with any translation work
        lmin = L
        for l in range(L + 1):
            if self.R[l] or (l >= 2):
                lmin = l
                break

        # Step 2: upward pass
        mult = [dict() for _ in range(L + 1)]
        for key, idx in t.leaves.items():
            cx, cy = t.centre(L, *key)
            dx = t.xy[idx, 0] - cx
            dy = t.xy[idx, 1] - cy
            rho = np.hypot(dx, dy)
            th = np.arctan2(dy, dx)
            m = np.arange(-p[L], p[L] + 1)
            basis = jv(m[:, None], k * rho[None, :]) * np.exp(-1j * m[:, None] * th[None, :])
            mult[L][key] = basis @ q[:, idx].T                     # [2p+1, nrhs]
        for l in range(L - 1, lmin - 1, -1):
            hc = t.h(l + 1)
            for (ix, iy) in ne[l]:
                acc = np.zeros((2 * p[l] + 1, nrhs), dtype=complex)
                for a in range(4):
                    c = (2 * ix + (a & 1), 2 * iy + (a >> 1))
                    if c not in mult[l + 1]:
                        continue
                    v = ((0.5 - (a & 1)) * hc, (0.5 - (a >> 1)) * hc)   # P - c
                    acc += m2m_matrix(p[l + 1], p[l], v, k) @ mult[l + 1][c]
                mult[l][(ix, iy)] = acc

        # Step 3: downward pass
        loc = [dict() for _ in range(L + 1)]
        for l in range(lmin, L + 1):
            h = t.h(l)
            for T in ne[l]:
                acc = np.zeros((2 * p[l] + 1, nrhs), dtype=complex)
                if l > lmin:
                    P = (T[0] >> 1, T[1] >> 1)
                    if P in loc[l - 1]:
                        a = (T[0] & 1) + 2 * (T[1] & 1)
                        v = (((a & 1) - 0.5) * h, ((a >> 1) - 0.5) * h)   # c - P
                        acc += l2l_matrix(p[l - 1], p[l], v, k) @ loc[l - 1][P]
                if l >= 2 and (parts & self.FAR_FREE):
                    for S in v_list(t, l, T, ne[l]):
                        D = ((T[0] - S[0]) * h, (T[1] - S[1]) * h)
                        acc += m2l_free_matrix(p[l], D, k) @ mult[l][S]
                loc[l][T] = acc
            for T, S in (self.R[l] if parts & self.FAR_REACT else []):
                An = self.A(l, T[0] - S[0], T[1] + S[1])
                loc[l][T] += m2l_reaction_matrix(p[l], An) @ mult[l][S]

        # Step 4: local expansions at the targets
        y = np.zeros((nrhs, t.xy.shape[0]), dtype=complex)
        for key, idx in t.leaves.items():
            cx, cy = t.centre(L, *key)
            dx = t.xy[idx, 0] - cx
            dy = t.xy[idx, 1] - cy
            rho = np.hypot(dx, dy)
            th = np.arctan2(dy, dx)
            m = np.arange(-p[L], p[L] + 1)
            basis = jv(m[None, :], k * rho[:, None]) * np.exp(1j * m[None, :] * th[:, None])
            y[:, idx] += 0.25j * (basis @ loc[L][key]).T

        # Step 5: direct interactions
        for T, idx in (t.leaves.items() if parts & self.NEAR_FREE else []):
            for S in u_list(t, T):
                jdx = t.leaves[S]
                r = np.hypot(t.xy[idx, 0][:, None] - t.xy[jdx, 0][None, :],
                             t.xy[idx, 1][:, None] - t.xy[jdx, 1][None, :])
                same = idx[:, None] == jdx[None, :]
                Gm = np.where(same, 0.0, 0.25j * hankel1(0, k * np.where(same, 1.0, r)))
                y[:, idx] += (Gm @ q[:, jdx].T).T
        for T, S in (self.direct_pairs if parts & self.NEAR_REACT else []):
            idx = t.leaves[T]
            jdx = t.leaves[S]
            Gm = self._direct_block(T, S, idx, jdx)
            y[:, idx] += (Gm @ q[:, jdx].T).T
        return y[0] if squeeze else y

    def _direct_block(self, T, S, idx, jdx):
        key = (T, S)
        if key not in self._direct_cache:
            xy = self.tree.xy
            X = xy[idx, 0][:, None] - xy[jdx, 0][None, :]
            Y = xy[idx, 1][:, None] + xy[jdx, 1][None, :]
            self._direct_cache[key] = green.green_reaction(self.medium, X, Y)
        return self._direct_cache[key]
