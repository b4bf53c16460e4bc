"""O(N M) direct sum y = G q on the CPU in FP64 (test infrastructure).

    y_i = sum_{j != i} (i/4) H0^(1)(k1 |x_i - x_j|) q_j
        + sum_j G^s(x_i - x_j, y_i + y_j) q_j

The free part uses SciPy's Hankel function (AMOS).  The reaction part is the
Sommerfeld integral of Eq. (eq:multisommer) / (eq:multitop) summed over the
sources under the integral sign, i.e. the "uncompressed" form of Eq.
(eq:uncompressed):
    sum_j q_j G^s = 1/(4 pi) int e^{-s1 y_i + i lambda x_i}
                    [sum_j q_j e^{-s1 y_j - i lambda x_j}] sigma / s1 dlambda,
on the same tau / t rules as oracle.green (lambda = -k1 cos tau with
dlambda / s1 = i dtau; lambda = +-xi(t) with dlambda / s1 = dt / xi).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import hankel1

from . import green


def free_sum(xy_t, xy_s, q, k, self_index=None, block=2048):
    """sum_j (i/4) H0(k r_ij) q_j; targets xy_t [M,2], sources xy_s [N,2],
    q [nrhs, N]; self_index[i] = source index equal to target i (skipped) or -1."""
    q = np.atleast_2d(q)
    M = xy_t.shape[0]
    out = np.zeros((q.shape[0], M), dtype=complex)
    for a in range(0, M, block):
        b = min(M, a + block)
        r = np.hypot(xy_t[a:b, 0][:, None] - xy_s[:, 0][None, :],
                     xy_t[a:b, 1][:, None] - xy_s[:, 1][None, :])
        if self_index is not None:
            si = self_index[a:b]
            rows = np.nonzero(si >= 0)[0]
            r[rows, si[rows]] = 1.0
        Gm = 0.25j * hankel1(0, k * r)
        if self_index is not None:
            Gm[rows, si[rows]] = 0.0
        out[:, a:b] = (Gm @ q.T).T
    return out


def reaction_sum(medium, xy_t, xy_s, q, refine=1, chunk=4096):
    """sum_j G^s(x_i - x_j, y_i + y_j) q_j for all targets i."""
    q = np.atleast_2d(q)
    k1 = medium.k1
    xmid = 0.5 * (min(xy_t[:, 0].min(), xy_s[:, 0].min()) + max(xy_t[:, 0].max(), xy_s[:, 0].max()))
    xt = xy_t[:, 0] - xmid
    xs = xy_s[:, 0] - xmid
    yt = xy_t[:, 1]
    ys = xy_s[:, 1]
    xmax = max(np.abs(xt).max(), np.abs(xs).max()) * 2.0
    ymin = yt.min() + ys.min()
    ymax = yt.max() + ys.max()
    out = np.zeros((q.shape[0], xy_t.shape[0]), dtype=complex)
    # propagating part
    tau, wtau = green.tau_rule(medium, xmax, ymax, 0, refine)
    lam = -k1 * np.cos(tau)
    sg = green.sigma(medium, lam * lam + 0j, -1j * k1 * np.sin(tau))
    coef = 1j * wtau * sg / (4 * math.pi)
    for a in range(0, tau.size, chunk):
        b = min(tau.size, a + chunk)
        st, ct = np.sin(tau[a:b]), np.cos(tau[a:b])
        Es = np.exp(1j * k1 * (ys[:, None] * st[None, :] + xs[:, None] * ct[None, :]))
        Et = np.exp(1j * k1 * (yt[:, None] * st[None, :] - xt[:, None] * ct[None, :]))
        Sn = q @ Es                                   # [nrhs, nodes]
        out += (Sn * coef[None, a:b]) @ Et.T
    # evanescent part, both signs of lambda
    t, wt = green.t_rule(medium, xmax, ymin, 0, refine)
    xi = np.sqrt(t * t + k1 * k1)
    sg = green.sigma(medium, xi * xi, t)
    coef = wt * sg / xi / (4 * math.pi)
    for a in range(0, t.size, chunk):
        b = min(t.size, a + chunk)
        tt, xx = t[a:b], xi[a:b]
        for sgn in (1.0, -1.0):
            Es = np.exp(-ys[:, None] * tt[None, :] - 1j * sgn * xs[:, None] * xx[None, :])
            Et = np.exp(-yt[:, None] * tt[None, :] + 1j * sgn * xt[:, None] * xx[None, :])
            Sn = q @ Es
            out += (Sn * coef[None, a:b]) @ Et.T
    return out


def direct_apply(medium, xy, q, targets=None, refine=1):
    """y = G q by direct summation; ``targets`` optionally selects the rows."""
    xy = np.asarray(xy, dtype=float)
    q = np.atleast_2d(np.asarray(q, dtype=complex))
    n = xy.shape[0]
    idx = np.arange(n) if targets is None else np.asarray(targets)
    xt = xy[idx]
    yf = free_sum(xt, xy, q, medium.k1, self_index=idx)
    yr = reaction_sum(medium, xt, xy, q, refine)
    return yf + yr


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


# ---------------------------------------------------------------------------
# field gradients and the position gradient of a real loss
# ---------------------------------------------------------------------------

def free_field_grad(xy_t, xy_s, v, k, self_index=None, block=1024):
    """grad_x sum_j (i/4) H0(k |x - x_j|) v_j at the targets (skipping j = self):
    (i/4) (-k H1(k r)) (x - x_j) / r.  Returns (gx, gy), each [nrhs, M]."""
    v = np.atleast_2d(v)
    M = xy_t.shape[0]
    gx = np.zeros((v.shape[0], M), dtype=complex)
    gy = np.zeros((v.shape[0], M), dtype=complex)
    for a in range(0, M, block):
        b = min(M, a + block)
        dx = xy_t[a:b, 0][:, None] - xy_s[:, 0][None, :]
        dy = xy_t[a:b, 1][:, None] - xy_s[:, 1][None, :]
        r = np.hypot(dx, dy)
        if self_index is not None:
            si = self_index[a:b]
            rows = np.nonzero(si >= 0)[0]
            r[rows, si[rows]] = 1.0
        c = 0.25j * (-k) * hankel1(1, k * r) / r
        if self_index is not None:
            c[rows, si[rows]] = 0.0
        gx[:, a:b] = ((c * dx) @ v.T).T
        gy[:, a:b] = ((c * dy) @ v.T).T
    return gx, gy


def reaction_field_grad(medium, xy_t, xy_s, v, refine=1, chunk=4096):
    """grad over the target point of sum_j G^s(x - x_j, y + y_j) v_j: the
    Sommerfeld integrand's target factor e^{-s1 y + i lambda x} contributes
    i lambda (d/dx) and -s1 (d/dy)."""
    v = np.atleast_2d(v)
    k1 = medium.k1
    xmid = 0.5 * (min(xy_t[:, 0].min(), xy_s[:, 0].min()) + max(xy_t[:, 0].max(), xy_s[:, 0].max()))
    xt, xs = xy_t[:, 0] - xmid, xy_s[:, 0] - xmid
    yt, ys = xy_t[:, 1], xy_s[:, 1]
    xmax = max(np.abs(xt).max(), np.abs(xs).max()) * 2.0
    ymin, ymax = yt.min() + ys.min(), yt.max() + ys.max()
    gx = np.zeros((v.shape[0], xy_t.shape[0]), dtype=complex)
    gy = np.zeros_like(gx)
    tau, wtau = green.tau_rule(medium, xmax, ymax, 1, refine)
    lam = -k1 * np.cos(tau)
    s1 = -1j * k1 * np.sin(tau)
    sg = green.sigma(medium, lam * lam + 0j, s1)
    coef = 1j * wtau * sg / (4 * math.pi)
    for a in range(0, tau.size, chunk):
        b = min(tau.size, a + chunk)
        st, ct = np.sin(tau[a:b]), np.cos(tau[a:b])
        Es = np.exp(1j * k1 * (ys[:, None] * st[None, :] + xs[:, None] * ct[None, :]))
        Et = np.exp(1j * k1 * (yt[:, None] * st[None, :] - xt[:, None] * ct[None, :]))
        Sn = (v @ Es) * coef[None, a:b]
        gx += (Sn * (1j * lam[None, a:b])) @ Et.T
        gy += (Sn * (-s1[None, a:b])) @ Et.T
    t, wt = green.t_rule(medium, xmax, ymin, 1, refine)
    xi = np.sqrt(t * t + k1 * k1)
    sg = green.sigma(medium, xi * xi, t)
    coef = wt * sg / xi / (4 * math.pi)
    for a in range(0, t.size, chunk):
        b = min(t.size, a + chunk)
        tt, xx = t[a:b], xi[a:b]
        for sgn in (1.0, -1.0):
            Es = np.exp(-ys[:, None] * tt[None, :] - 1j * sgn * xs[:, None] * xx[None, :])
            Et = np.exp(-yt[:, None] * tt[None, :] + 1j * sgn * xt[:, None] * xx[None, :])
            Sn = (v @ Es) * coef[None, a:b]
            gx += (Sn * (1j * sgn * xx[None, :])) @ Et.T
            gy += (Sn * (-tt[None, :])) @ Et.T
    return gx, gy


def field_grad(medium, xy, v):
    """grad_x of u(x) = sum_j G(x, x_j) v_j at every point x_i (free self term
    skipped, reaction self term kept)."""
    xy = np.asarray(xy, dtype=float)
    v = np.atleast_2d(np.asarray(v, dtype=complex))
    n = xy.shape[0]
    fx, fy = free_field_grad(xy, xy, v, medium.k1, self_index=np.arange(n))
    rx, ry = reaction_field_grad(medium, xy, xy, v)
    return fx + rx, fy + ry


def position_grad(medium, xy, q, g):
    """dL/dx_j, dL/dy_j of a real loss L(y), y = G(x) q, given
    g = dL/dRe(y) + i dL/dIm(y) (shape [nrhs, n]):
        dL/dx_j = Re sum_r [ conj(g_rj) d_x u_r(x_j) + q_rj d_x w_r(x_j) ],
    u_r = sum_k G(., x_k) q_rk, w_r = sum_k G(., x_k) conj(g_rk), which uses
    the reciprocity G(a, b) = G(b, a).  Returns [n, 2]."""
    q = np.atleast_2d(q)
    g = np.atleast_2d(g)
    ux, uy = field_grad(medium, xy, q)
    wx, wy = field_grad(medium, xy, np.conj(g))
    gx = np.real(np.conj(g) * ux + q * wx).sum(axis=0)
    gy = np.real(np.conj(g) * uy + q * wy).sum(axis=0)
    return np.stack([gx, gy], axis=1)
