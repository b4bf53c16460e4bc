"""CPU FP64 oracle for the top-layer domain Green's function (test infrastructure).

This package is the independent reference the CUDA path is checked against.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; nothing in the library calls it.  It is plain, slow NumPy /
SciPy code that follows the paper's formulas term by term.

Notation (paper, Sec. 2):
  * top layer y > 0 with wavenumber k1; sources and targets lie there;
  * s_j(lambda) = sqrt(lambda^2 - k_j^2) on the branch Re s >= 0, written
    s_j = -i sqrt(k_j^2 - lambda^2) with the principal square root, so that
    s = -i sqrt(k^2 - lambda^2) for |lambda| < k (outgoing waves, time factor
    e^{-i omega t}, Sommerfeld identity Eq. (eq:spectralfree));
  * the reaction (scattered) field of a unit source at x0 observed at x is
    G^s(X, Y) with X = x - x0, Y = y + y0 > 0 (Eq. (eq:multisommer), Eq.
    (eq:multitop)):
        G^s(X, Y) = 1/(4 pi) int e^{-s1 Y} / s1 e^{i lambda X} sigma(lambda) dlambda.
  * sigma is the only place the medium enters:
        impedance   sigma_hat = (s1 + i alpha) / (s1 - i alpha)   (Sec. 2.2)
        two layers  sigma_1   = (s1 - s2) / (s1 + s2)            (d -> inf of Sec. 2.3)
        three layers sigma_1 from the 4x4 system of Sec. 2.3, closed form
                    (r12 + r23 e^{-2 s2 d}) / (1 + r12 r23 e^{-2 s2 d}).

Readings of the paper taken here (each is pinned by a test):
  * the impedance condition du/dn - i alpha u = 0 uses the normal n = -y_hat
    (outward from y > 0); this is the normal that gives sigma_hat;
  * theta inside the plane-wave form of the M2L operator (Eq. (eq:m2loperator))
    is the integration variable tau;
  * real-axis poles of sigma_1 (guided modes of the middle layer) and the
    branch points of s2, s3 are avoided by deforming the evanescent variable t
    into Im t < 0 (limiting absorption: a lossy k_j moves them into Im > 0).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss
from scipy.special import hankel1

IMPEDANCE, TWO_LAYER, THREE_LAYER = 0, 1, 2

GL_POINTS = 20
_GL_X, _GL_W = leggauss(GL_POINTS)


# ---------------------------------------------------------------------------
# branches and sigma functions
# ---------------------------------------------------------------------------

def _plus_zero_imag(w):
    """Give purely real entries a +0 imaginary part so that the principal
    square root of a negative real number is +i sqrt(|w|)."""
    w = np.asarray(w, dtype=complex)
    return np.where(w.imag == 0.0, w.real + 0j, w)


def s_of(k, lam2):
    """s = -i sqrt(k^2 - lambda^2), principal sqrt; lam2 = lambda^2 (complex)."""
    return -1j * np.sqrt(_plus_zero_imag(k * k - np.asarray(lam2, dtype=complex)))


def sigma(medium, lam2, s1):
    """sigma(lambda) of the medium, given lambda^2 and the top-layer s1."""
    lam2 = np.asarray(lam2, dtype=complex)
    s1 = np.asarray(s1, dtype=complex)
    kind = medium.kind
    if kind == IMPEDANCE:
        a = medium.alpha
        return (s1 + 1j * a) / (s1 - 1j * a)
    if kind == TWO_LAYER:
        s2 = s_of(medium.k[1], lam2)
        return (s1 - s2) / (s1 + s2)
    if kind == THREE_LAYER:
        s2 = s_of(medium.k[1], lam2)
        s3 = s_of(medium.k[2], lam2)
        r12 = (s1 - s2) / (s1 + s2)
        r23 = (s2 - s3) / (s2 + s3)
        e = np.exp(-2.0 * s2 * medium.d)
        return (r12 + r23 * e) / (1.0 + r12 * r23 * e)
    raise ValueError(f"unknown medium kind {kind}")


def sigma_three_layer_4x4(k1, k2, k3, d, lam):
    """Solve the paper's printed 4x4 system (Sec. 2.3) at one real lambda and
    return (sigma_1, sigma_2^+, sigma_2^-, sigma_3).  The square roots
    sqrt(lambda^2 - k_j^2) are the branch s_j defined above."""
    l2 = complex(lam) ** 2
    s1, s2, s3 = (complex(s_of(k, l2)) for k in (k1, k2, k3))
    e = np.exp(-s2 * d)
    A = np.array([
        [1 / s1, -1 / s2, -e / s2, 0],
        [0, e / s2, 1 / s2, -1 / s3],
        [1, 1, -e, 0],
        [0, e, -1, -1],
    ], dtype=complex)
    b = np.array([-1 / s1, 0, 1, 0], dtype=complex)
    return np.linalg.solve(A, b)


def singular_t(medium):
    """Real t >= 0 (t = s1 on the evanescent branch, lambda^2 = t^2 + k1^2)
    where sigma is not analytic: branch points of s_j with k_j > k1 and, for
    three layers, guided-mode poles which lie between them."""
    k1 = medium.k1
    pts = []
    if medium.kind in (TWO_LAYER, THREE_LAYER):
        ks = medium.k[1:2] if medium.kind == TWO_LAYER else medium.k[1:3]
        for kj in ks:
            if kj > k1:
                pts.append(math.sqrt(kj * kj - k1 * k1))
    return pts


def tau_kinks(medium):
    """tau in (0, pi) where sigma(-k1 cos tau) has a square-root kink
    (branch points of s_j with k_j < k1 lie on the propagating range)."""
    k1 = medium.k1
    out = []
    if medium.kind in (TWO_LAYER, THREE_LAYER):
        ks = medium.k[1:2] if medium.kind == TWO_LAYER else medium.k[1:3]
        for kj in ks:
            if kj < k1:
                c = kj / k1
                out += [math.acos(c), math.acos(-c)]
    return sorted(out)


# ---------------------------------------------------------------------------
# quadrature rules for the propagating (tau) and evanescent (t) integrals
# ---------------------------------------------------------------------------

def _panels(a, b, n):
    """Composite Gauss-Legendre on [a, b] with n equal panels."""
    edges = np.linspace(a, b, n + 1)
    lo, hi = edges[:-1], edges[1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    x = (mid[:, None] + half[:, None] * _GL_X[None, :]).ravel()
    w = (half[:, None] * _GL_W[None, :]).ravel()
    return x, w


def _edge_panels(edges):
    """Gauss-Legendre nodes and weights on the panels between given edges."""
    edges = np.asarray(edges, dtype=float)
    lo, hi = edges[:-1], edges[1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    x = (mid[:, None] + half[:, None] * _GL_X[None, :]).ravel()
    w = (half[:, None] * _GL_W[None, :]).ravel()
    return x, w


def impedance_pole_tau(medium):
    """The impedance sigma_hat = (s1 + i alpha)/(s1 - i alpha) (Sec. 2.2) has a
    pole at s1 = i alpha.  On the propagating path s1 = -i k1 sin tau, so for
    0 < alpha < k1 the pole lies on the real tau axis at -delta and
    pi + delta, delta = asin(alpha / k1); returns delta (None otherwise)."""
    if medium.kind == IMPEDANCE and 0.0 < medium.alpha < medium.k1:
        return math.asin(medium.alpha / medium.k1)
    return None


def tau_rule(medium, xmax, ymax, nmax, refine=1):
    """Nodes and weights on [0, pi] for integrands e^{i k1 (Y sin - X cos)}
    e^{-i n tau} sigma with |X| <= xmax, Y <= ymax, |n| <= nmax.  Near an
    impedance pole no panel is wider than 1.5 times its distance to it."""
    k1 = medium.k1
    rate = k1 * (abs(xmax) + abs(ymax)) + nmax + 1.0
    if medium.kind == THREE_LAYER:
        rate += 2.0 * medium.d * max(abs(medium.k[1]), k1)   # e^{-2 s2 d} of sigma_1
    brk = [0.0] + tau_kinks(medium) + [math.pi]
    delta = impedance_pole_tau(medium)
    xs, ws = [], []
    for a, b in zip(brk[:-1], brk[1:]):
        n = refine * (int(math.ceil((b - a) * rate / 5.0)) + 2)
        if delta is None:
            x, w = _panels(a, b, n)
        else:
            width = (b - a) / n
            edges = [a]
            while edges[-1] < b:
                e = edges[-1]
                step = min(width, 1.5 * (e + delta) / refine, 0.6 * (math.pi + delta - e) / refine, b - e)
                edges.append(b if b - (e + step) < 1e-14 else e + step)
            x, w = _edge_panels(edges)
        xs.append(x)
        ws.append(w)
    return np.concatenate(xs), np.concatenate(ws)


def _log_envelope(t, k1, Y, nmax):
    xi = np.sqrt(t * t + k1 * k1)
    return -t * Y + nmax * np.log((xi + t) / k1) - np.log(xi)


def t_upper(k1, Y, nmax, digits=40.0):
    """Upper limit T of the evanescent integral: the envelope
    e^{-tY} ((xi + t)/k1)^nmax / xi has dropped e^{-digits} below its peak."""
    if Y <= 0:
        raise ValueError("the evanescent integral needs Y > 0")
    grid = np.concatenate([[0.0], np.geomspace(1e-3, 1e7, 4000)])
    env = _log_envelope(grid, k1, Y, nmax)
    ipk = int(np.argmax(env))
    target = env[ipk] - digits
    lo = grid[ipk]
    hi = max(lo * 2.0, 1.0)
    while _log_envelope(hi, k1, Y, nmax) > target:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _log_envelope(mid, k1, Y, nmax) > target:
            lo = mid
        else:
            hi = mid
    return hi


def t_rule(medium, xmax, ymin, nmax, refine=1):
    """Complex nodes t and weights dt (Jacobian included) for the evanescent
    integral over t in [0, T].  For layered media the path is deformed to
    t = u - i c sin(pi u / tb) on [0, tb], tb beyond every real singularity,
    then follows the real axis."""
    k1 = medium.k1
    xmax = abs(xmax)
    T = t_upper(k1, ymin, nmax)
    sing = singular_t(medium)
    ts, ws = [], []
    u0 = 0.0
    if sing:
        tb = 1.25 * max(sing) + 0.05 * k1
        c = min(0.15 * tb, 1.0 / max(xmax, 1e-12))
        wdef = 1.2 * c
        if medium.kind == THREE_LAYER and medium.d > 0:
            wdef = min(wdef, 2.5 / medium.d)
        npan = refine * (2 * int(math.ceil(tb / wdef)) + 8)
        u, wu = _panels(0.0, tb, npan)
        ph = math.pi / tb
        t = u - 1j * c * np.sin(ph * u)
        dt = 1.0 - 1j * c * ph * np.cos(ph * u)
        ts.append(t)
        ws.append(wu * dt)
        u0 = tb
        T = max(T, tb + 1.0)
    # real axis [u0, T]: panel width limited by decay, oscillation and the
    # power ((xi + t)/k1)^nmax
    wmax = 5.0 / max(ymin, 1e-300)
    if xmax > 0:
        wmax = min(wmax, 5.0 / xmax)
    if medium.kind == THREE_LAYER and medium.d > 0:
        wmax = min(wmax, 2.5 / medium.d)
    # impedance pole at t = i alpha (Sec. 2.2): panel width <= 1.5 x its distance
    alpha = medium.alpha if medium.kind == IMPEDANCE and medium.alpha > 0 else None
    edges = [u0]
    a = u0
    while a < T:
        w = min(wmax, max(5.0 * max(a, 0.5 / k1) / max(nmax, 1), 0.02 * wmax, 1e-3), T - a)
        if alpha is not None:
            w = min(w, 1.5 * math.hypot(a, alpha))
        # 1/xi, xi = sqrt(t^2 + k1^2), has branch points at t = +-i k1: at low
        # frequency they sit close to t = 0, so the panels there are graded too
        w = min(w, 1.5 * math.hypot(a, k1))
        w = max(w / refine, 1e-12)
        a = a + w
        edges.append(a)
    edges = np.array(edges)
    lo, hi = edges[:-1], edges[1:]
    half = 0.5 * (hi - lo)
    mid = 0.5 * (hi + lo)
    ts.append((mid[:, None] + half[:, None] * _GL_X[None, :]).ravel() + 0j)
    ws.append((half[:, None] * _GL_W[None, :]).ravel() + 0j)
    return np.concatenate(ts), np.concatenate(ws)


# ---------------------------------------------------------------------------
# G^s(X, Y) and the heterogeneous M2L kernel A_n(X, Y)
# ---------------------------------------------------------------------------

def green_reaction(medium, X, Y, refine=1):
    """G^s(X, Y) for arrays X, Y (Y > 0): propagating part over tau plus
    evanescent part over t (Eq. (eq:evanprop) with sigma inserted):
        (i / 4 pi) int_0^pi e^{i k1 (Y sin tau - X cos tau)} sigma(-k1 cos tau) dtau
      + (1 / 2 pi) int_0^inf e^{-t Y} cos(xi X) / xi sigma(xi) dt,  xi = sqrt(t^2 + k1^2).
    """
    X = np.atleast_1d(np.asarray(X, dtype=float))
    Y = np.atleast_1d(np.asarray(Y, dtype=float))
    X, Y = np.broadcast_arrays(X, Y)
    k1 = medium.k1
    tau, wtau = tau_rule(medium, np.max(np.abs(X)), np.max(Y), 0, refine)
    lam = -k1 * np.cos(tau)
    sg_tau = sigma(medium, lam * lam + 0j, -1j * k1 * np.sin(tau))
    t, wt = t_rule(medium, np.max(np.abs(X)), np.min(Y), 0, refine)
    xi = np.sqrt(t * t + k1 * k1)
    sg_t = sigma(medium, xi * xi, t)
    out = np.empty(X.shape, dtype=complex)
    for idx in np.ndindex(X.shape):
        x, y = X[idx], Y[idx]
        prop = np.sum(wtau * np.exp(1j * k1 * (y * np.sin(tau) - x * np.cos(tau))) * sg_tau)
        evan = np.sum(wt * np.exp(-t * y) * np.cos(xi * x) / xi * sg_t)
        out[idx] = 1j / (4 * math.pi) * prop + evan / (2 * math.pi)
    return out


def hetero_m2l_kernel(medium, X, Y, nmax, refine=1):
    """A_n(X, Y), n = -nmax..nmax (Eq. (eq:m2loperator), three-layer form of
    Sec. 5 with sigma of the medium; theta read as tau):
      A_n = i^n / pi int_0^pi e^{i k1 (Y sin tau - X cos tau)} e^{-i n tau} sigma(-k1 cos tau) dtau
          + (-i)^n / (i pi) int_0^inf e^{-tY} / xi [ e^{i xi X} ((xi - t)/k1)^n
                                                   + e^{-i xi X} ((-xi - t)/k1)^n ] sigma(xi) dt.
    With sigma = 1 this is H_n(k1 |D|) e^{i n angle(D)} for D = (X, Y).
    Returns an array of length 2 nmax + 1 (index n + nmax)."""
    k1 = medium.k1
    n = np.arange(-nmax, nmax + 1)
    tau, wtau = tau_rule(medium, abs(X), Y, nmax, refine)
    lam = -k1 * np.cos(tau)
    sg_tau = sigma(medium, lam * lam + 0j, -1j * k1 * np.sin(tau))
    base = wtau * np.exp(1j * k1 * (Y * np.sin(tau) - X * np.cos(tau))) * sg_tau
    prop = (np.exp(-1j * np.outer(n, tau)) @ base) * (1j ** n) / math.pi
    t, wt = t_rule(medium, abs(X), Y, nmax, refine)
    xi = np.sqrt(t * t + k1 * k1)
    sg_t = sigma(medium, xi * xi, t)
    zp = k1 / (xi + t)            # (xi - t)/k1 without cancellation
    zm = -(xi + t) / k1           # (-xi - t)/k1
    common = wt * np.exp(-t * Y) / xi * sg_t
    ep = np.exp(1j * xi * X) * common
    em = np.exp(-1j * xi * X) * common
    evan = np.empty(n.shape, dtype=complex)
    for i, nn in enumerate(n):
        evan[i] = np.sum(ep * zp ** nn + em * zm ** nn)
    evan *= ((-1j) ** n) / (1j * math.pi)
    return prop + evan


def hankel_cyl(nmax, X, Y, k):
    """H_n(k |D|) e^{i n angle(D)}, n = -nmax..nmax, via SciPy (AMOS)."""
    r = math.hypot(X, Y)
    th = math.atan2(Y, X)
    n = np.arange(-nmax, nmax + 1)
    return hankel1(n, k * r) * np.exp(1j * n * th)


# ---------------------------------------------------------------------------
# independent representation: complex line image (impedance, Sec. 2.2)
# ---------------------------------------------------------------------------

def green_reaction_line_image(k, alpha, X, Y):
    """Impedance G^s from the point image plus the line image
    mu(s) = 2 i alpha e^{i alpha s} (Eq. (Sfield)), with the line integral
    rotated to s = i v (both factors decay in the first quadrant):
      (i/4) H0(k r_im) + int_0^inf (i/4) H0(k sqrt(X^2 + (Y + i v)^2))
                                   2 i alpha e^{-alpha v} i dv."""
    from scipy.integrate import quad
    r_im = math.hypot(X, Y)
    point = 0.25j * hankel1(0, k * r_im)

    def f(v, part):
        w = np.sqrt(X * X + (Y + 1j * v) ** 2 + 0j)
        val = 0.25j * hankel1(0, k * w) * 2j * alpha * math.exp(-alpha * v) * 1j
        return val.real if part == 0 else val.imag

    upper = 60.0 / alpha
    re = quad(f, 0, upper, args=(0,), limit=400, epsabs=1e-15, epsrel=1e-13)[0]
    im = quad(f, 0, upper, args=(1,), limit=400, epsabs=1e-15, epsrel=1e-13)[0]
    return point + re + 1j * im


def green_free(k, r):
    """(i/4) H0^(1)(k r), Eq. (eq:freeGreen)."""
    return 0.25j * hankel1(0, k * np.asarray(r))
