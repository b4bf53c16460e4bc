"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers: point clouds, complex strengths and
medium parameters shaped like the workloads the H-FMM is measured on.  It
holds none of the method's arithmetic (no Green's function, no expansion, no
tree), so both the CUDA path and the CPU oracle may take their inputs from it.

Seeds: ``seed = 1000 * cfg + stream`` with stream 1 for positions, 2 for
strengths, 3 for anything else (sample indices, perturbations), drawn with
NumPy's PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Medium kinds, numbered as in the C header.
IMPEDANCE = 0
TWO_LAYER = 1
THREE_LAYER = 2


@dataclass(frozen=True)
class Medium:
    """Layered medium seen from the top layer (sources and targets have y > 0).

    kind      IMPEDANCE: half-space y > 0 with the impedance condition on y = 0.
              TWO_LAYER: k[0] for y > 0, k[1] for y < 0.
              THREE_LAYER: k[0] for y > 0, k[1] for -d < y < 0, k[2] for y < -d.
    k         wavenumbers (unused entries are ignored).
    d         thickness of the middle layer (THREE_LAYER only).
    alpha     real impedance parameter (IMPEDANCE only).
    """
    kind: int
    k: tuple
    d: float = 0.0
    alpha: float = 0.0

    @property
    def k1(self) -> float:
        return float(self.k[0])


@dataclass(frozen=True)
class Workload:
    name: str
    medium: Medium
    n: int
    box: tuple            # ((x0, x1), (y0, y1))
    nrhs: int
    tol: float
    leaf: int
    dist: str = "uniform"
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    1: Workload("impedance-1600-k20", Medium(IMPEDANCE, (20.0,), alpha=10.0),
                1600, ((0.0, 1.0), (0.05, 1.05)), 1, 1e-6, 32),
    2: Workload("impedance-6400-clusters-k40", Medium(IMPEDANCE, (40.0,), alpha=20.0),
                6400, ((0.0, 1.0), (0.05, 1.05)), 1, 1e-6, 32, "clusters"),
    3: Workload("two-layer-262144-k60-90", Medium(TWO_LAYER, (60.0, 90.0)),
                262144, ((0.0, 4.0), (0.02, 4.02)), 1, 1e-6, 32),
    4: Workload("three-layer-1048576-k40-80-60-64rhs",
                Medium(THREE_LAYER, (40.0, 80.0, 60.0), d=0.5),
                1048576, ((0.0, 8.0), (0.02, 8.02)), 64, 1e-6, 32),
    5: Workload("impedance-batch32-k40", Medium(IMPEDANCE, (40.0,), alpha=20.0),
                0, ((0.0, 1.0), (0.05, 1.05)), 1, 1e-6, 32, "batch",
                {"ninst": 32, "nmin": 4096, "nmax": 200000}),
    # the setting of the paper's timing table (Sec. 4): impedance alpha = 1,
    # low frequency, sources = targets in the unit box centred at (0, 1.5),
    # fixed order p = 39; N runs over the table's sizes
    6: Workload("impedance-table2-sweep", Medium(IMPEDANCE, (0.1,), alpha=1.0),
                0, ((-0.5, 0.5), (1.0, 2.0)), 1, 1e-6, 32, "sweep",
                {"p": 39, "k": (0.1, 1.0),
                 "n": (100, 6400, 10000, 90000, 360000, 640000, 810000, 1000000)}),
    # high frequency on the unit box (level-2 boxes 30 and 120 wavelengths
    # wide): the coarse levels' translations dominate the FP64 apply
    7: Workload("impedance-unit-box-high-frequency", Medium(IMPEDANCE, (400.0,), alpha=200.0),
                0, ((0.0, 1.0), (0.05, 1.05)), 1, 1e-6, 32, "uniform",
                {"cases": ((400.0, 65536), (1500.0, 65536), (1500.0, 262144))}),
    # particles on the surface of a scatterer (a five-lobed star curve in
    # config 1's box): the setting the paper's adaptive tree is made for
    8: Workload("impedance-star-curve-k40", Medium(IMPEDANCE, (40.0,), alpha=20.0),
                65536, ((0.0, 1.0), (0.05, 1.05)), 1, 1e-6, 32, "curve",
                {"centre": (0.5, 0.55), "R": 0.3, "a": 0.3, "lobes": 5, "bench_n": (65536, 262144)}),
}


def generator(cfg: int, stream: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * cfg + stream + 100000 * salt))


def _uniform(g, n, box):
    (x0, x1), (y0, y1) = box
    xy = np.empty((n, 2))
    xy[:, 0] = g.uniform(x0, x1, n)
    xy[:, 1] = g.uniform(y0, y1, n)
    return xy


def _clusters(g, n, box):
    """40% / 40% Gaussian blobs (sigma 0.1) at (0.3, 0.4) and (0.7, 0.9), 20%
    uniform; Gaussian samples outside the box are redrawn."""
    (x0, x1), (y0, y1) = box
    n1 = int(round(0.4 * n))
    n2 = int(round(0.4 * n))
    n3 = n - n1 - n2
    parts = []
    for centre, m in (((0.3, 0.4), n1), ((0.7, 0.9), n2)):
        got = np.empty((0, 2))
        while got.shape[0] < m:
            cand = g.normal(centre, 0.1, size=(2 * m, 2))
            ok = (cand[:, 0] >= x0) & (cand[:, 0] <= x1) & (cand[:, 1] >= y0) & (cand[:, 1] <= y1)
            got = np.concatenate([got, cand[ok]])
        parts.append(got[:m])
    parts.append(_uniform(g, n3, box))
    xy = np.concatenate(parts)
    return xy[g.permutation(n)]


def _curve(g, n, extra):
    """Points on the closed star curve r(t) = R (1 + a cos(m t)) about c,
    equally spaced in t with a uniform jitter of a quarter spacing: the
    surface of a scatterer discretised into particles."""
    cx, cy = extra["centre"]
    R, a, m = extra["R"], extra["a"], extra["lobes"]
    t = (np.arange(n) + 0.25 * g.uniform(-1.0, 1.0, n)) * (2.0 * math.pi / n)
    r = R * (1.0 + a * np.cos(m * t))
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def points(cfg: int, n: int | None = None, salt: int = 0) -> np.ndarray:
    """Point cloud [n, 2] (float64) of workload ``cfg``; ``n`` overrides the size."""
    w = WORKLOADS[cfg]
    n = w.n if n is None else int(n)
    g = generator(cfg, 1, salt)
    if w.dist == "clusters":
        return _clusters(g, n, w.box)
    if w.dist == "curve":
        return _curve(g, n, w.extra)
    return _uniform(g, n, w.box)


def points_in_box(cfg: int, n: int, box, salt: int = 0) -> np.ndarray:
    """Uniform points of workload ``cfg``'s seed family inside an explicit box."""
    return _uniform(generator(cfg, 1, salt), int(n), box)


def strengths(cfg: int, n: int, nrhs: int | None = None, salt: int = 0) -> np.ndarray:
    """Complex strengths [nrhs, n] (complex128) with i.i.d. N(0,1) real and
    imaginary parts; right-hand side r is row r (column-major [nrhs][n])."""
    w = WORKLOADS[cfg]
    nrhs = w.nrhs if nrhs is None else int(nrhs)
    g = generator(cfg, 2, salt)
    re = g.standard_normal((nrhs, n))
    im = g.standard_normal((nrhs, n))
    return re + 1j * im


def sample_indices(cfg: int, n: int, m: int, salt: int = 0) -> np.ndarray:
    """m distinct indices in [0, n), sorted."""
    g = generator(cfg, 3, salt)
    return np.sort(g.choice(n, size=min(m, n), replace=False))


def batch_sizes(cfg: int = 5) -> np.ndarray:
    """Instance sizes of the uneven batch: log-uniform in [nmin, nmax]."""
    w = WORKLOADS[cfg]
    g = generator(cfg, 3)
    lo, hi = math.log(w.extra["nmin"]), math.log(w.extra["nmax"])
    return np.floor(np.exp(g.uniform(lo, hi, w.extra["ninst"]))).astype(np.int64)


def perturb(cfg: int, xy: np.ndarray, sigma: float = 1e-3, salt: int = 0) -> np.ndarray:
    """Positions moved by i.i.d. N(0, sigma^2) per coordinate."""
    g = generator(cfg, 4, salt)
    return xy + g.normal(0.0, sigma, size=xy.shape)
