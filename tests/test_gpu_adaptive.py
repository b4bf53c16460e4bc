"""Adaptive trees (Sec. 3.1, HFMM_FLAG_ADAPTIVE) on the CUDA path against the
oracle's adaptive H-FMM (oracle/adaptive.py):

* boxes, point sets and the U / V / W / X, reaction and direct lists equal
  the oracle's as sets of (level, ix, iy) keys;
* each of the four terms at <= 1e-11 (relative to the full result) against
  the CPU FMM at equal p, on clustered clouds for the impedance and
  three-layer media;
* the whole apply against the O(N^2) direct sum at tol 1e-6 and 1e-10;
* adjoint, batches and the options that adaptive plans refuse;
* mixed precision (FP32 passes over plan-time bases) against FP64 and the
  oracle within 1e-5.
"""
import numpy as np
import pytest

import workloads as W
from workloads import Medium
from oracle import adaptive, direct

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1703_09136_gb300 import Batch, HfmmError, MIXED, Plan  # noqa: E402

PARITY_TOL = 1e-11
CFG4_MED = W.WORKLOADS[4].medium


def _near_interface(n, salt):
    """60% in a Gaussian blob (sigma 0.05) at (0.3, 0.08), redrawn below
    y = 0.02; 40% uniform in [0, 0.6] x [0.02, 0.62]."""
    g = np.random.Generator(np.random.PCG64(7000 + salt))
    n1 = int(0.6 * n)
    pts = []
    while len(pts) < n1:
        c = g.normal((0.3, 0.08), 0.05, size=(n1, 2))
        c = c[(c[:, 1] >= 0.02) & (c[:, 0] >= 0.0) & (c[:, 0] <= 0.6) & (c[:, 1] <= 0.62)]
        pts.extend(c.tolist())
    u = np.stack([g.uniform(0.0, 0.6, n - n1), g.uniform(0.02, 0.62, n - n1)], axis=1)
    return np.concatenate([np.array(pts[:n1]), u])


def _case(name):
    """(medium, xy, q, tol, leaf)"""
    if name == "cfg2-clusters":
        xy = W.points(2, 1200)
        return W.WORKLOADS[2].medium, xy, W.strengths(2, 1200, 2, salt=41), 1e-6, 12
    if name == "three-layer-near-interface":
        xy = _near_interface(700, 2)
        return CFG4_MED, xy, W.strengths(4, 700, 2, salt=42), 1e-6, 12
    if name == "star-curve":
        xy = W.points(8, 1500)
        return W.WORKLOADS[8].medium, xy, W.strengths(8, 1500, 2, salt=45), 1e-6, 16
    raise KeyError(name)


_cache = {}


def _oracle(name):
    if name not in _cache:
        med, xy, q, tol, leaf = _case(name)
        F = adaptive.AdaptiveCpuFmm(xy, med, tol=tol, leaf_size=leaf)
        _cache[name] = (F, {part: F.apply(q, parts=part) for part in (1, 2, 4, 8)})
    return _cache[name]


def _plan(name, **kw):
    med, xy, q, tol, leaf = _case(name)
    return Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=q.shape[0], adaptive=True, **kw)


@pytest.mark.parametrize("name", ["cfg2-clusters", "three-layer-near-interface", "star-curve"])
def test_adaptive_tree_and_lists_equal_the_oracle(name):
    F, _ = _oracle(name)
    med, xy, q, tol, leaf = _case(name)
    plan = _plan(name)
    boxes = plan.boxes()
    perm = plan.perm()
    inf = plan.info
    keys = [(int(b[0]), int(b[1]), int(b[2])) for b in boxes]
    t = F.tree
    assert set(keys) == set(t.boxes), "boxes"
    for b, key in zip(boxes, keys):
        pts = set(perm[b[3]:b[4]].tolist())
        assert pts == set(t.boxes[key].idx.tolist()), key
        assert bool(b[5]) == t.boxes[key].leaf, key
    assert inf["adaptive"] == 1 and inf["levels"] == t.L
    assert inf["nonempty_leaves"] == len(t.leaves())
    assert inf["p"] == list(F.p)

    def pairs(kind):
        return {(keys[a], keys[b]) for a, b in plan.lists(kind)}

    want_u = {(T.key, S.key) for T in t.leaves() for S in F.U[T.key]}
    want_v = {(k, S.key) for k, vs in F.V.items() for S in vs}
    want_w = {(T.key, D.key) for T in t.leaves() for D in F.W[T.key]}
    want_x = {(k, C.key) for k, cs in F.X.items() for C in cs}
    want_r = {(T.key, S.key) for l in F.R for T, S in F.R[l]}
    want_d = {(T.key, S.key) for T, S in F.direct_pairs}
    got = [pairs(k) for k in range(6)]
    assert got[0] == want_u and got[1] == want_v and got[2] == want_w
    assert got[3] == want_x and got[4] == want_r and got[5] == want_d
    assert inf["w_pairs"] == len(want_w) > 0 and inf["x_pairs"] == len(want_x) > 0
    plan.close()


@pytest.mark.parametrize("part", [1, 2, 4, 8])
@pytest.mark.parametrize("name", ["cfg2-clusters", "three-layer-near-interface", "star-curve"])
def test_adaptive_terms_match_cpu_fmm(name, part):
    """Each term (1 U-list H0, 2 free far field with V, W and X, 4 reaction
    M2L, 8 directly summed reaction) against the oracle's adaptive FMM."""
    F, parts = _oracle(name)
    med, xy, q, tol, leaf = _case(name)
    plan = _plan(name)
    y = plan.apply(torch.from_numpy(q).cuda(), parts=part).cpu().numpy()
    plan.close()
    full = sum(parts.values())
    err = np.linalg.norm(y - parts[part]) / np.linalg.norm(full)
    assert err < PARITY_TOL, (name, part, err)


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_adaptive_matches_direct_sum_on_config_2(tol):
    """Config 2 itself (6400 points, 80% in two Gaussian clusters) with the
    adaptive tree at tol 1e-6 and 1e-10."""
    w = W.WORKLOADS[2]
    xy = W.points(2)
    q = W.strengths(2, xy.shape[0], 1)
    yd = direct.direct_apply(w.medium, xy, q)
    plan = Plan(xy, w.medium, tol=tol, leaf_size=w.leaf, max_rhs=1, adaptive=True)
    inf = plan.info
    y = plan.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    plan.close()
    assert inf["w_pairs"] > 0 and inf["x_pairs"] > 0
    assert direct.rel_l2(y, yd) < tol, direct.rel_l2(y, yd)


def test_adaptive_adjoint_batch_and_refused_options():
    med, xy, q, tol, leaf = _case("three-layer-near-interface")
    plan = _plan("three-layer-near-interface")
    qd = torch.from_numpy(q).cuda()
    rng = np.random.default_rng(43)
    v = rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)
    Gq = plan.apply(qd).cpu().numpy()
    GHv = plan.adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    assert abs(np.vdot(v, Gq) - np.vdot(GHv, q)) < 1e-12 * abs(np.vdot(v, Gq))
    with pytest.raises(HfmmError):
        plan.grad(qd, qd)
    plan.close()
    # two adaptive instances through the batch graph equal their single plans
    xy2 = _near_interface(500, 3)
    q2 = W.strengths(4, 500, 2, salt=44)
    b = Batch([xy, xy2], med, tol=tol, leaf_size=leaf, max_rhs=2, adaptive=True)
    ys = b.apply([qd, torch.from_numpy(q2).cuda()])
    b.close()
    for x_, q_, y_ in ((xy, q, ys[0]), (xy2, q2, ys[1])):
        with Plan(x_, med, tol=tol, leaf_size=leaf, max_rhs=2, adaptive=True) as p1:
            assert np.array_equal(p1.apply(torch.from_numpy(q_).cuda()).cpu().numpy(), y_.cpu().numpy())
    with pytest.raises(HfmmError):
        Plan(xy, med, tol=tol, leaf_size=leaf, autotune=True, adaptive=True)


@pytest.mark.parametrize("case", ["n1", "n2", "n3", "n33", "collinear", "depth-cap"])
def test_adaptive_edge_cases_match_direct_sum(case):
    """Tiny and degenerate inputs on the adaptive tree against the direct
    sum: 1, 2, 3 and 33 points; 400 points on one horizontal line (the root
    square from the x extent); 60 points packed within 1e-9 of each other
    beside 300 spread ones, so boxes reach the depth cap (level 16) still
    holding more than leaf_size points and stay leaves."""
    med = W.WORKLOADS[1].medium
    g = np.random.Generator(np.random.PCG64(9100))
    if case.startswith("n"):
        n = int(case[1:])
        xy = W.points(1, n, salt=9)
    elif case == "collinear":
        xy = np.stack([np.linspace(0.0, 1.0, 400) + 1e-4 * g.uniform(-1, 1, 400), np.full(400, 0.3)], axis=1)
    else:
        base = W.points(1, 300, salt=10)
        tight = np.array([0.41, 0.57]) + 1e-9 * g.uniform(-1, 1, (60, 2))
        xy = np.concatenate([base, tight])
    q = W.strengths(1, xy.shape[0], 2, salt=11)
    yd = direct.direct_apply(med, xy, q)
    plan = Plan(xy, med, tol=1e-10, leaf_size=8, max_rhs=2, adaptive=True)
    inf = plan.info
    # host buffers (staged through the plan's device buffers)
    y = plan.apply(q)
    plan.close()
    if case == "depth-cap":
        assert inf["levels"] == 16
    assert direct.rel_l2(y, yd) < 1e-9, (case, direct.rel_l2(y, yd))


MIXED_TOL = 1e-5


@pytest.mark.parametrize("part", [1, 2, 4, 8])
@pytest.mark.parametrize("name", ["cfg2-clusters", "three-layer-near-interface", "star-curve"])
def test_adaptive_mixed_terms_match_cpu_fmm(name, part):
    """Mixed-precision adaptive plans (scaled FP32 expansions, plan-time FP32
    bases for P2M / L2P, M2P and P2L, FP32 near-field blocks): each term
    against the adaptive CPU FMM within 1e-5 of the full result."""
    F, parts = _oracle(name)
    med, xy, q, tol, leaf = _case(name)
    plan = Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=q.shape[0], adaptive=True, precision=MIXED)
    y = plan.apply(torch.from_numpy(q.astype(np.complex64)).cuda(), parts=part).cpu().numpy().astype(np.complex128)
    plan.close()
    full = sum(parts.values())
    err = np.linalg.norm(y - parts[part]) / np.linalg.norm(full)
    assert err < MIXED_TOL, (name, part, err)


def test_adaptive_mixed_matches_fp64_many_rhs_and_batch():
    """The star curve with 16 right-hand sides: mixed against FP64 adaptive
    per right-hand side within 1e-5, host buffers, the adjoint identity, and a
    batch of two mixed adaptive instances equal to their single plans."""
    med = W.WORKLOADS[8].medium
    xy = W.points(8, 3000)
    q = W.strengths(8, 3000, 16, salt=46)
    p64 = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=16, adaptive=True)
    y64 = p64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    p64.close()
    p32 = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=16, adaptive=True, precision=MIXED)
    q32 = q.astype(np.complex64)
    y32 = p32.apply(q32).astype(np.complex128)          # host buffers
    worst = max(direct.rel_l2(y32[r], y64[r]) for r in range(16))
    assert worst < MIXED_TOL, worst
    v = (W.strengths(8, 3000, 16, salt=47)).astype(np.complex64)
    Gq = p32.apply(q32).astype(np.complex128)
    GHv = p32.adjoint(v).astype(np.complex128)
    lhs, rhs = np.vdot(v.astype(np.complex128), Gq), np.vdot(GHv, q32.astype(np.complex128))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    p32.close()
    xy2 = W.points(8, 1200, salt=2)
    q2 = W.strengths(8, 1200, 16, salt=48).astype(np.complex64)
    b = Batch([xy, xy2], med, tol=1e-6, leaf_size=16, max_rhs=16, adaptive=True, precision=MIXED)
    ys = b.apply([torch.from_numpy(q32).cuda(), torch.from_numpy(q2).cuda()])
    b.close()
    for x_, q_, y_ in ((xy, q32, ys[0]), (xy2, q2, ys[1])):
        with Plan(x_, med, tol=1e-6, leaf_size=16, max_rhs=16, adaptive=True, precision=MIXED) as p1:
            assert np.array_equal(p1.apply(torch.from_numpy(q_).cuda()).cpu().numpy(), y_.cpu().numpy())


def test_adaptive_solve_and_layered_accuracy():
    """hfmm_solve with an adaptive plan as the operator: GMRES on (10 I + A) x
    = b for 1000 points of the star curve against numpy's dense solve of the
    oracle's matrix (FP64 to 1e-8, mixed to 1e-4); and the FP64 adaptive
    apply on a three-layer blob next to the interface against the direct sum
    at tol 1e-10."""
    med = W.WORKLOADS[8].medium
    xy = W.points(8, 1000)
    n = xy.shape[0]
    G = np.empty((n, n), dtype=complex)
    eye = np.eye(n, dtype=complex)
    for c0 in range(0, n, 250):
        G[:, c0:c0 + 250] = direct.direct_apply(med, xy, eye[c0:c0 + 250]).T
    b = W.strengths(8, n, 1, salt=49)[0]
    sigma = 10.0
    x_ref = np.linalg.solve(sigma * np.eye(n) + G, b)
    with Plan(xy, med, tol=1e-10, leaf_size=16, adaptive=True) as p64:
        x, it, rr = p64.solve(torch.from_numpy(b).cuda(), sigma=sigma, tol=1e-10, restart=100, maxit=600)
        assert rr <= 1e-10 and 0 < it <= 600
        assert direct.rel_l2(x.cpu().numpy(), x_ref) < 1e-8, direct.rel_l2(x.cpu().numpy(), x_ref)
    with Plan(xy, med, tol=1e-6, leaf_size=16, adaptive=True, precision=MIXED) as p32:
        x32, it32, rr32 = p32.solve(torch.from_numpy(b.astype(np.complex64)).cuda(), sigma=sigma, tol=1e-5,
                                    restart=100, maxit=600)
        assert rr32 <= 1e-5
        assert direct.rel_l2(x32.cpu().numpy().astype(np.complex128), x_ref) < 1e-4
    xy3 = _near_interface(900, 5)
    q3 = W.strengths(4, 900, 1, salt=50)
    yd = direct.direct_apply(CFG4_MED, xy3, q3)
    with Plan(xy3, CFG4_MED, tol=1e-10, leaf_size=12, adaptive=True) as p3:
        y3 = p3.apply(torch.from_numpy(q3).cuda()).cpu().numpy()
    assert direct.rel_l2(y3, yd) < 1e-10, direct.rel_l2(y3, yd)
