"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

* tree and interaction lists: bit-exact against the oracle's tree;
* expansion orders: equal integers;
* every term of the FP64 apply against the plain CPU FMM at equal p (1e-11,
  relative to the norm of the full result);
* whole apply against the O(N^2) direct sum within the FMM tolerance;
* the full-size workloads on sampled targets with sparse strengths.
"""
import math

import numpy as np
import pytest

import workloads as W
from workloads import Medium
from oracle import direct, fmm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1703_09136_gb300 import Plan, HfmmError  # noqa: E402
from paper_1703_09136_gb300 import build as _build  # noqa: E402

PARITY_TOL = 1e-11

CFG4_MED = W.WORKLOADS[4].medium
CFG3_MED = W.WORKLOADS[3].medium


def _case(name):
    """(medium, xy, q, tol, leaf, p) of a parity case."""
    if name == "cfg1":
        w = W.WORKLOADS[1]
        xy = W.points(1)
        return w.medium, xy, W.strengths(1, xy.shape[0], 2), 1e-6, 32, 0
    if name == "cfg2":
        w = W.WORKLOADS[2]
        xy = W.points(2)
        return w.medium, xy, W.strengths(2, xy.shape[0], 1), 1e-6, 32, 0
    if name == "cfg3-small":
        xy = W.points_in_box(3, 2048, ((0.0, 0.5), (0.02, 0.52)))
        return CFG3_MED, xy, W.strengths(3, 2048, 2), 1e-6, 16, 0
    if name == "cfg4-small":
        xy = W.points_in_box(4, 2048, ((0.0, 0.5), (0.02, 0.52)))
        return CFG4_MED, xy, W.strengths(4, 2048, 2), 1e-6, 16, 0
    raise KeyError(name)


CASES = ["cfg1", "cfg2", "cfg3-small", "cfg4-small"]
_cache = {}


def _oracle(name):
    if name not in _cache:
        med, xy, q, tol, leaf, p = _case(name)
        F = fmm.CpuFmm(xy, med, tol=tol, leaf_size=leaf, p=p)
        parts = {part: F.apply(q, parts=part) for part in (1, 2, 4, 8)}
        _cache[name] = (F, parts)
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _built():
    _build.build()


def _plan(name, **kw):
    med, xy, q, tol, leaf, p = _case(name)
    return Plan(xy, med, tol=tol, leaf_size=leaf, p=p, max_rhs=q.shape[0], **kw)


def _morton(ix, iy):
    out = np.zeros_like(ix, dtype=np.int64)
    for b in range(16):
        out |= ((ix >> b) & 1).astype(np.int64) << (2 * b)
        out |= ((iy >> b) & 1).astype(np.int64) << (2 * b + 1)
    return out


@pytest.mark.parametrize("name", CASES)
def test_tree_and_lists_match_oracle(name):
    F, _ = _oracle(name)
    t = F.tree
    plan = _plan(name)
    info = plan.info
    assert info["levels"] == t.L
    assert info["x0"] == t.x0 and info["y0"] == t.y0 and info["size"] == t.S
    perm, ix, iy = plan.tree()
    assert np.array_equal(ix, t.leaf_ix) and np.array_equal(iy, t.leaf_iy)
    want = np.lexsort((np.arange(len(ix)), _morton(t.leaf_ix, t.leaf_iy)))
    assert np.array_equal(perm, want)
    for l in range(t.L + 1):
        ne = t.nonempty(l)
        if l >= 2:
            v = {tuple(r) for r in plan.pairs(0, l)}
            v_or = {(T[0], T[1], S[0], S[1]) for T in ne for S in fmm.v_list(t, l, T, ne)}
            assert v == v_or, l
        r = {tuple(x) for x in plan.pairs(1, l)}
        assert r == {(T[0], T[1], S[0], S[1]) for T, S in F.R[l]}, l
    d = {tuple(x) for x in plan.pairs(2, t.L)}
    assert d == {(T[0], T[1], S[0], S[1]) for T, S in F.direct_pairs}
    u = {tuple(x) for x in plan.pairs(3, t.L)}
    assert u == {(T[0], T[1], S[0], S[1]) for T in t.leaves for S in fmm.u_list(t, T)}
    assert info["p"] == F.p
    plan.close()


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("part", [1, 2, 4, 8])
def test_fp64_terms_match_cpu_fmm(name, part):
    F, parts = _oracle(name)
    med, xy, q, tol, leaf, p = _case(name)
    full = sum(parts.values())
    plan = _plan(name)
    y = plan.apply(torch.from_numpy(q).cuda(), parts=part).cpu().numpy()
    err = np.linalg.norm(y - parts[part]) / np.linalg.norm(full)
    assert err < PARITY_TOL, (name, part, err)
    plan.close()


@pytest.mark.parametrize("name,tol", [("cfg1", 1e-6), ("cfg2", 1e-6), ("cfg2", 1e-10)])
def test_fp64_matches_direct_sum(name, tol):
    med, xy, q, _, leaf, p = _case(name)
    yd = direct.direct_apply(med, xy, q)
    plan = Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=q.shape[0])
    y = plan.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    assert direct.rel_l2(y, yd) < tol
    plan.close()


def test_adjoint_dot_product_and_conjugate_symmetry():
    med, xy, q, tol, leaf, p = _case("cfg1")
    rng = np.random.default_rng(11)
    v = rng.standard_normal(q.shape) + 1j * rng.standard_normal(q.shape)
    plan = _plan("cfg1")
    qd = torch.from_numpy(q).cuda()
    vd = torch.from_numpy(v).cuda()
    Gq = plan.apply(qd).cpu().numpy()
    GHv = plan.adjoint(vd).cpu().numpy()
    lhs = np.vdot(v, Gq)          # <v, G q>
    rhs = np.vdot(GHv, q)         # <G^H v, q>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    plan.close()


def test_multi_rhs_equals_single_rhs_and_host_pointers():
    med, xy, q1, tol, leaf, p = _case("cfg4-small")
    q = np.concatenate([q1, W.strengths(4, xy.shape[0], 2, salt=5)])
    plan = Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=q.shape[0])
    yall = plan.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    for r in range(q.shape[0]):
        yr = plan.apply(torch.from_numpy(q[r:r + 1].copy()).cuda()).cpu().numpy()
        assert np.max(np.abs(yr[0] - yall[r])) <= 1e-14 * np.max(np.abs(yall[r]))
    yh = plan.apply(q)            # numpy in/out: host pointers through the C ABI
    assert np.array_equal(yh, yall)
    plan.close()


@pytest.mark.parametrize("n", [1, 2, 3, 33])
def test_tiny_inputs_match_direct_sum(n):
    med = W.WORKLOADS[1].medium
    xy = W.points(1, n, salt=3)
    q = W.strengths(1, n, 1, salt=3)
    plan = Plan(xy, med, tol=1e-10, leaf_size=4)
    y = plan.apply(q)
    yd = direct.direct_apply(med, xy, q)
    assert direct.rel_l2(y, yd) < 1e-9
    plan.close()


@pytest.mark.parametrize("engine", ["small", "tensor"])
@pytest.mark.parametrize("n", [1, 2, 3, 33, 1000])
def test_tiny_and_ragged_inputs_on_the_mixed_path(n, engine):
    """Mixed precision on tiny and ragged inputs (leaves of 1..4 points, a
    ragged last tile, 3 right-hand sides) against the direct sum, on both
    mixed engines."""
    from paper_1703_09136_gb300 import MIXED
    med = W.WORKLOADS[4].medium
    xy = W.points_in_box(4, n, ((0.0, 0.5), (0.02, 0.52)), salt=3)
    q = W.strengths(4, n, 3, salt=3)
    plan = Plan(xy, med, tol=1e-6, leaf_size=4, max_rhs=3, precision=MIXED, small_rhs=0 if engine == "small" else -1)
    y = plan.apply(q.astype(np.complex64)).astype(np.complex128)
    assert plan.info["device_error"] == 0
    plan.close()
    yd = direct.direct_apply(med, xy, q)
    assert direct.rel_l2(y, yd) < MIXED_TOL, direct.rel_l2(y, yd)


def test_bounded_device_wait_gives_up_with_a_timeout_status():
    """The tensor-core kernels' bounded mbarrier wait: on a barrier that
    nothing completes it gives up after the given polls (HFMM_ERR_TIMEOUT,
    no fault); released, it completes.  A mixed plan with an explicit bound
    runs to completion with no device error."""
    from paper_1703_09136_gb300 import debug_wait_timeout, MIXED
    debug_wait_timeout(1000, arrive=True)
    with pytest.raises(HfmmError) as e:
        debug_wait_timeout(1000, arrive=False)
    assert e.value.status == 6
    med = W.WORKLOADS[5].medium
    xy = W.points(5, 3000)
    q = W.strengths(5, 3000, 4, salt=9).astype(np.complex64)
    plan = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=4, precision=MIXED, spin_limit=3_000_000, small_rhs=-1)
    ref = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=4, precision=MIXED, small_rhs=-1)
    assert np.array_equal(plan.apply(q), ref.apply(q))
    assert plan.info["device_error"] == 0
    # few leaf tiles: split steps, so the leaves' L2P runs on the SIMT kernel
    assert plan.info["leaf_l2p_fused"] == 0
    plan.close(); ref.close()


def test_device_side_input_errors():
    med = W.WORKLOADS[1].medium
    xy = W.points(1, 50)
    bad = xy.copy()
    bad[7, 1] = -0.01
    with pytest.raises(HfmmError) as e:
        Plan(bad, med)
    assert e.value.status == 1
    bad[7, 1] = float("nan")
    with pytest.raises(HfmmError):
        Plan(bad, med)
    plan = Plan(xy, med, max_rhs=1)
    with pytest.raises(HfmmError):
        plan.apply(np.zeros((2, 50), dtype=np.complex128))
    plan.close()


def _sparse_probe(cfg, n_src=1500, n_tgt=300):
    """Full-size point cloud, strengths on a random subset: the direct sum on
    sampled targets is cheap and the FMM still runs over the whole tree."""
    w = W.WORKLOADS[cfg]
    xy = W.points(cfg)
    n = xy.shape[0]
    src = W.sample_indices(cfg, n, n_src, salt=1)
    tgt = W.sample_indices(cfg, n, n_tgt, salt=2)
    q = np.zeros((1, n), dtype=np.complex128)
    q[0, src] = W.strengths(cfg, n_src, 1, salt=9)[0]
    self_index = np.where(np.isin(tgt, src), np.searchsorted(src, tgt), -1)
    yd = direct.free_sum(xy[tgt], xy[src], q[:, src], w.medium.k1, self_index=self_index)
    yd = yd + direct.reaction_sum(w.medium, xy[tgt], xy[src], q[:, src])
    return w, xy, q, tgt, yd


@pytest.mark.parametrize("cfg", [3, 4])
def test_full_size_workload_on_sampled_targets(cfg):
    w, xy, q, tgt, yd = _sparse_probe(cfg)
    plan = Plan(torch.from_numpy(xy).cuda(), w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=1)
    y = plan.apply(torch.from_numpy(q).cuda()).cpu().numpy()[:, tgt]
    err = direct.rel_l2(y, yd)
    assert err < w.tol, (cfg, err)
    plan.close()


def test_full_size_mixed_64_rhs_on_sampled_targets():
    """The benchmarked configuration itself (three layers, N = 1,048,576, 64
    right-hand sides, mixed precision with tensor cores on every level and the
    tensor-core near field) against the oracle's direct sum: every right-hand
    side has strengths on the same 1500 random sources (its own values), the
    300 sampled targets are compared element by element for all 64."""
    from paper_1703_09136_gb300 import MIXED
    cfg = 4
    w = W.WORKLOADS[cfg]
    xy = W.points(cfg)
    n = xy.shape[0]
    src = W.sample_indices(cfg, n, 1500, salt=4)
    tgt = W.sample_indices(cfg, n, 300, salt=5)
    qs = W.strengths(cfg, 1500, 64, salt=10)
    q = np.zeros((64, n), dtype=np.complex64)
    q[:, src] = qs.astype(np.complex64)
    qs = q[:, src].astype(np.complex128)
    self_index = np.where(np.isin(tgt, src), np.searchsorted(src, tgt), -1)
    yd = direct.free_sum(xy[tgt], xy[src], qs, w.medium.k1, self_index=self_index)
    yd = yd + direct.reaction_sum(w.medium, xy[tgt], xy[src], qs)
    plan = Plan(torch.from_numpy(xy).cuda(), w.medium, tol=w.tol, leaf_size=w.leaf, max_rhs=64, precision=MIXED)
    inf = plan.info
    assert inf["tensor_levels"] == inf["levels"] - inf["lmin"] + 1 and inf["leaf_l2p_fused"] == 1
    assert inf["near_tc_blocks"] > 0
    y = plan.apply(torch.from_numpy(q).cuda()).cpu().numpy()[:, tgt].astype(np.complex128)
    assert plan.info["device_error"] == 0
    plan.close()
    assert direct.rel_l2(y, yd) < MIXED_TOL, direct.rel_l2(y, yd)
    worst = max(direct.rel_l2(y[r], yd[r]) for r in range(64))
    assert worst < MIXED_TOL, worst


# --- adjoint against the oracle --------------------------------------------------

def _adjoint_case(name):
    if name == "cfg1":
        return W.WORKLOADS[1].medium, W.points(1)
    return CFG4_MED, W.points_in_box(4, 1200, ((0.0, 0.5), (0.02, 0.52)), salt=6)


_dense_cache = {}


def _dense_matrix(name):
    """G entry by entry from the oracle's direct sum (free H0 part plus the
    Sommerfeld-quadrature reaction, free self term dropped): column j is the
    direct sum of the unit strength e_j.  No symmetry is assumed."""
    if name not in _dense_cache:
        med, xy = _adjoint_case(name)
        n = xy.shape[0]
        _dense_cache[name] = direct.direct_apply(med, xy, np.eye(n, dtype=complex)).T
    return _dense_cache[name]


def _close(got, want, tol):
    """rel-l2 below tol, and every element within 10 tol of the largest entry."""
    got = np.asarray(got, dtype=np.complex128)
    e2 = direct.rel_l2(got, want)
    emax = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
    return e2 < tol and emax < 10 * tol, (e2, emax)


@pytest.mark.parametrize("name", ["cfg1", "cfg4-adjoint"])
def test_adjoint_matches_dense_oracle_matrix(name):
    """hfmm_apply_adjoint(v) against G^H v with G built densely from the oracle
    (Sec. 2.4: A_ij = u_{x_j}(x_i); G^H is formed explicitly, so a conjugation
    or transposition error in the adjoint cannot cancel): FP64 at tol 1e-10,
    mixed precision at tol 1e-6 within the mixed bound."""
    from paper_1703_09136_gb300 import MIXED
    med, xy = _adjoint_case(name)
    n = xy.shape[0]
    G = _dense_matrix(name)
    v = W.strengths(1, n, 2, salt=13)
    want = (G.conj().T @ v.T).T
    p64 = Plan(xy, med, tol=1e-10, leaf_size=16, max_rhs=2)
    ok, errs = _close(p64.adjoint(v), want, 1e-9)
    assert ok, ("fp64", errs)
    for sr in (0, -1):                         # warp-level and tensor-core engines
        p32 = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=2, precision=MIXED, small_rhs=sr)
        ok, errs = _close(p32.adjoint(v.astype(np.complex64)), want, MIXED_TOL)
        assert ok, ("mixed", sr, errs)
        p32.close()
    # the forward pass against the same matrix
    ok, errs = _close(p64.apply(v), (G @ v.T).T, 1e-9)
    assert ok, ("fp64 forward", errs)
    p64.close()


@pytest.mark.parametrize("name", ["cfg1", "cfg4-adjoint"])
def test_adjoint_matches_cpu_fmm_transposed(name):
    """The adjoint against the CPU FMM at equal p: conj(F conj v), which is
    F^H v because the CPU FMM's operator is symmetric (symmetric lists,
    transposition identities of its translations); FP64 per term 1e-11,
    mixed 1e-5."""
    from paper_1703_09136_gb300 import MIXED
    med, xy = _adjoint_case(name)
    n = xy.shape[0]
    v = W.strengths(1, n, 2, salt=14)
    F = fmm.CpuFmm(xy, med, tol=1e-6, leaf_size=16)
    want = np.conj(F.apply(np.conj(v)))
    p64 = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=2)
    got = p64.adjoint(v)
    assert direct.rel_l2(got, want) < PARITY_TOL, direct.rel_l2(got, want)
    p32 = Plan(xy, med, tol=1e-6, leaf_size=16, max_rhs=2, precision=MIXED)
    got32 = p32.adjoint(v.astype(np.complex64)).astype(np.complex128)
    assert direct.rel_l2(got32, want) < MIXED_TOL, direct.rel_l2(got32, want)
    p64.close(); p32.close()


# --- mixed precision ------------------------------------------------------------

MIXED_TOL = 1e-5


@pytest.mark.parametrize("engine", ["small", "tensor"])
@pytest.mark.parametrize("name", CASES)
def test_mixed_matches_fp64_and_oracle(name, engine):
    """FP32 expansions / near field with scaled FP32 translation matrices,
    on the warp-level few-RHS kernels and on the tensor-core passes: rel-l2
    against the FP64 GPU path and against the CPU FMM <= 1e-5, whole and per term."""
    from paper_1703_09136_gb300 import MIXED
    F, parts = _oracle(name)
    med, xy, q, tol, leaf, p = _case(name)
    full = sum(parts.values())
    sr = 0 if engine == "small" else -1
    plan = Plan(xy, med, tol=tol, leaf_size=leaf, p=p, max_rhs=q.shape[0], precision=MIXED, small_rhs=sr)
    y32 = plan.apply(torch.from_numpy(q.astype(np.complex64)).cuda()).cpu().numpy()
    plan.close()
    assert direct.rel_l2(y32, full) < MIXED_TOL, direct.rel_l2(y32, full)
    for part in (1, 2, 4, 8):
        plan = Plan(xy, med, tol=tol, leaf_size=leaf, p=p, max_rhs=q.shape[0], precision=MIXED, small_rhs=sr)
        yp = plan.apply(torch.from_numpy(q.astype(np.complex64)).cuda(), parts=part).cpu().numpy()
        plan.close()
        err = np.linalg.norm(yp - parts[part]) / np.linalg.norm(full)
        assert err < MIXED_TOL, (part, err)


def test_mixed_many_rhs_and_adjoint():
    from paper_1703_09136_gb300 import MIXED
    med, xy, q1, tol, leaf, p = _case("cfg4-small")
    nrhs = 70                      # more than one 64-wide right-hand-side pass
    q = W.strengths(4, xy.shape[0], nrhs, salt=8)
    plan64 = Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=nrhs)
    plan32 = Plan(xy, med, tol=tol, leaf_size=leaf, max_rhs=nrhs, precision=MIXED)
    y64 = plan64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    y32 = plan32.apply(torch.from_numpy(q.astype(np.complex64)).cuda()).cpu().numpy()
    assert direct.rel_l2(y32, y64) < MIXED_TOL
    v = W.strengths(4, xy.shape[0], nrhs, salt=9).astype(np.complex64)
    w32 = plan32.adjoint(torch.from_numpy(v).cuda()).cpu().numpy()
    lhs = np.vdot(v.astype(np.complex128), y32.astype(np.complex128))
    rhs = np.vdot(w32.astype(np.complex128), q)
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    plan64.close()
    plan32.close()


def test_tensor_core_downward_pass_matches_simt_and_fp64():
    """tcgen05 3xF16 M2M and downward passes (every level, wide coarse
    levels in column blocks; the leaves' L2P in the downward epilogue)
    against the FP32 SIMT passes (same plan otherwise) and against the FP64
    path, 64 right-hand sides (one full M = 128 tile of two target boxes)."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 8192, ((0.0, 1.0), (0.02, 1.02)))
    q = W.strengths(4, 8192, 64, salt=3)
    q32 = torch.from_numpy(q.astype(np.complex64)).cuda()
    tc = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=64, precision=MIXED)
    si = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=64, precision=MIXED, simt_m2l=True)
    f64 = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=4)
    assert tc.info["tensor_levels"] == tc.info["levels"] - tc.info["lmin"] + 1
    assert si.info["tensor_levels"] == 0
    assert tc.info["leaf_l2p_fused"] == 1 and si.info["leaf_l2p_fused"] == 0
    y_tc = tc.apply(q32).cpu().numpy()
    y_si = si.apply(q32).cpu().numpy()
    y64 = f64.apply(torch.from_numpy(q[:4].copy()).cuda()).cpu().numpy()
    assert tc.info["device_error"] == 0
    e_tc = direct.rel_l2(y_tc[:4], y64)
    e_si = direct.rel_l2(y_si[:4], y64)
    assert e_tc < MIXED_TOL and e_si < MIXED_TOL, (e_tc, e_si)
    # 3xF16 drops the lo*lo term and truncates inside TMEM between drains:
    # a little above the SIMT FP32 error, never far above it
    assert e_tc < 2.5 * e_si, (e_tc, e_si)
    assert direct.rel_l2(y_tc, y_si) < 2.0 * (e_tc + e_si)
    for p in (tc, si, f64):
        p.close()


def test_profile_plan_reports_stage_and_leaf_kernel_times():
    """Profile plans: per-stage event times of the last apply, and the
    leaf-level tensor-core downward launch's own time and algorithmic flops
    (the downward stage's flops minus the other levels', plus the L2P)."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 8192, ((0.0, 1.0), (0.02, 1.02)))
    q = torch.from_numpy(W.strengths(4, 8192, 64, salt=6).astype(np.complex64)).cuda()
    plan = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=64, precision=MIXED, profile=True)
    plan.apply(q)
    st = plan.stage_times()
    ms, fl = plan.leaf_down_time()
    inf = plan.info
    assert st["down"] > 0.0 and st["p2p"] > 0.0 and st["gather"] > 0.0
    assert 0.0 < ms <= st["down"]
    assert inf["leaf_l2p_fused"] == 1 and inf["leaf_tc_width"] % 16 == 0
    # leaf flops: part of the downward stage's count plus the L2P (8 nrhs (2p+1) per point)
    l2p = 8.0 * 64 * 8192 * (2 * inf["p"][inf["levels"]] + 1)
    assert 0.0 < fl - l2p < inf["flops_last_apply"]["down"] - l2p
    # a plan without profiling refuses
    plain = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=64, precision=MIXED)
    with pytest.raises(HfmmError):
        plain.leaf_down_time()
    plan.close(); plain.close()


def test_level_wide_scales_with_spread_and_spiked_right_hand_sides():
    """The leaves and the level above them carry one f16 exponent per
    right-hand side (from the bound 2 max|q_r| sum|B|) so that a tile's free
    and reaction steps accumulate in TMEM: right-hand sides scaled from 1e-20
    to 1e20, an all-zero one and ones with a single strength 1e6 times the
    rest (a bound far above most leaves' multipoles) against the FP64 path,
    right-hand side by right-hand side."""
    from paper_1703_09136_gb300 import MIXED
    n, nrhs = 16384, 64
    xy = W.points_in_box(4, n, ((0.0, 1.0), (0.02, 1.02)), salt=41)
    q = W.strengths(4, n, nrhs, salt=42)
    q *= (10.0 ** np.linspace(-20, 20, nrhs))[:, None]
    q[7] = 0.0
    rng = np.random.default_rng(43)
    for r in (11, 40):
        q[r, rng.integers(n)] *= 1e6
    mp = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=nrhs, precision=MIXED)
    f64 = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=nrhs)
    assert mp.info["tensor_levels"] > 0 and mp.info["tc_run_levels"] == 2
    y = mp.apply(torch.from_numpy(q.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
    ref = f64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    assert not np.any(y[7])
    for r in range(nrhs):
        if r == 7:
            continue
        assert np.all(np.isfinite(y[r])), r
        assert direct.rel_l2(y[r], ref[r]) < MIXED_TOL, (r, direct.rel_l2(y[r], ref[r]))
    mp.close()
    f64.close()


def test_tensor_core_ragged_rhs_blocks_and_changing_width():
    """Two 64-row right-hand-side blocks with a ragged second block (70 RHS),
    then a narrower apply (5 RHS) on the same plan: every column agrees with
    the FP64 path, so rows beyond nrhs never leak into the next apply."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 6000, ((0.0, 1.0), (0.02, 1.02)))
    tc = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=70, precision=MIXED)
    f64 = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=70)
    assert tc.info["tensor_levels"] == tc.info["levels"] - tc.info["lmin"] + 1
    for nrhs, salt in ((70, 11), (5, 12), (70, 13)):
        q = W.strengths(4, 6000, nrhs, salt=salt)
        y_tc = tc.apply(torch.from_numpy(q.astype(np.complex64)).cuda()).cpu().numpy()
        y64 = f64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
        for r in range(nrhs):
            assert direct.rel_l2(y_tc[r], y64[r]) < MIXED_TOL, (nrhs, r)
    assert tc.info["device_error"] == 0
    tc.close()
    f64.close()


def test_autotune_keeps_fastest_depth_and_same_result():
    """HFMM_FLAG_AUTOTUNE tries the leaf levels around the leaf_size choice,
    keeps the fastest, and the kept plan gives the result of a plan built
    with that depth directly."""
    med = W.WORKLOADS[2].medium
    xy = W.points(2, 20000)
    q = torch.from_numpy(W.strengths(2, 20000, 2)).cuda()
    tuned = Plan(xy, med, tol=1e-6, leaf_size=32, max_rhs=2, autotune=True)
    inf = tuned.info
    tried = inf["tune"]
    assert len(tried) >= 2 and all(ms > 0 for ms in tried.values())
    assert inf["levels"] == min(tried, key=tried.get)
    fixed = Plan(xy, med, tol=1e-6, levels=inf["levels"], max_rhs=2)
    y_t = tuned.apply(q)
    y_f = fixed.apply(q)
    assert torch.equal(y_t, y_f)
    tuned.close()
    fixed.close()


def test_near_field_tensor_blocks_and_simt_fallback():
    """Clustered points: the tensor-core near field (precomputed tiles) and
    the SIMT kernel for blocks wider than 128 padded targets both run, and
    every term matches the FP64 path."""
    from paper_1703_09136_gb300 import MIXED
    med = W.WORKLOADS[2].medium
    xy = W.points(2, 6400)
    q = W.strengths(2, 6400, 2)
    tc = Plan(xy, med, tol=1e-6, leaf_size=24, max_rhs=2, precision=MIXED, small_rhs=-1)
    f64 = Plan(xy, med, tol=1e-6, leaf_size=24, max_rhs=2)
    inf = tc.info
    assert inf["near_tc_blocks"] > 0 and inf["near_simt_leaves"] > 0, inf
    full = f64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    for part in (1, 2, 4, 8, 15):
        a = tc.apply(torch.from_numpy(q.astype(np.complex64)).cuda(), parts=part).cpu().numpy()
        b = f64.apply(torch.from_numpy(q).cuda(), parts=part).cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(full) < MIXED_TOL, part
    tc.close()
    f64.close()


def test_page_locked_host_buffers_match_device_buffers():
    """Page-locked host q / y (used in place by the permutation kernels) give
    the device-buffer result, FP64 and mixed; pageable host buffers too."""
    from paper_1703_09136_gb300 import MIXED
    med = W.WORKLOADS[2].medium
    xy = W.points(2, 5000)
    q = W.strengths(2, 5000, 3)
    for prec, cdt in ((0, torch.complex128), (MIXED, torch.complex64)):
        plan = Plan(xy, med, tol=1e-6, max_rhs=3, precision=prec)
        qd = torch.from_numpy(q).to(cdt).cuda()
        yd = plan.apply(qd).cpu()
        qh = torch.from_numpy(q).to(cdt).pin_memory()
        yh = torch.empty_like(qh).pin_memory()
        plan.apply(qh, out=yh)
        assert torch.equal(yh, yd)
        yp = plan.apply(torch.from_numpy(q).to(cdt))
        assert torch.equal(yp, yd)
        plan.close()


# --- gradients ---------------------------------------------------------------------

def test_position_gradient_matches_oracle_direct_sum_gradient():
    med = W.WORKLOADS[1].medium
    xy = W.points(1, 400)
    q = W.strengths(1, 400, 2, salt=1)
    y_obs = direct.direct_apply(med, W.perturb(1, xy), q)
    plan = Plan(xy, med, tol=1e-10, leaf_size=16, max_rhs=2)
    y = plan.apply(q)
    g = 2.0 * (y - y_obs)
    got = plan.grad(q, g)
    want = direct.position_grad(med, xy, q, g)
    assert np.linalg.norm(got - want) < 1e-8 * np.linalg.norm(want)
    plan.close()


def test_mixed_plan_position_gradient_runs_the_fp64_tree_pass():
    """A mixed plan's position gradient widens its complex64 q and g and runs
    the FP64 pass: it equals an FP64 plan's gradient of the same rounded
    inputs (same tree, same orders) and the oracle's direct-sum gradient."""
    from paper_1703_09136_gb300 import MIXED
    for wl in (1, 5):
        med = W.WORKLOADS[wl].medium
        n = 700
        xy = W.points(wl, n)
        q32 = W.strengths(wl, n, 3, salt=4).astype(np.complex64)
        g32 = W.strengths(wl, n, 3, salt=5).astype(np.complex64)
        p32 = Plan(xy, med, tol=1e-6, leaf_size=24, max_rhs=3, precision=MIXED)
        p64 = Plan(xy, med, tol=1e-6, leaf_size=24, max_rhs=3)
        got = p32.grad(q32, g32)
        ref = p64.grad(q32.astype(np.complex128), g32.astype(np.complex128))
        assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref), wl
        want = direct.position_grad(med, xy, q32.astype(np.complex128), g32.astype(np.complex128))
        assert np.linalg.norm(got - want) < 1e-4 * np.linalg.norm(want), wl
        gt = p32.grad(torch.from_numpy(q32).cuda(), torch.from_numpy(g32).cuda())
        assert torch.equal(gt.cpu(), torch.from_numpy(got)), wl
        p32.close(); p64.close()


def test_autograd_gradients_match_finite_differences():
    """torch.autograd through the C ABI (adjoint for strengths, field
    gradients for positions) against central differences, h = 1e-6."""
    from paper_1703_09136_gb300 import matvec
    med = W.WORKLOADS[5].medium
    xy0 = W.points(5, 300)
    q0 = W.strengths(5, 300, 1, salt=2)
    y_obs = torch.from_numpy(direct.direct_apply(med, W.perturb(5, xy0), q0)).cuda()
    xy = torch.from_numpy(xy0).cuda().requires_grad_(True)
    q = torch.from_numpy(q0).cuda().requires_grad_(True)
    opts = dict(tol=1e-12, leaf_size=16)
    loss = (matvec(xy, q, med, **opts) - y_obs).abs().pow(2).sum()
    loss.backward()
    def L(z, qq):
        with torch.no_grad():
            return float((matvec(z, qq, med, **opts) - y_obs).abs().pow(2).sum())
    h = 1e-6
    for j, d in ((3, 0), (3, 1), (150, 0), (299, 1)):
        zp = xy.detach().clone(); zp[j, d] += h
        zm = xy.detach().clone(); zm[j, d] -= h
        fd = (L(zp, q.detach()) - L(zm, q.detach())) / (2 * h)
        assert abs(fd - float(xy.grad[j, d])) < 1e-5 * max(1.0, abs(fd))
    for j in (0, 77):
        for part in (1.0, 1j):
            qp = q.detach().clone(); qp[0, j] += h * part
            qm = q.detach().clone(); qm[0, j] -= h * part
            fd = (L(xy.detach(), qp) - L(xy.detach(), qm)) / (2 * h)
            g = q.grad[0, j]
            want = float(g.real) if part == 1.0 else float(g.imag)
            assert abs(fd - want) < 1e-5 * max(1.0, abs(fd))


# --- batched uneven instances ------------------------------------------------------

def test_batch_graph_equals_individual_plans():
    """Uneven instances in one captured CUDA graph give exactly the results of
    their single-plan applies (FP64 and mixed), on the first (recording) call
    and on a replay."""
    from paper_1703_09136_gb300 import Batch, MIXED
    med = W.WORKLOADS[5].medium
    sizes = [3000, 700, 12000, 1500, 5000]
    xys = [W.points(5, n, salt=i) for i, n in enumerate(sizes)]
    for prec, cdt in ((0, torch.complex128), (MIXED, torch.complex64)):
        qs = [torch.from_numpy(W.strengths(5, n, 2, salt=i)).cuda().to(cdt) for i, n in enumerate(sizes)]
        batch = Batch(xys, med, leaf_size=32, precision=prec, max_rhs=2)
        ys = [torch.empty_like(q) for q in qs]
        for rep in range(2):
            for y in ys:
                y.zero_()
            batch.apply(qs, ys)
            torch.cuda.synchronize()
            for xy, q, y in zip(xys, qs, ys):
                single = Plan(xy, med, leaf_size=32, precision=prec, max_rhs=2)
                ref = single.apply(q)
                single.close()
                assert torch.equal(ref, y)
        # and against the oracle's direct sum (two instances)
        for i in (1, 3):
            yd = direct.direct_apply(med, xys[i], W.strengths(5, sizes[i], 2, salt=i))
            err = direct.rel_l2(ys[i].cpu().numpy().astype(np.complex128), yd)
            assert err < (1e-6 if prec == 0 else MIXED_TOL), (prec, i, err)
        batch.close()


def test_batch_graph_captures_the_concurrent_near_field():
    """An instance large enough for the fused leaf L2P runs its near field on
    a low-priority stream concurrently with the far-field chain; captured into
    the batch graph, that fork-join gives exactly the single-plan result."""
    from paper_1703_09136_gb300 import Batch, MIXED
    med = W.WORKLOADS[5].medium
    sizes = [60000, 2000]
    xys = [W.points(5, n, salt=10 + i) for i, n in enumerate(sizes)]
    qs = [torch.from_numpy(W.strengths(5, n, 4, salt=i)).cuda().to(torch.complex64) for i, n in enumerate(sizes)]
    singles = [Plan(xy, med, leaf_size=16, precision=MIXED, max_rhs=4, small_rhs=-1) for xy in xys]
    assert singles[0].info["leaf_l2p_fused"] == 1 and singles[1].info["leaf_l2p_fused"] == 0
    refs = [p.apply(q) for p, q in zip(singles, qs)]
    batch = Batch(xys, med, leaf_size=16, precision=MIXED, max_rhs=4, small_rhs=-1)
    ys = [torch.empty_like(q) for q in qs]
    for rep in range(3):
        for y in ys:
            y.zero_()
        batch.apply(qs, ys)
        torch.cuda.synchronize()
        for ref, y in zip(refs, ys):
            assert torch.equal(ref, y), rep
    batch.close()
    for p in singles:
        p.close()


# --- table quadrature convergence ----------------------------------------------

@pytest.mark.parametrize("name", ["cfg1", "cfg3-small", "cfg4-small", "near-interface", "small-alpha"])
def test_table_quadrature_is_checked_against_its_node_doubled_rule(name):
    """Every reaction table entry A_n (Eq. (eq:m2loperator)) and every directly
    summed G^s block is recomputed at plan time on the rule with twice the
    panels; the converged rules agree far below 1e-12 (weighted by what the
    normalised expansions reach), and rules coarsened through quad_scale are
    rejected with HFMM_ERR_NUMERICS instead of giving a silently worse result."""
    if name == "near-interface":
        med = CFG4_MED
        xy = W.points_in_box(4, 2048, ((0.0, 0.5), (0.002, 0.502)), salt=8)
        leaf = 16
    elif name == "small-alpha":
        med = Medium(W.IMPEDANCE, (20.0,), alpha=0.5)
        xy = W.points(1)
        leaf = 32
    else:
        med, xy, q, tol, leaf, p = _case(name)
    plan = Plan(xy, med, tol=1e-6, leaf_size=leaf)
    inf = plan.info
    assert 0.0 < inf["table_check"] < 1e-12, inf["table_check"]
    if name == "near-interface":
        assert inf["direct_leaf_pairs"] > 0
    plan.close()
    with pytest.raises(HfmmError) as e:
        Plan(xy, med, tol=1e-6, leaf_size=leaf, quad_scale=0.05)
    assert e.value.status == 5 and "node-doubled" in str(e.value)


def test_impedance_with_small_alpha_matches_direct_sum():
    """alpha / k = 0.025: the pole of sigma_hat at s1 = i alpha (Sec. 2.2)
    sits close to both quadrature paths of the tables and of the directly
    summed blocks; FP64 at tol 1e-10 against the oracle's direct sum."""
    med = Medium(W.IMPEDANCE, (20.0,), alpha=0.5)
    xy = W.points(1)
    q = W.strengths(1, xy.shape[0], 1, salt=15)
    plan = Plan(xy, med, tol=1e-10, leaf_size=32)
    assert plan.info["direct_leaf_pairs"] > 0
    y = plan.apply(q)
    plan.close()
    err = direct.rel_l2(y, direct.direct_apply(med, xy, q))
    assert err < 1e-10, err


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4, 7])
def test_small_rhs_engine_matches_tensor_engine_and_fp64(nrhs):
    """The warp-level kernels for few right-hand sides (default for nrhs <= 4,
    forced here up to 7: passes of 8, 4, 2, 1 right-hand sides and ragged
    passes) against the tensor-core engine and the FP64 path, right-hand
    side by right-hand side, on the three-layer medium with every level,
    the reaction lists and the fused near field involved."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 8192, ((0.0, 1.0), (0.02, 1.02)), salt=2)
    q = W.strengths(4, 8192, nrhs, salt=16)
    sm = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=nrhs, precision=MIXED, small_rhs=8)
    tc = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=nrhs, precision=MIXED, small_rhs=-1)
    f64 = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=nrhs)
    q32 = torch.from_numpy(q.astype(np.complex64)).cuda()
    y_sm = sm.apply(q32).cpu().numpy().astype(np.complex128)
    y_tc = tc.apply(q32).cpu().numpy().astype(np.complex128)
    y64 = f64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
    for r in range(nrhs):
        assert direct.rel_l2(y_sm[r], y64[r]) < MIXED_TOL, (r, direct.rel_l2(y_sm[r], y64[r]))
        assert direct.rel_l2(y_sm[r], y_tc[r]) < MIXED_TOL
    # deterministic: the same apply twice gives the same bits
    assert torch.equal(sm.apply(q32), sm.apply(q32))
    for p in (sm, tc, f64):
        p.close()


@pytest.mark.parametrize("p_fixed", [0, 18, 28])
def test_blocked_few_rhs_downward_pass_matches_fp64_per_part(p_fixed):
    """Few right-hand sides at a level of 4,096 boxes: L2L and the V lists run
    on the blocked kernel (32 target boxes per CTA sharing each staged
    matrix; 2, 3 and 4 output coefficients per lane for nc up to 32, 48, 64),
    the reaction lists on the per-box kernel added on top.  Each far-field
    part, the whole apply and the adjoint against the FP64 path at the same
    p, right-hand side by right-hand side; two applies give the same bits."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 65536, ((0.0, 1.0), (0.02, 1.02)), salt=31)
    nrhs = 2
    q = W.strengths(4, 65536, nrhs, salt=32)
    sm = Plan(xy, CFG4_MED, tol=1e-6, p=p_fixed, leaf_size=16, max_rhs=nrhs, precision=MIXED)
    f64 = Plan(xy, CFG4_MED, tol=1e-6, p=p_fixed, leaf_size=16, max_rhs=nrhs)
    info = sm.info
    assert info["levels"] == 6
    nc = 2 * info["p"][6] + 1
    lo, hi = {0: (1, 32), 18: (33, 48), 28: (49, 64)}[p_fixed]
    assert lo <= nc <= hi, nc
    q32 = torch.from_numpy(q.astype(np.complex64)).cuda()
    q64 = torch.from_numpy(q).cuda()
    full = f64.apply(q64).cpu().numpy()
    for part in (2, 4, 6, 15):
        y = sm.apply(q32, parts=part).cpu().numpy().astype(np.complex128)
        ref = f64.apply(q64, parts=part).cpu().numpy()
        for r in range(nrhs):
            err = np.linalg.norm(y[r] - ref[r]) / np.linalg.norm(full[r])
            assert err < MIXED_TOL, (part, r, err)
    ya = sm.adjoint(q32).cpu().numpy().astype(np.complex128)
    ra = f64.adjoint(q64).cpu().numpy()
    for r in range(nrhs):
        assert direct.rel_l2(ya[r], ra[r]) < MIXED_TOL
    assert torch.equal(sm.apply(q32), sm.apply(q32))
    sm.close()
    f64.close()


def test_persistent_batch_forward_and_adjoint_match_single_plans():
    """Uneven mixed-precision instances (1 and 3 right-hand sides) through the
    persistent batch kernel: every stage of every instance from one device
    work queue; forward and adjoint against single-plan applies and the FP64
    path, on the recording call and on a replay."""
    from paper_1703_09136_gb300 import Batch, MIXED
    med = W.WORKLOADS[5].medium
    sizes = [4100, 900, 30000, 1500, 12000, 60]
    xys = [W.points(5, n, salt=20 + i) for i, n in enumerate(sizes)]
    for nrhs in (1, 3):
        qs = [torch.from_numpy(W.strengths(5, n, nrhs, salt=i)).cuda().to(torch.complex64)
              for i, n in enumerate(sizes)]
        batch = Batch(xys, med, leaf_size=32, precision=MIXED, max_rhs=nrhs, persistent=True)
        singles = [Plan(xy, med, leaf_size=32, precision=MIXED, max_rhs=nrhs) for xy in xys]
        f64 = [Plan(xy, med, leaf_size=32, max_rhs=nrhs) for xy in xys]
        for adjoint in (False, True):
            ys = [torch.empty_like(q) for q in qs]
            for rep in range(2):
                for y in ys:
                    y.fill_(float("nan"))
                batch.apply(qs, ys, adjoint=adjoint)
                torch.cuda.synchronize()
                assert batch.device_error == 0
                for sp, p64, q, y in zip(singles, f64, qs, ys):
                    ref = sp.adjoint(q) if adjoint else sp.apply(q)
                    err = float(torch.linalg.norm(ref - y) / torch.linalg.norm(ref))
                    assert err < 1e-6, (nrhs, adjoint, rep, err)
                    q64 = q.to(torch.complex128)
                    r64 = p64.adjoint(q64) if adjoint else p64.apply(q64)
                    assert float(torch.linalg.norm(y.to(torch.complex128) - r64) / torch.linalg.norm(r64)) < MIXED_TOL
        batch.close()
        for p in singles + f64:
            p.close()


def test_persistent_batch_wait_limit_reports_instead_of_hanging():
    """Every dependency wait of the persistent batch kernel is bounded: with a
    one-poll limit, items that find their inputs unfinished give up, the batch
    reports a device error, and the kernel still finishes (no hang, no fault);
    with the default limit the same batch reports none."""
    from paper_1703_09136_gb300 import Batch, MIXED
    med = W.WORKLOADS[5].medium
    sizes = [40000, 30000, 20000, 10000]
    xys = [W.points(5, n, salt=30 + i) for i, n in enumerate(sizes)]
    qs = [torch.from_numpy(W.strengths(5, n, 1, salt=i)).cuda().to(torch.complex64) for i, n in enumerate(sizes)]
    ys = [torch.empty_like(q) for q in qs]
    tight = Batch(xys, med, leaf_size=32, precision=MIXED, max_rhs=1, spin_limit=1, persistent=True)
    tight.apply(qs, ys)
    tight.apply(qs, ys)
    assert tight.device_error == 1
    tight.close()
    ok = Batch(xys, med, leaf_size=32, precision=MIXED, max_rhs=1, persistent=True)
    ok.apply(qs, ys)
    ok.apply(qs, ys)
    assert ok.device_error == 0
    ok.close()


def test_low_frequency_deep_tree_with_the_papers_order():
    """The setting of the paper's timing table (Sec. 4: impedance alpha = 1,
    k = 0.1, p = 39) on a deep tree: the order is capped where the unscaled
    translation entries would leave the double range, both precisions stay
    finite and match the oracle's direct sum."""
    from paper_1703_09136_gb300 import MIXED
    med = Medium(W.IMPEDANCE, (0.1,), alpha=1.0)
    xy = W.points_in_box(6, 3000, ((-0.5, 0.5), (1.0, 2.0)))
    q = W.strengths(6, 3000, 1)
    yd = direct.direct_apply(med, xy, q)
    F = fmm.CpuFmm(xy, med, p=38, L=7)
    p64 = Plan(xy, med, p=38, levels=7)
    assert p64.info["p"] == F.p and min(F.p) < 39
    y64 = p64.apply(q)
    assert np.all(np.isfinite(y64)) and direct.rel_l2(y64, yd) < 1e-8, direct.rel_l2(y64, yd)
    p32 = Plan(xy, med, p=38, levels=7, precision=MIXED)
    y32 = p32.apply(q.astype(np.complex64)).astype(np.complex128)
    assert np.all(np.isfinite(y32)) and direct.rel_l2(y32, yd) < MIXED_TOL, direct.rel_l2(y32, yd)
    p64.close(); p32.close()


def test_batch_gradients_at_the_uneven_batch_spec():
    """Differentiation on an uneven impedance batch (k = 40, alpha = 20): loss
    L = sum_i |A_i(x_i) q_i - y_obs_i|^2 with y_obs_i from positions moved by
    N(0, (1e-3)^2); the strength gradient through the batch adjoint and the
    position gradient through hfmm_batch_apply_grad, FP64 against central
    differences (h = 1e-6) and both precisions against the oracle's
    direct-sum gradient on two instances (Sec. 2.4: A_ij = u_{x_j}(x_i))."""
    from paper_1703_09136_gb300 import Batch, MIXED
    med = W.WORKLOADS[5].medium
    sizes = [1500, 400, 2600, 800]
    xys = [W.points(5, n, salt=40 + i) for i, n in enumerate(sizes)]
    q_h = [W.strengths(5, n, 1, salt=40 + i) for i, n in enumerate(sizes)]
    y_obs = []
    for i, n in enumerate(sizes):
        p = Plan(W.perturb(5, xys[i], 1e-3, salt=i), med, tol=1e-12, leaf_size=32)
        y_obs.append(p.apply(q_h[i]))
        p.close()
    opts = dict(tol=1e-12, leaf_size=32)

    def loss_i(i, xy, q):
        p = Plan(xy, med, **opts)
        r = p.apply(q) - y_obs[i]
        p.close()
        return float(np.sum(np.abs(r) ** 2))

    grads = {}
    for prec, cdt, tol in ((0, torch.complex128, 1e-12), (MIXED, torch.complex64, 1e-6)):
        batch = Batch(xys, med, tol=tol, leaf_size=32, precision=prec, max_rhs=1)
        qs = [torch.from_numpy(q).to(cdt).cuda() for q in q_h]
        ys = batch.apply(qs)
        gs = [2.0 * (y - torch.from_numpy(yo).to(cdt).cuda()) for y, yo in zip(ys, y_obs)]
        gq = [t.cpu().numpy() for t in batch.apply(gs, adjoint=True)]
        gx = [t.cpu().numpy() for t in batch.grad(qs, gs)]
        torch.cuda.synchronize()
        grads[prec] = (gq, gx, [g.cpu().numpy().astype(np.complex128) for g in gs])
        batch.close()
    gq, gx, g64 = grads[0]
    h = 1e-6
    for i, j, d in ((0, 5, 0), (0, 1200, 1), (2, 77, 0), (3, 0, 1)):
        zp = xys[i].copy(); zp[j, d] += h
        zm = xys[i].copy(); zm[j, d] -= h
        fd = (loss_i(i, zp, q_h[i]) - loss_i(i, zm, q_h[i])) / (2 * h)
        assert abs(fd - gx[i][j, d]) < 1e-5 * max(1.0, abs(fd)), (i, j, d, fd, gx[i][j, d])
    for i, j in ((1, 3), (2, 2000)):
        for part in (1.0, 1j):
            qp = q_h[i].copy(); qp[0, j] += h * part
            qm = q_h[i].copy(); qm[0, j] -= h * part
            fd = (loss_i(i, xys[i], qp) - loss_i(i, xys[i], qm)) / (2 * h)
            want = gq[i][0, j].real if part == 1.0 else gq[i][0, j].imag
            assert abs(fd - want) < 1e-5 * max(1.0, abs(fd)), (i, j, part)
    for i in (1, 3):
        ref = direct.position_grad(med, xys[i], q_h[i], g64[i])
        assert np.linalg.norm(gx[i] - ref) < 1e-8 * np.linalg.norm(ref), i
        gq32, gx32, g32 = grads[MIXED]
        ref32 = direct.position_grad(med, xys[i], q_h[i].astype(np.complex64).astype(np.complex128), g32[i])
        assert np.linalg.norm(gx32[i] - ref32) < 1e-4 * np.linalg.norm(ref32), i
        assert np.linalg.norm(gq32[i] - gq[i]) < 1e-4 * np.linalg.norm(gq[i]), i


def test_autotune_picks_the_engine_crossover_for_mixed_plans():
    """A mixed autotuned plan also times the warp-level and the tensor-core
    engines at nrhs = 1, 2, 4, ... and keeps the crossover as small_rhs; its
    applies stay within the mixed bound of FP64 on both sides of it."""
    from paper_1703_09136_gb300 import MIXED
    xy = W.points_in_box(4, 30000, ((0.0, 2.0), (0.02, 2.02)), salt=3)
    tuned = Plan(xy, CFG4_MED, tol=1e-6, leaf_size=16, max_rhs=16, precision=MIXED, autotune=True)
    inf = tuned.info
    assert inf["small_rhs"] in (0, 1, 2, 4, 8, 16), inf["small_rhs"]
    f64 = Plan(xy, CFG4_MED, tol=1e-6, levels=inf["levels"], max_rhs=16)
    for nrhs in (1, 16):
        q = W.strengths(4, 30000, nrhs, salt=nrhs)
        y = tuned.apply(torch.from_numpy(q.astype(np.complex64)).cuda()).cpu().numpy().astype(np.complex128)
        y64 = f64.apply(torch.from_numpy(q).cuda()).cpu().numpy()
        assert direct.rel_l2(y, y64) < MIXED_TOL, (nrhs, direct.rel_l2(y, y64))
    tuned.close(); f64.close()


@pytest.mark.parametrize("sigma", [1.0, 10 + 5j])
def test_gmres_solve_matches_dense_oracle_solve(sigma):
    """hfmm_solve: restarted GMRES on (sigma I + A) x = b with the plan's apply
    as the operator (Sec. 2.4, the matrix of a discretised integral equation),
    against numpy's dense solve with A built entry by entry from the oracle
    (condition numbers 110 and 7.5); FP64 and mixed precision."""
    from paper_1703_09136_gb300 import MIXED
    med, xy = _adjoint_case("cfg1")
    n = xy.shape[0]
    G = _dense_matrix("cfg1")
    b = W.strengths(1, n, 1, salt=17)[0]
    x_ref = np.linalg.solve(sigma * np.eye(n) + G, b)
    p64 = Plan(xy, med, tol=1e-10, leaf_size=32)
    x, it, rr = p64.solve(torch.from_numpy(b).cuda(), sigma=sigma, tol=1e-10, restart=200, maxit=1500)
    assert rr <= 1e-10 and 0 < it <= 1500
    assert direct.rel_l2(x.cpu().numpy(), x_ref) < 1e-7, direct.rel_l2(x.cpu().numpy(), x_ref)
    p32 = Plan(xy, med, tol=1e-6, leaf_size=32, precision=MIXED)
    x32, it32, rr32 = p32.solve(torch.from_numpy(b.astype(np.complex64)).cuda(), sigma=sigma, tol=1e-5,
                                restart=200, maxit=1500)
    assert rr32 <= 1e-5
    err = direct.rel_l2(x32.cpu().numpy().astype(np.complex128), x_ref)
    assert err < (5e-4 if sigma == 1.0 else 1e-4), err
    with pytest.raises(HfmmError) as e:                # too few iterations: reported, not hidden
        p64.solve(torch.from_numpy(b).cuda(), sigma=sigma, tol=1e-12, restart=5, maxit=5)
    assert e.value.status == 5
    p64.close(); p32.close()


# ---------------------------------------------------------------------------
# Diagonal form of the FP64 translations (Sec. 3.3: the free and reaction
# operators depend on m - p only).  k = 400 on the unit box makes the level-2
# boxes ~70 wavelengths wide, where the plan keeps the circulant form.
# ---------------------------------------------------------------------------
HF_MED = Medium(W.IMPEDANCE, (400.0,), alpha=200.0)
_hf = {}


def _hf_case():
    if not _hf:
        xy = W.points_in_box(1, 2000, ((0.0, 1.0), (0.05, 1.05)), salt=7)
        q = W.strengths(1, 2000, 2, salt=7)
        F = fmm.CpuFmm(xy, HF_MED, tol=1e-6, leaf_size=32)
        _hf.update(xy=xy, q=q, parts={part: F.apply(q, parts=part) for part in (1, 2, 4, 8)})
    return _hf["xy"], _hf["q"], _hf["parts"]


@pytest.mark.parametrize("part", [2, 4])
def test_diagonal_translations_match_cpu_fmm(part):
    """Free (2) and reaction (4) far-field terms with level 2 (and any other
    level that passes the plan-time check) in diagonal form, against the CPU
    FMM's dense translations at equal p: 1e-11 relative to the full result."""
    xy, q, parts = _hf_case()
    plan = Plan(xy, HF_MED, tol=1e-6, leaf_size=32, max_rhs=2)
    inf = plan.info
    assert inf["diag_levels"] & (1 << 2), inf["diag_levels"]
    assert 0.0 <= inf["diag_check"] <= 1e-12
    y = plan.apply(torch.from_numpy(q).cuda(), parts=part).cpu().numpy()
    plan.close()
    full = sum(parts.values())
    err = np.linalg.norm(y - parts[part]) / np.linalg.norm(full)
    assert err < PARITY_TOL, (part, err)


def test_diagonal_translations_equal_dense_plan_forward_adjoint_gradient():
    """The same plan with HFMM_FLAG_DENSE_M2L: forward and adjoint agree to
    1e-12, position gradients to 1e-10; low-frequency plans keep every level
    dense (the check fails there)."""
    xy, q, _ = _hf_case()
    a = Plan(xy, HF_MED, tol=1e-6, leaf_size=32, max_rhs=2)
    b = Plan(xy, HF_MED, tol=1e-6, leaf_size=32, max_rhs=2, dense_m2l=True)
    assert a.info["diag_levels"] != 0 and b.info["diag_levels"] == 0
    qd = torch.from_numpy(q).cuda()
    ya, yb = a.apply(qd).cpu().numpy(), b.apply(qd).cpu().numpy()
    assert direct.rel_l2(ya, yb) < 1e-12, direct.rel_l2(ya, yb)
    wa, wb = a.adjoint(qd).cpu().numpy(), b.adjoint(qd).cpu().numpy()
    assert direct.rel_l2(wa, wb) < 1e-12, direct.rel_l2(wa, wb)
    g = torch.from_numpy(W.strengths(1, xy.shape[0], 2, salt=8)).cuda()
    ga, gb = a.grad(qd, g).cpu().numpy(), b.grad(qd, g).cpu().numpy()
    assert np.linalg.norm(ga - gb) < 1e-10 * np.linalg.norm(gb)
    a.close()
    b.close()
    med, xy1, q1, tol, leaf, p = _case("cfg1")
    with Plan(xy1, med, tol=tol, leaf_size=leaf, max_rhs=2) as c:
        assert c.info["diag_levels"] == 0
