"""GB300 heterogeneous FMM for the 2-D layered-media Helmholtz equation.

Thin Python binding of the C ABI in include/hfmm.h: argument marshalling
only; every step of the computation runs in the native CUDA library
``libhfmm.so`` (built by ``paper_1703_09136_gb300.build``).  There is no
fallback: if the library is missing or fails to load, an ImportError is
raised on first use.

    from paper_1703_09136_gb300 import Plan, Medium
    plan = Plan(xy, Medium.three_layer(40, 80, 60, d=0.5), tol=1e-6, max_rhs=64)
    y = plan.apply(q)            # q: [nrhs, n] complex tensor or array
    w = plan.adjoint(v)          # A^H v
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _native as _n
from ._native import (HfmmError, PART_ALL, PART_FAR_FREE, PART_FAR_REACT, PART_NEAR_FREE,
                      PART_NEAR_REACT, FP64, MIXED, IMPEDANCE, TWO_LAYER, THREE_LAYER)

__all__ = ["Plan", "Medium", "HfmmError", "library", "PART_ALL", "PART_FAR_FREE",
           "PART_FAR_REACT", "PART_NEAR_FREE", "PART_NEAR_REACT", "FP64", "MIXED",
           "IMPEDANCE", "TWO_LAYER", "THREE_LAYER"]


def library():
    """The loaded ctypes handle of libhfmm.so (raises ImportError if absent)."""
    return _n.lib()


class Medium:
    """Medium description (see hfmm_medium in include/hfmm.h)."""

    def __init__(self, kind, k, d=0.0, alpha=0.0):
        self.kind = int(kind)
        k = list(k) + [0.0] * (3 - len(k))
        self.k = tuple(float(v) for v in k[:3])
        self.d = float(d)
        self.alpha = float(alpha)

    @classmethod
    def impedance(cls, k, alpha):
        return cls(IMPEDANCE, (k,), alpha=alpha)

    @classmethod
    def two_layer(cls, k1, k2):
        return cls(TWO_LAYER, (k1, k2))

    @classmethod
    def three_layer(cls, k1, k2, k3, d):
        return cls(THREE_LAYER, (k1, k2, k3), d=d)

    @classmethod
    def of(cls, m):
        if isinstance(m, cls):
            return m
        return cls(m.kind, tuple(m.k), getattr(m, "d", 0.0), getattr(m, "alpha", 0.0))

    def _c(self):
        c = _n.hfmm_medium()
        c.kind = self.kind
        for i in range(3):
            c.k[i] = self.k[i]
        c.d = self.d
        c.alpha = self.alpha
        return c


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _stream_handle(stream):
    if stream is None:
        torch = _torch()
        if torch is not None and torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(a):
    """(pointer, keepalive) of a contiguous numpy array or torch tensor."""
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a)
    return ctypes.c_void_p(a.ctypes.data), a


class Plan:
    """An H-FMM plan for fixed points: y = A q with A_ij = u_{x_j}(x_i)."""

    def __init__(self, xy, medium, tol=1e-6, p=0, leaf_size=32, levels=0, precision=FP64,
                 max_rhs=1, stream=None, profile=False, simt_m2l=False, autotune=False, spin_limit=0,
                 quad_scale=0.0, small_rhs=0, dense_m2l=False, adaptive=False):
        lib = _n.lib()
        m = Medium.of(medium)
        opts = _n.hfmm_options()
        lib.hfmm_options_default(ctypes.byref(opts))
        opts.tol = float(tol)
        opts.p = int(p)
        opts.leaf_size = int(leaf_size)
        opts.levels = int(levels)
        opts.precision = int(precision)
        opts.max_rhs = int(max_rhs)
        opts.flags = ((_n.FLAG_PROFILE if profile else 0) | (_n.FLAG_SIMT_M2L if simt_m2l else 0) |
                      (_n.FLAG_AUTOTUNE if autotune else 0) | (_n.FLAG_DENSE_M2L if dense_m2l else 0) |
                      (_n.FLAG_ADAPTIVE if adaptive else 0))
        opts.spin_limit = int(spin_limit)
        opts.quad_scale = float(quad_scale)
        opts.small_rhs = int(small_rhs)
        torch = _torch()
        if torch is not None and isinstance(xy, torch.Tensor):
            if xy.dtype != torch.float64:
                raise ValueError("xy must be float64")
            xy = xy.contiguous()
            n = xy.shape[0]
        else:
            xy = np.ascontiguousarray(xy, dtype=np.float64)
            n = xy.shape[0]
        if xy.shape[-1] != 2:
            raise ValueError("xy must have shape [n, 2]")
        ptr, keep = _ptr(xy)
        h = _n.hfmm_plan_t()
        _n.check(lib.hfmm_plan_create(ctypes.byref(h), ctypes.c_int64(n), ptr, ctypes.byref(m._c()),
                                      ctypes.byref(opts), _stream_handle(stream)))
        del keep
        self._h = h
        self.n = int(n)
        self.medium = m
        self.precision = int(precision)
        self.max_rhs = int(max_rhs)

    # ------------------------------------------------------------------
    def _complex_dtype(self):
        return np.complex128 if self.precision == FP64 else np.complex64

    def _run(self, fn, q, out, stream, *extra):
        torch = _torch()
        is_t = torch is not None and isinstance(q, torch.Tensor)
        want = self._complex_dtype()
        if is_t:
            tdt = torch.complex128 if want == np.complex128 else torch.complex64
            if q.dtype != tdt:
                raise ValueError(f"q must be {tdt}")
            q = q.contiguous()
            shape = q.shape
            if out is None:
                out = torch.empty_like(q)
        else:
            q = np.ascontiguousarray(q)
            if q.dtype != want:
                raise ValueError(f"q must be {np.dtype(want)}")
            shape = q.shape
            if out is None:
                out = np.empty_like(q)
        if shape[-1] != self.n:
            raise ValueError(f"last dimension must be n = {self.n}")
        nrhs = 1 if len(shape) == 1 else int(np.prod(shape[:-1]))
        qp, kq = _ptr(q)
        yp, ky = _ptr(out)
        _n.check(fn(self._h, ctypes.c_int32(nrhs), qp, yp, *extra, _stream_handle(stream)))
        if not is_t and ky is not out:
            out[...] = ky
        return out

    def apply(self, q, out=None, stream=None, parts=PART_ALL):
        """y = A q (parts: sum of PART_* flags selects terms)."""
        lib = _n.lib()
        if parts == PART_ALL:
            return self._run(lib.hfmm_apply, q, out, stream)
        return self._run(lib.hfmm_apply_parts, q, out, stream, ctypes.c_int32(parts))

    def adjoint(self, v, out=None, stream=None):
        """w = A^H v."""
        return self._run(_n.lib().hfmm_apply_adjoint, v, out, stream)

    def grad(self, q, g, out=None, stream=None):
        """dL/dx_j, dL/dy_j ([n, 2] float64) of a real loss of y = A q, given
        g = dL/dRe(y) + i dL/dIm(y) (hfmm_apply_grad)."""
        torch = _torch()
        is_t = torch is not None and isinstance(q, torch.Tensor)
        want = self._complex_dtype()
        if is_t:
            tdt = torch.complex128 if want == np.complex128 else torch.complex64
            if q.dtype != tdt:
                raise ValueError(f"q must be {tdt}")
            q = q.contiguous()
            g = g.contiguous().to(q.dtype)
            if out is None:
                out = torch.empty((self.n, 2), dtype=torch.float64, device=q.device)
        else:
            q = np.ascontiguousarray(q, dtype=want)
            g = np.ascontiguousarray(g, dtype=want)
            if out is None:
                out = np.empty((self.n, 2), dtype=np.float64)
        nrhs = 1 if q.ndim == 1 else int(np.prod(q.shape[:-1]))
        qp, kq = _ptr(q)
        gp, kg = _ptr(g)
        op, ko = _ptr(out)
        _n.check(_n.lib().hfmm_apply_grad(self._h, ctypes.c_int32(nrhs), qp, gp, op, _stream_handle(stream)))
        return out

    def solve(self, b, sigma=1.0, x0=None, tol=1e-8, restart=50, maxit=1000, stream=None):
        """x with (sigma I + A) x = b by restarted GMRES (hfmm_solve); b a
        device tensor of n complex values.  Returns (x, iterations, relative
        residual); raises HfmmError (HFMM_ERR_NUMERICS) if tol is not reached."""
        torch = _torch()
        b = b.contiguous().reshape(-1)
        x = torch.zeros_like(b) if x0 is None else x0.clone().contiguous().reshape(-1)
        sg = (ctypes.c_double * 2)(complex(sigma).real, complex(sigma).imag)
        it = ctypes.c_int32(0)
        rr = ctypes.c_double(0.0)
        _n.check(_n.lib().hfmm_solve(self._h, sg, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_double(tol), ctypes.c_int32(restart), ctypes.c_int32(maxit),
                                     ctypes.byref(it), ctypes.byref(rr), _stream_handle(stream)))
        return x, int(it.value), float(rr.value)

    # ------------------------------------------------------------------
    @property
    def info(self):
        inf = _n.hfmm_plan_info()
        _n.check(_n.lib().hfmm_plan_get_info(self._h, ctypes.byref(inf)))
        d = {name: getattr(inf, name) for name, _ in inf._fields_
             if name not in ("p", "flops_last_apply", "bytes_last_apply", "tune_levels", "tune_ms")}
        d["tune"] = {int(inf.tune_levels[c]): float(inf.tune_ms[c]) for c in range(3) if inf.tune_levels[c]}
        d["p"] = [inf.p[l] for l in range(inf.levels + 1)]
        d["flops_last_apply"] = dict(zip(_n.STAGES, list(inf.flops_last_apply)))
        d["bytes_last_apply"] = dict(zip(_n.STAGES, list(inf.bytes_last_apply)))
        return d

    def leaf_down_time(self):
        """(ms, flops) of the leaf-level tensor-core downward launch of the last
        apply (profile plans, hfmm_plan_get_leaf_down)."""
        ms, fl = ctypes.c_double(), ctypes.c_double()
        _n.check(_n.lib().hfmm_plan_get_leaf_down(self._h, ctypes.byref(ms), ctypes.byref(fl)))
        return float(ms.value), float(fl.value)

    def stage_times(self):
        """Per-stage milliseconds of the last apply (plan built with profile=True)."""
        ms = (ctypes.c_double * _n.NUM_STAGES)()
        _n.check(_n.lib().hfmm_plan_get_stage_times(self._h, ms))
        return dict(zip(_n.STAGES, list(ms)))

    def tree(self):
        """(perm, leaf_ix, leaf_iy) as numpy arrays."""
        perm = np.empty(self.n, dtype=np.int64)
        ix = np.empty(self.n, dtype=np.int32)
        iy = np.empty(self.n, dtype=np.int32)
        _n.check(_n.lib().hfmm_plan_get_tree(self._h, perm.ctypes.data_as(ctypes.c_void_p),
                                             ix.ctypes.data_as(ctypes.c_void_p),
                                             iy.ctypes.data_as(ctypes.c_void_p)))
        return perm, ix, iy

    def pairs(self, kind, level):
        """Interaction pairs [(tx, ty, sx, sy)] of a level: kind 0 V list,
        1 reaction M2L, 2 direct reaction, 3 neighbouring leaves."""
        lib = _n.lib()
        cnt = ctypes.c_int64(0)
        st = lib.hfmm_plan_get_pairs(self._h, kind, level, None, ctypes.c_int64(0), ctypes.byref(cnt))
        if st not in (0, 1):
            _n.check(st)
        out = np.empty((max(cnt.value, 1), 4), dtype=np.int32)
        _n.check(lib.hfmm_plan_get_pairs(self._h, kind, level, out.ctypes.data_as(ctypes.c_void_p),
                                         ctypes.c_int64(cnt.value), ctypes.byref(cnt)))
        return out[:cnt.value]

    def perm(self):
        """perm[i] = caller index of the i-th point in the tree's sorted order."""
        perm = np.empty(self.n, dtype=np.int64)
        _n.check(_n.lib().hfmm_plan_get_tree(self._h, perm.ctypes.data_as(ctypes.c_void_p), None, None))
        return perm

    def boxes(self):
        """Adaptive plans: boxes [nbox, 6] int32 = (level, ix, iy, first sorted
        point, end, leaf) (hfmm_plan_get_boxes)."""
        lib = _n.lib()
        cnt = ctypes.c_int64(0)
        _n.check(lib.hfmm_plan_get_boxes(self._h, None, ctypes.c_int64(0), ctypes.byref(cnt)))
        out = np.empty((max(cnt.value, 1), 6), dtype=np.int32)
        _n.check(lib.hfmm_plan_get_boxes(self._h, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(cnt.value),
                                         ctypes.byref(cnt)))
        return out[:cnt.value]

    def lists(self, kind):
        """Adaptive plans: (target box, source box) index pairs [npairs, 2] of
        list kind 0 U, 1 V, 2 W, 3 X, 4 reaction M2L, 5 direct reaction."""
        lib = _n.lib()
        cnt = ctypes.c_int64(0)
        _n.check(lib.hfmm_plan_get_lists(self._h, kind, None, ctypes.c_int64(0), ctypes.byref(cnt)))
        out = np.empty((max(cnt.value, 1), 2), dtype=np.int32)
        _n.check(lib.hfmm_plan_get_lists(self._h, kind, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(cnt.value),
                                         ctypes.byref(cnt)))
        return out[:cnt.value]

    def close(self):
        if getattr(self, "_h", None):
            _n.lib().hfmm_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent problems of uneven sizes applied through one CUDA graph
    (hfmm_batch_*).  xys: list of [n_i, 2] float64 arrays / tensors.
    persistent=True runs mixed-precision applies with few right-hand sides as
    one persistent kernel over a device work queue."""

    def __init__(self, xys, medium, tol=1e-6, p=0, leaf_size=32, levels=0, precision=FP64, max_rhs=1,
                 stream=None, simt_m2l=False, spin_limit=0, small_rhs=0, persistent=False, adaptive=False):
        lib = _n.lib()
        m = Medium.of(medium)
        opts = _n.hfmm_options()
        lib.hfmm_options_default(ctypes.byref(opts))
        opts.tol, opts.p, opts.leaf_size, opts.levels = float(tol), int(p), int(leaf_size), int(levels)
        opts.precision, opts.max_rhs = int(precision), int(max_rhs)
        opts.small_rhs = int(small_rhs)
        opts.flags = ((_n.FLAG_SIMT_M2L if simt_m2l else 0) | (_n.FLAG_PERSISTENT if persistent else 0) |
                      (_n.FLAG_ADAPTIVE if adaptive else 0))
        opts.spin_limit = int(spin_limit)
        keep = [_ptr(np.ascontiguousarray(x, dtype=np.float64) if not hasattr(x, "data_ptr") else x.contiguous())
                for x in xys]
        ns = (ctypes.c_int64 * len(xys))(*[int(x.shape[0]) for x in xys])
        ptrs = (ctypes.c_void_p * len(xys))(*[k[0].value for k in keep])
        h = ctypes.c_void_p()
        _n.check(lib.hfmm_batch_create(ctypes.byref(h), len(xys), ns, ptrs, ctypes.byref(m._c()),
                                       ctypes.byref(opts), _stream_handle(stream)))
        self._h = h
        self.sizes = [int(x.shape[0]) for x in xys]
        self.precision = int(precision)

    def apply(self, qs, ys=None, adjoint=False, stream=None):
        """ys[i] = A_i qs[i] (device tensors [nrhs, n_i]); returns ys."""
        if ys is None:
            ys = [q.new_empty(q.shape) for q in qs]
        nrhs = 1 if qs[0].dim() == 1 else int(qs[0].shape[0])
        qp = (ctypes.c_void_p * len(qs))(*[q.data_ptr() for q in qs])
        yp = (ctypes.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        _n.check(_n.lib().hfmm_batch_apply(self._h, nrhs, qp, yp, 1 if adjoint else 0, _stream_handle(stream)))
        return ys

    def grad(self, qs, gs, outs=None, stream=None):
        """Position gradients [n_i, 2] (float64) of every instance for a real
        loss of y_i = A_i q_i, given g_i = dL/dRe(y_i) + i dL/dIm(y_i)
        (hfmm_batch_apply_grad); device tensors."""
        if outs is None:
            outs = [torch_empty2(q) for q in qs]
        nrhs = 1 if qs[0].dim() == 1 else int(qs[0].shape[0])
        gs = [g.contiguous().to(q.dtype) for g, q in zip(gs, qs)]
        qp = (ctypes.c_void_p * len(qs))(*[q.data_ptr() for q in qs])
        gp = (ctypes.c_void_p * len(gs))(*[g.data_ptr() for g in gs])
        op = (ctypes.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        _n.check(_n.lib().hfmm_batch_apply_grad(self._h, nrhs, qp, gp, op, _stream_handle(stream)))
        return outs

    @property
    def device_error(self):
        """Flag of the last persistent-kernel apply (a bounded wait gave up); synchronises."""
        e = ctypes.c_int32(0)
        _n.check(_n.lib().hfmm_batch_device_error(self._h, ctypes.byref(e)))
        return int(e.value)

    def close(self):
        if getattr(self, "_h", None):
            _n.lib().hfmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def torch_empty2(q):
    """[n, 2] float64 tensor on q's device for the gradient of q's points."""
    torch = _torch()
    return torch.empty((int(q.shape[-1]), 2), dtype=torch.float64, device=q.device)


def matvec(xy, q, medium, **plan_options):
    """Differentiable y = A(xy) q (torch tensors on one CUDA device).

    Builds a plan for the positions, applies it, and in backward returns
    A^H g for q (hfmm_apply_adjoint) and the position gradient of
    hfmm_apply_grad for xy.  Both precisions support both gradients (the
    position gradient of a mixed plan is computed in FP64 from its complex64
    q and g); plan_options are passed to Plan (tol, leaf_size, ...)."""
    return _MatvecFn.apply(xy, q, medium, plan_options)


def _make_fn():
    torch = _torch()
    if torch is None:  # pragma: no cover
        return None

    class MatvecFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, xy, q, medium, opts):
            nrhs = 1 if q.dim() == 1 else int(np.prod(q.shape[:-1]))
            plan = Plan(xy.detach().contiguous(), medium, max_rhs=max(nrhs, 1), **opts)
            y = plan.apply(q.detach().contiguous())
            ctx.plan = plan
            ctx.save_for_backward(q.detach())
            return y

        @staticmethod
        def backward(ctx, gy):
            (q,) = ctx.saved_tensors
            plan = ctx.plan
            gy = gy.contiguous()
            gq = plan.adjoint(gy) if ctx.needs_input_grad[1] else None
            gxy = plan.grad(q, gy) if ctx.needs_input_grad[0] else None
            plan.close()
            return gxy, gq, None, None

    return MatvecFn


_MatvecFn = _make_fn()


def debug_wait_timeout(spin, arrive):
    """One bounded device wait of at most `spin` polls on a barrier that
    completes only when `arrive` (hfmm_debug_wait_timeout): raises HfmmError
    (HFMM_ERR_TIMEOUT) when the wait gave up."""
    _n.check(_n.lib().hfmm_debug_wait_timeout(ctypes.c_int64(int(spin)), ctypes.c_int32(1 if arrive else 0)))
