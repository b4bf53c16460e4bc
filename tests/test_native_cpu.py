"""Host-side checks of the native library (no GPU needed): it builds, loads,
exports every entry point of include/hfmm.h, rejects bad arguments before
touching the device, and its Bessel code agrees with SciPy (AMOS)."""
import ctypes
import os
import re

import numpy as np
import pytest
from scipy.special import hankel1, jv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_09136_gb300 import build, _native
    build.build()
    return _native.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "hfmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hfmm_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function(lib):
    from paper_1703_09136_gb300 import _native
    names = header_functions()
    assert len(names) >= 12
    assert sorted(_native.EXPORTS) == names
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(7):
        assert lib.hfmm_status_string(s)
    assert b"unknown" in lib.hfmm_status_string(99)


@pytest.mark.parametrize("x", [1e-4, 0.3, 2.404825557695773, 5.0, 9.7, 40.0, 250.0])
def test_bessel_sequences_match_scipy(lib, x):
    nmax = 50
    j = np.zeros(nmax + 1)
    h = np.zeros(2 * (nmax + 1))
    assert lib.hfmm_debug_bessel(x, nmax, j.ctypes.data_as(ctypes.c_void_p),
                                 h.ctypes.data_as(ctypes.c_void_p)) == 0
    n = np.arange(nmax + 1)
    jr = jv(n, x)
    ok = np.abs(jr) > 1e-250
    # relative to the larger of |J_n| and the local scale of the sequence
    scale = np.maximum(np.abs(jr), 1e-3 * np.max(np.abs(jr)))
    assert np.max(np.abs(j[ok] - jr[ok]) / scale[ok]) < 1e-12
    H = h[0::2] + 1j * h[1::2]
    hr = hankel1(n, x)
    fin = np.isfinite(hr)
    assert np.max(np.abs(H[fin] - hr[fin]) / np.abs(hr[fin])) < 1e-12


def test_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_1703_09136_gb300 import _native as N
    h = N.hfmm_plan_t()
    m = N.hfmm_medium()
    m.kind = 0
    m.k[0] = 20.0
    m.alpha = 10.0
    xy = np.array([[0.1, 0.2], [0.3, 0.4]])
    vp = ctypes.c_void_p
    p = xy.ctypes.data_as(vp)
    # n < 1
    assert lib.hfmm_plan_create(ctypes.byref(h), 0, p, ctypes.byref(m), None, None) == 1
    # null points
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, None, ctypes.byref(m), None, None) == 1
    # negative impedance is a real-axis pole of sigma: unsupported
    m.alpha = -1.0
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), None, None) == 2
    assert b"alpha" in lib.hfmm_last_error()
    m.alpha = 10.0
    m.k[0] = 0.0
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), None, None) == 2
    m.k[0] = 20.0
    m.kind = 2
    m.k[1], m.k[2], m.d = 80.0, 60.0, 0.0
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), None, None) == 2
    m.kind = 7
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), None, None) == 1
    # a negative bound on device waits
    m.kind = 0
    m.k[1], m.k[2], m.d = 0.0, 0.0, 0.0
    o = N.hfmm_options()
    lib.hfmm_options_default(ctypes.byref(o))
    o.spin_limit = -1
    assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), ctypes.byref(o), None) == 1
    assert b"spin_limit" in lib.hfmm_last_error()
    # a negative or non-finite quadrature panel scale
    o.spin_limit = 0
    for bad in (-0.5, float("nan"), 1e9):
        o.quad_scale = bad
        assert lib.hfmm_plan_create(ctypes.byref(h), 2, p, ctypes.byref(m), ctypes.byref(o), None) == 1
        assert b"quad_scale" in lib.hfmm_last_error()
    # apply on a null plan
    q = np.zeros(2, dtype=np.complex128)
    assert lib.hfmm_apply(None, 1, q.ctypes.data_as(vp), q.ctypes.data_as(vp), None) == 1
    # leaf-kernel timing of a null plan, a wait probe without polls
    ms, fl = ctypes.c_double(), ctypes.c_double()
    assert lib.hfmm_plan_get_leaf_down(None, ctypes.byref(ms), ctypes.byref(fl)) == 1
    assert lib.hfmm_debug_wait_timeout(0, 0) == 1
    assert b"spin" in lib.hfmm_last_error()
    assert lib.hfmm_plan_destroy(None) == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_1703_09136_gb300 import _native as N
    monkeypatch.setattr(N, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(N, "_lib", None)
    with pytest.raises(ImportError):
        N.lib()


def test_options_and_info_layout_match_the_header(lib):
    """The ctypes mirrors of hfmm_options and hfmm_plan_info end with the
    fields the header declares last (quad_scale, table_check), and
    hfmm_options_default leaves the quadrature scale at 0 (= 1)."""
    from paper_1703_09136_gb300 import _native as N
    text = open(os.path.join(ROOT, "include", "hfmm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for struct, cls in (("hfmm_options", N.hfmm_options), ("hfmm_plan_info", N.hfmm_plan_info)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        flat = []
        for decl in body.split(";"):
            words = decl.split()
            if len(words) < 2:
                continue
            names = " ".join(words[1:]).split(",")        # "x0, y0, size" on one line
            flat += [re.sub(r"\[.*\]", "", nm).strip() for nm in names]
        assert [f[0] for f in cls._fields_] == flat, struct
    o = N.hfmm_options()
    o.quad_scale = 5.0
    lib.hfmm_options_default(ctypes.byref(o))
    assert o.quad_scale == 0.0 and o.tol == 1e-6
