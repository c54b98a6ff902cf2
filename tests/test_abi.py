"""The C-ABI library loads, exports every symbol `include/rt.h` declares, and rejects invalid
arguments on the host (no GPU needed: validation precedes any CUDA call)."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(rt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    from paper_2509_03623_b300 import _rt, build
    build.build()
    return _rt.lib()


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "rt_render" in names and "rt_last_error" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_version(L):
    from paper_2509_03623_b300 import _rt
    assert "sm_103a" in _rt.version()


def _structs(**over):
    from paper_2509_03623_b300 import _rt
    v = np.linspace(-4, 4, 16).astype(np.float32)
    g = _rt.rt_grid(64, 32, 1, 10.0, 600.0, 0.5)
    f = _rt.rt_fields(16, 16, 16, 16, 16, 1e-4, 0.01, 0)  # dummy device pointers
    o = _rt.rt_geom(45.0, 0.0, 100.0, 2.0, 0.0)
    vw = _rt.rt_view(64, 64, 0.0, 16, v.ctypes.data_as(C.POINTER(C.c_float)), 128, 0.0, 0)
    ln = _rt.rt_line(230.538e9, 7.16e-7, 0.0, 28.0101, 2.388, 2)
    objs = dict(g=g, f=f, o=o, vw=vw, ln=ln)
    for k, val in over.items():
        obj, field = k.split("__")
        setattr(objs[obj], field, val)
    return g, f, o, vw, ln, v


@pytest.mark.parametrize("over", [
    dict(g__nr=1), dict(g__nz=0), dict(g__r_in_au=0.0), dict(g__r_out_au=5.0),
    dict(g__zr_max=-1.0), dict(f__T_K=0), dict(f__edge_w=-0.1), dict(f__x_co=float("nan")),
    dict(o__incl_deg=float("inf")), dict(o__mstar_msun=-1.0), dict(vw__nx=-3),
    dict(vw__nch=257), dict(vw__n_samples=0), dict(vw__n_samples=(1 << 20) + 1),
    dict(vw__units=2), dict(ln__J_u=0), dict(ln__nu0_hz=0.0), dict(ln__m_co_amu=0.0),
])
def test_invalid_arguments_rejected(L, over):
    g, f, o, vw, ln, keep = _structs(**over)
    rc = L.rt_render(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                     C.c_void_p(16), None)
    assert rc == -1
    assert len(L.rt_last_error()) > 0


def test_null_structs_and_cube_rejected(L):
    g, f, o, vw, ln, keep = _structs()
    assert L.rt_render(None, C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                       C.c_void_p(16), None) == -1
    assert L.rt_render(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                       None, None) == -1
    assert b"cube" in L.rt_last_error()
    assert L.rt_count_gas_samples(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                  C.byref(ln), None, None) == -1


def test_empty_image_is_a_no_op(L):
    # nothing to render: returns RT_OK without touching the device
    g, f, o, vw, ln, keep = _structs(vw__nx=0)
    assert L.rt_render(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                       None, None) == 0
    g, f, o, vw, ln, keep = _structs(vw__nch=0)
    assert L.rt_render(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                       None, None) == 0


@pytest.mark.parametrize("over", [
    dict(nr=1), dict(nth=1), dict(nph=0), dict(r_in_au=-1.0), dict(r_out_au=5.0),
    dict(r_log=1, r_in_au=0.0), dict(th0_rad=-0.1), dict(th1_rad=4.0), dict(th1_rad=0.5),
    dict(r_out_au=float("nan")),
])
def test_spherical_grid_invalid_arguments_rejected(L, over):
    from paper_2509_03623_b300 import _rt
    _, _, o, vw, ln, keep = _structs()
    g = _rt.rt_grid_sph(8, 8, 8, 1, 10.0, 600.0, 1.0, 2.0)
    for k, val in over.items():
        setattr(g, k, val)
    f = _rt.rt_fields_sph(16, 16, 16, 16, 16, 16, 16, 0)  # dummy device pointers
    rc = L.rt_render_sph(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                         C.c_void_p(16), None)
    assert rc == -1
    assert len(L.rt_last_error()) > 0


def test_spherical_grid_null_field_rejected(L):
    from paper_2509_03623_b300 import _rt
    _, _, o, vw, ln, keep = _structs()
    g = _rt.rt_grid_sph(8, 8, 8, 1, 10.0, 600.0, 1.0, 2.0)
    f = _rt.rt_fields_sph(16, 16, 16, 16, 16, 0, 16, 0)
    assert L.rt_render_sph(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                           C.c_void_p(16), None) == -1
    assert b"field" in L.rt_last_error()


def test_plain_march_rejects_rotation_field(L):
    g, f, o, vw, ln, keep = _structs()
    f.vphi_kms = 16  # a rotation field: the plain march takes Keplerian rotation only
    assert L.rt_render_plain(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                             C.c_void_p(16), None) == -1
    assert b"Keplerian" in L.rt_last_error()


def test_pipe_probe_rejects_bad_arguments(L):
    import ctypes as C
    d = C.c_double()
    assert L.rt_pipe_peak(99, 1024, C.byref(d), C.byref(d), C.byref(d), None) == -1
    assert L.rt_pipe_peak(0, 1, C.byref(d), C.byref(d), C.byref(d), None) == -1
    assert L.rt_pipe_peak(0, 1024, None, C.byref(d), C.byref(d), None) == -1
