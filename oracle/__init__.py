"""FP64 CPU oracle of the line radiative-transfer march -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import
this package. It wraps `rt_oracle.c` (plain C, double precision, OpenMP over pixel rows)
with ctypes and shares no code with the CUDA library.

Problems are passed as any object with the attributes of the C struct `orc_problem`
(grid, node fields, geometry, view and line constants); arrays are converted to float64.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_HDR = os.path.join(_HERE, "rt_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE semantics, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("nr", C.c_int), ("nz", C.c_int), ("r_log", C.c_int),
        ("r_in_au", C.c_double), ("r_out_au", C.c_double), ("zr_max", C.c_double),
        ("T", C.POINTER(C.c_double)), ("n_h2", C.POINTER(C.c_double)),
        ("vturb", C.POINTER(C.c_double)), ("h_lo", C.POINTER(C.c_double)),
        ("h_hi", C.POINTER(C.c_double)),
        ("x_co", C.c_double), ("edge_w", C.c_double), ("vturb_mach", C.c_int),
        ("incl_deg", C.c_double), ("pa_deg", C.c_double), ("dist_pc", C.c_double),
        ("mstar_msun", C.c_double), ("vsys_kms", C.c_double),
        ("nx", C.c_int), ("ny", C.c_int), ("half_fov_au", C.c_double), ("nch", C.c_int),
        ("v_kms", C.POINTER(C.c_double)), ("n_samples", C.c_int), ("I0", C.c_double),
        ("units", C.c_int),
        ("nu0_hz", C.c_double), ("A_ul", C.c_double), ("B_rot_hz", C.c_double),
        ("m_co_amu", C.c_double), ("m_mol_amu", C.c_double), ("J_u", C.c_int),
        ("vphi", C.POINTER(C.c_double)),
        ("g3", C.c_void_p),
        ("gs", C.c_void_p),
    ]


class _Grid3(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
        ("z0", C.c_double), ("z1", C.c_double),
        ("T", C.POINTER(C.c_double)), ("n_h2", C.POINTER(C.c_double)),
        ("vturb", C.POINTER(C.c_double)), ("x_co", C.POINTER(C.c_double)),
        ("vx", C.POINTER(C.c_double)), ("vy", C.POINTER(C.c_double)),
        ("vz", C.POINTER(C.c_double)),
    ]


class _GridSph(C.Structure):
    _fields_ = [
        ("nr", C.c_int), ("nth", C.c_int), ("nph", C.c_int), ("r_log", C.c_int),
        ("r_in", C.c_double), ("r_out", C.c_double), ("th0", C.c_double), ("th1", C.c_double),
        ("T", C.POINTER(C.c_double)), ("n_h2", C.POINTER(C.c_double)),
        ("vturb", C.POINTER(C.c_double)), ("x_co", C.POINTER(C.c_double)),
        ("vr", C.POINTER(C.c_double)), ("vth", C.POINTER(C.c_double)),
        ("vph", C.POINTER(C.c_double)),
    ]


class _MLP(C.Structure):
    _fields_ = [
        ("n_freq", C.c_int), ("B", C.POINTER(C.c_double)), ("n_layers", C.c_int),
        ("dims", C.POINTER(C.c_int)), ("W", C.POINTER(C.POINTER(C.c_double))),
        ("b", C.POINTER(C.POINTER(C.c_double))), ("h_scale", C.c_double),
    ]


class _Chain(C.Structure):
    _fields_ = [
        ("sigma0_gcm2", C.c_double), ("r_c_au", C.c_double), ("gamma", C.c_double),
        ("T_freeze", C.c_double), ("N_dissoc_cm2", C.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            pp = C.POINTER(_Problem)
            lib.orc_render.argtypes = [pp, dp, C.c_int]
            lib.orc_render_pixels.argtypes = [pp, C.POINTER(C.c_longlong), C.c_int, dp, C.c_int]
            lib.orc_ray.argtypes = [pp, C.c_int, C.c_int, dp, dp, dp, dp]
            lib.orc_point.argtypes = [pp, C.c_double, C.c_double, C.c_double, C.c_double, dp]
            lib.orc_partition.argtypes = [C.c_double, C.c_double]
            lib.orc_partition.restype = C.c_double
            lib.orc_render_adjoint.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
            lib.orc_render_adjoint_vphi.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
            lib.orc_render_adjoint3.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
            lib.orc_mlp_eval.argtypes = [C.POINTER(_MLP), dp, C.c_int, dp]
            lib.orc_mlp_grad.argtypes = [C.POINTER(_MLP), dp, dp, C.c_int, dp, dp]
            lib.orc_render_mlp.argtypes = [pp, C.POINTER(_MLP), C.POINTER(C.c_longlong),
                                           C.c_int, dp, C.c_int]
            lib.orc_render_mlp_adjoint.argtypes = [pp, C.POINTER(_MLP), dp, dp, dp, dp, dp, dp,
                                                   dp, dp, dp, C.c_int]
            lib.orc_field_chain.argtypes = [pp, C.POINTER(_Chain), dp, dp, dp, dp, dp]
            lib.orc_pressure_vphi.argtypes = [pp, dp, dp, dp]
            lib.orc_pressure_vphi_adjoint.argtypes = [pp, dp, dp, dp, dp, dp]
            lib.orc_field_chain_adjoint.argtypes = [pp, C.POINTER(_Chain), dp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Packed:
    """Keeps the float64 copies alive while the struct is in use."""

    def __init__(self, p):
        self.keep = []

        def arr(x):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
            self.keep.append(a)
            return _dptr(a)

        s = _Problem()
        s.nr, s.nz, s.r_log = int(p.nr), int(p.nz), int(p.r_log)
        s.r_in_au, s.r_out_au, s.zr_max = float(p.r_in_au), float(p.r_out_au), float(p.zr_max)
        s.T, s.n_h2, s.vturb = arr(p.T), arr(p.n_h2), arr(p.vturb)
        s.h_lo, s.h_hi = arr(p.h_lo), arr(p.h_hi)
        s.x_co, s.edge_w, s.vturb_mach = float(p.x_co), float(p.edge_w), int(p.vturb_mach)
        s.incl_deg, s.pa_deg, s.dist_pc = float(p.incl_deg), float(p.pa_deg), float(p.dist_pc)
        s.mstar_msun, s.vsys_kms = float(p.mstar_msun), float(p.vsys_kms)
        s.nx, s.ny, s.half_fov_au = int(p.nx), int(p.ny), float(p.half_fov_au)
        v = np.asarray(p.v_kms, dtype=np.float64)
        s.nch, s.v_kms = int(v.size), arr(v)
        s.n_samples, s.I0, s.units = int(p.n_samples), float(p.I0), int(p.units)
        s.nu0_hz, s.A_ul, s.B_rot_hz = float(p.nu0_hz), float(p.A_ul), float(p.B_rot_hz)
        s.m_co_amu, s.m_mol_amu, s.J_u = float(p.m_co_amu), float(p.m_mol_amu), int(p.J_u)
        vphi = getattr(p, "vphi", None)
        s.vphi = arr(vphi) if vphi is not None else C.POINTER(C.c_double)()
        g3 = getattr(p, "g3", None)
        if g3 is not None:
            g = _Grid3()
            g.nx, g.ny, g.nz = int(g3.nx), int(g3.ny), int(g3.nz)
            g.x0, g.x1, g.y0, g.y1, g.z0, g.z1 = (float(v) for v in g3.extent)
            g.T, g.n_h2, g.vturb, g.x_co = arr(g3.T), arr(g3.n_h2), arr(g3.vturb), arr(g3.x_co)
            g.vx, g.vy, g.vz = arr(g3.vx), arr(g3.vy), arr(g3.vz)
            self.keep.append(g)
            s.g3 = C.cast(C.pointer(g), C.c_void_p)
        else:
            s.g3 = None
        gs = getattr(p, "gs", None)
        if gs is not None:
            g = _GridSph()
            g.nr, g.nth, g.nph, g.r_log = int(gs.nr), int(gs.nth), int(gs.nph), int(gs.r_log)
            g.r_in, g.r_out, g.th0, g.th1 = (float(gs.r_in), float(gs.r_out), float(gs.th0),
                                             float(gs.th1))
            g.T, g.n_h2, g.vturb, g.x_co = arr(gs.T), arr(gs.n_h2), arr(gs.vturb), arr(gs.x_co)
            g.vr, g.vth, g.vph = arr(gs.vr), arr(gs.vth), arr(gs.vph)
            self.keep.append(g)
            s.gs = C.cast(C.pointer(g), C.c_void_p)
        else:
            s.gs = None
        self.s = s
        self.nch = s.nch


class _PackedMLP:
    def __init__(self, w):
        self.keep = []
        B = np.ascontiguousarray(np.asarray(w.B, dtype=np.float64))
        Ws = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in w.W]
        bs = [np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in w.b]
        dims = np.array([Ws[0].shape[1]] + [x.shape[0] for x in Ws], dtype=np.int32)
        Wp = (C.POINTER(C.c_double) * len(Ws))(*[_dptr(x) for x in Ws])
        bp = (C.POINTER(C.c_double) * len(bs))(*[_dptr(x) for x in bs])
        self.keep += [B, Ws, bs, dims, Wp, bp]
        m = _MLP()
        m.n_freq = int(B.shape[0])
        m.B = _dptr(B)
        m.n_layers = len(Ws)
        m.dims = dims.ctypes.data_as(C.POINTER(C.c_int))
        m.W = Wp
        m.b = bp
        m.h_scale = float(getattr(w, "h_scale", 0.02))
        self.m = m
        self.n_out = int(dims[-1])


def _threads(nthreads):
    return int(nthreads) if nthreads else 0


def render(p, nthreads: int = 0) -> np.ndarray:
    """Cube [nch][ny][nx] in float64."""
    lib = _load()
    pk = _Packed(p)
    cube = np.zeros((pk.nch, int(p.ny), int(p.nx)), dtype=np.float64)
    rc = lib.orc_render(C.byref(pk.s), _dptr(cube), _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem")
    return cube


def render_pixels(p, pix, nthreads: int = 0) -> np.ndarray:
    """Spectra [npix][nch] of flat pixel indices pix = iy*nx + ix."""
    lib = _load()
    pk = _Packed(p)
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
    out = np.zeros((pix.size, pk.nch), dtype=np.float64)
    rc = lib.orc_render_pixels(C.byref(pk.s), pix.ctypes.data_as(C.POINTER(C.c_longlong)),
                               int(pix.size), _dptr(out), _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem")
    return out


def ray(p, ix: int, iy: int):
    """(hit, s_in, s_out, P0[3], omega[3]) of one pixel's ray (au)."""
    lib = _load()
    pk = _Packed(p)
    s0, s1 = C.c_double(), C.c_double()
    P0 = np.zeros(3)
    om = np.zeros(3)
    hit = lib.orc_ray(C.byref(pk.s), int(ix), int(iy), C.byref(s0), C.byref(s1), _dptr(P0),
                      _dptr(om))
    return bool(hit), s0.value, s1.value, P0, om


POINT_KEYS = ("j", "beta", "T", "n_h2", "X_co", "v_los_kms", "alpha_kms", "n_u", "n_l",
              "phi", "S", "vturb")


def point(p, x: float, y: float, z: float, v_kms: float) -> dict:
    """Local quantities at a disk-frame point (au) for one channel velocity."""
    lib = _load()
    pk = _Packed(p)
    out = np.zeros(12)
    gas = lib.orc_point(C.byref(pk.s), float(x), float(y), float(z), float(v_kms), _dptr(out))
    d = dict(zip(POINT_KEYS, out.tolist()))
    d["gas"] = bool(gas)
    return d


def partition(T: float, B_rot_hz: float) -> float:
    return float(_load().orc_partition(float(T), float(B_rot_hz)))


def render_adjoint(p, dL_dcube: np.ndarray, nthreads: int = 0):
    """(cube, grads) with grads = dict(T, n_h2, vturb [nz][nr], h_lo, h_hi [nr])."""
    lib = _load()
    pk = _Packed(p)
    g = np.ascontiguousarray(np.asarray(dL_dcube, dtype=np.float64))
    cube = np.zeros((pk.nch, int(p.ny), int(p.nx)), dtype=np.float64)
    shp = (int(p.nz), int(p.nr))
    dT, dn, dvt = np.zeros(shp), np.zeros(shp), np.zeros(shp)
    dlo, dhi = np.zeros(int(p.nr)), np.zeros(int(p.nr))
    rc = lib.orc_render_adjoint(C.byref(pk.s), _dptr(g), _dptr(cube), _dptr(dT), _dptr(dn),
                                _dptr(dvt), _dptr(dlo), _dptr(dhi), _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem")
    return cube, dict(T=dT, n_h2=dn, vturb=dvt, h_lo=dlo, h_hi=dhi)


def render_adjoint_vphi(p, dL_dcube: np.ndarray, nthreads: int = 0):
    """render_adjoint for a problem with a rotation field: grads also hold vphi [nz][nr]."""
    lib = _load()
    pk = _Packed(p)
    g = np.ascontiguousarray(np.asarray(dL_dcube, dtype=np.float64))
    cube = np.zeros((pk.nch, int(p.ny), int(p.nx)), dtype=np.float64)
    shp = (int(p.nz), int(p.nr))
    dT, dn, dvt, dvp = np.zeros(shp), np.zeros(shp), np.zeros(shp), np.zeros(shp)
    dlo, dhi = np.zeros(int(p.nr)), np.zeros(int(p.nr))
    rc = lib.orc_render_adjoint_vphi(C.byref(pk.s), _dptr(g), _dptr(cube), _dptr(dT), _dptr(dn),
                                     _dptr(dvt), _dptr(dlo), _dptr(dhi), _dptr(dvp),
                                     _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem (a rotation field is required)")
    return cube, dict(T=dT, n_h2=dn, vturb=dvt, h_lo=dlo, h_hi=dhi, vphi=dvp)


def render_adjoint3(p, dL_dcube: np.ndarray, nthreads: int = 0):
    """Reverse mode of the 3-D grid marches: (cube, grads) with grads a dict of T, n_h2,
    vturb, x_co and the velocity fields (vx, vy, vz on a Cartesian grid p.g3, [nz][ny][nx];
    vr, vth, vph on a spherical grid p.gs, [nph][nth][nr]), like the grid's fields."""
    lib = _load()
    pk = _Packed(p)
    g = np.ascontiguousarray(np.asarray(dL_dcube, dtype=np.float64))
    cube = np.zeros((pk.nch, int(p.ny), int(p.nx)), dtype=np.float64)
    if getattr(p, "gs", None) is not None:
        gs = p.gs
        shp = (int(gs.nph), int(gs.nth), int(gs.nr))
        keys = ("T", "n_h2", "vturb", "x_co", "vr", "vth", "vph")
    else:
        g3 = p.g3
        shp = (int(g3.nz), int(g3.ny), int(g3.nx))
        keys = ("T", "n_h2", "vturb", "x_co", "vx", "vy", "vz")
    out = {k: np.zeros(shp) for k in keys}
    rc = lib.orc_render_adjoint3(C.byref(pk.s), _dptr(g), _dptr(cube),
                                 *[_dptr(out[k]) for k in keys], _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem (one 3-D grid is required)")
    return cube, out


def mlp_eval(w, x: np.ndarray) -> np.ndarray:
    """Network outputs [npts][n_out] at inputs x [npts][2] = (rhat, zhat)."""
    lib = _load()
    pm = _PackedMLP(w)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 2))
    out = np.zeros((x.shape[0], pm.n_out))
    rc = lib.orc_mlp_eval(C.byref(pm.m), _dptr(x), int(x.shape[0]), _dptr(out))
    if rc:
        raise ValueError("oracle: invalid network")
    return out


def render_mlp(p, w, pix=None, nthreads: int = 0) -> np.ndarray:
    """Neural-field render: full cube [nch][ny][nx] (pix None) or spectra [npix][nch]."""
    lib = _load()
    pk = _Packed(p)
    pm = _PackedMLP(w)
    if pix is None:
        out = np.zeros((pk.nch, int(p.ny), int(p.nx)))
        rc = lib.orc_render_mlp(C.byref(pk.s), C.byref(pm.m), None, 0, _dptr(out),
                                _threads(nthreads))
    else:
        pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int64))
        out = np.zeros((pix.size, pk.nch))
        rc = lib.orc_render_mlp(C.byref(pk.s), C.byref(pm.m),
                                pix.ctypes.data_as(C.POINTER(C.c_longlong)), int(pix.size),
                                _dptr(out), _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem or network")
    return out


def render_mlp_adjoint(p, w, dL_dcube: np.ndarray, nthreads: int = 0):
    """(cube, grads): grads = dict(T, n_h2, vturb [nz][nr], h_lo, h_hi [nr] w.r.t. the grid
    fields under the network modulation, W = [dL/dW_l], b = [dL/db_l])."""
    lib = _load()
    pk = _Packed(p)
    pm = _PackedMLP(w)
    g = np.ascontiguousarray(np.asarray(dL_dcube, dtype=np.float64))
    cube = np.zeros((pk.nch, int(p.ny), int(p.nx)), dtype=np.float64)
    shp = (int(p.nz), int(p.nr))
    dT, dn, dvt = np.zeros(shp), np.zeros(shp), np.zeros(shp)
    dlo, dhi = np.zeros(int(p.nr)), np.zeros(int(p.nr))
    shapes = [np.asarray(x).shape for x in w.W]
    dW = np.zeros(sum(a * b for a, b in shapes))
    db = np.zeros(sum(a for a, _ in shapes))
    rc = lib.orc_render_mlp_adjoint(C.byref(pk.s), C.byref(pm.m), _dptr(g), _dptr(cube),
                                    _dptr(dT), _dptr(dn), _dptr(dvt), _dptr(dlo), _dptr(dhi),
                                    _dptr(dW), _dptr(db), _threads(nthreads))
    if rc:
        raise ValueError("oracle: invalid problem or network")
    Ws, bs, ow, ob = [], [], 0, 0
    for a, b in shapes:
        Ws.append(dW[ow:ow + a * b].reshape(a, b))
        bs.append(db[ob:ob + a])
        ow += a * b
        ob += a
    return cube, dict(T=dT, n_h2=dn, vturb=dvt, h_lo=dlo, h_hi=dhi, W=Ws, b=bs)


def mlp_grad(w, x: np.ndarray, gout: np.ndarray):
    """(dW list, db list) of sum_i gout[i] . net(x[i]) with respect to the weights."""
    lib = _load()
    pm = _PackedMLP(w)
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 2))
    gout = np.ascontiguousarray(np.asarray(gout, dtype=np.float64).reshape(x.shape[0], -1))
    shapes = [np.asarray(a).shape for a in w.W]
    dW = np.zeros(sum(a * b for a, b in shapes))
    db = np.zeros(sum(a for a, _ in shapes))
    rc = lib.orc_mlp_grad(C.byref(pm.m), _dptr(x), _dptr(gout), int(x.shape[0]), _dptr(dW),
                          _dptr(db))
    if rc:
        raise ValueError("oracle: invalid network")
    Ws, bs, ow, ob = [], [], 0, 0
    for a, b in shapes:
        Ws.append(dW[ow:ow + a * b].reshape(a, b))
        bs.append(db[ob:ob + a])
        ow += a * b
        ob += a
    return Ws, bs


def field_chain(p, chain, T=None):
    """Physics-constrained field chain (rt_oracle.h, orc_field_chain) on the grid of p with
    the temperature grid T [nz][nr] (p.T when None): dict(n_h2, N_h2 [nz][nr], h_lo, h_hi
    [nr]). `chain` has the attributes sigma0_gcm2, r_c_au, gamma, T_freeze, N_dissoc_cm2."""
    lib = _load()
    q = p if T is None else p.replace(T=np.asarray(T, dtype=np.float64))
    pk = _Packed(q)
    Tg = np.ascontiguousarray(np.asarray(q.T, dtype=np.float64))
    c = _Chain(float(chain.sigma0_gcm2), float(chain.r_c_au), float(chain.gamma),
               float(chain.T_freeze), float(chain.N_dissoc_cm2))
    n = np.zeros((q.nz, q.nr))
    N = np.zeros((q.nz, q.nr))
    lo = np.zeros(q.nr)
    hi = np.zeros(q.nr)
    rc = lib.orc_field_chain(C.byref(pk.s), C.byref(c), _dptr(Tg), _dptr(n), _dptr(N),
                             _dptr(lo), _dptr(hi))
    if rc != 0:
        raise ValueError("orc_field_chain: invalid arguments")
    return dict(n_h2=n, N_h2=N, h_lo=lo, h_hi=hi)


def field_chain_adjoint(p, chain, T=None, g_n=None, g_lo=None, g_hi=None):
    """Reverse mode of field_chain (rt_oracle.h, orc_field_chain_adjoint): dL/dT [nz][nr]
    from dL/dn_h2 [nz][nr] and dL/dh_lo, dL/dh_hi [nr] (None: zero)."""
    lib = _load()
    q = p if T is None else p.replace(T=np.asarray(T, dtype=np.float64))
    pk = _Packed(q)
    Tg = np.ascontiguousarray(np.asarray(q.T, dtype=np.float64))
    c = _Chain(float(chain.sigma0_gcm2), float(chain.r_c_au), float(chain.gamma),
               float(chain.T_freeze), float(chain.N_dissoc_cm2))
    keep = []

    def opt(a, shape):
        if a is None:
            return C.POINTER(C.c_double)()
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shape))
        keep.append(a)
        return _dptr(a)

    gT = np.zeros((q.nz, q.nr))
    rc = lib.orc_field_chain_adjoint(C.byref(pk.s), C.byref(c), _dptr(Tg),
                                     opt(g_n, (q.nz, q.nr)), opt(g_lo, (q.nr,)),
                                     opt(g_hi, (q.nr,)), _dptr(gT))
    if rc != 0:
        raise ValueError("orc_field_chain_adjoint: invalid arguments")
    return gT


def pressure_vphi_adjoint(p, g_v, n_h2=None, T=None):
    """Reverse mode of pressure_vphi: (dL/dn_h2, dL/dT) [nz][nr] from dL/dvphi [nz][nr]."""
    lib = _load()
    pk = _Packed(p)
    n = np.ascontiguousarray(np.asarray(p.n_h2 if n_h2 is None else n_h2, dtype=np.float64))
    Tg = np.ascontiguousarray(np.asarray(p.T if T is None else T, dtype=np.float64))
    gv = np.ascontiguousarray(np.asarray(g_v, dtype=np.float64))
    gn, gT = np.zeros((p.nz, p.nr)), np.zeros((p.nz, p.nr))
    if lib.orc_pressure_vphi_adjoint(C.byref(pk.s), _dptr(n), _dptr(Tg), _dptr(gv), _dptr(gn),
                                     _dptr(gT)) != 0:
        raise ValueError("orc_pressure_vphi_adjoint: invalid arguments")
    return gn, gT


def pressure_vphi(p, n_h2=None, T=None):
    """Pressure-corrected rotation [nz][nr] km/s (rt_oracle.h, orc_pressure_vphi) from the
    node fields n_h2 and T (p's when None)."""
    lib = _load()
    pk = _Packed(p)
    n = np.ascontiguousarray(np.asarray(p.n_h2 if n_h2 is None else n_h2, dtype=np.float64))
    Tg = np.ascontiguousarray(np.asarray(p.T if T is None else T, dtype=np.float64))
    out = np.zeros((p.nz, p.nr))
    if lib.orc_pressure_vphi(C.byref(pk.s), _dptr(n), _dptr(Tg), _dptr(out)) != 0:
        raise ValueError("orc_pressure_vphi: invalid arguments")
    return out
