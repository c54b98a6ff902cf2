"""ctypes binding of librt_b300.so (argument marshalling only).

Every function here fills the C structs of `include/rt.h` from a problem description and
torch CUDA tensors, then calls the library on the current torch stream. There is no CPU
fallback: if the shared library is missing or fails to load, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librt_b300.so")

RT_OK, RT_EINVAL, RT_ENOMEM, RT_EBUSY, RT_ETIMEDOUT, RT_ECUDA, RT_ENOTFOUND = (
    0, -1, -2, -3, -4, -5, -6)
RT_MAX_CH = 256


class RTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


class rt_grid(C.Structure):
    _fields_ = [("nr", C.c_int), ("nz", C.c_int), ("r_log", C.c_int),
                ("r_in_au", C.c_double), ("r_out_au", C.c_double), ("zr_max", C.c_double)]


class rt_fields(C.Structure):
    _fields_ = [("T_K", C.c_void_p), ("n_h2_cm3", C.c_void_p), ("vturb", C.c_void_p),
                ("h_lo", C.c_void_p), ("h_hi", C.c_void_p), ("x_co", C.c_double),
                ("edge_w", C.c_double), ("vturb_mach", C.c_int), ("vphi_kms", C.c_void_p)]


class rt_geom(C.Structure):
    _fields_ = [("incl_deg", C.c_double), ("pa_deg", C.c_double), ("dist_pc", C.c_double),
                ("mstar_msun", C.c_double), ("vsys_kms", C.c_double)]


class rt_view(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("half_fov_au", C.c_double),
                ("nch", C.c_int), ("v_kms", C.POINTER(C.c_float)), ("n_samples", C.c_int),
                ("I0", C.c_double), ("units", C.c_int)]


class rt_line(C.Structure):
    _fields_ = [("nu0_hz", C.c_double), ("A_ul", C.c_double), ("B_rot_hz", C.c_double),
                ("m_co_amu", C.c_double), ("m_mol_amu", C.c_double), ("J_u", C.c_int)]


class rt_grads(C.Structure):
    _fields_ = [("dT", C.c_void_p), ("dn", C.c_void_p), ("dvt", C.c_void_p),
                ("dh_lo", C.c_void_p), ("dh_hi", C.c_void_p), ("loss", C.c_void_p),
                ("dvphi", C.c_void_p)]


class rt_mlp(C.Structure):
    _fields_ = [("n_freq", C.c_int), ("width", C.c_int), ("hidden", C.c_int), ("n_out", C.c_int),
                ("B", C.c_void_p), ("W", C.c_void_p * 5), ("b", C.c_void_p * 5),
                ("h_scale", C.c_double), ("precision", C.c_int)]


RT_MLP_F16, RT_MLP_BF16 = 0, 1


class rt_mlp_grads(C.Structure):
    _fields_ = [("dW", C.c_void_p * 5), ("db", C.c_void_p * 5)]


_lock = threading.Lock()
_lib = None


class rt_grid3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("x0_au", C.c_double), ("x1_au", C.c_double), ("y0_au", C.c_double),
                ("y1_au", C.c_double), ("z0_au", C.c_double), ("z1_au", C.c_double)]


class rt_fields3(C.Structure):
    _fields_ = [("T_K", C.c_void_p), ("n_h2_cm3", C.c_void_p), ("vturb", C.c_void_p),
                ("x_co", C.c_void_p), ("vx_kms", C.c_void_p), ("vy_kms", C.c_void_p),
                ("vz_kms", C.c_void_p), ("vturb_mach", C.c_int)]


class rt_grads3(C.Structure):
    _fields_ = [("dT", C.c_void_p), ("dn_h2", C.c_void_p), ("dvturb", C.c_void_p),
                ("dx_co", C.c_void_p), ("dvx", C.c_void_p), ("dvy", C.c_void_p),
                ("dvz", C.c_void_p), ("loss", C.c_void_p)]


class rt_grid_sph(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("nph", C.c_int), ("r_log", C.c_int),
                ("r_in_au", C.c_double), ("r_out_au", C.c_double), ("th0_rad", C.c_double),
                ("th1_rad", C.c_double)]


class rt_fields_sph(C.Structure):
    _fields_ = [("T_K", C.c_void_p), ("n_h2_cm3", C.c_void_p), ("vturb", C.c_void_p),
                ("x_co", C.c_void_p), ("vr_kms", C.c_void_p), ("vth_kms", C.c_void_p),
                ("vph_kms", C.c_void_p), ("vturb_mach", C.c_int)]


class rt_chain(C.Structure):
    _fields_ = [("sigma0_gcm2", C.c_double), ("r_c_au", C.c_double), ("gamma", C.c_double),
                ("T_freeze_K", C.c_double), ("N_dissoc_cm2", C.c_double)]


def lib():
    """Load librt_b300.so (after torch, so that one CUDA runtime serves both)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -m paper_2509_03623_b300.build`"
                    " (there is no CPU fallback)")
            import torch  # noqa: F401  (loads libcudart first)
            L = C.CDLL(LIB_PATH, mode=C.RTLD_GLOBAL)
            P = C.POINTER
            base = [P(rt_grid), P(rt_fields), P(rt_geom), P(rt_view), P(rt_line)]
            L.rt_render.argtypes = base + [C.c_void_p, C.c_void_p]
            L.rt_render.restype = C.c_int
            L.rt_count_gas_samples.argtypes = base + [C.c_void_p, C.c_void_p]
            L.rt_count_gas_samples.restype = C.c_int
            L.rt_render_work.argtypes = base + [C.c_void_p, C.c_void_p, C.c_void_p]
            L.rt_render_work.restype = C.c_int
            L.rt_render_adjoint.argtypes = base + [C.c_void_p, C.c_void_p, C.c_void_p,
                                                   P(rt_grads), C.c_void_p]
            L.rt_render_adjoint.restype = C.c_int
            L.rt_render_adjoint_work.argtypes = base + [C.c_void_p, C.c_void_p, C.c_void_p,
                                                        P(rt_grads), C.c_void_p, C.c_void_p]
            L.rt_render_adjoint_work.restype = C.c_int
            L.rt_render_adjoint_noalloc.argtypes = L.rt_render_adjoint.argtypes
            L.rt_render_adjoint_noalloc.restype = C.c_int
            L.rt_surface_powerlaw_grad.argtypes = [P(rt_grid), C.c_void_p, C.c_void_p,
                                                   C.c_double, C.c_void_p, C.c_void_p]
            L.rt_surface_powerlaw_grad.restype = C.c_int
            L.rt_mlp_eval.argtypes = [P(rt_mlp), C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]
            L.rt_mlp_eval.restype = C.c_int
            L.rt_render_mlp.argtypes = base + [P(rt_mlp), C.c_void_p, C.c_void_p]
            L.rt_render_mlp.restype = C.c_int
            L.rt_mlp_backward.argtypes = [P(rt_mlp), C.c_void_p, C.c_void_p, C.c_longlong,
                                          P(rt_mlp_grads), C.c_void_p]
            L.rt_mlp_backward.restype = C.c_int
            L.rt_render_mlp_adjoint.argtypes = base + [P(rt_mlp), C.c_void_p, C.c_void_p,
                                                       C.c_void_p, P(rt_grads),
                                                       P(rt_mlp_grads), C.c_void_p]
            L.rt_render_mlp_adjoint.restype = C.c_int
            L.rt_sample_coords.argtypes = base + [C.c_void_p, C.c_void_p]
            L.rt_sample_coords.restype = C.c_int
            L.rt_render_modulated.argtypes = base + [C.c_void_p, C.c_double, C.c_void_p,
                                                     C.c_void_p]
            L.rt_render_modulated.restype = C.c_int
            L.rt_field_chain.argtypes = [P(rt_grid), P(rt_geom), P(rt_line), P(rt_chain),
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p]
            L.rt_field_chain.restype = C.c_int
            L.rt_field_chain_adjoint.argtypes = [P(rt_grid), P(rt_geom), P(rt_line),
                                                 P(rt_chain), C.c_void_p, C.c_void_p,
                                                 C.c_void_p, C.c_void_p, C.c_void_p,
                                                 C.c_void_p]
            L.rt_field_chain_adjoint.restype = C.c_int
            L.rt_pressure_vphi.argtypes = [P(rt_grid), P(rt_geom), P(rt_line), C.c_void_p,
                                           C.c_void_p, C.c_void_p, C.c_void_p]
            L.rt_pressure_vphi.restype = C.c_int
            L.rt_pressure_vphi_adjoint.argtypes = [P(rt_grid), P(rt_geom), P(rt_line), C.c_void_p,
                                                   C.c_void_p, C.c_void_p, C.c_void_p,
                                                   C.c_void_p, C.c_void_p]
            L.rt_pressure_vphi_adjoint.restype = C.c_int
            L.rt_render3d.argtypes = [P(rt_grid3), P(rt_fields3), P(rt_geom), P(rt_view),
                                      P(rt_line), C.c_void_p, C.c_void_p]
            L.rt_render3d.restype = C.c_int
            L.rt_render3d_adjoint.argtypes = [P(rt_grid3), P(rt_fields3), P(rt_geom),
                                              P(rt_view), P(rt_line), C.c_void_p, C.c_void_p,
                                              C.c_void_p, P(rt_grads3), C.c_void_p]
            L.rt_render3d_adjoint.restype = C.c_int
            L.rt_render_sph.argtypes = [P(rt_grid_sph), P(rt_fields_sph), P(rt_geom),
                                        P(rt_view), P(rt_line), C.c_void_p, C.c_void_p]
            L.rt_render_sph.restype = C.c_int
            L.rt_render_sph_adjoint.argtypes = [P(rt_grid_sph), P(rt_fields_sph), P(rt_geom),
                                                P(rt_view), P(rt_line), C.c_void_p, C.c_void_p,
                                                C.c_void_p, P(rt_grads3), C.c_void_p]
            L.rt_render_sph_adjoint.restype = C.c_int
            L.rt_pack_nodes3.argtypes = [P(rt_fields3), C.c_longlong, C.c_void_p, C.c_void_p]
            L.rt_pack_nodes3.restype = C.c_int
            L.rt_render3d_packed.argtypes = [P(rt_grid3), C.c_void_p, C.c_int, P(rt_geom),
                                             P(rt_view), P(rt_line), C.c_void_p, C.c_void_p]
            L.rt_render3d_packed.restype = C.c_int
            L.rt_render_sph_packed.argtypes = [P(rt_grid_sph), C.c_void_p, C.c_int, P(rt_geom),
                                               P(rt_view), P(rt_line), C.c_void_p, C.c_void_p]
            L.rt_render_sph_packed.restype = C.c_int
            for nm, G in (("rt_render3d_adjoint_packed", rt_grid3),
                          ("rt_render_sph_adjoint_packed", rt_grid_sph)):
                fn = getattr(L, nm)
                fn.argtypes = [P(G), C.c_void_p, C.c_int, P(rt_geom), P(rt_view), P(rt_line),
                               C.c_void_p, C.c_void_p, C.c_void_p, P(rt_grads3), C.c_void_p]
                fn.restype = C.c_int
            L.rt_render_plain.argtypes = base + [C.c_void_p, C.c_void_p]
            L.rt_render_plain.restype = C.c_int
            L.rt_render_dense.argtypes = base + [C.c_void_p, C.c_void_p]
            L.rt_render_dense.restype = C.c_int
            L.rt_render_launch_count.argtypes = base + [P(C.c_int)]
            L.rt_render_launch_count.restype = C.c_int
            L.rt_pipe_peak.argtypes = [C.c_int, C.c_int, P(C.c_double), P(C.c_double),
                                       P(C.c_double), C.c_void_p]
            L.rt_pipe_peak.restype = C.c_int
            L.rt_kernel_timing.argtypes = [C.c_int]
            L.rt_kernel_timing.restype = C.c_int
            L.rt_kernel_time.argtypes = [P(C.c_double), P(C.c_int)]
            L.rt_kernel_time.restype = C.c_int
            L.rt_mlp_status.argtypes = [P(C.c_int)]
            L.rt_mlp_status.restype = C.c_int
            L.rt_last_error.restype = C.c_char_p
            L.rt_version.restype = C.c_char_p
            _lib = L
    return _lib


def check(rc: int):
    if rc != RT_OK:
        raise RTError(rc, lib().rt_last_error().decode())


def stream_handle(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class DeviceDisk:
    """Device-resident float32 node fields and surfaces of one problem."""

    FIELDS = ("T", "n_h2", "vturb", "h_lo", "h_hi")

    def __init__(self, problem, device="cuda"):
        import torch
        self.problem = problem
        self.device = torch.device(device)
        for k in self.FIELDS:
            setattr(self, k, torch.as_tensor(
                np.ascontiguousarray(getattr(problem, k), dtype=np.float32), device=self.device))
        vphi = getattr(problem, "vphi", None)  # optional rotation field (None: Keplerian)
        self.vphi = (torch.as_tensor(np.ascontiguousarray(vphi, dtype=np.float32),
                                     device=self.device) if vphi is not None else None)

    def tensors(self):
        return tuple(getattr(self, k) for k in self.FIELDS)


def structs(problem, T, n, vt, hlo, hhi, vphi=None):
    """C structs for `problem` with field tensors (CUDA float32, contiguous); vphi: optional
    rotation field [nz][nr] km/s (None: Keplerian)."""
    for t, shp in ((T, (problem.nz, problem.nr)), (n, (problem.nz, problem.nr)),
                   (vt, (problem.nz, problem.nr)), (hlo, (problem.nr,)), (hhi, (problem.nr,))):
        if (not t.is_cuda or t.dtype.itemsize != 4 or not t.is_floating_point()
                or not t.is_contiguous() or tuple(t.shape) != shp):
            raise ValueError(f"field tensors must be contiguous CUDA float32 of shape {shp}")
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    if vphi is not None and (not vphi.is_cuda or vphi.dtype.itemsize != 4 or not vphi.is_contiguous()
                             or tuple(vphi.shape) != (problem.nz, problem.nr)):
        raise ValueError("vphi must be a contiguous CUDA float32 tensor of shape [nz][nr]")
    f = rt_fields(T.data_ptr(), n.data_ptr(), vt.data_ptr(), hlo.data_ptr(), hhi.data_ptr(),
                  float(problem.x_co), float(problem.edge_w), int(problem.vturb_mach),
                  vphi.data_ptr() if vphi is not None else None)
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    v = np.ascontiguousarray(np.asarray(problem.v_kms, dtype=np.float32))
    vw = rt_view(int(problem.nx), int(problem.ny), float(problem.half_fov_au), int(v.size),
                 v.ctypes.data_as(C.POINTER(C.c_float)), int(problem.n_samples),
                 float(problem.I0), int(problem.units))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    return g, f, o, vw, ln, v


def rt_render(problem, fields=None, out=None, stream=None):
    """Forward render through the C ABI; returns the cube tensor [nch][ny][nx] float32."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    check(lib().rt_render(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                          C.c_void_p(out.data_ptr()), stream_handle(stream)))
    return out


def rt_render_plain(problem, fields=None, out=None, stream=None):
    """The plain FP32 comparison march (rt_render_plain); returns the cube tensor."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    check(lib().rt_render_plain(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                                C.c_void_p(out.data_ptr()), stream_handle(stream)))
    return out


def rt_render_dense(problem, fields=None, out=None, stream=None):
    """The dense FP32 comparison march (rt_render_dense); returns the cube tensor."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    check(lib().rt_render_dense(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                                C.c_void_p(out.data_ptr()), stream_handle(stream)))
    return out


def rt_render_launch_count(problem, fields=None) -> int:
    """Kernel launches rt_render makes for `problem` (2 with the corner-quad packing)."""
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi, getattr(dd, "vphi", None))
    c = C.c_int()
    check(lib().rt_render_launch_count(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                       C.byref(ln), C.byref(c)))
    return c.value


def rt_count_gas_samples(problem, fields=None, stream=None) -> int:
    """Number of (ray, sample) pairs inside the gas grid (executed samples of a render)."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    cnt = torch.zeros(1, dtype=torch.int64, device=T.device)
    check(lib().rt_count_gas_samples(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                     C.byref(ln), C.c_void_p(cnt.data_ptr()),
                                     stream_handle(stream)))
    return int(cnt.item())


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _cube_arg(t, shape, name):
    if t is None:
        return None
    if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous() or tuple(t.shape) != shape:
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of shape {shape}")
    return t


def rt_render_work(problem, fields=None, out=None, stream=None):
    """rt_render plus its work counts: (cube, physics samples with gas, sample-channel
    evaluations computed after the channel window)."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    work = torch.zeros(2, dtype=torch.int64, device=T.device)
    check(lib().rt_render_work(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                               _ptr(out), _ptr(work), stream_handle(stream)))
    w = work.cpu().tolist()
    return out, int(w[0]), int(w[1])


def rt_render_adjoint(problem, fields=None, dL_dcube=None, target=None, cube_out=True,
                      stream=None, work=None):
    """Fused forward + reverse march through the C ABI.

    Give exactly one of dL_dcube (gradient of a loss w.r.t. the cube) or target (loss =
    sum (cube - target)^2). Returns (cube or None, grads) with grads a dict of float64 CUDA
    tensors T, n_h2, vturb [nz][nr], h_lo, h_hi [nr] and loss (1 element). With `work` (a
    CUDA int64 tensor of 4 elements) the call is rt_render_adjoint_work, which also counts the
    kernel's work into it."""
    import torch
    dd = fields if fields is not None else DeviceDisk(problem)
    T, n, vt, hlo, hhi = dd.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(dd, "vphi", None))
    shape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, shape, "dL_dcube")
    target = _cube_arg(target, shape, "target")
    dev = T.device
    cube = None
    if cube_out is True:
        cube = torch.empty(shape, dtype=torch.float32, device=dev)
    elif cube_out is not None and cube_out is not False:
        cube = _cube_arg(cube_out, shape, "cube_out")
    out = {k: torch.empty(tuple(t.shape), dtype=torch.float64, device=dev)
           for k, t in zip(DeviceDisk.FIELDS, (T, n, vt, hlo, hhi))}
    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
    vp = getattr(dd, "vphi", None)
    if vp is not None:  # a rotation field: its gradient too
        out["vphi"] = torch.empty(tuple(vp.shape), dtype=torch.float64, device=dev)
    gr = rt_grads(out["T"].data_ptr(), out["n_h2"].data_ptr(), out["vturb"].data_ptr(),
                  out["h_lo"].data_ptr(), out["h_hi"].data_ptr(), out["loss"].data_ptr(),
                  out["vphi"].data_ptr() if vp is not None else None)
    if work is not None:
        assert work.is_cuda and work.dtype == torch.int64 and work.numel() >= 4
        check(lib().rt_render_adjoint_work(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                           C.byref(ln), _ptr(dL_dcube), _ptr(target),
                                           _ptr(cube), C.byref(gr), _ptr(work),
                                           stream_handle(stream)))
    else:
        check(lib().rt_render_adjoint(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                      C.byref(ln), _ptr(dL_dcube), _ptr(target), _ptr(cube),
                                      C.byref(gr), stream_handle(stream)))
    return cube, out


def rt_render_adjoint_noalloc(problem, fields, cube_out, grads, dL_dcube=None, target=None,
                              stream=None):
    """rt_render_adjoint without any allocation inside the library: for callers that must
    not allocate device memory while running. Every buffer (cube_out and the float64
    gradient tensors in `grads`, keys T, n_h2, vturb, h_lo, h_hi, loss) is supplied by the
    caller; the library uses its fixed 32 MiB device array for checkpoints and gradient copies."""
    T, n, vt, hlo, hhi = fields.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(fields, "vphi", None))
    shape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, shape, "dL_dcube")
    target = _cube_arg(target, shape, "target")
    cube_out = _cube_arg(cube_out, shape, "cube_out")
    gr = rt_grads(grads["T"].data_ptr(), grads["n_h2"].data_ptr(), grads["vturb"].data_ptr(),
                  grads["h_lo"].data_ptr(), grads["h_hi"].data_ptr(),
                  grads["loss"].data_ptr() if grads.get("loss") is not None else None,
                  grads["vphi"].data_ptr() if grads.get("vphi") is not None else None)
    check(lib().rt_render_adjoint_noalloc(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                          C.byref(ln), _ptr(dL_dcube), _ptr(target),
                                          _ptr(cube_out), C.byref(gr), stream_handle(stream)))


def rt_surface_powerlaw_grad(problem, dh, h, c, stream=None):
    """(dL/dc, dL/dp) of a surface h = c (r/100 au)^p m(r) from node gradients dh."""
    import torch
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    dh = dh.contiguous().to(torch.float64)
    h = h.contiguous().to(torch.float32)
    out = torch.empty(2, dtype=torch.float64, device=dh.device)
    check(lib().rt_surface_powerlaw_grad(C.byref(g), _ptr(dh), _ptr(h), float(c), _ptr(out),
                                         stream_handle(stream)))
    return out


def rt_field_chain(problem, T, chain, column=True, stream=None, out=None):
    """Physics-constrained field chain on the grid of `problem` from the temperature grid T
    (CUDA float32 [nz][nr]): dict(n_h2, N_h2 (None unless column), h_lo, h_hi), written into
    `out` (a dict of that form) when given. `chain` has the attributes sigma0_gcm2, r_c_au,
    gamma, T_freeze, N_dissoc_cm2."""
    import torch
    shp = (int(problem.nz), int(problem.nr))
    if not T.is_cuda or T.dtype != torch.float32 or not T.is_contiguous() or tuple(T.shape) != shp:
        raise ValueError(f"T must be a contiguous CUDA float32 tensor of shape {shp}")
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    c = rt_chain(float(chain.sigma0_gcm2), float(chain.r_c_au), float(chain.gamma),
                 float(chain.T_freeze), float(chain.N_dissoc_cm2))
    if out is not None:
        n, N, lo, hi = out["n_h2"], out["N_h2"], out["h_lo"], out["h_hi"]
    else:
        n = torch.empty(shp, dtype=torch.float32, device=T.device)
        N = torch.empty(shp, dtype=torch.float32, device=T.device) if column else None
        lo = torch.empty(shp[1], dtype=torch.float32, device=T.device)
        hi = torch.empty(shp[1], dtype=torch.float32, device=T.device)
    check(lib().rt_field_chain(C.byref(g), C.byref(o), C.byref(ln), C.byref(c), _ptr(T),
                               _ptr(n), _ptr(N) if N is not None else None, _ptr(lo), _ptr(hi),
                               stream_handle(stream)))
    return dict(n_h2=n, N_h2=N, h_lo=lo, h_hi=hi)


def rt_field_chain_adjoint(problem, T, chain, g_n=None, g_lo=None, g_hi=None, out=None,
                           stream=None):
    """Reverse mode of rt_field_chain: dL/dT (CUDA float64 [nz][nr], written into `out` when
    given) from dL/dn_h2 (float64 [nz][nr]) and dL/dh_lo, dL/dh_hi (float64 [nr]); None for
    zero."""
    import torch
    shp = (int(problem.nz), int(problem.nr))
    if not T.is_cuda or T.dtype != torch.float32 or not T.is_contiguous() or tuple(T.shape) != shp:
        raise ValueError(f"T must be a contiguous CUDA float32 tensor of shape {shp}")
    for name, t, sh in (("g_n", g_n, shp), ("g_lo", g_lo, shp[1:]), ("g_hi", g_hi, shp[1:])):
        if t is not None and (not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()
                              or tuple(t.shape) != sh):
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor of shape {sh}")
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    c = rt_chain(float(chain.sigma0_gcm2), float(chain.r_c_au), float(chain.gamma),
                 float(chain.T_freeze), float(chain.N_dissoc_cm2))
    if out is None:
        out = torch.empty(shp, dtype=torch.float64, device=T.device)
    opt = lambda t: _ptr(t) if t is not None else None
    check(lib().rt_field_chain_adjoint(C.byref(g), C.byref(o), C.byref(ln), C.byref(c), _ptr(T),
                                       opt(g_n), opt(g_lo), opt(g_hi), _ptr(out),
                                       stream_handle(stream)))
    return out


def rt_pressure_vphi_adjoint(problem, n_h2, T, g_vphi, stream=None):
    """Reverse mode of rt_pressure_vphi: (dL/dn_h2, dL/dT), CUDA float64 [nz][nr], from
    dL/dvphi (CUDA float64 [nz][nr])."""
    import torch
    shp = (int(problem.nz), int(problem.nr))
    for name, t, dt in (("n_h2", n_h2, torch.float32), ("T", T, torch.float32),
                        ("g_vphi", g_vphi, torch.float64)):
        if not t.is_cuda or t.dtype != dt or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"{name} must be a contiguous CUDA {dt} tensor of shape {shp}")
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    gn = torch.empty(shp, dtype=torch.float64, device=T.device)
    gT = torch.empty(shp, dtype=torch.float64, device=T.device)
    check(lib().rt_pressure_vphi_adjoint(C.byref(g), C.byref(o), C.byref(ln), _ptr(n_h2), _ptr(T),
                                         _ptr(g_vphi), _ptr(gn), _ptr(gT), stream_handle(stream)))
    return gn, gT


def rt_pressure_vphi(problem, n_h2, T, out=None, stream=None):
    """Pressure-corrected rotation [nz][nr] km/s from the node fields n_h2 and T (CUDA
    float32 [nz][nr])."""
    import torch
    shp = (int(problem.nz), int(problem.nr))
    for t in (n_h2, T):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"n_h2 and T must be contiguous CUDA float32 tensors of shape {shp}")
    g = rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log), float(problem.r_in_au),
                float(problem.r_out_au), float(problem.zr_max))
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    if out is None:
        out = torch.empty(shp, dtype=torch.float32, device=T.device)
    check(lib().rt_pressure_vphi(C.byref(g), C.byref(o), C.byref(ln), _ptr(n_h2), _ptr(T),
                                 _ptr(out), stream_handle(stream)))
    return out


class DeviceGrid3:
    """Device-resident float32 fields [nz][ny][nx] of a 3-D grid (problem.g3)."""

    FIELDS = ("T", "n_h2", "vturb", "x_co", "vx", "vy", "vz")

    def __init__(self, problem, device="cuda"):
        import torch
        g = problem.g3
        self.problem = problem
        for k in self.FIELDS:
            setattr(self, k, torch.as_tensor(np.ascontiguousarray(getattr(g, k), dtype=np.float32),
                                             device=device))


def _view_line_geom(problem):
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    v = np.ascontiguousarray(np.asarray(problem.v_kms, dtype=np.float32))
    vw = rt_view(int(problem.nx), int(problem.ny), float(problem.half_fov_au), int(v.size),
                 v.ctypes.data_as(C.POINTER(C.c_float)), int(problem.n_samples),
                 float(problem.I0), int(problem.units))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    return o, v, vw, ln


class DeviceGridSph:
    """Device-resident float32 fields [nph][nth][nr] of a spherical grid (problem.gs)."""

    FIELDS = ("T", "n_h2", "vturb", "x_co", "vr", "vth", "vph")

    def __init__(self, problem, device="cuda"):
        import torch
        g = problem.gs
        self.problem = problem
        for k in self.FIELDS:
            setattr(self, k, torch.as_tensor(np.ascontiguousarray(getattr(g, k), dtype=np.float32),
                                             device=device))


def rt_render_sph(problem, grid=None, out=None, stream=None):
    """Forward render through a 3-D spherical grid (problem.gs); returns the cube tensor
    [nch][ny][nx] float32."""
    import torch
    gs = problem.gs
    dg = grid if grid is not None else DeviceGridSph(problem)
    shp = (int(gs.nph), int(gs.nth), int(gs.nr))
    for k in DeviceGridSph.FIELDS:
        t = getattr(dg, k)
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"spherical field {k} must be a contiguous CUDA float32 tensor of "
                             f"shape {shp}")
    gg = rt_grid_sph(int(gs.nr), int(gs.nth), int(gs.nph), int(gs.r_log), float(gs.r_in),
                     float(gs.r_out), float(gs.th0), float(gs.th1))
    f = rt_fields_sph(*(getattr(dg, k).data_ptr() for k in DeviceGridSph.FIELDS),
                      int(problem.vturb_mach))
    o, v, vw, ln = _view_line_geom(problem)
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=dg.T.device)
    check(lib().rt_render_sph(C.byref(gg), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                              _ptr(out), stream_handle(stream)))
    return out


def rt_render_sph_adjoint(problem, grid=None, dL_dcube=None, target=None, cube_out=True,
                          stream=None):
    """Fused forward + reverse march through a 3-D spherical grid (problem.gs), through the C
    ABI. Give exactly one of dL_dcube or target (loss = sum (cube - target)^2). Returns
    (cube or None, grads) with grads a dict of float64 CUDA tensors T, n_h2, vturb, x_co, vr,
    vth, vph [nph][nth][nr] and loss (1 element)."""
    import torch
    gs = problem.gs
    dg = grid if grid is not None else DeviceGridSph(problem)
    shp = (int(gs.nph), int(gs.nth), int(gs.nr))
    for k in DeviceGridSph.FIELDS:
        t = getattr(dg, k)
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"spherical field {k} must be a contiguous CUDA float32 tensor of "
                             f"shape {shp}")
    gg = rt_grid_sph(int(gs.nr), int(gs.nth), int(gs.nph), int(gs.r_log), float(gs.r_in),
                     float(gs.r_out), float(gs.th0), float(gs.th1))
    f = rt_fields_sph(*(getattr(dg, k).data_ptr() for k in DeviceGridSph.FIELDS),
                      int(problem.vturb_mach))
    o, v, vw, ln = _view_line_geom(problem)
    cshape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, cshape, "dL_dcube")
    target = _cube_arg(target, cshape, "target")
    dev = dg.T.device
    cube = None
    if cube_out is True:
        cube = torch.empty(cshape, dtype=torch.float32, device=dev)
    elif cube_out is not None and cube_out is not False:
        cube = _cube_arg(cube_out, cshape, "cube_out")
    out = {k: torch.empty(shp, dtype=torch.float64, device=dev) for k in DeviceGridSph.FIELDS}
    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
    gr = rt_grads3(*(out[k].data_ptr() for k in DeviceGridSph.FIELDS), out["loss"].data_ptr())
    check(lib().rt_render_sph_adjoint(C.byref(gg), C.byref(f), C.byref(o), C.byref(vw),
                                      C.byref(ln), _ptr(dL_dcube), _ptr(target), _ptr(cube),
                                      C.byref(gr), stream_handle(stream)))
    return cube, out


def rt_pack_nodes3(problem, grid=None, out=None, stream=None):
    """Node records of the problem's 3-D grid (Cartesian problem.g3 or spherical problem.gs)
    packed once through rt_pack_nodes3: a CUDA float32 tensor [2][nodes][4] for
    rt_render3d_packed / rt_render_sph_packed."""
    import torch
    sph = getattr(problem, "gs", None) is not None
    if sph:
        dg = grid if grid is not None else DeviceGridSph(problem)
        keys, g = DeviceGridSph.FIELDS, problem.gs
        nodes = int(g.nr) * int(g.nth) * int(g.nph)
    else:
        dg = grid if grid is not None else DeviceGrid3(problem)
        keys, g = DeviceGrid3.FIELDS, problem.g3
        nodes = int(g.nx) * int(g.ny) * int(g.nz)
    for k in keys:
        t = getattr(dg, k)
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != nodes:
            raise ValueError(f"3-D field {k} must be a contiguous CUDA float32 tensor of {nodes} nodes")
    f = rt_fields3(*(getattr(dg, k).data_ptr() for k in keys), int(problem.vturb_mach))
    if out is None:
        out = torch.empty((2, nodes, 4), dtype=torch.float32, device=dg.T.device)
    check(lib().rt_pack_nodes3(C.byref(f), nodes, _ptr(out), stream_handle(stream)))
    return out


def rt_render_packed(problem, records, out=None, stream=None):
    """Forward render through the problem's 3-D grid from records of rt_pack_nodes3
    (rt_render3d_packed or rt_render_sph_packed); returns the cube [nch][ny][nx] float32."""
    import torch
    if not records.is_cuda or not records.is_contiguous() or records.dtype != torch.float32:
        raise ValueError("records must be a contiguous CUDA float32 tensor from rt_pack_nodes3")
    o, v, vw, ln = _view_line_geom(problem)
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=records.device)
    if getattr(problem, "gs", None) is not None:
        gs = problem.gs
        if records.numel() != 8 * int(gs.nr) * int(gs.nth) * int(gs.nph):
            raise ValueError("records do not match the spherical grid")
        gg = rt_grid_sph(int(gs.nr), int(gs.nth), int(gs.nph), int(gs.r_log), float(gs.r_in),
                         float(gs.r_out), float(gs.th0), float(gs.th1))
        check(lib().rt_render_sph_packed(C.byref(gg), _ptr(records), int(problem.vturb_mach),
                                         C.byref(o), C.byref(vw), C.byref(ln), _ptr(out),
                                         stream_handle(stream)))
    else:
        g3 = problem.g3
        if records.numel() != 8 * int(g3.nx) * int(g3.ny) * int(g3.nz):
            raise ValueError("records do not match the 3-D grid")
        gg = rt_grid3(int(g3.nx), int(g3.ny), int(g3.nz), *(float(v) for v in g3.extent))
        check(lib().rt_render3d_packed(C.byref(gg), _ptr(records), int(problem.vturb_mach),
                                       C.byref(o), C.byref(vw), C.byref(ln), _ptr(out),
                                       stream_handle(stream)))
    return out


def rt_render_adjoint_packed(problem, records, dL_dcube=None, target=None, cube_out=True,
                             stream=None):
    """Fused forward + reverse march through the problem's 3-D grid from records of
    rt_pack_nodes3 (rt_render3d_adjoint_packed / rt_render_sph_adjoint_packed). Returns
    (cube or None, grads) as rt_render3d_adjoint / rt_render_sph_adjoint."""
    import torch
    if not records.is_cuda or not records.is_contiguous() or records.dtype != torch.float32:
        raise ValueError("records must be a contiguous CUDA float32 tensor from rt_pack_nodes3")
    sph = getattr(problem, "gs", None) is not None
    if sph:
        gs = problem.gs
        shp = (int(gs.nph), int(gs.nth), int(gs.nr))
        keys = DeviceGridSph.FIELDS
        gg = rt_grid_sph(int(gs.nr), int(gs.nth), int(gs.nph), int(gs.r_log), float(gs.r_in),
                         float(gs.r_out), float(gs.th0), float(gs.th1))
    else:
        g3 = problem.g3
        shp = (int(g3.nz), int(g3.ny), int(g3.nx))
        keys = DeviceGrid3.FIELDS
        gg = rt_grid3(int(g3.nx), int(g3.ny), int(g3.nz), *(float(v) for v in g3.extent))
    if records.numel() != 8 * shp[0] * shp[1] * shp[2]:
        raise ValueError("records do not match the grid")
    o, v, vw, ln = _view_line_geom(problem)
    cshape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, cshape, "dL_dcube")
    target = _cube_arg(target, cshape, "target")
    dev = records.device
    cube = None
    if cube_out is True:
        cube = torch.empty(cshape, dtype=torch.float32, device=dev)
    elif cube_out is not None and cube_out is not False:
        cube = _cube_arg(cube_out, cshape, "cube_out")
    out = {k: torch.empty(shp, dtype=torch.float64, device=dev) for k in keys}
    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
    gr = rt_grads3(*(out[k].data_ptr() for k in keys), out["loss"].data_ptr())
    fn = lib().rt_render_sph_adjoint_packed if sph else lib().rt_render3d_adjoint_packed
    check(fn(C.byref(gg), _ptr(records), int(problem.vturb_mach), C.byref(o), C.byref(vw),
             C.byref(ln), _ptr(dL_dcube), _ptr(target), _ptr(cube), C.byref(gr),
             stream_handle(stream)))
    return cube, out


def rt_render3d(problem, grid=None, out=None, stream=None):
    """Forward render through a 3-D Cartesian grid (problem.g3); returns the cube tensor
    [nch][ny][nx] float32."""
    import torch
    g3 = problem.g3
    dg = grid if grid is not None else DeviceGrid3(problem)
    shp = (int(g3.nz), int(g3.ny), int(g3.nx))
    for k in DeviceGrid3.FIELDS:
        t = getattr(dg, k)
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"3-D field {k} must be a contiguous CUDA float32 tensor of shape {shp}")
    gg = rt_grid3(*shp[::-1], *(float(v) for v in g3.extent))
    f = rt_fields3(*(getattr(dg, k).data_ptr() for k in DeviceGrid3.FIELDS),
                   int(problem.vturb_mach))
    o = rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                float(problem.mstar_msun), float(problem.vsys_kms))
    v = np.ascontiguousarray(np.asarray(problem.v_kms, dtype=np.float32))
    vw = rt_view(int(problem.nx), int(problem.ny), float(problem.half_fov_au), int(v.size),
                 v.ctypes.data_as(C.POINTER(C.c_float)), int(problem.n_samples),
                 float(problem.I0), int(problem.units))
    ln = rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                 float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=dg.T.device)
    check(lib().rt_render3d(C.byref(gg), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                            _ptr(out), stream_handle(stream)))
    return out


def rt_render3d_adjoint(problem, grid=None, dL_dcube=None, target=None, cube_out=True,
                        stream=None):
    """Fused forward + reverse march through a 3-D Cartesian grid (problem.g3), through the C
    ABI. Give exactly one of dL_dcube or target (loss = sum (cube - target)^2). Returns
    (cube or None, grads) with grads a dict of float64 CUDA tensors T, n_h2, vturb, x_co, vx,
    vy, vz [nz][ny][nx] and loss (1 element)."""
    import torch
    g3 = problem.g3
    dg = grid if grid is not None else DeviceGrid3(problem)
    shp = (int(g3.nz), int(g3.ny), int(g3.nx))
    for k in DeviceGrid3.FIELDS:
        t = getattr(dg, k)
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != shp:
            raise ValueError(f"3-D field {k} must be a contiguous CUDA float32 tensor of shape {shp}")
    gg = rt_grid3(*shp[::-1], *(float(v) for v in g3.extent))
    f = rt_fields3(*(getattr(dg, k).data_ptr() for k in DeviceGrid3.FIELDS),
                   int(problem.vturb_mach))
    o, v, vw, ln = _view_line_geom(problem)
    cshape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, cshape, "dL_dcube")
    target = _cube_arg(target, cshape, "target")
    dev = dg.T.device
    cube = None
    if cube_out is True:
        cube = torch.empty(cshape, dtype=torch.float32, device=dev)
    elif cube_out is not None and cube_out is not False:
        cube = _cube_arg(cube_out, cshape, "cube_out")
    out = {k: torch.empty(shp, dtype=torch.float64, device=dev) for k in DeviceGrid3.FIELDS}
    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
    gr = rt_grads3(*(out[k].data_ptr() for k in DeviceGrid3.FIELDS), out["loss"].data_ptr())
    check(lib().rt_render3d_adjoint(C.byref(gg), C.byref(f), C.byref(o), C.byref(vw),
                                    C.byref(ln), _ptr(dL_dcube), _ptr(target), _ptr(cube),
                                    C.byref(gr), stream_handle(stream)))
    return cube, out


class DeviceMLP:
    """Device-resident float32 network (master weights) in the layout of rt_mlp."""

    def __init__(self, w, device="cuda", precision="f16"):
        import torch
        self.precision = {"f16": RT_MLP_F16, "bf16": RT_MLP_BF16}[precision]
        self.B = torch.as_tensor(np.ascontiguousarray(w.B, dtype=np.float32), device=device)
        self.W = [torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device=device)
                  for x in w.W]
        self.b = [torch.as_tensor(np.ascontiguousarray(x, dtype=np.float32), device=device)
                  for x in w.b]
        self.h_scale = float(getattr(w, "h_scale", 0.02))

    def struct(self):
        m = rt_mlp()
        m.n_freq = int(self.B.shape[0])
        m.width = int(self.W[0].shape[0])
        m.hidden = len(self.W) - 1
        m.n_out = int(self.W[-1].shape[0])
        m.B = self.B.data_ptr()
        for i in range(5):
            m.W[i] = self.W[i].data_ptr() if i < len(self.W) else None
            m.b[i] = self.b[i].data_ptr() if i < len(self.b) else None
        m.h_scale = self.h_scale
        m.precision = self.precision
        return m


def rt_mlp_eval(net, xy, out=None, stream=None):
    """Tensor-core (BF16, FP32 accumulate) network outputs [n][4] for inputs xy [n][2]."""
    import torch
    xy = xy.contiguous().float()
    n = xy.shape[0]
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float32, device=xy.device)
    m = net.struct()
    check(lib().rt_mlp_eval(C.byref(m), _ptr(xy), _ptr(out), int(n), stream_handle(stream)))
    return out


def rt_render_mlp(problem, fields, net, out=None, stream=None):
    """Forward render with the tensor-core neural field modulating the grid fields."""
    import torch
    T, n, vt, hlo, hhi = fields.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(fields, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    m = net.struct()
    check(lib().rt_render_mlp(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                              C.byref(m), _ptr(out), stream_handle(stream)))
    return out


def _mlp_grad_buffers(net):
    """float64 CUDA tensors shaped like the network's weights and biases, and their rt_mlp_grads."""
    import torch
    dW = [torch.empty(tuple(w.shape), dtype=torch.float64, device=w.device) for w in net.W]
    db = [torch.empty(tuple(b.shape), dtype=torch.float64, device=b.device) for b in net.b]
    g = rt_mlp_grads()
    for i in range(5):
        g.dW[i] = dW[i].data_ptr() if i < len(dW) else None
        g.db[i] = db[i].data_ptr() if i < len(db) else None
    return dW, db, g


def rt_mlp_backward(net, xy, dout, stream=None):
    """Reverse mode of rt_mlp_eval on the tensor cores: (dW, db) summed over the inputs xy
    [n][2] for dL/d(outputs) dout [n][4] (float64 CUDA tensors shaped like the weights)."""
    xy = xy.contiguous().float()
    dout = dout.contiguous().float()
    dW, db, g = _mlp_grad_buffers(net)
    m = net.struct()
    check(lib().rt_mlp_backward(C.byref(m), _ptr(xy), _ptr(dout), int(xy.shape[0]), C.byref(g),
                                stream_handle(stream)))
    return dW, db


def rt_render_mlp_adjoint(problem, fields, net, dL_dcube=None, target=None, cube_out=True,
                          stream=None):
    """Neural-field render plus its adjoint: (cube or None, grads, (dW, db)) with grads as in
    rt_render_adjoint (w.r.t. the grid fields under the modulation) and the network's
    parameter gradients."""
    import torch
    T, n, vt, hlo, hhi = fields.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(fields, "vphi", None))
    shape = (vw.nch, vw.ny, vw.nx)
    dL_dcube = _cube_arg(dL_dcube, shape, "dL_dcube")
    target = _cube_arg(target, shape, "target")
    dev = T.device
    cube = None
    if cube_out is True:
        cube = torch.empty(shape, dtype=torch.float32, device=dev)
    elif cube_out is not None and cube_out is not False:
        cube = _cube_arg(cube_out, shape, "cube_out")
    out = {k: torch.empty(tuple(t.shape), dtype=torch.float64, device=dev)
           for k, t in zip(DeviceDisk.FIELDS, (T, n, vt, hlo, hhi))}
    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
    gr = rt_grads(out["T"].data_ptr(), out["n_h2"].data_ptr(), out["vturb"].data_ptr(),
                  out["h_lo"].data_ptr(), out["h_hi"].data_ptr(), out["loss"].data_ptr())
    dW, db, mg = _mlp_grad_buffers(net)
    m = net.struct()
    check(lib().rt_render_mlp_adjoint(C.byref(g), C.byref(f), C.byref(o), C.byref(vw),
                                      C.byref(ln), C.byref(m), _ptr(dL_dcube), _ptr(target),
                                      _ptr(cube), C.byref(gr), C.byref(mg),
                                      stream_handle(stream)))
    return cube, out, (dW, db)


def rt_sample_coords(problem, fields, out=None, stream=None):
    """Network inputs (rhat, zhat) of every (pixel, sample): [npix][n_samples][2]."""
    import torch
    T, n, vt, hlo, hhi = fields.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(fields, "vphi", None))
    if out is None:
        out = torch.empty((vw.nx * vw.ny, vw.n_samples, 2), dtype=torch.float32, device=T.device)
    check(lib().rt_sample_coords(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                                 _ptr(out), stream_handle(stream)))
    return out


def rt_render_modulated(problem, fields, mod, h_scale, out=None, stream=None):
    """Forward render with per-sample network outputs mod [npix][n_samples][4]."""
    import torch
    T, n, vt, hlo, hhi = fields.tensors()
    g, f, o, vw, ln, keep = structs(problem, T, n, vt, hlo, hhi,
                                       getattr(fields, "vphi", None))
    if out is None:
        out = torch.empty((vw.nch, vw.ny, vw.nx), dtype=torch.float32, device=T.device)
    mod = mod.contiguous().float()
    check(lib().rt_render_modulated(C.byref(g), C.byref(f), C.byref(o), C.byref(vw), C.byref(ln),
                                    _ptr(mod), float(h_scale), _ptr(out), stream_handle(stream)))
    return out


PIPE_OPS = {"ffma": 0, "ffma2": 1, "ex2": 2, "rsqrt": 3, "lg2": 4, "rcp": 5, "sqrt": 6,
            "tanh": 7, "tanh_f16x2": 8}


def rt_pipe_peak(op: str, iters: int = 8192, stream=None) -> dict:
    """Measured rate of one operation (rt_pipe_peak): results per second per SM, the
    launch's CUDA-event time [ms] and the rate of the per-SM cycle counter [MHz]."""
    r, ms, mhz = C.c_double(), C.c_double(), C.c_double()
    check(lib().rt_pipe_peak(PIPE_OPS[op], int(iters), C.byref(r), C.byref(ms), C.byref(mhz),
                             stream_handle(stream)))
    return {"per_s_sm": r.value, "ms": ms.value, "counter_mhz": mhz.value}


def rt_kernel_timing(on: bool) -> None:
    """Switch the CUDA-event timing of forward march launches on or off (rt_kernel_timing)."""
    check(lib().rt_kernel_timing(1 if on else 0))


def rt_kernel_time() -> tuple:
    """Summed milliseconds and count of the march launches timed since the last read
    (rt_kernel_time)."""
    ms, n = C.c_double(), C.c_int()
    check(lib().rt_kernel_time(C.byref(ms), C.byref(n)))
    return ms.value, n.value


def rt_mlp_status() -> int:
    v = C.c_int()
    check(lib().rt_mlp_status(C.byref(v)))
    return v.value


def version() -> str:
    return lib().rt_version().decode()
