"""Serving: Python handle of the library's continuous-batching request loop (rt_server_*).

Argument marshalling only: admission, scheduling, streams and completion tracking all run in
the C++ scheduler inside librt_b300.so. The handle keeps the tensors of every unfinished
request alive until the request finishes.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _rt

STATE_NAMES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}
REQ_RENDER, REQ_ADJOINT = 0, 1
FAKE_DEVICE = 1


class rt_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("grid", _rt.rt_grid), ("fields", _rt.rt_fields),
                ("geom", _rt.rt_geom), ("view", _rt.rt_view), ("line", _rt.rt_line),
                ("cube", C.c_void_p), ("dL_dcube", C.c_void_p), ("target", C.c_void_p),
                ("grads", _rt.rt_grads), ("fake_us", C.c_int)]


def _declare(L):
    if getattr(L, "_serve_declared", False):
        return L
    P = C.POINTER
    L.rt_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.c_int, P(C.c_void_p)]
    L.rt_submit.argtypes = [C.c_void_p, P(rt_request), P(C.c_uint64)]
    L.rt_poll.argtypes = [C.c_void_p, C.c_uint64, P(C.c_int), P(C.c_double)]
    L.rt_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_double, P(C.c_int), P(C.c_double)]
    L.rt_cancel.argtypes = [C.c_void_p, C.c_uint64]
    L.rt_request_error.argtypes = [C.c_void_p, C.c_uint64, C.c_char_p, C.c_size_t]
    L.rt_server_stats.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_size_t),
                                  P(C.c_uint64)]
    L.rt_server_destroy.argtypes = [C.c_void_p]
    L.rt_request_device_times.argtypes = [C.c_void_p, C.c_uint64, P(C.c_double), P(C.c_double)]
    for f in ("rt_server_create", "rt_submit", "rt_poll", "rt_wait", "rt_cancel",
              "rt_request_error", "rt_server_stats", "rt_server_destroy",
              "rt_request_device_times"):
        getattr(L, f).restype = C.c_int
    L._serve_declared = True
    return L


def max_overlap(intervals):
    """Largest number of (start, end) intervals that contain a common instant."""
    ev = sorted([(a, 1) for a, _ in intervals] + [(b, -1) for _, b in intervals],
                key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


class Server:
    """Continuous-batching server on the current CUDA device (or a fake device)."""

    def __init__(self, mem_budget_bytes=40 << 30, max_inflight=8, max_queue=4096, fake=False):
        self.L = _declare(_rt.lib())
        h = C.c_void_p()
        _rt.check(self.L.rt_server_create(int(mem_budget_bytes), int(max_inflight),
                                          int(max_queue), FAKE_DEVICE if fake else 0,
                                          C.byref(h)))
        self.h = h
        self.fake = fake
        self._keep = {}

    # -- request construction -------------------------------------------------------------
    def _request(self, kind, problem, fields, cube=None, dL_dcube=None, target=None,
                 grads=None, fake_us=0, keep=()):
        if self.fake:
            g, f, o, vw, ln, v = _fake_structs(problem)
        else:
            if fields is None:
                raise ValueError("fields are required")
            g, f, o, vw, ln, v = _rt.structs(problem, *fields.tensors(),
                                             getattr(fields, "vphi", None))
        r = rt_request()
        r.kind, r.grid, r.fields, r.geom, r.view, r.line = kind, g, f, o, vw, ln
        r.cube, r.dL_dcube, r.target = _addr(cube), _addr(dL_dcube), _addr(target)
        if grads is not None:
            r.grads = _rt.rt_grads(*[_addr(grads.get(k))
                                     for k in ("T", "n_h2", "vturb", "h_lo", "h_hi", "loss",
                                               "vphi")])
        r.fake_us = int(fake_us)
        return r, (v, fields, cube, dL_dcube, target, grads) + tuple(keep)

    def submit(self, req, keep=()):
        t = C.c_uint64()
        _rt.check(self.L.rt_submit(self.h, C.byref(req), C.byref(t)))
        self._keep[t.value] = keep
        return t.value

    def submit_render(self, problem, fields, cube, fake_us=0):
        r, keep = self._request(REQ_RENDER, problem, fields, cube=cube, fake_us=fake_us)
        return self.submit(r, keep)

    def submit_adjoint(self, problem, fields, grads, dL_dcube=None, target=None, cube=None,
                       fake_us=0):
        r, keep = self._request(REQ_ADJOINT, problem, fields, cube=cube, dL_dcube=dL_dcube,
                                target=target, grads=grads, fake_us=fake_us)
        return self.submit(r, keep)

    # -- status ---------------------------------------------------------------------------
    def poll(self, ticket):
        s, lat = C.c_int(), C.c_double()
        _rt.check(self.L.rt_poll(self.h, C.c_uint64(ticket), C.byref(s), C.byref(lat)))
        if s.value >= 2:
            self._keep.pop(ticket, None)
        return STATE_NAMES[s.value], lat.value

    def wait(self, ticket, timeout_ms=60000.0):
        s, lat = C.c_int(), C.c_double()
        rc = self.L.rt_wait(self.h, C.c_uint64(ticket), float(timeout_ms), C.byref(s),
                            C.byref(lat))
        if rc == _rt.RT_ETIMEDOUT:
            raise TimeoutError(self.L.rt_last_error().decode())
        _rt.check(rc)
        self._keep.pop(ticket, None)
        return STATE_NAMES[s.value], lat.value

    def cancel(self, ticket):
        _rt.check(self.L.rt_cancel(self.h, C.c_uint64(ticket)))

    def error(self, ticket):
        buf = C.create_string_buffer(512)
        _rt.check(self.L.rt_request_error(self.h, C.c_uint64(ticket), buf, 512))
        return buf.value.decode()

    def device_times(self, ticket):
        """(start, end) [ms] of a finished request's work on the device, relative to the
        server's creation."""
        a, b = C.c_double(), C.c_double()
        _rt.check(self.L.rt_request_device_times(self.h, C.c_uint64(ticket), C.byref(a),
                                                 C.byref(b)))
        return a.value, b.value

    def stats(self):
        q, r, b, c = C.c_int(), C.c_int(), C.c_size_t(), C.c_uint64()
        _rt.check(self.L.rt_server_stats(self.h, C.byref(q), C.byref(r), C.byref(b), C.byref(c)))
        return dict(queued=q.value, running=r.value, bytes_in_use=b.value, completed=c.value)

    def close(self):
        if self.h:
            self.L.rt_server_destroy(self.h)
            self.h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _fake_structs(problem):
    """Structs with placeholder field pointers (fake device: nothing is dereferenced)."""
    g = _rt.rt_grid(int(problem.nr), int(problem.nz), int(problem.r_log),
                    float(problem.r_in_au), float(problem.r_out_au), float(problem.zr_max))
    f = _rt.rt_fields(16, 16, 16, 16, 16, float(problem.x_co), float(problem.edge_w),
                      int(problem.vturb_mach))
    o = _rt.rt_geom(float(problem.incl_deg), float(problem.pa_deg), float(problem.dist_pc),
                    float(problem.mstar_msun), float(problem.vsys_kms))
    v = np.ascontiguousarray(np.asarray(problem.v_kms, dtype=np.float32))
    vw = _rt.rt_view(int(problem.nx), int(problem.ny), float(problem.half_fov_au), int(v.size),
                     v.ctypes.data_as(C.POINTER(C.c_float)), int(problem.n_samples),
                     float(problem.I0), int(problem.units))
    ln = _rt.rt_line(float(problem.nu0_hz), float(problem.A_ul), float(problem.B_rot_hz),
                     float(problem.m_co_amu), float(problem.m_mol_amu), int(problem.J_u))
    return g, f, o, vw, ln, v


def _addr(x):
    """Device address of a tensor (or an integer placeholder on the fake device)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()
