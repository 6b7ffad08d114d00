"""Python binding of the C ABI (include/dvm.h), function for function, plus a small
``Solver`` convenience wrapper.  Argument marshalling only: numpy arrays on the host,
raw device pointers (ints) where the ABI takes them.  Every computation happens in the
CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native as _n


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class Handle:
    """Owns a ``dvm_ctx*`` and the input arrays referenced while it is created."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep
        self.n_cell = 0
        self.N = (0, 0, 0)

    def __bool__(self):
        return bool(self.ptr)


def dvm_create(xyz, hex8, bface, bface_group, N, lo, hi, Pr, omega, Kn, format=0,
               precision=0, rank_cap=8, tol=1e-5, cfl=0.5, dt=0.0, stream=0, variant=0,
               max_chunk=0, engine=0, scheme=0):
    L = N_lib()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    hex8 = np.ascontiguousarray(hex8, dtype=np.int64)
    bface = np.ascontiguousarray(bface, dtype=np.int64).reshape(-1, 2)
    bgroup = np.ascontiguousarray(bface_group, dtype=np.int32)
    mesh = _n.dvm_mesh(xyz.shape[0], _dp(xyz), hex8.shape[0], _i64p(hex8), bface.shape[0],
                      _i64p(bface), _i32p(bgroup))
    vg = _n.dvm_vgrid((ctypes.c_int32 * 3)(*[int(v) for v in N_tuple(N)]),
                     (ctypes.c_double * 3)(*[float(v) for v in lo]),
                     (ctypes.c_double * 3)(*[float(v) for v in hi]))
    gas = _n.dvm_gas(float(Pr), float(omega), float(Kn))
    opts = _n.dvm_opts(int(format), int(precision), int(rank_cap), float(tol), float(cfl),
                      float(dt), ctypes.c_void_p(int(stream)), int(variant), int(max_chunk),
                      int(engine), int(scheme))
    out = ctypes.c_void_p()
    _n.check(L.dvm_create(ctypes.byref(out), ctypes.byref(mesh), ctypes.byref(vg),
                         ctypes.byref(gas), ctypes.byref(opts)), "dvm_create")
    h = Handle(out, (xyz, hex8, bface, bgroup))
    h.n_cell = int(hex8.shape[0])
    h.N = N_tuple(N)
    return h


def N_tuple(N):
    return tuple(int(v) for v in N)


def N_lib():
    return _n.load()


def dvm_set_bc(h, group, bc_type, params=None):
    p = np.zeros(8) if params is None else np.ascontiguousarray(params, dtype=np.float64)
    return _n.check(N_lib().dvm_set_bc(h.ptr, int(group), int(bc_type), _dp(p)), "dvm_set_bc")


def dvm_init_maxwellian(h, n, u, T):
    n = np.ascontiguousarray(n, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    return _n.check(N_lib().dvm_init_maxwellian(h.ptr, _dp(n), _dp(u), _dp(T)),
                   "dvm_init_maxwellian")


def dvm_init_f(h, f=None, device_ptr=None):
    """Initial full tensors from a host array ``f`` or a device pointer (int)."""
    L = N_lib()
    if device_ptr is not None:
        return _n.check(L.dvm_init_f(h.ptr, ctypes.cast(ctypes.c_void_p(int(device_ptr)),
                                                       ctypes.POINTER(ctypes.c_double)), 1),
                       "dvm_init_f")
    f = np.ascontiguousarray(f, dtype=np.float64)
    return _n.check(L.dvm_init_f(h.ptr, _dp(f), 0), "dvm_init_f")


def dvm_step(h, nsteps=1, residual=True):
    r = ctypes.c_double(0.0)
    _n.check(N_lib().dvm_step(h.ptr, int(nsteps), ctypes.byref(r) if residual else None),
            "dvm_step")
    return r.value if residual else None


def dvm_moments(h):
    out = np.empty((h.n_cell, 8))
    _n.check(N_lib().dvm_moments(h.ptr, _dp(out)), "dvm_moments")
    return out


def dvm_solve(h, tol, max_steps, check_every=10):
    steps = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    rc = _n.check(N_lib().dvm_solve(h.ptr, float(tol), int(max_steps), int(check_every),
                                   ctypes.byref(steps), ctypes.byref(res)), "dvm_solve")
    return rc == _n.DVM_OK, int(steps.value), float(res.value)


def dvm_get_f(h, cell0=0, ncell=None):
    ncell = h.n_cell - cell0 if ncell is None else ncell
    out = np.empty((ncell,) + tuple(h.N))
    _n.check(N_lib().dvm_get_f(h.ptr, int(cell0), int(ncell), _dp(out)), "dvm_get_f")
    return out


def dvm_get_dt(h):
    v = ctypes.c_double(0.0)
    _n.check(N_lib().dvm_get_dt(h.ptr, ctypes.byref(v)), "dvm_get_dt")
    return v.value


def dvm_get_step_count(h):
    v = ctypes.c_int64(0)
    _n.check(N_lib().dvm_get_step_count(h.ptr, ctypes.byref(v)), "dvm_get_step_count")
    return v.value


def dvm_get_num_faces(h):
    v = ctypes.c_int64(0)
    _n.check(N_lib().dvm_get_num_faces(h.ptr, ctypes.byref(v)), "dvm_get_num_faces")
    return v.value


def dvm_get_geometry(h):
    nf = dvm_get_num_faces(h)
    vol = np.empty(h.n_cell)
    fcell = np.empty((nf, 3), dtype=np.int64)
    fgeo = np.empty((nf, 4))
    _n.check(N_lib().dvm_get_geometry(h.ptr, _dp(vol), _i64p(fcell), _dp(fgeo)),
            "dvm_get_geometry")
    return vol, fcell, fgeo


def dvm_get_ranks(h):
    r = np.empty((h.n_cell, 3), dtype=np.int32)
    _n.check(N_lib().dvm_get_ranks(h.ptr, _i32p(r)), "dvm_get_ranks")
    return r


def dvm_get_launch_config(h):
    g = ctypes.c_int32(0)
    t = (ctypes.c_float * 5)()
    _n.check(N_lib().dvm_get_launch_config(h.ptr, ctypes.byref(g), t), "dvm_get_launch_config")
    return int(g.value), [float(v) for v in t]


def dvm_get_tucker(h, R):
    """Current Tucker state (ranks [nc,3], core [nc,R^3], factors [nc,N_a,R]), host arrays in
    the solver's layout."""
    nc = h.n_cell
    ranks = np.empty((nc, 3), dtype=np.int32)
    core = np.empty((nc, R * R * R))
    fac = [np.empty((nc, h.N[a], R)) for a in range(3)]
    _n.check(N_lib().dvm_get_tucker(h.ptr, _i32p(ranks), _dp(core), _dp(fac[0]), _dp(fac[1]),
                                    _dp(fac[2])), "dvm_get_tucker")
    return ranks, core, fac


def dvm_init_tucker(h, ranks, core, fac):
    """Set the Tucker state from host arrays in the layout of ``dvm_get_tucker``."""
    ranks = np.ascontiguousarray(ranks, dtype=np.int32)
    core = np.ascontiguousarray(core, dtype=np.float64)
    fac = [np.ascontiguousarray(u, dtype=np.float64) for u in fac]
    return _n.check(N_lib().dvm_init_tucker(h.ptr, _i32p(ranks), _dp(core), _dp(fac[0]),
                                            _dp(fac[1]), _dp(fac[2]), 0), "dvm_init_tucker")


def dvm_init_tucker_device(h, ranks_ptr, core_ptr, fac_ptrs):
    """Set the Tucker state from device pointers (ints) in the layout of ``dvm_get_tucker``:
    ranks int32 [nc,3], core float64 [nc,R^3], factors float64 [nc,N_a,R]."""
    v = ctypes.c_void_p
    return _n.check(N_lib().dvm_init_tucker(h.ptr, ctypes.cast(v(int(ranks_ptr)), _n._c_i32p),
                                            ctypes.cast(v(int(core_ptr)), _n._c_dp),
                                            ctypes.cast(v(int(fac_ptrs[0])), _n._c_dp),
                                            ctypes.cast(v(int(fac_ptrs[1])), _n._c_dp),
                                            ctypes.cast(v(int(fac_ptrs[2])), _n._c_dp), 1),
                    "dvm_init_tucker")


def dvm_set_kernel_timing(h, on):
    _n.check(N_lib().dvm_set_kernel_timing(h.ptr, int(bool(on))), "dvm_set_kernel_timing")


def dvm_get_kernel_timing(h):
    """{class name: (total ms, launches)} since timing was switched on."""
    ms = (ctypes.c_double * _n.DVM_KERNEL_CLASSES)()
    nl = (ctypes.c_int64 * _n.DVM_KERNEL_CLASSES)()
    _n.check(N_lib().dvm_get_kernel_timing(h.ptr, ms, nl), "dvm_get_kernel_timing")
    return {name: (float(ms[k]), int(nl[k])) for k, name in enumerate(_n.KERNEL_CLASS_NAMES)}


def dvm_memory(h):
    fb = ctypes.c_size_t(0)
    tb = ctypes.c_size_t(0)
    _n.check(N_lib().dvm_memory(h.ptr, ctypes.byref(fb), ctypes.byref(tb)), "dvm_memory")
    return int(fb.value), int(tb.value)


def dvm_save(h, path):
    return _n.check(N_lib().dvm_save(h.ptr, str(path).encode()), "dvm_save")


def dvm_load(h, path):
    return _n.check(N_lib().dvm_load(h.ptr, str(path).encode()), "dvm_load")


def dvm_full_macro_noalloc(f_ptr, n_cell, N, lo, hi, macro_ptr, stream=0):
    """Macroparameters of n_cell device-resident full tensors (device pointer f_ptr)
    into the device buffer macro_ptr ([n_cell][8] doubles), enqueued on ``stream``;
    the library allocates no device memory for it."""
    vg = _n.dvm_vgrid((ctypes.c_int32 * 3)(*[int(v) for v in N_tuple(N)]),
                      (ctypes.c_double * 3)(*[float(v) for v in lo]),
                      (ctypes.c_double * 3)(*[float(v) for v in hi]))
    return _n.check(N_lib().dvm_full_macro_noalloc(ctypes.c_void_p(int(f_ptr)), int(n_cell),
                                                   ctypes.byref(vg),
                                                   ctypes.c_void_p(int(macro_ptr)),
                                                   ctypes.c_void_p(int(stream))),
                    "dvm_full_macro_noalloc")


def dvm_destroy(h):
    if h.ptr:
        N_lib().dvm_destroy(h.ptr)
        h.ptr = None


def dvm_last_error():
    return N_lib().dvm_last_error().decode(errors="replace")


class Solver:
    """One solve on one workload (``workloads.Workload``): create, set BCs, init."""

    def __init__(self, wl, format=_n.DVM_FORMAT_FULL, precision=_n.DVM_PREC_FP64,
                 rank_cap=None, tol=None, dt=0.0, stream=0, init=True,
                 variant=_n.DVM_VARIANT_AUTO, max_chunk=0, engine=_n.DVM_ENGINE_AUTO,
                 scheme=_n.DVM_SCHEME_EXPLICIT, cfl=None):
        self.wl = wl
        self.h = dvm_create(wl.xyz, wl.hex8, wl.bface, wl.bgroup, wl.N, wl.lo, wl.hi, wl.Pr,
                            wl.omega, wl.Kn, format=format, precision=precision,
                            rank_cap=wl.rank_cap if rank_cap is None else rank_cap,
                            tol=wl.tol if tol is None else tol,
                            cfl=wl.cfl if cfl is None else cfl, dt=dt,
                            stream=stream, variant=variant, max_chunk=max_chunk,
                            engine=engine, scheme=scheme)
        for g, t, p in wl.bcs:
            dvm_set_bc(self.h, g, t, p)
        if init:
            dvm_init_maxwellian(self.h, wl.n0, wl.u0, wl.T0)

    def close(self):
        dvm_destroy(self.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, residual=True):
        return dvm_step(self.h, n, residual)

    def moments(self):
        return dvm_moments(self.h)

    def f(self, cell0=0, ncell=None):
        return dvm_get_f(self.h, cell0, ncell)

    @property
    def dt(self):
        return dvm_get_dt(self.h)


# --------------------------------------------------------------------------
# Serving (continuous batching of steady-state solves)

def _request(wl, format, precision, rank_cap, tol, res_tol, max_steps, check_every, keep,
             scheme=_n.DVM_SCHEME_EXPLICIT, cfl=None):
    xyz = np.ascontiguousarray(wl.xyz, dtype=np.float64)
    hex8 = np.ascontiguousarray(wl.hex8, dtype=np.int64)
    bface = np.ascontiguousarray(wl.bface, dtype=np.int64).reshape(-1, 2)
    bgroup = np.ascontiguousarray(wl.bgroup, dtype=np.int32)
    groups = np.ascontiguousarray([g for g, _, _ in wl.bcs], dtype=np.int32)
    types = np.ascontiguousarray([t for _, t, _ in wl.bcs], dtype=np.int32)
    params = np.ascontiguousarray(np.stack([np.asarray(p, float) for _, _, p in wl.bcs]),
                                  dtype=np.float64)
    n0 = np.ascontiguousarray(wl.n0, dtype=np.float64)
    u0 = np.ascontiguousarray(wl.u0, dtype=np.float64)
    T0 = np.ascontiguousarray(wl.T0, dtype=np.float64)
    keep.extend([xyz, hex8, bface, bgroup, groups, types, params, n0, u0, T0])
    req = _n.dvm_request()
    req.mesh = _n.dvm_mesh(xyz.shape[0], _dp(xyz), hex8.shape[0], _i64p(hex8), bface.shape[0],
                           _i64p(bface), _i32p(bgroup))
    req.vgrid = _n.dvm_vgrid((ctypes.c_int32 * 3)(*[int(v) for v in wl.N]),
                             (ctypes.c_double * 3)(*[float(v) for v in wl.lo]),
                             (ctypes.c_double * 3)(*[float(v) for v in wl.hi]))
    req.gas = _n.dvm_gas(float(wl.Pr), float(wl.omega), float(wl.Kn))
    req.opts = _n.dvm_opts(int(format), int(precision), int(rank_cap), float(tol),
                           float(wl.cfl if cfl is None else cfl), 0.0, None,
                           _n.DVM_VARIANT_AUTO, 0, _n.DVM_ENGINE_AUTO, int(scheme))
    req.n_bc = len(wl.bcs)
    req.bc_group, req.bc_type, req.bc_params = _i32p(groups), _i32p(types), _dp(params)
    req.n0, req.u0, req.T0 = _dp(n0), _dp(u0), _dp(T0)
    req.tol = float(res_tol)
    req.max_steps = int(max_steps)
    req.check_every = int(check_every)
    return req


def dvm_estimate_memory(wl, format=0, precision=0, rank_cap=8, tol=1e-5, scheme=0):
    keep = []
    req = _request(wl, format, precision, rank_cap, tol, 1e-6, 1, 1, keep, scheme=scheme)
    b = ctypes.c_size_t(0)
    _n.check(N_lib().dvm_estimate_memory(ctypes.byref(req), ctypes.byref(b)),
             "dvm_estimate_memory")
    return int(b.value)


class Server:
    """``dvm_server_*``: admits requests by device-memory budget and free slots, runs their
    steps interleaved on separate streams, retires them at their residual target."""

    def __init__(self, hbm_budget, max_slots):
        self.ptr = ctypes.c_void_p()
        _n.check(N_lib().dvm_server_create(ctypes.byref(self.ptr), int(hbm_budget),
                                           int(max_slots)), "dvm_server_create")

    def submit(self, wl, format=0, precision=0, rank_cap=8, tol=1e-5, res_tol=1e-6,
               max_steps=10000, check_every=10, scheme=0, cfl=None):
        keep = []
        req = _request(wl, format, precision, rank_cap, tol, res_tol, max_steps, check_every,
                       keep, scheme=scheme, cfl=cfl)
        t = ctypes.c_int64(0)
        _n.check(N_lib().dvm_server_submit(self.ptr, ctypes.byref(req), ctypes.byref(t)),
                 "dvm_server_submit")
        return int(t.value)

    def run(self, max_seconds):
        p = ctypes.c_int64(0)
        _n.check(N_lib().dvm_server_run(self.ptr, float(max_seconds), ctypes.byref(p)),
                 "dvm_server_run")
        return int(p.value)

    def poll(self, ticket):
        st, steps = ctypes.c_int32(0), ctypes.c_int64(0)
        res, lat = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _n.check(N_lib().dvm_server_poll(self.ptr, int(ticket), ctypes.byref(st),
                                         ctypes.byref(steps), ctypes.byref(res),
                                         ctypes.byref(lat)), "dvm_server_poll")
        return {"state": int(st.value), "steps": int(steps.value), "residual": float(res.value),
                "latency_s": float(lat.value)}

    def error(self, ticket):
        return N_lib().dvm_server_error(self.ptr, int(ticket)).decode(errors="replace")

    def cancel(self, ticket):
        return _n.check(N_lib().dvm_server_cancel(self.ptr, int(ticket)), "dvm_server_cancel")

    def result(self, ticket, n_cell):
        out = np.empty((n_cell, 8))
        _n.check(N_lib().dvm_server_result(self.ptr, int(ticket), _dp(out)), "dvm_server_result")
        return out

    def close(self):
        if self.ptr:
            N_lib().dvm_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dvm_server_create(hbm_budget, max_slots):
    return Server(hbm_budget, max_slots)


def dvm_server_submit(srv, wl, **kw):
    return srv.submit(wl, **kw)


def dvm_server_run(srv, max_seconds):
    return srv.run(max_seconds)


def dvm_server_poll(srv, ticket):
    return srv.poll(ticket)


def dvm_server_result(srv, ticket, n_cell):
    return srv.result(ticket, n_cell)


def dvm_server_error(srv, ticket):
    return srv.error(ticket)


def dvm_server_cancel(srv, ticket):
    return srv.cancel(ticket)


def dvm_server_destroy(srv):
    srv.close()


def dvm_gram_tc(x_ptr, ncell, n, K, c_ptr, status_ptr, stream=0):
    """Tensor-core Gram matrices of ncell device-resident n x K FP32 matrices (device
    pointer x_ptr) into the device buffer c_ptr ([ncell][n][n] doubles); status_ptr is a
    device int the kernel ORs 2 into if a bounded wait runs out.  Enqueued on ``stream``."""
    return _n.check(N_lib().dvm_gram_tc(ctypes.c_void_p(int(x_ptr)), int(ncell), int(n), int(K),
                                        ctypes.c_void_p(int(c_ptr)),
                                        ctypes.c_void_p(int(status_ptr)),
                                        ctypes.c_void_p(int(stream))), "dvm_gram_tc")


def dvm_fault_inject(kind, count=0):
    """Arm a host-side injected failure (``_native.DVM_FAULT_*``); see include/dvm.h."""
    return _n.check(N_lib().dvm_fault_inject(int(kind), int(count)), "dvm_fault_inject")


def dvm_lusgs_wavefronts(nb, forward=True):
    """Schedule of one sweep of the implicit LU-SGS step (host only): ``nb`` is the
    [n_cell, 6] neighbour table (-1 on the boundary).  Returns (order, offsets): the
    cells by wavefront and the wavefront boundaries; see include/dvm.h."""
    nb = np.ascontiguousarray(nb, dtype=np.int32).reshape(-1, 6)
    n = nb.shape[0]
    order = np.empty(n, dtype=np.int32)
    off = np.empty(n + 1, dtype=np.int64)
    nw = ctypes.c_int64(0)
    _n.check(N_lib().dvm_lusgs_wavefronts(n, _i32p(nb), 1 if forward else 0, _i32p(order),
                                          _i64p(off), ctypes.byref(nw)), "dvm_lusgs_wavefronts")
    return order, off[:nw.value + 1].copy()
