"""Python binding of libtursca_gb (C ABI in include/tursca.h).

The functions below carry the C names and only marshal arguments; every step
of the path runs in the library's CUDA kernels.  There is no fallback: if the
shared library is missing or fails to load, every call raises.

``Runner`` strings the stages together for one scene on torch device memory
and the current torch CUDA stream (torch supplies memory and streams only).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtursca_gb.so")

FP64, FP32_REFINE = 0, 1
COUPLING_NONE, COUPLING_WEIGHT = 0, 1
SOLVER_AUTO, SOLVER_NEUMANN, SOLVER_GMRES, SOLVER_CHEBYSHEV = 0, 1, 2, 3

OK, E_INVALID, E_NOMEM, E_CUDA, E_NOT_CONVERGED, E_TIMEOUT, E_STATE, E_UNSUPPORTED = range(8)

F_ROW_PTR, F_COL, F_VAL, F_SLOT_DIR, F_SLOT_K, F_TSUN, F_E1, F_S, F_X, F_EMIS, F_GSUN, F_Q_ISO, F_Q_LAMB, \
    F_Q_SUN, F_DIRS, F_ANISO_X = range(16)


class TurscaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class tursca_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("n_species", C.c_int), ("stencil_radius", C.c_int), ("fib_points", C.c_int),
                ("coupling_mode", C.c_int), ("precision", C.c_int)]


class tursca_geometry(C.Structure):
    _fields_ = [("sza", C.c_double), ("saa", C.c_double), ("vza", C.c_double), ("vaa", C.c_double),
                ("f0", C.c_double), ("npx", C.c_int), ("npy", C.c_int)]


class tursca_request_info(C.Structure):
    _fields_ = [("submit_ms", C.c_double), ("start_ms", C.c_double), ("end_ms", C.c_double),
                ("slot_reused", C.c_int), ("iters", C.c_int), ("rel_resid64", C.c_double), ("status", C.c_int)]


class tursca_server_stats(C.Structure):
    _fields_ = [("budget_bytes", C.c_size_t), ("used_bytes", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("slots", C.c_int), ("busy_slots", C.c_int), ("pending", C.c_int), ("evictions", C.c_int),
                ("slots_built", C.c_int), ("batches", C.c_longlong), ("batched_refinements", C.c_longlong),
                ("max_batch", C.c_int)]


class tursca_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("rel_resid64", C.c_double),
                ("rho_est", C.c_double), ("solver", C.c_int)]


class tursca_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_longlong), ("total_ms", C.c_double)]


class tursca_graph_stats(C.Structure):
    _fields_ = [("n_atm", C.c_int), ("n_ground", C.c_int), ("n_nodes", C.c_int),
                ("n_dirs", C.c_int), ("n_up_dirs", C.c_int), ("n_gdirs", C.c_int), ("n_gmembers", C.c_int),
                ("nnz", C.c_longlong), ("nnz_edges", C.c_longlong), ("n_classes", C.c_int), ("max_row", C.c_int)]


_lib = None
_lock = threading.Lock()
_vp = C.c_void_p


def lib() -> C.CDLL:
    """Load libtursca_gb.so (built by ``build.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtursca_gb.so is not built (run paper_2503_16037_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        st = C.c_int
        sig = {
            "tursca_scene_create": (st, [C.POINTER(tursca_grid_desc), _vp, C.POINTER(_vp)]),
            "tursca_scene_destroy": (st, [_vp]),
            "tursca_set_medium": (st, [_vp, _vp, _vp, C.POINTER(C.c_double), C.c_double]),
            "tursca_build_graph": (st, [_vp]),
            "tursca_assemble_flux": (st, [_vp, C.POINTER(tursca_geometry)]),
            "tursca_solve": (st, [_vp, C.c_double, C.c_int, C.POINTER(tursca_solve_info)]),
            "tursca_solve_with": (st, [_vp, C.c_int, C.c_double, C.c_int, C.POINTER(tursca_solve_info)]),
            "tursca_render_radiance": (st, [_vp, _vp, _vp]),
            "tursca_run": (st, [_vp, _vp, _vp, C.POINTER(C.c_double), C.c_double, C.POINTER(tursca_geometry), C.c_int,
                                C.c_double, C.c_int, _vp, _vp, C.POINTER(tursca_solve_info)]),
            "tursca_adjoint": (st, [_vp, _vp, _vp]),
            "tursca_get": (st, [_vp, C.c_int, _vp, C.c_size_t]),
            "tursca_launch_count": (C.c_longlong, [_vp]),
            "tursca_scene_device_bytes": (C.c_size_t, [_vp]),
            "tursca_server_create": (st, [C.c_size_t, C.c_int, C.POINTER(_vp)]),
            "tursca_server_submit": (st, [_vp, C.POINTER(tursca_grid_desc), C.POINTER(tursca_geometry), _vp, _vp,
                                          C.POINTER(C.c_double), C.c_double, C.c_double, _vp,
                                          C.POINTER(C.c_longlong)]),
            "tursca_server_wait": (st, [_vp, C.c_longlong, C.POINTER(tursca_request_info)]),
            "tursca_server_stats_get": (st, [_vp, C.POINTER(tursca_server_stats)]),
            "tursca_server_configure": (st, [_vp, C.c_int, C.c_double]),
            "tursca_selftest_barrier": (st, [_vp, C.c_int, C.c_int]),
            "tursca_selftest_aniso_contract": (st, [_vp, C.c_int, C.c_int, _vp, _vp]),
            "tursca_server_destroy": (st, [_vp]),
            "tursca_graph_info": (st, [C.POINTER(tursca_grid_desc), C.POINTER(tursca_graph_stats)]),
            "tursca_graph_structure": (st, [C.POINTER(tursca_grid_desc), _vp, _vp, _vp, _vp]),
            "tursca_quadrature": (st, [C.POINTER(tursca_grid_desc), _vp, _vp]),
            "tursca_profile_enable": (st, [_vp, C.c_int]),
            "tursca_set_option": (st, [_vp, C.c_int, C.c_double]),
            "tursca_selection_info": (st, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                           C.POINTER(C.c_longlong)]),
            "tursca_profile_read": (st, [_vp, C.POINTER(tursca_kernel_stat), C.c_int, C.POINTER(C.c_int)]),
            "tursca_csr_solve_noalloc": (st, [_vp, _vp, _vp, C.c_int, _vp, _vp, C.c_int, C.c_int, _vp, _vp]),
            "tursca_selftest_wait": (st, [_vp, C.c_int, C.POINTER(C.c_double)]),
            "tursca_status_string": (C.c_char_p, [C.c_int]),
            "tursca_last_error": (st, [_vp, C.c_char_p, C.c_size_t]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def _err(scene, status: int):
    buf = C.create_string_buffer(512)
    lib().tursca_last_error(scene, buf, 512)
    return TurscaError(status, buf.value.decode() or lib().tursca_status_string(status).decode())


def _check(scene, status: int):
    if status != OK:
        raise _err(scene, status)


def _ptr(a) -> int:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a)


# ---- same-name wrappers ----------------------------------------------------

def tursca_scene_create(desc: tursca_grid_desc, cuda_stream: int = 0):
    out = _vp()
    _check(None, lib().tursca_scene_create(C.byref(desc), cuda_stream or None, C.byref(out)))
    return out


def tursca_scene_destroy(scene):
    _check(None, lib().tursca_scene_destroy(scene))


def tursca_set_medium(scene, mu_abs, mu_sca, g, albedo: float):
    gg = (C.c_double * len(g))(*[float(v) for v in g])
    _check(scene, lib().tursca_set_medium(scene, _ptr(mu_abs), _ptr(mu_sca), gg, float(albedo)))


def tursca_build_graph(scene):
    _check(scene, lib().tursca_build_graph(scene))


def tursca_assemble_flux(scene, geom: tursca_geometry):
    _check(scene, lib().tursca_assemble_flux(scene, C.byref(geom)))


def tursca_solve(scene, rtol: float, max_iter: int) -> tursca_solve_info:
    info = tursca_solve_info()
    _check(scene, lib().tursca_solve(scene, float(rtol), int(max_iter), C.byref(info)))
    return info


def tursca_solve_with(scene, solver: int, rtol: float, max_iter: int) -> tursca_solve_info:
    info = tursca_solve_info()
    _check(scene, lib().tursca_solve_with(scene, int(solver), float(rtol), int(max_iter), C.byref(info)))
    return info


def tursca_render_radiance(scene, radiance, reflectance=None):
    _check(scene, lib().tursca_render_radiance(scene, _ptr(radiance), _ptr(reflectance)))


def tursca_run(scene, mu_abs, mu_sca, g, albedo: float, geom: tursca_geometry, solver: int, rtol: float,
               max_iter: int, radiance, reflectance=None) -> tursca_solve_info:
    gg = (C.c_double * len(g))(*[float(v) for v in g])
    info = tursca_solve_info()
    _check(scene, lib().tursca_run(scene, _ptr(mu_abs), _ptr(mu_sca), gg, float(albedo), C.byref(geom), int(solver),
                                   float(rtol), int(max_iter), _ptr(radiance), _ptr(reflectance), C.byref(info)))
    return info


def tursca_adjoint(scene, dJ_dL, dJ_dmu_abs):
    _check(scene, lib().tursca_adjoint(scene, _ptr(dJ_dL), _ptr(dJ_dmu_abs)))


def tursca_get(scene, which: int, dst, nbytes: int):
    _check(scene, lib().tursca_get(scene, int(which), _ptr(dst), int(nbytes)))


def tursca_launch_count(scene) -> int:
    return int(lib().tursca_launch_count(scene))


OPT_RESIDUAL_FP64 = 1
OPT_GROUP_WARPS = 2
OPT_STAGE_VALUES = 3
OPT_L2_RESIDENT = 4
OPT_GATHER_TILE = 5
OPT_SINGLE_SCATTER = 6
OPT_COUPLING_MIN = 7
OPT_ANISO = 8
OPT_MAX_COUPLINGS = 9
SERVER_BATCH_SOLVES = 1


def tursca_set_option(scene, option: int, value: float):
    _check(scene, lib().tursca_set_option(scene, int(option), float(value)))


def tursca_selftest_barrier(blocks: int, arrive: bool, stream: int = 0) -> int:
    """Status of the batched refinements' barrier self-test (OK or E_TIMEOUT)."""
    return int(lib().tursca_selftest_barrier(C.c_void_p(stream), int(blocks), 1 if arrive else 0))


def tursca_selftest_aniso_contract(scene, which: int, tensor_cores: bool, X, out):
    """Raw dense contraction of the anisotropic mode (0: leave, 1: routing
    denominators) into the device tensor ``out`` ([N][n_atm], float32)."""
    xp = None if X is None else C.c_void_p(X.data_ptr())
    _check(scene, lib().tursca_selftest_aniso_contract(scene, int(which), 1 if tensor_cores else 0, xp,
                                                       C.c_void_p(out.data_ptr())))


def tursca_selection_info(scene) -> dict:
    thr = C.c_double(0.0)
    nc = C.c_longlong(0)
    nk = C.c_longlong(0)
    _check(scene, lib().tursca_selection_info(scene, C.byref(thr), C.byref(nc), C.byref(nk)))
    return {"threshold": thr.value, "n_couplings": nc.value, "n_kept": nk.value}


def tursca_profile_enable(scene, on: bool):
    _check(scene, lib().tursca_profile_enable(scene, 1 if on else 0))


def tursca_profile_read(scene) -> dict:
    arr = (tursca_kernel_stat * 16)()
    n = C.c_int(0)
    _check(scene, lib().tursca_profile_read(scene, arr, 16, C.byref(n)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(n.value)}


def tursca_graph_info(desc: tursca_grid_desc) -> tursca_graph_stats:
    out = tursca_graph_stats()
    _check(None, lib().tursca_graph_info(C.byref(desc), C.byref(out)))
    return out


def tursca_graph_structure(desc: tursca_grid_desc):
    st = tursca_graph_info(desc)
    row_ptr = np.zeros(st.n_nodes + 1, np.int32)
    col = np.zeros(st.nnz, np.int32)
    dr = np.zeros(st.nnz, np.int16)
    k = np.zeros(st.nnz, np.int8)
    _check(None, lib().tursca_graph_structure(C.byref(desc), row_ptr.ctypes.data, col.ctypes.data, dr.ctypes.data,
                                              k.ctypes.data))
    return row_ptr, col, dr, k


def tursca_quadrature(desc: tursca_grid_desc):
    st = tursca_graph_info(desc)
    qi = np.zeros(st.n_dirs)
    ql = np.zeros(st.n_gdirs)
    _check(None, lib().tursca_quadrature(C.byref(desc), qi.ctypes.data, ql.ctypes.data))
    return qi, ql


def tursca_csr_solve_noalloc(row_ptr, col, val, n_nodes: int, s, x, sweeps: int, refinements: int, resid2=None,
                             cuda_stream: int = 0):
    """Allocation-free refined solve on caller device arrays (see tursca.h)."""
    _check(None, lib().tursca_csr_solve_noalloc(_ptr(row_ptr), _ptr(col), _ptr(val), int(n_nodes), _ptr(s), _ptr(x),
                                                int(sweeps), int(refinements), _ptr(resid2), cuda_stream or None))


def tursca_selftest_wait(arrive: bool, cuda_stream: int = 0):
    """(status, seconds) of the bounded-wait self-test; the status is
    returned, not raised."""
    sec = C.c_double(0.0)
    rc = lib().tursca_selftest_wait(C.c_void_p(cuda_stream), int(bool(arrive)), C.byref(sec))
    return int(rc), float(sec.value)


def tursca_status_string(status: int) -> str:
    return lib().tursca_status_string(int(status)).decode()


# ---- helpers ----------------------------------------------------------------

def grid_desc(sc, precision: Optional[int] = None) -> tursca_grid_desc:
    """Descriptor for a ``scenes.Scene``."""
    d = tursca_grid_desc()
    d.nx, d.ny, d.nz = sc.nx, sc.ny, sc.nz
    d.hx, d.hy, d.hz = sc.hx, sc.hy, sc.hz
    d.n_species = sc.n_species
    d.stencil_radius = sc.R
    d.fib_points = sc.M
    d.coupling_mode = sc.coupling
    d.precision = sc.precision if precision is None else precision
    return d


def geometry(sc) -> tursca_geometry:
    g = tursca_geometry()
    g.sza, g.saa, g.vza, g.vaa, g.f0 = sc.sza, sc.saa, sc.vza, sc.vaa, sc.f0
    g.npx, g.npy = sc.npx, sc.npy
    return g


class Runner:
    """One scene on the current CUDA device and torch stream.

    Fields are torch tensors (device or host); results are torch tensors on
    the device.  ``run()`` executes set_medium -> assemble -> solve -> render.
    """

    def __init__(self, sc, precision: Optional[int] = None, stream=None):
        import torch
        self.torch = torch
        self.sc = sc
        self.desc = grid_desc(sc, precision)
        self.dtype = torch.float64 if self.desc.precision == FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.handle = tursca_scene_create(self.desc, self.stream.cuda_stream)
        self.stats = tursca_graph_info(self.desc)
        self.geom = geometry(sc)
        tursca_build_graph(self.handle)
        if getattr(sc, "c_min", 0.0) > 0.0:
            tursca_set_option(self.handle, OPT_COUPLING_MIN, sc.c_min)
        if getattr(sc, "max_couplings", 0) > 0:
            tursca_set_option(self.handle, OPT_MAX_COUPLINGS, sc.max_couplings)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.rad = torch.empty((sc.npy, sc.npx), dtype=self.dtype, device=dev)
        self.refl = torch.empty((sc.npy, sc.npx), dtype=self.dtype, device=dev)
        self.info = None

    def fields(self, device="cuda"):
        t = self.torch
        mu_a = t.as_tensor(np.ascontiguousarray(self.sc.mu_a), dtype=self.dtype).to(device)
        mu_s = t.as_tensor(np.ascontiguousarray(self.sc.mu_s), dtype=self.dtype).to(device)
        return mu_a.contiguous(), mu_s.contiguous()

    def set_medium(self, mu_a, mu_s):
        tursca_set_medium(self.handle, mu_a, mu_s, list(self.sc.g), self.sc.albedo)

    def assemble(self):
        tursca_assemble_flux(self.handle, self.geom)

    def solve(self, rtol=1e-10, max_iter=5000, solver=SOLVER_AUTO):
        self.info = tursca_solve_with(self.handle, solver, rtol, max_iter)
        return self.info

    def render(self, rad=None, refl=None):
        rad = self.rad if rad is None else rad
        refl = self.refl if refl is None else refl
        tursca_render_radiance(self.handle, rad, refl)
        return rad, refl

    def run(self, mu_a, mu_s, rtol=1e-10, max_iter=5000, solver=SOLVER_AUTO):
        """set_medium -> assemble -> solve -> render in one library call."""
        self.info = tursca_run(self.handle, mu_a, mu_s, list(self.sc.g), self.sc.albedo, self.geom, solver, rtol,
                               max_iter, self.rad, self.refl)
        return self.rad, self.refl

    def adjoint(self, dJ_dL):
        """dJ/dmu_abs (per voxel, C order (z, y, x), compute type) for the
        detector-radiance adjoint dJ/dL of the last render."""
        t = self.torch
        dl = t.as_tensor(dJ_dL, dtype=self.dtype, device=self.rad.device).contiguous()
        if dl.numel() != self.rad.numel():
            raise ValueError("dJ_dL must have one entry per detector pixel")
        out = t.empty((self.sc.nz, self.sc.ny, self.sc.nx), dtype=self.dtype, device=self.rad.device)
        tursca_adjoint(self.handle, dl, out)
        return out

    def get(self, which: int, n: int, dtype):
        t = self.torch
        out = t.empty(n, dtype=dtype)
        tursca_get(self.handle, which, out.data_ptr(), out.numel() * out.element_size())
        return out.numpy()

    def launches(self) -> int:
        return tursca_launch_count(self.handle)

    def close(self):
        if self.handle:
            tursca_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class TurscaRender(torch.autograd.Function):
        """Detector radiance of a scene as a differentiable function of the
        per-voxel absorption coefficient: forward runs set_medium ->
        assemble -> solve -> render on the Runner's scene, backward runs the
        library's adjoint (K^T solve and reverse edge march)."""

        @staticmethod
        def forward(ctx, mu_a, runner, mu_s, rtol):
            runner.run(mu_a.detach().contiguous(), mu_s, rtol=rtol)
            ctx.runner = runner
            return runner.rad.clone()

        @staticmethod
        def backward(ctx, grad_rad):
            g = ctx.runner.adjoint(grad_rad.contiguous())
            return g, None, None, None

    return TurscaRender


_TurscaRender = None


def render(mu_a, runner, mu_s, rtol=1e-10):
    """Differentiable detector radiance (see TurscaRender)."""
    global _TurscaRender
    if _TurscaRender is None:
        _TurscaRender = _autograd()
    return _TurscaRender.apply(mu_a, runner, mu_s, rtol)


class Server:
    """Continuous-batching server of scene solves (the tursca_server_* calls):
    requests are queued at once, run on resident slots by the library's
    worker threads, and collected with wait().  Inputs are copied to pinned
    host buffers at submit and kept alive until wait() returns."""

    def __init__(self, budget_bytes: int, workers: int, batch_solves: bool = False):
        import torch
        self.torch = torch
        h = _vp()
        st = lib().tursca_server_create(C.c_size_t(int(budget_bytes)), int(workers), C.byref(h))
        if st != OK:
            raise TurscaError(st, "tursca_server_create failed")
        self.handle = h.value
        self._live = {}
        st = lib().tursca_server_configure(self.handle, SERVER_BATCH_SOLVES, 1.0 if batch_solves else 0.0)
        if st != OK:
            raise TurscaError(st, "tursca_server_configure failed")

    def submit(self, sc, precision: Optional[int] = None, rtol: float = 1e-10, fields=None, out=None) -> int:
        """Queue scene ``sc``; fields = (mu_a, mu_s) tensors (host pinned or
        device) or None to take them from ``sc``; out = radiance tensor or None."""
        t = self.torch
        desc = grid_desc(sc, precision)
        dtype = t.float64 if desc.precision == FP64 else t.float32
        if fields is None:
            mu_a = t.as_tensor(np.ascontiguousarray(sc.mu_a), dtype=dtype).pin_memory()
            mu_s = t.as_tensor(np.ascontiguousarray(sc.mu_s), dtype=dtype).pin_memory()
        else:
            mu_a, mu_s = fields
        if out is None:
            out = t.empty((sc.npy, sc.npx), dtype=dtype).pin_memory()
        g = (C.c_double * len(sc.g))(*[float(v) for v in sc.g])
        geom = geometry(sc)
        tk = C.c_longlong()
        st = lib().tursca_server_submit(self.handle, C.byref(desc), C.byref(geom), _ptr(mu_a), _ptr(mu_s), g,
                                        float(sc.albedo), float(rtol), _ptr(out), C.byref(tk))
        if st != OK:
            raise TurscaError(st, "tursca_server_submit failed")
        self._live[tk.value] = (mu_a, mu_s, out, g, desc, geom)
        return tk.value

    def wait(self, ticket: int):
        info = tursca_request_info()
        st = lib().tursca_server_wait(self.handle, C.c_longlong(ticket), C.byref(info))
        keep = self._live.pop(ticket)
        if st != OK:
            raise TurscaError(st, "request %d failed" % ticket)
        d = {k: getattr(info, k) for k, _ in tursca_request_info._fields_}
        return keep[2], d

    def stats(self) -> dict:
        s = tursca_server_stats()
        _check(None, lib().tursca_server_stats_get(self.handle, C.byref(s)))
        return {k: getattr(s, k) for k, _ in tursca_server_stats._fields_}

    def close(self):
        if self.handle:
            lib().tursca_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

