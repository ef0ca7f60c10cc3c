"""FP64 CPU oracle of the scattering-graph voxel path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It wraps ``tursca_oracle.c`` (plain C,
FP64, OpenMP), which shares no code with the CUDA library.

``run(scene)`` returns every intermediate the method defines: quadrature
tables, sun transmittances, the first-order source e1, the matrices K and
K^sun as slot lists (one slot per receiver, source, direction and chain
index), s = K^sun e1, the solution of (I - K) x = s (Eq. flux_system),
the emission split E_i and the detector radiance (final radiance sum of
Sec. 2 integrated over voxel segments).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tursca_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtursca_oracle.so")
_lock = threading.Lock()
_lib = None

SINGLE_SCATTER = 1
NO_SOLVE = 2
ANISO = 4
K_SELF = 0
K_GROUND = 7
MAXDIR = 128
MAXGDIR = 64


class OrcDesc(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
        ("R", C.c_int), ("M", C.c_int), ("coupling", C.c_int), ("S", C.c_int),
        ("albedo", C.c_double),
        ("sza", C.c_double), ("saa", C.c_double), ("vza", C.c_double), ("vaa", C.c_double),
        ("f0", C.c_double),
        ("npx", C.c_int), ("npy", C.c_int),
        ("flags", C.c_int), ("threads", C.c_int),
        ("gmres_tol", C.c_double), ("gmres_restart", C.c_int), ("gmres_maxit", C.c_int),
        ("c_min", C.c_double),
        ("max_couplings", C.c_long),
    ]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class OrcResult(C.Structure):
    _fields_ = [
        ("n_atm", C.c_int), ("n_ground", C.c_int), ("n_nodes", C.c_int),
        ("n_dirs", C.c_int), ("n_gdirs", C.c_int),
        ("dirs", C.c_int * (MAXDIR * 3)),
        ("kmax", C.c_int * MAXDIR),
        ("gdir_nmem", C.c_int * MAXGDIR),
        ("gdir_mem", C.c_int * (MAXGDIR * 4 * 3)),
        ("q_iso", C.c_double * MAXDIR),
        ("q_lamb", C.c_double * MAXGDIR),
        ("q_sun", _dp),
        ("mu_s_lamb", C.c_double),
        ("tsun", _dp), ("e1", _dp),
        ("z_iso", _dp), ("z_sun", _dp),
        ("esc_iso", _dp), ("esc_sun", _dp),
        ("n_slots", C.c_long),
        ("slot_row", _ip), ("slot_col", _ip),
        ("slot_dir", C.POINTER(C.c_int16)), ("slot_k", C.POINTER(C.c_int8)),
        ("slot_dep", _dp), ("slot_depsun", _dp),
        ("slot_val", _dp), ("slot_valsun", _dp),
        ("s", _dp), ("x", _dp),
        ("emis1", _dp), ("emis_sun", _dp), ("emis_ms", _dp),
        ("rad", _dp), ("refl", _dp),
        ("gmres_iters", C.c_int),
        ("rel_resid", C.c_double),
        ("slot_P", _dp),
        ("chain_C", _dp), ("chain_E", _dp),
        ("X", _dp),
        ("arrive", _dp), ("esc_out", _dp),
        ("aniso_iters", C.c_int),
        ("c_min_used", C.c_double),
        ("n_couplings", C.c_long), ("n_kept", C.c_long),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_run.argtypes = [C.POINTER(OrcDesc), _dp, _dp, _dp, C.POINTER(C.POINTER(OrcResult))]
        lib.orc_run.restype = C.c_int
        lib.orc_free.argtypes = [C.POINTER(OrcResult)]
        lib.orc_tau_segment.argtypes = [C.POINTER(OrcDesc), _dp, _dp, _dp, C.c_double, C.c_double]
        lib.orc_tau_segment.restype = C.c_double
        lib.orc_fibonacci.argtypes = [C.c_int, C.c_int, _dp]
        lib.orc_partition.argtypes = [C.POINTER(OrcDesc), _dp, C.c_int, _ip, _dp, _dp]
        lib.orc_partition.restype = C.c_int
        lib.orc_phase_quadrature.argtypes = [C.POINTER(OrcDesc), _dp, _dp, C.POINTER(C.c_int)]
        lib.orc_phase_quadrature.restype = C.c_int
        lib.orc_aniso_rows.argtypes = [C.POINTER(OrcDesc), _dp, _dp, _dp, _dp, _ip, C.c_int, _dp]
        lib.orc_aniso_rows.restype = C.c_int
        lib.orc_result_size.restype = C.c_int
        lib.orc_desc_size.restype = C.c_int
        assert lib.orc_result_size() == C.sizeof(OrcResult), "OrcResult layout mismatch"
        assert lib.orc_desc_size() == C.sizeof(OrcDesc), "OrcDesc layout mismatch"
        _lib = lib
    return _lib


def _desc(sc, flags=0, threads=0, gmres_tol=1e-13):
    d = OrcDesc()
    d.nx, d.ny, d.nz = sc.nx, sc.ny, sc.nz
    d.hx, d.hy, d.hz = sc.hx, sc.hy, sc.hz
    d.R, d.M, d.coupling, d.S = sc.R, sc.M, sc.coupling, sc.n_species
    d.albedo = sc.albedo
    d.sza, d.saa, d.vza, d.vaa = sc.sza, sc.saa, sc.vza, sc.vaa
    d.f0 = sc.f0
    d.npx, d.npy = sc.npx, sc.npy
    d.flags, d.threads = flags, threads
    d.gmres_tol, d.gmres_restart, d.gmres_maxit = gmres_tol, 60, 20000
    d.c_min = getattr(sc, "c_min", 0.0)
    d.max_couplings = int(getattr(sc, "max_couplings", 0))
    return d


def _arr(ptr, n, dtype=np.float64):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def aniso_rows(sc, X: np.ndarray, rows, threads: int = 0) -> np.ndarray:
    """The edge form's fixed-point map F(X) (Eq. flux_system with the arrival
    direction kept) at the receiver rows ``rows``: X is [n_nodes][n_dirs +
    n_gdirs] in FP64 (the oracle's arrival-direction order); returns
    [len(rows)][n_dirs + n_gdirs].  A solution of the series satisfies
    F(X) = X."""
    lib = _load()
    d = _desc(sc, ANISO, threads, 1e-13)
    mu_a = np.ascontiguousarray(sc.mu_a, dtype=np.float64).ravel()
    mu_s = np.ascontiguousarray(sc.mu_s, dtype=np.float64).ravel()
    g = np.ascontiguousarray(sc.g, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    nin = X.shape[1]
    out = np.zeros((len(rows), nin), dtype=np.float64)
    rc = lib.orc_aniso_rows(C.byref(d), mu_a.ctypes.data_as(_dp), mu_s.ctypes.data_as(_dp), g.ctypes.data_as(_dp),
                            X.ctypes.data_as(_dp), rows.ctypes.data_as(_ip), C.c_int(len(rows)),
                            out.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError("oracle rejected the scene (code %d)" % rc)
    return out


def run(sc, flags: int = 0, threads: int = 0, gmres_tol: float = 1e-13) -> dict:
    """Run the whole path on scene ``sc`` (a ``scenes.Scene``) in FP64."""
    lib = _load()
    d = _desc(sc, flags, threads, gmres_tol)
    mu_a = np.ascontiguousarray(sc.mu_a, dtype=np.float64).ravel()
    mu_s = np.ascontiguousarray(sc.mu_s, dtype=np.float64).ravel()
    g = np.ascontiguousarray(sc.g, dtype=np.float64)
    out = C.POINTER(OrcResult)()
    rc = lib.orc_run(C.byref(d), mu_a.ctypes.data_as(_dp), mu_s.ctypes.data_as(_dp), g.ctypes.data_as(_dp),
                     C.byref(out))
    if rc != 0:
        raise ValueError("oracle rejected the scene (code %d)" % rc)
    r = out.contents
    try:
        na, ng, nn, nd, ngd = r.n_atm, r.n_ground, r.n_nodes, r.n_dirs, r.n_gdirs
        ns = r.n_slots
        res = {
            "n_atm": na, "n_ground": ng, "n_nodes": nn, "n_dirs": nd, "n_gdirs": ngd,
            "dirs": np.array(r.dirs[: 3 * nd], dtype=np.int64).reshape(nd, 3),
            "kmax": np.array(r.kmax[:nd], dtype=np.int64),
            "gdir_nmem": np.array(r.gdir_nmem[:ngd], dtype=np.int64),
            "gdir_mem": np.array(r.gdir_mem[: ngd * 12], dtype=np.int64).reshape(ngd, 4, 3),
            "q_iso": np.array(r.q_iso[:nd]),
            "q_lamb": np.array(r.q_lamb[:ngd]),
            "q_sun": _arr(r.q_sun, sc.n_species * nd).reshape(sc.n_species, nd),
            "mu_s_lamb": r.mu_s_lamb,
            "tsun": _arr(r.tsun, nn), "e1": _arr(r.e1, nn),
            "z_iso": _arr(r.z_iso, nn), "z_sun": _arr(r.z_sun, nn),
            "esc_iso": _arr(r.esc_iso, nn), "esc_sun": _arr(r.esc_sun, nn),
            "n_slots": ns,
            "slot_row": _arr(r.slot_row, ns, np.int64), "slot_col": _arr(r.slot_col, ns, np.int64),
            "slot_dir": _arr(r.slot_dir, ns, np.int64), "slot_k": _arr(r.slot_k, ns, np.int64),
            "slot_dep": _arr(r.slot_dep, ns), "slot_depsun": _arr(r.slot_depsun, ns),
            "slot_val": _arr(r.slot_val, ns), "slot_valsun": _arr(r.slot_valsun, ns),
            "s": _arr(r.s, nn),
            "c_min_used": r.c_min_used, "n_couplings": int(r.n_couplings), "n_kept": int(r.n_kept),
        }
        if not flags & NO_SOLVE:
            res.update({
                "x": _arr(r.x, nn),
                "emis1": _arr(r.emis1, na), "emis_sun": _arr(r.emis_sun, na), "emis_ms": _arr(r.emis_ms, na),
                "rad": _arr(r.rad, sc.npx * sc.npy).reshape(sc.npy, sc.npx),
                "refl": _arr(r.refl, sc.npx * sc.npy).reshape(sc.npy, sc.npx),
                "gmres_iters": r.gmres_iters, "rel_resid": r.rel_resid,
            })
            res["emis"] = res["emis1"] + res["emis_sun"] + res["emis_ms"]
            if flags & ANISO and not flags & SINGLE_SCATTER:
                res.update({
                    "X": _arr(r.X, nn * (nd + ngd)).reshape(nn, nd + ngd),
                    "arrive": _arr(r.arrive, nn), "esc_out": _arr(r.esc_out, nn),
                    "aniso_iters": r.aniso_iters,
                })
        return res
    finally:
        lib.orc_free(out)


def tau_segment(sc, mu_e, P, V, tend, lphys) -> float:
    """Optical depth of one straight segment (cell-unit start P, cell-unit
    direction V per unit parameter, parameter range [0, tend], physical length
    per unit parameter lphys), horizontally periodic."""
    lib = _load()
    d = _desc(sc)
    me = np.ascontiguousarray(mu_e, dtype=np.float64).ravel()
    P = np.ascontiguousarray(P, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    return lib.orc_tau_segment(C.byref(d), me.ctypes.data_as(_dp), P.ctypes.data_as(_dp), V.ctypes.data_as(_dp),
                               float(tend), float(lphys))


def partition(sc, kept, ground: bool = False):
    """Quadrature weights of one source that keeps the directions where
    ``kept`` is true (coupling selection): (q_iso, q_sun[S][n_dirs]) for the
    atmospheric set, q_lamb for the ground set (``ground``)."""
    lib = _load()
    d = _desc(sc)
    k = np.ascontiguousarray(kept, dtype=np.int32)
    g = np.ascontiguousarray(sc.g, dtype=np.float64)
    qi = np.zeros(MAXDIR)
    qs = np.zeros(sc.n_species * MAXDIR)
    n = lib.orc_partition(C.byref(d), g.ctypes.data_as(_dp), int(ground), k.ctypes.data_as(_ip),
                          qi.ctypes.data_as(_dp), qs.ctypes.data_as(_dp))
    if len(k) != n:
        raise ValueError("kept has %d entries for %d directions" % (len(k), n))
    if ground:
        return qi[:n]
    return qi[:n], qs[: sc.n_species * n].reshape(sc.n_species, n)


def phase_quadrature(sc) -> np.ndarray:
    """Q[S][n_dirs + n_gdirs][n_dirs]: HG of each species integrated over the
    cell of each atmospheric direction, by arrival direction (atmospheric
    directions, then the ground chains' directions); rows sum to one."""
    lib = _load()
    d = _desc(sc)
    g = np.ascontiguousarray(sc.g, dtype=np.float64)
    buf = np.zeros(sc.n_species * (MAXDIR + MAXGDIR) * MAXDIR)
    nd = C.c_int(0)
    nin = lib.orc_phase_quadrature(C.byref(d), g.ctypes.data_as(_dp), buf.ctypes.data_as(_dp), C.byref(nd))
    return buf[: sc.n_species * nin * nd.value].reshape(sc.n_species, nin, nd.value)


def fibonacci(M: int) -> np.ndarray:
    lib = _load()
    out = np.zeros((M, 3))
    buf = (C.c_double * 3)()
    for m in range(M):
        lib.orc_fibonacci(m, M, buf)
        out[m] = buf[:]
    return out


def csr(res: dict, which: str = "slot_val"):
    """Row-major CSR (rowptr, col, val) of a slot list (slots are row-sorted)."""
    nn = res["n_nodes"]
    rowptr = np.zeros(nn + 1, dtype=np.int64)
    np.add.at(rowptr, res["slot_row"] + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, res["slot_col"], res[which]


def dense(res: dict, which: str = "slot_val") -> np.ndarray:
    nn = res["n_nodes"]
    K = np.zeros((nn, nn))
    np.add.at(K, (res["slot_row"], res["slot_col"]), res[which])
    return K
