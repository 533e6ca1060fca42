"""Python binding of the GB300 DDA library (include/dda.h).

Thin ctypes marshalling over the C ABI: every step of the hot path runs in
the CUDA library ``libdda_gb300.so`` built in-tree by ``build.py``.  There is
no CPU fallback: if the library is missing or no GPU is present, the calls
raise.  Functions carry the names of the C entry points; :class:`Context`
bundles them for convenience.

Array conventions (see include/dda.h): composition grids are uint8
``[nz, ny, nx]``; vectors are complex128 ``[R, 3, N]`` with sites in the
grid's row-major scan order; ``khat`` is float ``[R, 3]``; ``e`` is complex
``[R, 3]``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "DdaError", "Precision", "Context", "load_library", "library_path",
    "dda_create", "dda_destroy", "dda_last_error", "dda_set_stream", "dda_set_target", "dda_set_materials",
    "dda_prepare", "dda_get_info", "dda_solve", "dda_solve_device", "dda_matvec", "dda_matvec_device",
    "dda_incident_field", "dda_grad_qabs", "dda_matvec_device_noalloc", "dda_set_schedule", "dda_get_schedule",
    "dda_nearfield", "dda_nearfield_dims", "dda_set_slice_passes", "dda_scattering_directions", "dda_farfield",
    "dda_angular_averages", "dda_mueller", "dda_set_anisotropic_materials", "dda_set_xpass", "dda_get_xpass",
    "dda_set_site_materials", "dda_get_solve_schedule", "dda_set_ypass", "dda_get_ypass",
]

STATUS = {0: "DDA_OK", 1: "DDA_ERR_ARG", 2: "DDA_ERR_CUDA", 3: "DDA_ERR_OOM", 4: "DDA_ERR_SIZE",
          5: "DDA_ERR_NOT_CONVERGED", 6: "DDA_ERR_BREAKDOWN", 7: "DDA_ERR_NONFINITE"}


class Precision:
    FP64 = 0
    FP32_REFINED = 1
    FP32 = 2
    DF64 = 3  # matvec only: double-float arithmetic on complex128 vectors


class DdaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.status_name = STATUS.get(status, str(status))


class dda_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("normal_eq", ctypes.c_int),
                ("x0", ctypes.POINTER(ctypes.c_double)), ("residual_fp64", ctypes.c_int), ("solver", ctypes.c_int)]


class dda_result(ctypes.Structure):
    _fields_ = [("qext", ctypes.c_double), ("qabs", ctypes.c_double), ("qsca", ctypes.c_double),
                ("resid_rel", ctypes.c_double), ("resid_normal_eq", ctypes.c_double), ("iters", ctypes.c_int),
                ("outer_iters", ctypes.c_int), ("matvecs", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["status_name"] = STATUS.get(self.status, str(self.status))
        return d


class dda_info(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("Lx", ctypes.c_int),
                ("Ly", ctypes.c_int), ("Lz", ctypes.c_int), ("ndipoles", ctypes.c_int64), ("ncomp", ctypes.c_int),
                ("aeff_lattice", ctypes.c_double), ("kd", ctypes.c_double), ("x", ctypes.c_double)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load (building first if needed) the in-tree CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not _build.up_to_date():
        if not build_if_missing and not os.path.exists(path):
            raise DdaError(2, f"CUDA library not built: {path}")
        path = _build.build()
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sig = {
        "dda_create": ([ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "dda_destroy": ([vp], ctypes.c_int),
        "dda_last_error": ([vp], ctypes.c_char_p),
        "dda_set_stream": ([vp, vp], ctypes.c_int),
        "dda_set_target": ([vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8)], ctypes.c_int),
        "dda_set_materials": ([vp, ctypes.c_int, _D, ctypes.c_double], ctypes.c_int),
        "dda_set_anisotropic_materials": ([vp, ctypes.c_int, _D, _D, ctypes.c_double], ctypes.c_int),
        "dda_prepare": ([vp, ctypes.c_double, ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "dda_get_info": ([vp, ctypes.POINTER(dda_info)], ctypes.c_int),
        "dda_solve": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.POINTER(dda_opts), _D, ctypes.POINTER(dda_result)],
                      ctypes.c_int),
        "dda_solve_device": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.POINTER(dda_opts), vp,
                              ctypes.POINTER(dda_result)], ctypes.c_int),
        "dda_matvec": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D], ctypes.c_int),
        "dda_matvec_device": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, vp, vp], ctypes.c_int),
        "dda_matvec_device_noalloc": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, vp, vp], ctypes.c_int),
        "dda_incident_field": ([vp, ctypes.c_int, _D, _D, _D], ctypes.c_int),
        "dda_grad_qabs": ([vp, ctypes.c_int, _D, _D, ctypes.POINTER(dda_opts), _D, _D, _D, ctypes.POINTER(dda_result)],
                          ctypes.c_int),
        "dda_set_schedule": ([vp, ctypes.c_int], ctypes.c_int),
        "dda_set_slice_passes": ([vp, ctypes.c_int], ctypes.c_int),
        "dda_scattering_directions": ([ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D, _D,
                                       ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "dda_farfield": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_int, _D, _D, _D], ctypes.c_int),
        "dda_mueller": ([vp, ctypes.c_int, _D, _D, _D, _D, ctypes.c_int, _D, _D, _D, _D], ctypes.c_int),
        "dda_angular_averages": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, ctypes.c_double, _D,
                                  ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "dda_nearfield_dims": ([vp, _D, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "dda_nearfield": ([vp, ctypes.c_int, ctypes.c_int, _D, _D, _D, _D, _D, _D], ctypes.c_int),
        "dda_get_schedule": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                             ctypes.c_int),
        "dda_set_xpass": ([vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "dda_set_site_materials": ([vp, _D, ctypes.c_double], ctypes.c_int),
        "dda_get_solve_schedule": ([vp, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4, ctypes.c_int),
        "dda_set_ypass": ([vp, ctypes.c_int], ctypes.c_int),
        "dda_get_ypass": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "dda_get_xpass": ([vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
                          ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _check(ctx, status: int):
    if status != 0:
        msg = dda_last_error(ctx) if ctx else ""
        raise DdaError(status, msg)


def _rhs(khat, e):
    k = np.ascontiguousarray(np.atleast_2d(np.asarray(khat, dtype=np.float64)))
    ev = np.ascontiguousarray(np.atleast_2d(np.asarray(e, dtype=np.complex128)))
    if k.shape[1] != 3 or ev.shape != k.shape:
        raise ValueError("khat must be (R,3) real and e (R,3) complex")
    return k, ev.view(np.float64).reshape(k.shape[0], 6).copy(), k.shape[0]


SOLVERS = {"bicgstab": 0, "bicgstab2": 1, "qmr": 2}


def _opts(tol=1e-5, maxit=1000, use_graph=True, inner_tol=0.0, max_outer=0, normal_eq=False, x0=None,
          residual_fp64=False, solver="bicgstab"):
    o = dda_opts()
    o.tol = tol
    o.maxit = maxit
    o.use_graph = 1 if use_graph else 0
    o.inner_tol = inner_tol
    o.max_outer = max_outer
    o.normal_eq = 1 if normal_eq else 0
    o.residual_fp64 = 1 if residual_fp64 else 0
    if solver not in SOLVERS:
        raise ValueError(f"solver must be one of {sorted(SOLVERS)}")
    o.solver = SOLVERS[solver]
    keep = None
    if x0 is not None:
        keep = np.ascontiguousarray(x0, dtype=np.complex128).view(np.float64)
        o.x0 = _dptr(keep)
    return o, keep


# ---------------------------------------------------------------- C names --
def dda_create(device: int = 0):
    lib = load_library()
    h = ctypes.c_void_p()
    st = lib.dda_create(device, ctypes.byref(h))
    if st != 0:
        raise DdaError(st, f"dda_create(device={device}) failed (no usable CUDA device?)")
    return h


def dda_destroy(ctx):
    if ctx:
        load_library().dda_destroy(ctx)


def dda_last_error(ctx) -> str:
    msg = load_library().dda_last_error(ctx)
    return msg.decode() if msg else ""


def dda_set_stream(ctx, stream_ptr: int | None):
    _check(ctx, load_library().dda_set_stream(ctx, ctypes.c_void_p(stream_ptr or 0)))


def dda_set_target(ctx, grid: np.ndarray):
    g = np.ascontiguousarray(grid, dtype=np.uint8)
    if g.ndim != 3:
        raise ValueError("grid must be [nz, ny, nx]")
    nz, ny, nx = g.shape
    _check(ctx, load_library().dda_set_target(ctx, nx, ny, nz, g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))))


def dda_set_materials(ctx, m, m_ambient: float = 1.0):
    mm = np.ascontiguousarray(np.atleast_1d(np.asarray(m, dtype=np.complex128)))
    _check(ctx, load_library().dda_set_materials(ctx, mm.size, _dptr(mm.view(np.float64)), float(m_ambient)))


def dda_set_anisotropic_materials(ctx, m_principal, df_angles, m_ambient: float = 1.0):
    """m_principal (ncomp, 3) complex refractive indices along e_1, e_2, e_3;
    df_angles (ncomp, 3) = (theta_DF, phi_DF, beta_DF) in radians."""
    mm = np.ascontiguousarray(np.asarray(m_principal, dtype=np.complex128).reshape(-1, 3))
    aa = np.ascontiguousarray(np.asarray(df_angles, dtype=np.float64).reshape(-1, 3))
    if aa.shape[0] != mm.shape[0]:
        raise ValueError("one (theta_DF, phi_DF, beta_DF) per composition")
    _check(ctx, load_library().dda_set_anisotropic_materials(ctx, mm.shape[0], _dptr(mm.view(np.float64)),
                                                              _dptr(aa), float(m_ambient)))


def dda_set_site_materials(ctx, m_site, m_ambient: float = 1.0):
    """One complex refractive index per occupied site (site order of
    dda_set_target); no limit on the number of distinct values."""
    mm = np.ascontiguousarray(np.asarray(m_site, dtype=np.complex128).ravel())
    N = dda_get_info(ctx)["ndipoles"]
    if mm.size != N:
        raise ValueError(f"{mm.size} indices for {N} occupied sites")
    _check(ctx, load_library().dda_set_site_materials(ctx, _dptr(mm.view(np.float64)), float(m_ambient)))


def dda_prepare(ctx, lambda_vac: float, aeff: float, precision: int = Precision.FP64):
    _check(ctx, load_library().dda_prepare(ctx, float(lambda_vac), float(aeff), int(precision)))


def dda_get_info(ctx) -> dict:
    info = dda_info()
    _check(ctx, load_library().dda_get_info(ctx, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in info._fields_}


def dda_solve(ctx, precision, khat, e, want_P=True, **opts):
    """Returns (results list of dicts, P complex [R,3,N] or None, status)."""
    k, ev, R = _rhs(khat, e)
    N = dda_get_info(ctx)["ndipoles"]
    o, keep = _opts(**opts)
    res = (dda_result * R)()
    P = np.empty((R, 3, N), dtype=np.complex128) if want_P else None
    st = load_library().dda_solve(ctx, int(precision), R, _dptr(k), _dptr(ev), ctypes.byref(o),
                                  _dptr(P.view(np.float64)) if want_P else None, res)
    if st not in (0, 5, 6):
        _check(ctx, st)
    return [r.as_dict() for r in res], P, st


def dda_solve_device(ctx, precision, khat, e, P_out, **opts):
    """P_out: a CUDA tensor (complex128, R*3*N elements) or a raw device pointer."""
    k, ev, R = _rhs(khat, e)
    o, keep = _opts(**opts)
    res = (dda_result * R)()
    ptr = P_out.data_ptr() if hasattr(P_out, "data_ptr") else int(P_out)
    st = load_library().dda_solve_device(ctx, int(precision), R, _dptr(k), _dptr(ev), ctypes.byref(o),
                                         ctypes.c_void_p(ptr), res)
    if st not in (0, 5, 6):
        _check(ctx, st)
    return [r.as_dict() for r in res], st


def dda_matvec(ctx, precision, khat, e, x: np.ndarray) -> np.ndarray:
    k, ev, R = _rhs(khat, e)
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    y = np.empty_like(xx)
    _check(ctx, load_library().dda_matvec(ctx, int(precision), R, _dptr(k), _dptr(ev), _dptr(xx.view(np.float64)),
                                          _dptr(y.view(np.float64))))
    return y


def dda_matvec_device(ctx, precision, khat, e, x_dev, y_dev):
    """x_dev, y_dev: CUDA tensors (complex128 for FP64, complex64 for FP32) or device pointers."""
    k, ev, R = _rhs(khat, e)
    xp = x_dev.data_ptr() if hasattr(x_dev, "data_ptr") else int(x_dev)
    yp = y_dev.data_ptr() if hasattr(y_dev, "data_ptr") else int(y_dev)
    _check(ctx, load_library().dda_matvec_device(ctx, int(precision), R, _dptr(k), _dptr(ev), ctypes.c_void_p(xp),
                                                 ctypes.c_void_p(yp)))


def dda_matvec_device_noalloc(ctx, precision, khat, e, x_dev, y_dev):
    """As dda_matvec_device, but the call allocates no device memory: its
    scratch is a fixed 64 MiB array inside the library (see include/dda.h)."""
    k, ev, R = _rhs(khat, e)
    xp = x_dev.data_ptr() if hasattr(x_dev, "data_ptr") else int(x_dev)
    yp = y_dev.data_ptr() if hasattr(y_dev, "data_ptr") else int(y_dev)
    _check(ctx, load_library().dda_matvec_device_noalloc(ctx, int(precision), R, _dptr(k), _dptr(ev),
                                                         ctypes.c_void_p(xp), ctypes.c_void_p(yp)))


def dda_incident_field(ctx, khat, e) -> np.ndarray:
    k, ev, R = _rhs(khat, e)
    N = dda_get_info(ctx)["ndipoles"]
    E = np.empty((R, 3, N), dtype=np.complex128)
    _check(ctx, load_library().dda_incident_field(ctx, R, _dptr(k), _dptr(ev), _dptr(E.view(np.float64))))
    return E


def dda_grad_qabs(ctx, precision, khat, e, **opts):
    """Returns (dQ/dRe eps [N], dQ/dIm eps [N], P [3,N], (forward result, adjoint result))."""
    k, ev, R = _rhs(khat, e)
    if R != 1:
        raise ValueError("dda_grad_qabs takes one right-hand side")
    N = dda_get_info(ctx)["ndipoles"]
    o, keep = _opts(**opts)
    gre = np.empty(N)
    gim = np.empty(N)
    P = np.empty((3, N), dtype=np.complex128)
    res = (dda_result * 2)()
    _check(ctx, load_library().dda_grad_qabs(ctx, int(precision), _dptr(k), _dptr(ev), ctypes.byref(o), _dptr(gre),
                                             _dptr(gim), _dptr(P.view(np.float64)), res))
    return gre, gim, P, (res[0].as_dict(), res[1].as_dict())


def dda_nearfield_dims(ctx, ext):
    """(dims (x, y, z), offset (x, y, z)) of the extended near-field box."""
    e6 = np.ascontiguousarray(np.asarray(ext, dtype=np.float64).reshape(6))
    d = (ctypes.c_int * 3)()
    o = (ctypes.c_int * 3)()
    _check(ctx, load_library().dda_nearfield_dims(ctx, _dptr(e6), d, o))
    return tuple(d), tuple(o)


def dda_nearfield(ctx, precision, khat, e, P, ext, want_inc=True):
    """E_inc, E_sca on the extended box, each (R, 3, Ne) complex128 (x fastest);
    P (R, 3, N) complex.  Returns (E_inc or None, E_sca, dims, offset)."""
    k, ev, R = _rhs(khat, e)
    dims, off = dda_nearfield_dims(ctx, ext)
    ne = dims[0] * dims[1] * dims[2]
    PP = np.ascontiguousarray(P, dtype=np.complex128)
    if PP.ndim == 2:
        PP = PP[None]
    e6 = np.ascontiguousarray(np.asarray(ext, dtype=np.float64).reshape(6))
    Es = np.empty((R, 3, ne), dtype=np.complex128)
    Ei = np.empty((R, 3, ne), dtype=np.complex128) if want_inc else None
    _check(ctx, load_library().dda_nearfield(ctx, int(precision), R, _dptr(k), _dptr(ev), _dptr(PP.view(np.float64)),
                                             _dptr(e6), _dptr(Ei.view(np.float64)) if want_inc else None,
                                             _dptr(Es.view(np.float64))))
    return Ei, Es, dims, off


def dda_scattering_directions(x: float, eta: float):
    """The guide's scattering directions for angular averages: (theta, phi, omega) arrays."""
    lib = load_library()
    n = ctypes.c_int(0)
    st = lib.dda_scattering_directions(float(x), float(eta), 0, None, None, None, ctypes.byref(n))
    if st != 0:
        raise DdaError(st, "bad x or eta")
    t, p, w = (np.empty(n.value) for _ in range(3))
    _check(None, lib.dda_scattering_directions(float(x), float(eta), n.value, _dptr(t), _dptr(p), _dptr(w),
                                               ctypes.byref(n)))
    return t, p, w


def _khat_P(khat, P):
    k = np.ascontiguousarray(np.atleast_2d(np.asarray(khat, dtype=np.float64)))
    PP = np.ascontiguousarray(P, dtype=np.complex128)
    if PP.ndim == 2:
        PP = PP[None]
    if k.shape[1] != 3 or PP.shape[0] != k.shape[0] or PP.shape[1] != 3:
        raise ValueError("khat (R,3) and P (R,3,N) expected")
    return k, PP, k.shape[0]


def dda_farfield(ctx, precision, khat, P, theta, phi):
    """F (R, ndir, 3) complex128: k^2 (I - n n) sum_j P_j exp(-i k n.r_j) in each RHS's Lab Frame."""
    k, PP, R = _khat_P(khat, P)
    t = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    p = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    F = np.empty((R, t.size, 3), dtype=np.complex128)
    _check(ctx, load_library().dda_farfield(ctx, int(precision), R, _dptr(k), _dptr(PP.view(np.float64)), t.size,
                                            _dptr(t), _dptr(p), _dptr(F.view(np.float64))))
    return F


def dda_mueller(ctx, precision, khat, e01, e02, P, theta, phi):
    """Mueller matrices (ndir, 4, 4) and amplitudes (ndir, 4) complex S1..S4 for
    one incident direction and the two incident states e01, e02; P (2, 3, N)."""
    k = np.ascontiguousarray(np.asarray(khat, dtype=np.float64).reshape(3))
    a = np.ascontiguousarray(np.asarray(e01, dtype=np.complex128).reshape(3))
    b = np.ascontiguousarray(np.asarray(e02, dtype=np.complex128).reshape(3))
    PP = np.ascontiguousarray(P, dtype=np.complex128)
    if PP.shape[0] != 2 or PP.shape[1] != 3:
        raise ValueError("P must be (2, 3, N)")
    t = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    p = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    M = np.empty((t.size, 4, 4))
    S = np.empty((t.size, 4), dtype=np.complex128)
    _check(ctx, load_library().dda_mueller(ctx, int(precision), _dptr(k), _dptr(a.view(np.float64)),
                                           _dptr(b.view(np.float64)), _dptr(PP.view(np.float64)), t.size, _dptr(t),
                                           _dptr(p), _dptr(M), _dptr(S.view(np.float64))))
    return M, S


def dda_angular_averages(ctx, precision, khat, P, eta=0.5):
    """(R, 6) array of Q_sca, <cos>, <cos^2>, g_x, g_y, g_z, and the number of directions used."""
    k, PP, R = _khat_P(khat, P)
    out = np.empty((R, 6))
    n = ctypes.c_int(0)
    _check(ctx, load_library().dda_angular_averages(ctx, int(precision), R, _dptr(k), _dptr(PP.view(np.float64)),
                                                    float(eta), _dptr(out), ctypes.byref(n)))
    return out, n.value


def dda_set_schedule(ctx, zpass: int):
    """Force the complex64 z-pass schedule (0, 1 or 2) or restore autotuning (-1)."""
    _check(ctx, load_library().dda_set_schedule(ctx, int(zpass)))


def dda_set_slice_passes(ctx, on: int):
    """Fused x+y slice passes: -1 timed, 0 never (default), 1 wherever built."""
    _check(ctx, load_library().dda_set_slice_passes(ctx, int(on)))


def dda_get_schedule(ctx, R: int, with_slices: bool = False):
    """The z-pass schedule complex64 matvecs of R RHS use (timed now if
    needed); with_slices=True returns (zpass, slice passes used)."""
    out = ctypes.c_int(-1)
    sl = ctypes.c_int(-1)
    _check(ctx, load_library().dda_get_schedule(ctx, int(R), ctypes.byref(out), ctypes.byref(sl)))
    return (out.value, sl.value) if with_slices else out.value


def dda_set_xpass(ctx, xpass):
    """Force the complex64 x-pass schedules (0 staged rows, 1 + V warp-local
    rows with radix plan V) or restore autotuning (-1): one value for both
    x passes, or an (x-forward, x-inverse) pair."""
    f, i = (xpass, xpass) if np.ndim(xpass) == 0 else xpass
    _check(ctx, load_library().dda_set_xpass(ctx, int(f), int(i)))


def dda_get_xpass(ctx, R: int):
    """(x-forward, x-inverse) schedules complex64 matvecs of R RHS use
    (timed now if needed)."""
    f, i = ctypes.c_int(-1), ctypes.c_int(-1)
    _check(ctx, load_library().dda_get_xpass(ctx, int(R), ctypes.byref(f), ctypes.byref(i)))
    return f.value, i.value


def dda_get_solve_schedule(ctx, R: int):
    """{"zpass", "xfwd", "xinv", "ypass"}: the schedules of the complex64
    matvecs in a solve of R RHS (timed now if needed)."""
    z, f, i, y = ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1), ctypes.c_int(-1)
    _check(ctx, load_library().dda_get_solve_schedule(ctx, int(R), ctypes.byref(z), ctypes.byref(f),
                                                      ctypes.byref(i), ctypes.byref(y)))
    return {"zpass": z.value, "xfwd": f.value, "xinv": i.value, "ypass": y.value}


def dda_set_ypass(ctx, ypass: int):
    """Force the complex64 y-pass radix plan (0 or 1) or restore autotuning (-1)."""
    _check(ctx, load_library().dda_set_ypass(ctx, int(ypass)))


def dda_get_ypass(ctx, R: int):
    """The y-pass radix plan complex64 matvecs of R RHS use (timed now if needed)."""
    y = ctypes.c_int(-1)
    _check(ctx, load_library().dda_get_ypass(ctx, int(R), ctypes.byref(y)))
    return y.value


class Context:
    """Owns one dda_ctx (one GPU)."""

    def __init__(self, device: int = 0):
        self.handle = dda_create(device)

    def close(self):
        if self.handle:
            dda_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_target(self, grid):
        dda_set_target(self.handle, grid)

    def set_materials(self, m, m_ambient=1.0):
        dda_set_materials(self.handle, m, m_ambient)

    def set_anisotropic_materials(self, m_principal, df_angles, m_ambient=1.0):
        dda_set_anisotropic_materials(self.handle, m_principal, df_angles, m_ambient)

    def set_site_materials(self, m_site, m_ambient=1.0):
        dda_set_site_materials(self.handle, m_site, m_ambient)

    def prepare(self, lambda_vac, aeff, precision=Precision.FP64):
        dda_prepare(self.handle, lambda_vac, aeff, precision)

    def prepare_size_parameter(self, x, precision=Precision.FP64):
        """Prepare for size parameter x = 2 pi a_eff / lambda (aeff = 1, lambda = 2 pi / x)."""
        dda_prepare(self.handle, 2.0 * np.pi / x, 1.0, precision)

    def info(self):
        return dda_get_info(self.handle)

    def solve(self, precision, khat, e, want_P=True, **opts):
        return dda_solve(self.handle, precision, khat, e, want_P=want_P, **opts)

    def matvec(self, precision, khat, e, x):
        return dda_matvec(self.handle, precision, khat, e, x)

    def incident_field(self, khat, e):
        return dda_incident_field(self.handle, khat, e)

    def nearfield(self, precision, khat, e, P, ext, want_inc=True):
        return dda_nearfield(self.handle, precision, khat, e, P, ext, want_inc)

    def nearfield_dims(self, ext):
        return dda_nearfield_dims(self.handle, ext)

    def farfield(self, precision, khat, P, theta, phi):
        return dda_farfield(self.handle, precision, khat, P, theta, phi)

    def mueller(self, precision, khat, e01, e02, P, theta, phi):
        return dda_mueller(self.handle, precision, khat, e01, e02, P, theta, phi)

    def angular_averages(self, precision, khat, P, eta=0.5):
        return dda_angular_averages(self.handle, precision, khat, P, eta)

    def set_schedule(self, zpass):
        dda_set_schedule(self.handle, zpass)

    def set_xpass(self, xpass):
        dda_set_xpass(self.handle, xpass)

    def get_xpass(self, R):
        return dda_get_xpass(self.handle, R)

    def get_solve_schedule(self, R):
        return dda_get_solve_schedule(self.handle, R)

    def set_ypass(self, ypass):
        dda_set_ypass(self.handle, ypass)

    def get_ypass(self, R):
        return dda_get_ypass(self.handle, R)

    def set_slice_passes(self, on):
        dda_set_slice_passes(self.handle, on)

    def get_schedule(self, R, with_slices=False):
        return dda_get_schedule(self.handle, R, with_slices)

    def grad_qabs(self, precision, khat, e, **opts):
        return dda_grad_qabs(self.handle, precision, khat, e, **opts)
