"""Thin ctypes binding of libmrcm.so (include/mrcm.h): argument marshalling only.

Every function keeps the C name.  Arrays may be numpy arrays (host) or torch
CUDA tensors (device); the binding passes their data pointers and the
current CUDA stream.  A missing library raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libmrcm.so")
LIBPATH_CHECK = os.path.join(HERE, "libmrcm_check.so")   # the bounds-check build (MRCM_CHECK=1)

MRCM_OK = 0
MRCM_NEUMANN, MRCM_DIRICHLET = 0, 1
MRCM_P0, MRCM_P1 = 0, 1
MRCM_FP64, MRCM_MIXED = 0, 1
MRCM_PARTICULAR_OMEGA, MRCM_PARTICULAR_HAT = 0, 1
ERRORS = {
    -1: "MRCM_ERR_BAD_INPUT", -2: "MRCM_ERR_STATE", -3: "MRCM_ERR_CUDA", -4: "MRCM_ERR_NOT_SPD",
    -5: "MRCM_ERR_NO_CONVERGENCE", -6: "MRCM_ERR_SINGULAR", -7: "MRCM_ERR_UNSUPPORTED",
    -8: "MRCM_ERR_NOMEM", -9: "MRCM_ERR_TIMEOUT", -10: "MRCM_ERR_CHECK",
}


class mrcm_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3)]


class mrcm_bc(C.Structure):
    _fields_ = [("kind", C.c_int * 6), ("value", C.c_double * 6)]


class mrcm_partition(C.Structure):
    _fields_ = [("sub", C.c_int * 3), ("overlap", C.c_int)]


class mrcm_params(C.Structure):
    _fields_ = [("space", C.c_int), ("alpha_basis", C.c_double), ("alpha_smooth", C.c_double),
                ("precision", C.c_int), ("ir_tol", C.c_double), ("max_ir", C.c_int),
                ("particular", C.c_int)]


EXPORTS = ["mrcm_create", "mrcm_create_batch", "mrcm_build_basis", "mrcm_solve_interface",
           "mrcm_smooth", "mrcm_run", "mrcm_fluxes", "mrcm_fluxes_static", "mrcm_set_permeability",
           "mrcm_adjoint", "mrcm_backward", "mrcm_stats", "mrcm_profile", "mrcm_timings", "mrcm_measure_fma_peaks",
           "mrcm_destroy", "mrcm_last_error"]
SLAB_INVERSES = {0: "gauss-jordan", 1: "lu", 2: "gauss-jordan-registers"}
PHASES = ["local_basis", "interface_factor", "interface_refine", "assemble", "smooth", "graph", "interface_lu"]

_lib = None


class MrcmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path=None):
    """Loads the library (raises OSError if it was not built): libmrcm.so, or
    the bounds-check build libmrcm_check.so when the environment has
    MRCM_CHECK=1."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIBPATH_CHECK if os.environ.get("MRCM_CHECK") == "1" else LIBPATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_2404_13811_gb300.build.build()")
    lib = C.CDLL(path)
    vp = C.c_void_p
    lib.mrcm_create.argtypes = [C.POINTER(mrcm_grid), vp, vp, C.POINTER(mrcm_bc),
                                C.POINTER(mrcm_partition), C.POINTER(mrcm_params), C.c_int, vp,
                                C.POINTER(vp)]
    lib.mrcm_create_batch.argtypes = [C.c_int, C.POINTER(mrcm_grid), C.POINTER(vp), C.POINTER(vp),
                                      C.POINTER(mrcm_bc), C.POINTER(mrcm_partition),
                                      C.POINTER(mrcm_params), C.c_int, vp, C.POINTER(vp)]
    for name in ("mrcm_build_basis", "mrcm_solve_interface", "mrcm_destroy"):
        getattr(lib, name).argtypes = [vp]
    lib.mrcm_smooth.argtypes = [vp, C.c_int]
    lib.mrcm_run.argtypes = [vp, C.c_int, C.c_int]
    lib.mrcm_fluxes.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    lib.mrcm_fluxes_static.argtypes = [vp, C.c_int, vp, vp]
    lib.mrcm_set_permeability.argtypes = [vp, vp, C.c_int, C.c_int]
    lib.mrcm_adjoint.argtypes = [vp, vp, vp, vp, C.c_int]
    lib.mrcm_backward.argtypes = [vp, vp, vp, vp]
    lib.mrcm_stats.argtypes = [vp, C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_double), C.c_int]
    lib.mrcm_profile.argtypes = [vp, C.c_int]
    lib.mrcm_timings.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]
    lib.mrcm_last_error.argtypes = [vp]
    lib.mrcm_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name != "mrcm_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(lib, h, rc):
    if rc != MRCM_OK:
        msg = lib.mrcm_last_error(h).decode() if h else ""
        raise MrcmError(rc, msg)


def make_structs(dim, n, h, bc_kind, bc_value, sub, overlap):
    g = mrcm_grid()
    g.dim = dim
    for a in range(dim):
        g.n[a] = int(n[a])
        g.h[a] = float(h[a])
    b = mrcm_bc()
    for s in range(2 * dim):
        b.kind[s] = int(bc_kind[s])
        b.value[s] = float(bc_value[s])
    p = mrcm_partition()
    for a in range(dim):
        p.sub[a] = int(sub[a])
    p.overlap = int(overlap)
    return g, b, p


def make_params(space, alpha_basis, alpha_smooth, precision, ir_tol=1e-12, max_ir=30, particular=0):
    q = mrcm_params()
    q.space = int(space)
    q.alpha_basis = float(alpha_basis)
    q.alpha_smooth = float(alpha_smooth)
    q.precision = int(precision)
    q.ir_tol = float(ir_tol)
    q.max_ir = int(max_ir)
    q.particular = int(particular)
    return q


def _ptr(a):
    """(data pointer, is_device) of a numpy array or torch tensor (C-contiguous float64)."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), bool(a.is_cuda)
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous and a.dtype == np.float64):
        raise ValueError("need a C-contiguous float64 numpy array")
    return a.ctypes.data, False


def mrcm_create(grid, K, f, bc, part, params, device_ptrs, stream):
    lib = load()
    h = C.c_void_p()
    rc = lib.mrcm_create(C.byref(grid), C.c_void_p(K), C.c_void_p(f), C.byref(bc), C.byref(part),
                         C.byref(params), int(device_ptrs), C.c_void_p(stream), C.byref(h))
    if rc != MRCM_OK:
        msg = lib.mrcm_last_error(h).decode() if h.value else ""
        if h.value:
            lib.mrcm_destroy(h)
        raise MrcmError(rc, msg)
    return h


def mrcm_create_batch(grids, Ks, fs, bcs, parts, params, device_ptrs, stream):
    lib = load()
    count = len(grids)
    GA = (mrcm_grid * count)(*grids)
    BA = (mrcm_bc * count)(*bcs)
    PA = (mrcm_partition * count)(*parts)
    KA = (C.c_void_p * count)(*[C.c_void_p(k) for k in Ks])
    FA = (C.c_void_p * count)(*[C.c_void_p(x) for x in fs])
    h = C.c_void_p()
    rc = lib.mrcm_create_batch(count, GA, KA, FA, BA, PA, C.byref(params), int(device_ptrs),
                               C.c_void_p(stream), C.byref(h))
    if rc != MRCM_OK:
        msg = lib.mrcm_last_error(h).decode() if h.value else ""
        if h.value:
            lib.mrcm_destroy(h)
        raise MrcmError(rc, msg)
    return h


def mrcm_build_basis(h):
    lib = load()
    _check(lib, h, lib.mrcm_build_basis(h))


def mrcm_solve_interface(h):
    lib = load()
    _check(lib, h, lib.mrcm_solve_interface(h))


def mrcm_smooth(h, n_steps):
    lib = load()
    _check(lib, h, lib.mrcm_smooth(h, int(n_steps)))


def mrcm_run(h, n_steps, use_graph):
    lib = load()
    _check(lib, h, lib.mrcm_run(h, int(n_steps), int(use_graph)))


def mrcm_fluxes(h, member, u_cellfaces, p_cells):
    """u_cellfaces / p_cells: both numpy (host) or both torch CUDA tensors (device); either may be None."""
    lib = load()
    up, ud = _ptr(u_cellfaces) if u_cellfaces is not None else (None, None)
    pp, pd = _ptr(p_cells) if p_cells is not None else (None, None)
    dev = ud if ud is not None else bool(pd)
    _check(lib, h, lib.mrcm_fluxes(h, int(member), C.c_void_p(up), C.c_void_p(pp), int(dev)))


def mrcm_fluxes_static(h, member, u_cellfaces, p_cells):
    """Device tensors only (either may be None); allocates nothing (see include/mrcm.h)."""
    lib = load()
    up = _ptr(u_cellfaces)[0] if u_cellfaces is not None else None
    pp = _ptr(p_cells)[0] if p_cells is not None else None
    _check(lib, h, lib.mrcm_fluxes_static(h, int(member), C.c_void_p(up), C.c_void_p(pp)))


def mrcm_set_permeability(h, values, is_log):
    """values: K or log K of all members (numpy on the host or a CUDA tensor)."""
    lib = load()
    vp_, dev = _ptr(values)
    _check(lib, h, lib.mrcm_set_permeability(h, C.c_void_p(vp_), int(is_log), int(dev)))


def mrcm_adjoint(h, gp, gu, g_logK):
    """gp / gu (either may be None) and the output g_logK: all numpy or all CUDA tensors."""
    lib = load()
    op, dev = _ptr(g_logK)
    pp = _ptr(gp)[0] if gp is not None else None
    up = _ptr(gu)[0] if gu is not None else None
    _check(lib, h, lib.mrcm_adjoint(h, C.c_void_p(pp), C.c_void_p(up), C.c_void_p(op), int(dev)))


def mrcm_backward(h, dL_du, dL_dp, dL_dlogK):
    """Host (numpy) seeds in (velocity, pressure) order; either may be None."""
    lib = load()
    up = _ptr(dL_du)[0] if dL_du is not None else None
    pp = _ptr(dL_dp)[0] if dL_dp is not None else None
    _check(lib, h, lib.mrcm_backward(h, C.c_void_p(up), C.c_void_p(pp), C.c_void_p(_ptr(dL_dlogK)[0])))


def mrcm_stats(h):
    lib = load()
    ints = (C.c_int * 8)()
    dbl = (C.c_double * 4)()
    _check(lib, h, lib.mrcm_stats(h, ints, 8, dbl, 4))
    return {"subdomains": ints[0], "interface_unknowns": ints[1], "interface_ir_steps": ints[2],
            "local_ir_steps": ints[3], "local_solves": ints[4],
            "slab_inverse": SLAB_INVERSES.get(ints[5], ints[5]), "interface_gmres": bool(ints[6]),
            "slab_inverse_source": {0: "fixed", 1: "cache", 2: "measured"}.get(ints[7], ints[7]),
            "interface_residual": dbl[0],
            "tune_ms": {"gauss-jordan": dbl[1], "lu": dbl[2], "gauss-jordan-registers": dbl[3]}}


def mrcm_profile(h, enable):
    lib = load()
    _check(lib, h, lib.mrcm_profile(h, int(enable)))


def mrcm_timings(h):
    """{phase: (device ms, launches)} since the last mrcm_profile call."""
    lib = load()
    n = len(PHASES)
    ms = (C.c_double * n)()
    ln = (C.c_longlong * n)()
    _check(lib, h, lib.mrcm_timings(h, ms, ln, n))
    return {PHASES[i]: (ms[i], ln[i]) for i in range(n)}


def mrcm_destroy(h):
    lib = load()
    lib.mrcm_destroy(h)


def mrcm_last_error(h):
    return load().mrcm_last_error(h).decode()


def mrcm_measure_fma_peaks(stream=0):
    """(FP32, FP64) FMA throughput of the current device in TFLOP/s."""
    lib = load()
    lib.mrcm_measure_fma_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]
    a, b = C.c_double(), C.c_double()
    rc = lib.mrcm_measure_fma_peaks(C.byref(a), C.byref(b), C.c_void_p(int(stream)))
    _check(lib, None, rc)
    return a.value, b.value
