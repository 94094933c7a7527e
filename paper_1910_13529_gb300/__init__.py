"""Python binding of libpic, the GB300 (sm_103a) relativistic-beam EM PIC step.

Thin ctypes marshalling over the C ABI in include/pic.h: the functions below carry the C
names and arguments; every step of the PIC loop runs in the CUDA kernels of csrc/.  PyTorch
is used only for device memory and streams (see runtime.py).  The first call raises
ImportError if the compiled library is missing -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpic.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_CUDA, PIC_ERR_OOM, PIC_ERR_TIMEOUT, PIC_ERR_STATE, PIC_ERR_CAPACITY = range(8)
STATUS_NAMES = ["PIC_OK", "PIC_ERR_ARG", "PIC_ERR_CFL", "PIC_ERR_CUDA", "PIC_ERR_OOM", "PIC_ERR_TIMEOUT",
                "PIC_ERR_STATE", "PIC_ERR_CAPACITY"]
PIC_SOLVER_YEE, PIC_SOLVER_CUSTOM, PIC_SOLVER_SPECTRAL, PIC_SOLVER_KT, PIC_SOLVER_PSATD = 0, 1, 2, 3, 4
PIC_FILTER_NONE, PIC_FILTER_5PASS = 0, 1
PIC_MAX_M, PIC_MAX_HLEN, PIC_MAX_SPECIES, PIC_DIAG_N = 16, 24, 4, 10
PIC_STATIC_RHO_CELLS = 1 << 20
DIAG_KEYS = ["gauss_max", "gauss_rms", "rho_max", "field_energy", "kinetic", "count", "step", "shifts",
             "status", "interior"]

# exported symbols declared in include/pic.h
EXPORTS = ["pic_create", "pic_destroy", "pic_last_error", "pic_fit_coefficients", "pic_fit_coefficients_b",
           "pic_correction_taps",
           "pic_cfl_dt", "pic_cfl_dt_split", "pic_cfl_dt_kspace", "pic_get_coefficients", "pic_get_coefficients_b", "pic_bind_fields", "pic_bind_species", "pic_gather_push",
           "pic_deposit", "pic_field_advance", "pic_step", "pic_filter_current", "pic_sort", "pic_diag", "pic_rho", "pic_gauss",
           "pic_get_count", "pic_get_state", "pic_sync", "pic_timing", "pic_timing_read", "pic_gauss_static",
           "pic_batch_create", "pic_batch_instance", "pic_batch_step", "pic_batch_destroy", "pic_batch_get_tuning",
           "pic_autotune", "pic_get_tuning", "pic_set_tuning", "pic_adjoint_step",
           "pic_set_state", "pic_get_next_id"]
TIMING_KEYS = ["particles", "deposit", "correction", "fields", "sort", "window", "diag", "filter"]


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class pic_config(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int), ("nz", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("dz", ctypes.c_double), ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dt", ctypes.c_double),
        ("solver", ctypes.c_int), ("M", ctypes.c_int), ("coef", ctypes.POINTER(ctypes.c_double)),
        ("fit_wk", ctypes.c_double), ("fit_n", ctypes.c_double), ("shape", ctypes.c_int),
        ("moving_window", ctypes.c_int), ("inject_species", ctypes.c_int), ("inject_ppc", ctypes.c_int * 3),
        ("rho_bg", ctypes.c_double), ("sort_every", ctypes.c_int), ("current_filter", ctypes.c_int),
        ("coef_b", ctypes.POINTER(ctypes.c_double)), ("precision", ctypes.c_int),
    ]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libpic.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_int64)
    sig = {
        "pic_create": ([ctypes.POINTER(pic_config), ctypes.POINTER(vp)], ctypes.c_int),
        "pic_destroy": ([vp], ctypes.c_int),
        "pic_last_error": ([vp], ctypes.c_char_p),
        "pic_fit_coefficients": ([ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp], ctypes.c_int),
        "pic_fit_coefficients_b": ([ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int,
                                    dp], ctypes.c_int),
        "pic_correction_taps": ([dp, ctypes.c_int, ctypes.c_int, dp], ctypes.c_int),
        "pic_cfl_dt": ([ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int, dp],
                       ctypes.c_int),
        "pic_get_coefficients": ([vp, dp, ip, dp, ip], ctypes.c_int),
        "pic_get_coefficients_b": ([vp, dp, ip], ctypes.c_int),
        "pic_cfl_dt_split": ([ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp,
                              ctypes.c_int, dp], ctypes.c_int),
        "pic_cfl_dt_kspace": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp],
                              ctypes.c_int),
        "pic_bind_fields": ([vp, vp, vp, vp], ctypes.c_int),
        "pic_bind_species": ([vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double], ctypes.c_int),
        "pic_gather_push": ([vp, vp], ctypes.c_int),
        "pic_deposit": ([vp, vp], ctypes.c_int),
        "pic_field_advance": ([vp, vp], ctypes.c_int),
        "pic_step": ([vp, ctypes.c_int, vp], ctypes.c_int),
        "pic_sort": ([vp, vp], ctypes.c_int),
        "pic_filter_current": ([vp, vp], ctypes.c_int),
        "pic_diag": ([vp, dp, vp], ctypes.c_int),
        "pic_rho": ([vp, vp, vp], ctypes.c_int),
        "pic_gauss": ([vp, vp, vp], ctypes.c_int),
        "pic_get_count": ([vp, ctypes.c_int, i64p, vp], ctypes.c_int),
        "pic_get_state": ([vp, i64p, i64p, ip], ctypes.c_int),
        "pic_sync": ([vp, vp], ctypes.c_int),
        "pic_timing": ([vp, ctypes.c_int], ctypes.c_int),
        "pic_timing_read": ([vp, dp, i64p, vp], ctypes.c_int),
        "pic_gauss_static": ([vp, vp, vp], ctypes.c_int),
        "pic_batch_create": ([ctypes.POINTER(pic_config), ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "pic_batch_instance": ([vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "pic_batch_step": ([vp, ctypes.c_int, vp], ctypes.c_int),
        "pic_batch_destroy": ([vp], ctypes.c_int),
        "pic_autotune": ([vp, vp], ctypes.c_int),
        "pic_get_tuning": ([vp, ip, dp, ip], ctypes.c_int),
        "pic_set_tuning": ([vp, ctypes.c_int], ctypes.c_int),
        "pic_adjoint_step": ([vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "pic_batch_get_tuning": ([vp, ip, dp], ctypes.c_int),
        "pic_set_state": ([vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int64], ctypes.c_int),
        "pic_get_next_id": ([vp, i64p], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


class _Lib:
    """libpic, loaded on first use (so that the build module can be imported before it exists);
    a missing library raises ImportError at that point -- there is no fallback."""

    _L = None

    def __getattr__(self, name):
        if _Lib._L is None:
            _Lib._L = _load()
        return getattr(_Lib._L, name)


lib = _Lib()


def _check(st, h=None):
    if st != PIC_OK:
        raise PicError(st, lib.pic_last_error(h).decode())


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- C ABI wrappers ----

def pic_create(cfg: pic_config):
    h = ctypes.c_void_p()
    _check(lib.pic_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def pic_destroy(h):
    _check(lib.pic_destroy(h), h)


def pic_last_error(h=None):
    return lib.pic_last_error(h).decode()


def pic_fit_coefficients(kappa, M=16, wk=0.0, n=0.0):
    C = np.zeros(M)
    _check(lib.pic_fit_coefficients(float(kappa), int(M), float(wk), float(n), _dptr(C)))
    return C


def pic_fit_coefficients_b(kappa, CE, M=16, wk=0.0, n=0.0):
    CE = np.ascontiguousarray(CE, dtype=np.float64)
    C = np.zeros(M)
    _check(lib.pic_fit_coefficients_b(float(kappa), int(M), float(wk), float(n), _dptr(CE), len(CE), _dptr(C)))
    return C


def pic_correction_taps(C, hlen=PIC_MAX_HLEN):
    C = np.ascontiguousarray(C, dtype=np.float64)
    h = np.zeros(2 * hlen + 1)
    _check(lib.pic_correction_taps(_dptr(C), len(C), int(hlen), _dptr(h)))
    return h


def pic_cfl_dt(ndim, dz, dx, dy, C):
    C = np.ascontiguousarray(C, dtype=np.float64)
    out = ctypes.c_double()
    _check(lib.pic_cfl_dt(int(ndim), float(dz), float(dx), float(dy), _dptr(C), len(C), ctypes.byref(out)))
    return out.value


def pic_cfl_dt_split(ndim, dz, dx, dy, CE, CB):
    M = max(len(CE), len(CB))
    CE = np.ascontiguousarray(np.pad(np.asarray(CE, dtype=np.float64), (0, M - len(CE))))
    CB = np.ascontiguousarray(np.pad(np.asarray(CB, dtype=np.float64), (0, M - len(CB))))
    out = ctypes.c_double()
    _check(lib.pic_cfl_dt_split(int(ndim), float(dz), float(dx), float(dy), _dptr(CE), _dptr(CB), M,
                                ctypes.byref(out)))
    return out.value


def pic_cfl_dt_kspace(ndim, solver, dz, dx, dy=1.0):
    out = ctypes.c_double()
    _check(lib.pic_cfl_dt_kspace(int(ndim), int(solver), float(dz), float(dx), float(dy), ctypes.byref(out)))
    return out.value


def pic_get_coefficients_b(h):
    Cb = np.zeros(PIC_MAX_M)
    split = ctypes.c_int()
    _check(lib.pic_get_coefficients_b(h, _dptr(Cb), ctypes.byref(split)), h)
    return Cb, bool(split.value)


def pic_get_coefficients(h):
    C = np.zeros(PIC_MAX_M)
    taps = np.zeros(2 * PIC_MAX_HLEN + 1)
    M, hl = ctypes.c_int(), ctypes.c_int()
    _check(lib.pic_get_coefficients(h, _dptr(C), ctypes.byref(M), _dptr(taps), ctypes.byref(hl)), h)
    return C[:M.value], taps[PIC_MAX_HLEN - hl.value: PIC_MAX_HLEN + hl.value + 1]


def pic_bind_fields(h, E_ptr, B_ptr, J_ptr):
    _check(lib.pic_bind_fields(h, E_ptr, B_ptr, J_ptr), h)


def pic_bind_species(h, s, cell_ptr, off_ptr, u_ptr, id_ptr, n, cap, q, m, w):
    _check(lib.pic_bind_species(h, int(s), cell_ptr, off_ptr, u_ptr, id_ptr, int(n), int(cap), float(q),
                                float(m), float(w)), h)


def pic_gather_push(h, stream):
    _check(lib.pic_gather_push(h, stream), h)


def pic_deposit(h, stream):
    _check(lib.pic_deposit(h, stream), h)


def pic_field_advance(h, stream):
    _check(lib.pic_field_advance(h, stream), h)


def pic_step(h, nsteps, stream):
    _check(lib.pic_step(h, int(nsteps), stream), h)


def pic_sort(h, stream):
    _check(lib.pic_sort(h, stream), h)


def pic_filter_current(h, stream):
    _check(lib.pic_filter_current(h, stream), h)


def pic_diag(h, stream):
    out = np.zeros(PIC_DIAG_N)
    _check(lib.pic_diag(h, _dptr(out), stream), h)
    return dict(zip(DIAG_KEYS, out.tolist()))


def pic_rho(h, rho_ptr, stream):
    _check(lib.pic_rho(h, rho_ptr, stream), h)


def pic_gauss(h, G_ptr, stream):
    _check(lib.pic_gauss(h, G_ptr, stream), h)


def pic_gauss_static(h, G_ptr, stream):
    """pic_gauss without allocating: scratch in a fixed in-library array (grids up to 2^20 nodes)."""
    _check(lib.pic_gauss_static(h, G_ptr, stream), h)


def pic_get_count(h, s, stream):
    n = ctypes.c_int64()
    _check(lib.pic_get_count(h, int(s), ctypes.byref(n), stream), h)
    return n.value


def pic_get_state(h):
    st, sh, pend = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
    _check(lib.pic_get_state(h, ctypes.byref(st), ctypes.byref(sh), ctypes.byref(pend)), h)
    return st.value, sh.value, pend.value


def pic_sync(h, stream):
    _check(lib.pic_sync(h, stream), h)


def pic_timing(h, enable):
    _check(lib.pic_timing(h, int(enable)), h)


def pic_timing_read(h, stream):
    ms = np.zeros(len(TIMING_KEYS))
    n = (ctypes.c_int64 * len(TIMING_KEYS))()
    _check(lib.pic_timing_read(h, _dptr(ms), n, stream), h)
    return dict(zip(TIMING_KEYS, ms.tolist())), dict(zip(TIMING_KEYS, list(n)))


def pic_autotune(h, stream):
    _check(lib.pic_autotune(h, stream), h)


def pic_get_tuning(h):
    v, nv = ctypes.c_int(), ctypes.c_int()
    ms = np.zeros(16)
    _check(lib.pic_get_tuning(h, ctypes.byref(v), _dptr(ms), ctypes.byref(nv)), h)
    return v.value, ms[: nv.value]


def pic_set_tuning(h, variant):
    _check(lib.pic_set_tuning(h, int(variant)), h)


def pic_adjoint_step(h, E_ptr, B_ptr, J_ptr, aE_ptr, aB_ptr, grad_ptr, stream):
    _check(lib.pic_adjoint_step(h, E_ptr, B_ptr, J_ptr, aE_ptr, aB_ptr, grad_ptr, stream), h)


def pic_set_state(h, step, shifts, pending_shift, next_id):
    _check(lib.pic_set_state(h, int(step), int(shifts), int(pending_shift), int(next_id)), h)


def pic_get_next_id(h):
    n = ctypes.c_int64()
    _check(lib.pic_get_next_id(h, ctypes.byref(n)), h)
    return n.value


def pic_batch_get_tuning(b):
    """(variant per stencil class [4], ms per class and variant (4, 3)) of the batched field advance."""
    v = (ctypes.c_int * 4)()
    ms = np.zeros(12)
    _check(lib.pic_batch_get_tuning(b, v, _dptr(ms)))
    return list(v), ms.reshape(4, 3)


def pic_batch_create(cfgs):
    arr = (pic_config * len(cfgs))(*cfgs)
    b = ctypes.c_void_p()
    _check(lib.pic_batch_create(arr, len(cfgs), ctypes.byref(b)))
    return b


def pic_batch_instance(b, i):
    h = ctypes.c_void_p()
    _check(lib.pic_batch_instance(b, int(i), ctypes.byref(h)))
    return h


def pic_batch_step(b, nsteps, stream):
    _check(lib.pic_batch_step(b, int(nsteps), stream))


def pic_batch_destroy(b):
    _check(lib.pic_batch_destroy(b))


def encode_cells(iz, ix, iy, nz, nx):
    """Guarded linear cell index of include/pic.h: (iz + 1) + (nz + 2) (ix + nx iy)."""
    iz, ix, iy = (np.asarray(a, dtype=np.int64) for a in (iz, ix, iy))
    return ((iz + 1) + (nz + 2) * (ix + nx * iy)).astype(np.int32)


def decode_cells(cell, nz, nx):
    cell = np.asarray(cell, dtype=np.int64)
    izg = cell % (nz + 2)
    r = cell // (nz + 2)
    return izg - 1, r % nx, r // nx
