"""Thin ctypes binding of the C-ABI in include/pic.h (libpic.so).

Functions carry the C names (pic_create, pic_add_species, pic_add_laser,
pic_step, pic_diag, ...) and only marshal arguments; every step of the PIC
path runs in the CUDA kernels of libpic.so.  PyTorch supplies device memory
(through the pic_alloc hooks) and the CUDA stream.  There is no CPU
fallback: loading fails loudly when the library or a GPU is missing.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PIC_OK = 0
ERRORS = {-1: "PIC_ERR_ARG", -2: "PIC_ERR_CUDA", -3: "PIC_ERR_OOM", -4: "PIC_ERR_CAPACITY",
          -5: "PIC_ERR_TIMEOUT", -6: "PIC_ERR_NUMERIC", -7: "PIC_ERR_STATE"}
PIC_FP64, PIC_FP32 = 0, 1
PIC_BC_PERIODIC, PIC_BC_OPEN = 0, 1
PIC_SOLVER_PERFECT, PIC_SOLVER_YEE = 0, 1
PIC_LOAD_RANDOM, PIC_LOAD_LATTICE = 0, 1
PIC_LASER_AUTO, PIC_LASER_HARD_SOURCE, PIC_LASER_IN_BOX = 0, 1, 2
PIC_DIAG_EX_LINEOUT, PIC_DIAG_FIELD_ENERGY, PIC_DIAG_CHARGE, PIC_DIAG_SPECTRUM = 0, 1, 2, 3
PIC_DIAG_EMITTANCE, PIC_DIAG_PHASE_X_PX, PIC_DIAG_DENSITY_XY = 4, 5, 6
PIC_DIAG_DIVE_RESIDUAL = 7
PIC_FLAG_TRACK_IDS = 1
COMPONENTS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class pic_alloc(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class pic_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("lambda0", C.c_double), ("x0", C.c_double),
                ("precision", C.c_int), ("bc_x", C.c_int), ("solver", C.c_int),
                ("seed", C.c_uint64),
                ("flags", C.c_uint32), ("max_particles", C.c_int64),
                ("alloc", C.POINTER(pic_alloc)), ("pml", C.c_int)]


class pic_window(C.Structure):
    _fields_ = [("v", C.c_double), ("t_start", C.c_double)]


class pic_profile(C.Structure):
    _fields_ = [("n", C.c_int), ("x", C.POINTER(C.c_double)), ("dens", C.POINTER(C.c_double))]


class pic_laser_opts(C.Structure):
    _fields_ = [("x_focus", C.c_double), ("t_peak", C.c_double), ("mode", C.c_int)]


class pic_diag_args(C.Structure):
    _fields_ = [("gamma_min", C.c_double), ("e_min", C.c_double), ("e_max", C.c_double),
                ("p_min", C.c_double), ("p_max", C.c_double)]


class pic_info(C.Structure):
    _fields_ = [("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("t", C.c_double), ("step", C.c_int64), ("shifts", C.c_int64), ("np", C.c_int64),
                ("capacity", C.c_int64), ("pushed", C.c_int64), ("precision", C.c_int)]


class pic_timing(C.Structure):
    _fields_ = [("ms", C.c_double * 4), ("launches", C.c_int64 * 4), ("kernels", C.c_int64)]


TIMING_GROUPS = ["gather_push_deposit", "field_update", "window_inject_bin", "other"]


class pic_particles(C.Structure):
    _fields_ = [("n", C.c_int64), ("xi", C.POINTER(C.c_double) * 3),
                ("u", C.POINTER(C.c_double) * 3), ("w", C.POINTER(C.c_double)),
                ("id", C.POINTER(C.c_uint32))]


_lib = None
_SIGS = {
    "pic_version": (C.c_char_p, []),
    "pic_last_error": (C.c_char_p, [C.c_void_p]),
    "pic_create": (C.c_int, [C.POINTER(pic_grid), C.c_double, C.POINTER(pic_window),
                             C.POINTER(C.c_void_p)]),
    "pic_add_species": (C.c_int, [C.c_void_p, C.POINTER(pic_profile), C.c_int, C.c_int,
                                  C.c_double, C.c_double, C.c_int]),
    "pic_add_laser": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.POINTER(pic_laser_opts)]),
    "pic_step": (C.c_int, [C.c_void_p, C.c_int]),
    "pic_diag": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t,
                           C.POINTER(pic_diag_args)]),
    "pic_get_info": (C.c_int, [C.c_void_p, C.POINTER(pic_info)]),
    "pic_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "pic_get_field": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "pic_set_field": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "pic_get_particles": (C.c_int, [C.c_void_p, C.POINTER(pic_particles)]),
    "pic_set_particles": (C.c_int, [C.c_void_p, C.POINTER(pic_particles)]),
    "pic_destroy": (C.c_int, [C.c_void_p]),
    "pic_diag_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_size_t,
                                   C.POINTER(pic_diag_args)]),
    "pic_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "pic_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "pic_timing_start": (C.c_int, [C.c_void_p, C.c_int]),
    "pic_timing_read": (C.c_int, [C.c_void_p, C.POINTER(pic_timing)]),
    "pic_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "pic_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "pic_batch_diag": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double),
                                 C.c_size_t, C.POINTER(pic_diag_args)]),
    "pic_batch_destroy": (C.c_int, [C.c_void_p]),
    "pic_batch_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_double)]),
    "pic_set_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "pic_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_char_p, C.POINTER(C.c_int),
                               C.POINTER(C.c_double)]),
}


def library_path():
    return _build.LIB


def lib(build_if_missing=True):
    """Load libpic.so (building it in-tree first if needed); raises if absent."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if build_if_missing and not os.path.exists(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpic.so is not built: run paper_1204_0838_gb300/build.py")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PicError(RuntimeError):
    def __init__(self, code, where, msg=""):
        super().__init__("%s returned %s %s" % (where, ERRORS.get(code, code), msg))
        self.code = code


def _check(rc, where, h=None):
    if rc != PIC_OK:
        msg = ""
        if h:
            m = lib().pic_last_error(h)
            msg = "(" + (m.decode() if m else "") + ")"
        raise PicError(rc, where, msg)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# Device memory and stream from PyTorch
# ---------------------------------------------------------------------------
class TorchMemory:
    """pic_alloc hooks backed by torch.cuda tensors (kept alive until freed)."""

    def __init__(self):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA device required: the library has no CPU path")
        self._torch = torch
        self._live = {}
        self._alloc_cb = _ALLOC_FN(self._alloc)
        self._free_cb = _FREE_FN(self._free)
        self.struct = pic_alloc(self._alloc_cb, self._free_cb, None)

    def _alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda")
        except RuntimeError:
            return None
        self._live[t.data_ptr()] = t
        return t.data_ptr()

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)


def torch_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------------------
# C-named wrappers
# ---------------------------------------------------------------------------
def pic_create(grid, dt=0.0, window=None):
    h = C.c_void_p()
    w = C.byref(window) if window is not None else None
    _check(lib().pic_create(C.byref(grid), float(dt), w, C.byref(h)), "pic_create")
    return h


def pic_add_species(h, prof_x, prof_n, ppc, spline_order=3, q=-1.0, m=1.0,
                    loading=PIC_LOAD_RANDOM):
    px = np.ascontiguousarray(prof_x, dtype=np.float64)
    pn = np.ascontiguousarray(prof_n, dtype=np.float64)
    prof = pic_profile(len(px), _dp(px), _dp(pn))
    _check(lib().pic_add_species(h, C.byref(prof), int(ppc), int(spline_order), float(q),
                                 float(m), int(loading)), "pic_add_species", h)


def pic_add_laser(h, a0, waist, duration_fwhm, lambda0, x_focus=0.0, t_peak=0.0,
                  mode=PIC_LASER_AUTO):
    opts = pic_laser_opts(float(x_focus), float(t_peak), int(mode))
    _check(lib().pic_add_laser(h, float(a0), float(waist), float(duration_fwhm), float(lambda0),
                               C.byref(opts)), "pic_add_laser", h)


def pic_step(h, n=1):
    _check(lib().pic_step(h, int(n)), "pic_step", h)


def pic_diag(h, kind, length=1, gamma_min=0.0, e_min=0.0, e_max=0.0, p_min=0.0, p_max=0.0):
    out = np.zeros(max(int(length), 1))
    a = pic_diag_args(float(gamma_min), float(e_min), float(e_max), float(p_min), float(p_max))
    _check(lib().pic_diag(h, int(kind), _dp(out), out.size, C.byref(a)), "pic_diag", h)
    return out


def pic_diag_noalloc(h, kind, length=1, gamma_min=0.0, e_min=0.0, e_max=0.0):
    """pic_diag without any device allocation (scratch in a fixed device array)."""
    out = np.zeros(max(int(length), 1))
    a = pic_diag_args(float(gamma_min), float(e_min), float(e_max), 0.0, 0.0)
    _check(lib().pic_diag_noalloc(h, int(kind), _dp(out), out.size, C.byref(a)), "pic_diag_noalloc", h)
    return out


def pic_get_info(h):
    i = pic_info()
    _check(lib().pic_get_info(h, C.byref(i)), "pic_get_info", h)
    return {f: getattr(i, f) for f, _ in pic_info._fields_}


def pic_set_stream(h, stream):
    _check(lib().pic_set_stream(h, stream), "pic_set_stream", h)


def pic_get_field(h, comp, shape):
    out = np.zeros(shape, dtype=np.float64)
    _check(lib().pic_get_field(h, int(comp), _dp(out)), "pic_get_field", h)
    return out


def pic_set_field(h, comp, arr):
    a = np.ascontiguousarray(arr, dtype=np.float64)
    _check(lib().pic_set_field(h, int(comp), _dp(a)), "pic_set_field", h)


def pic_get_particles(h, capacity=None):
    if capacity is None:
        capacity = pic_get_info(h)["np"]
    n = int(capacity)
    xi = np.zeros((3, max(n, 1)))
    u = np.zeros((3, max(n, 1)))
    w = np.zeros(max(n, 1))
    ids = np.zeros(max(n, 1), dtype=np.uint32)
    p = pic_particles()
    p.n = n
    for c in range(3):
        p.xi[c] = _dp(xi[c])
        p.u[c] = _dp(u[c])
    p.w = _dp(w)
    p.id = ids.ctypes.data_as(C.POINTER(C.c_uint32))
    _check(lib().pic_get_particles(h, C.byref(p)), "pic_get_particles", h)
    m = p.n
    return {"xi": xi[:, :m].copy(), "u": u[:, :m].copy(), "w": w[:m].copy(), "id": ids[:m].copy()}


def pic_set_particles(h, xi, u, w, ids=None):
    xi = [np.ascontiguousarray(xi[c], dtype=np.float64) for c in range(3)]
    u = [np.ascontiguousarray(u[c], dtype=np.float64) for c in range(3)]
    w = np.ascontiguousarray(w, dtype=np.float64)
    p = pic_particles()
    p.n = len(w)
    for c in range(3):
        p.xi[c] = _dp(xi[c])
        p.u[c] = _dp(u[c])
    p.w = _dp(w)
    if ids is not None:
        ids = np.ascontiguousarray(ids, dtype=np.uint32)
        p.id = ids.ctypes.data_as(C.POINTER(C.c_uint32))
    _check(lib().pic_set_particles(h, C.byref(p)), "pic_set_particles", h)


def pic_save(h, path):
    _check(lib().pic_save(h, str(path).encode()), "pic_save", h)


def pic_load(h, path):
    _check(lib().pic_load(h, str(path).encode()), "pic_load", h)


def pic_timing_start(h, enable=True):
    _check(lib().pic_timing_start(h, 1 if enable else 0), "pic_timing_start", h)


def pic_timing_read(h):
    t = pic_timing()
    _check(lib().pic_timing_read(h, C.byref(t)), "pic_timing_read", h)
    return {"ms": {TIMING_GROUPS[i]: t.ms[i] for i in range(4)},
            "launches": {TIMING_GROUPS[i]: t.launches[i] for i in range(4)},
            "kernels": t.kernels}


def pic_destroy(h):
    if h:
        _check(lib().pic_destroy(h), "pic_destroy")


def pic_batch_create(handles):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    b = C.c_void_p()
    _check(lib().pic_batch_create(len(handles), arr, C.byref(b)), "pic_batch_create")
    return b


def pic_batch_step(b, n=1):
    _check(lib().pic_batch_step(b, int(n)), "pic_batch_step")


def pic_batch_diag(b, instance, kind, length=1, gamma_min=0.0, e_min=0.0, e_max=0.0):
    out = np.zeros(max(int(length), 1))
    a = pic_diag_args(float(gamma_min), float(e_min), float(e_max), 0.0, 0.0)
    _check(lib().pic_batch_diag(b, int(instance), int(kind), _dp(out), out.size, C.byref(a)),
           "pic_batch_diag")
    return out


def pic_batch_info(b):
    g, k, ms = C.c_int64(), C.c_int64(), C.c_double()
    _check(lib().pic_batch_info(b, C.byref(g), C.byref(k), C.byref(ms)), "pic_batch_info")
    return {"graph_launches": g.value, "kernel_launches": k.value, "last_step_ms": ms.value}


def pic_set_tiles(h, tx, ty, tz):
    _check(lib().pic_set_tiles(h, int(tx), int(ty), int(tz)), "pic_set_tiles", h)


def pic_autotune(h, steps=2, cache_path=None):
    t = (C.c_int * 3)()
    ms = C.c_double()
    cp = cache_path.encode() if cache_path else None
    _check(lib().pic_autotune(h, int(steps), cp, t, C.byref(ms)), "pic_autotune", h)
    return (t[0], t[1], t[2]), ms.value


def pic_batch_destroy(b):
    if b:
        _check(lib().pic_batch_destroy(b), "pic_batch_destroy")


# ---------------------------------------------------------------------------
# Convenience object
# ---------------------------------------------------------------------------
class Sim:
    """One simulation on the GPU; SI set-up, normalised state accessors."""

    def __init__(self, nx, ny, nz, dx, dy, dz, lambda0, x0=0.0, periodic_x=True,
                 precision="fp64", seed=12040838, dt=0.0, window=None, track_ids=False,
                 max_particles=0, use_torch=True, solver="perfect", pml=0, memory=None):
        # memory: an object with a pic_alloc `struct` (default: TorchMemory)
        self._mem = memory if memory is not None else (TorchMemory() if use_torch else None)
        g = pic_grid(nx, ny, nz, dx, dy, dz, lambda0, x0,
                     PIC_FP64 if precision == "fp64" else PIC_FP32,
                     PIC_BC_PERIODIC if periodic_x else PIC_BC_OPEN,
                     PIC_SOLVER_YEE if solver == "yee" else PIC_SOLVER_PERFECT, seed,
                     PIC_FLAG_TRACK_IDS if track_ids else 0, int(max_particles),
                     C.pointer(self._mem.struct) if self._mem else None, int(pml))
        w = pic_window(window[0], window[1]) if window is not None else None
        self.h = pic_create(g, dt, w)
        self.shape = (nx, ny, nz)
        if use_torch:
            pic_set_stream(self.h, torch_stream())

    def close(self):
        if getattr(self, "h", None):
            pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_species(self, prof_x, prof_n, ppc, q=-1.0, m=1.0, loading="random"):
        pic_add_species(self.h, prof_x, prof_n, ppc, 3, q, m,
                        PIC_LOAD_LATTICE if loading == "lattice" else PIC_LOAD_RANDOM)

    def add_laser(self, a0, waist, fwhm, lambda_l, x_focus=0.0, t_peak=None, mode="auto"):
        modes = {"auto": PIC_LASER_AUTO, "hard_source": PIC_LASER_HARD_SOURCE,
                 "in_box": PIC_LASER_IN_BOX}
        pic_add_laser(self.h, a0, waist, fwhm, lambda_l, x_focus,
                      2 * fwhm if t_peak is None else t_peak, modes[mode])

    def step(self, n=1):
        pic_step(self.h, n)

    def info(self):
        return pic_get_info(self.h)

    def field(self, comp):
        return pic_get_field(self.h, comp, self.shape)

    def fields(self):
        return np.stack([self.field(c) for c in range(9)])

    def set_field(self, comp, arr):
        pic_set_field(self.h, comp, np.broadcast_to(arr, self.shape))

    def set_fields(self, arr):
        for c in range(9):
            self.set_field(c, arr[c])

    def particles(self):
        return pic_get_particles(self.h)

    def set_particles(self, xi, u, w, ids=None):
        pic_set_particles(self.h, xi, u, w, ids)

    def diag(self, kind, length=1, p0=0.0, p1=0.0):
        kinds = {"ex_lineout": PIC_DIAG_EX_LINEOUT, "field_energy": PIC_DIAG_FIELD_ENERGY,
                 "charge": PIC_DIAG_CHARGE, "spectrum": PIC_DIAG_SPECTRUM,
                 "emittance": PIC_DIAG_EMITTANCE, "phase_x_px": PIC_DIAG_PHASE_X_PX,
                 "density_xy": PIC_DIAG_DENSITY_XY, "dive_residual": PIC_DIAG_DIVE_RESIDUAL}
        k = kinds[kind]
        if k == PIC_DIAG_DIVE_RESIDUAL:
            return pic_diag(self.h, k, max(length, 1))
        if k == PIC_DIAG_EMITTANCE:
            return pic_diag(self.h, k, 2, gamma_min=p0)
        if k == PIC_DIAG_PHASE_X_PX:
            return pic_diag(self.h, k, length, p_min=p0, p_max=p1)
        if k == PIC_DIAG_DENSITY_XY:
            return pic_diag(self.h, k, self.shape[0] * self.shape[1])
        if k == PIC_DIAG_EX_LINEOUT:
            return pic_diag(self.h, k, max(length, self.shape[0]))
        if k == PIC_DIAG_CHARGE:
            return pic_diag(self.h, k, 1, gamma_min=p0)
        if k == PIC_DIAG_SPECTRUM:
            return pic_diag(self.h, k, length, e_min=p0, e_max=p1)
        return pic_diag(self.h, k, 1)
