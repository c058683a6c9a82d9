"""ctypes wrapper of the C oracle (oracle/pic_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU
baseline leg of bench.py, never by the product path.  Units of the state
accessors are the normalised ones of pic_oracle.h; set-up takes SI.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
COMP_NAMES = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]
LOAD = {"random": 0, "lattice": 1}
LASER = {"auto": 0, "hard_source": 1, "in_box": 2}
DIAG = {"ex_lineout": 0, "field_energy": 1, "charge": 2, "spectrum": 3, "dive_residual": 4,
        "emittance": 5, "phase_x_px": 6, "density_xy": 7}


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("lambda0", C.c_double), ("x0", C.c_double),
                ("periodic_x", C.c_int), ("seed", C.c_uint64), ("solver", C.c_int), ("pml", C.c_int)]


class _Window(C.Structure):
    _fields_ = [("v", C.c_double), ("t_start", C.c_double)]


class _Profile(C.Structure):
    _fields_ = [("n", C.c_int), ("x", C.POINTER(C.c_double)), ("dens", C.POINTER(C.c_double))]


class _Info(C.Structure):
    _fields_ = [("dt", C.c_double), ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("t", C.c_double), ("step", C.c_longlong), ("shifts", C.c_longlong),
                ("np", C.c_size_t)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Grid), C.c_double, C.POINTER(_Window)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_add_species.argtypes = [C.c_void_p, C.POINTER(_Profile), C.c_int, C.c_double,
                                     C.c_double, C.c_int]
        L.or_add_laser.argtypes = [C.c_void_p] + [C.c_double] * 6 + [C.c_int]
        L.or_step.argtypes = [C.c_void_p, C.c_int]
        L.or_diag.argtypes = [C.c_void_p, C.c_int, dp, C.c_size_t, C.c_double, C.c_double]
        L.or_info_get.argtypes = [C.c_void_p, C.POINTER(_Info)]
        L.or_field.restype = dp
        L.or_field.argtypes = [C.c_void_p, C.c_int]
        L.or_particles.restype = C.c_size_t
        L.or_particles.argtypes = [C.c_void_p, C.POINTER(dp), C.POINTER(dp), C.POINTER(dp),
                                   C.POINTER(C.POINTER(C.c_uint32))]
        L.or_set_particles.argtypes = [C.c_void_p, C.c_size_t, C.POINTER(dp), C.POINTER(dp), dp,
                                       C.POINTER(C.c_uint32)]
        L.or_m4.restype = C.c_double
        L.or_m4.argtypes = [C.c_double]
        L.or_smoothing.argtypes = [C.c_void_p, dp]
        L.or_boris.argtypes = [dp, dp, dp, C.c_double]
        L.or_gather.argtypes = [C.c_void_p, dp, dp, dp]
        L.or_rho.argtypes = [C.c_void_p, dp]
        L.or_div_e.argtypes = [C.c_void_p, dp]
        L.or_deposit_one.argtypes = [C.c_void_p, dp, dp, C.c_double]
        L.or_field_update.argtypes = [C.c_void_p]
        L.or_splitmix64.restype = C.c_uint64
        L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.or_laser_ey.restype = C.c_double
        L.or_laser_ey.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def m4(d):
    """Cubic B-spline kernel of the oracle."""
    return lib().or_m4(float(d))


def splitmix64(seed, n):
    return int(lib().or_splitmix64(seed, n))


def boris(u, E, B, h):
    """One Boris push of momentum u (3,) with h = q dt / (2 m); returns new u."""
    u = np.array(u, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lib().or_boris(_dp(u), _dp(E), _dp(B), float(h))
    return u


class Sim:
    """One oracle simulation (SI set-up, normalised state)."""

    def __init__(self, nx, ny, nz, dx, dy, dz, lambda0, x0=0.0, periodic_x=True, seed=12040838,
                 dt=0.0, window=None, solver="perfect", pml=0):
        g = _Grid(nx, ny, nz, dx, dy, dz, lambda0, x0, 1 if periodic_x else 0, seed,
                  1 if solver == "yee" else 0, int(pml))
        w = None
        if window is not None:
            w = C.pointer(_Window(float(window[0]), float(window[1])))
        self._h = lib().or_create(C.byref(g), float(dt), w)
        if not self._h:
            raise ValueError("oracle rejected the grid/time step/window")
        self.shape = (nx, ny, nz)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def add_species(self, prof_x, prof_n, ppc, q=-1.0, m=1.0, loading="random"):
        px = np.ascontiguousarray(prof_x, dtype=np.float64)
        pn = np.ascontiguousarray(prof_n, dtype=np.float64)
        p = _Profile(len(px), _dp(px), _dp(pn))
        if lib().or_add_species(self._h, C.byref(p), int(ppc), float(q), float(m), LOAD[loading]):
            raise ValueError("oracle rejected the species")

    def add_laser(self, a0, waist, fwhm, lambda_l, x_focus=0.0, t_peak=None, mode="auto"):
        if t_peak is None:
            t_peak = 2.0 * fwhm
        if lib().or_add_laser(self._h, a0, waist, fwhm, lambda_l, x_focus, t_peak, LASER[mode]):
            raise ValueError("oracle rejected the laser")

    def step(self, n=1):
        lib().or_step(self._h, int(n))

    def info(self):
        i = _Info()
        lib().or_info_get(self._h, C.byref(i))
        return {"dt": i.dt, "dx": i.dx, "dy": i.dy, "dz": i.dz, "t": i.t, "step": i.step,
                "shifts": i.shifts, "np": i.np}

    def field(self, comp):
        """Writable numpy view (nx, ny, nz) of a component array."""
        p = lib().or_field(self._h, int(comp))
        n = self.shape[0] * self.shape[1] * self.shape[2]
        return np.ctypeslib.as_array(p, shape=(n,)).reshape(self.shape)

    def fields(self):
        return np.stack([self.field(c).copy() for c in range(9)])

    def set_fields(self, arr):
        for c in range(9):
            self.field(c)[...] = arr[c]

    def particles(self):
        xi = (C.POINTER(C.c_double) * 3)()
        u = (C.POINTER(C.c_double) * 3)()
        w = C.POINTER(C.c_double)()
        i = C.POINTER(C.c_uint32)()
        n = lib().or_particles(self._h, xi, u, C.byref(w), C.byref(i))
        out = {"xi": np.zeros((3, n)), "u": np.zeros((3, n)), "w": np.zeros(n),
               "id": np.zeros(n, dtype=np.uint32)}
        if n:
            for c in range(3):
                out["xi"][c] = np.ctypeslib.as_array(xi[c], shape=(n,))
                out["u"][c] = np.ctypeslib.as_array(u[c], shape=(n,))
            out["w"][:] = np.ctypeslib.as_array(w, shape=(n,))
            out["id"][:] = np.ctypeslib.as_array(i, shape=(n,))
        return out

    def set_particles(self, xi, u, w, ids=None):
        xi = [np.ascontiguousarray(xi[c], dtype=np.float64) for c in range(3)]
        u = [np.ascontiguousarray(u[c], dtype=np.float64) for c in range(3)]
        w = np.ascontiguousarray(w, dtype=np.float64)
        n = len(w)
        xa = (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in xi])
        ua = (C.POINTER(C.c_double) * 3)(*[_dp(a) for a in u])
        ip = None
        if ids is not None:
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
            ip = ids.ctypes.data_as(C.POINTER(C.c_uint32))
        if lib().or_set_particles(self._h, n, xa, ua, _dp(w), ip):
            raise ValueError("particle outside the allowed range")

    def diag(self, kind, length=1, p0=0.0, p1=0.0):
        out = np.zeros(length)
        if lib().or_diag(self._h, DIAG[kind], _dp(out), length, float(p0), float(p1)):
            raise ValueError("bad diagnostic request")
        return out

    def smoothing(self):
        out = np.zeros(12)
        lib().or_smoothing(self._h, _dp(out))
        return out.reshape(3, 4)

    def gather(self, xi):
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        E = np.zeros(3)
        B = np.zeros(3)
        lib().or_gather(self._h, _dp(xi), _dp(E), _dp(B))
        return E, B

    def rho(self):
        out = np.zeros(self.shape)
        lib().or_rho(self._h, _dp(out))
        return out

    def div_e(self):
        out = np.zeros(self.shape)
        lib().or_div_e(self._h, _dp(out))
        return out

    def deposit_one(self, xi0, xi1, qw):
        a = np.ascontiguousarray(xi0, dtype=np.float64)
        b = np.ascontiguousarray(xi1, dtype=np.float64)
        lib().or_deposit_one(self._h, _dp(a), _dp(b), float(qw))

    def field_update(self):
        lib().or_field_update(self._h)

    def laser_ey(self, x, y, z, t):
        return lib().or_laser_ey(self._h, x, y, z, t)
