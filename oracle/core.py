"""ctypes wrappers around the FP64 C oracle and the plain step driver.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg import this module; the CUDA library never does.

The step follows the order of the PIC loop in Sec. 1 (deposit -> solve -> interpolate
-> push, started at the interpolation so that E and B sit at integer times):

    gather E^n, B^n at x^n -> Boris u^{n-1/2} -> u^{n+1/2} -> x^{n+1}
    -> Esirkepov J^{n+1/2} (x^n -> x^{n+1}) -> [filter] J <- F J along z
    -> [customised] J1 <- h * J1 (Sec. 3)
    -> B^{n+1/2}, E^{n+1}, B^{n+1} (Eq. 1) -> drop particles outside 0 <= z < nz
    -> [moving window] shift one cell when n dt >= (s+1) dz, inject cold plasma.
"""
import ctypes
import math

import numpy as np

from . import build as _build

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        L = _lib
        L.or_field_advance.argtypes = [_ip, _dp, _dp, _dp, _dp, _dp]
        L.or_faraday_half.argtypes = [_ip, _dp, _dp, _dp, _dp]
        L.or_ampere.argtypes = [_ip, _dp, _dp, _dp, _dp, _dp]
        L.or_correct_j1.argtypes = [_ip, _dp, ctypes.c_int, _dp]
        L.or_gather.argtypes = [_ip, _dp, _dp, _dp, ctypes.c_long, _dp, _dp]
        L.or_boris.argtypes = [ctypes.c_long, _dp, _dp, ctypes.c_double]
        L.or_move.argtypes = [_ip, _dp, ctypes.c_long, _dp, _dp, _dp]
        L.or_deposit.argtypes = [_ip, _dp, ctypes.c_long, _dp, _dp, _dp, ctypes.c_double, _dp]
        L.or_rho.argtypes = [_ip, _dp, ctypes.c_long, _dp, ctypes.c_double, _dp]
        L.or_gauss.argtypes = [_ip, _dp, _dp, _dp, _dp, _dp]
        L.or_shift_z.argtypes = [_ip, ctypes.c_int, _dp]
        L.or_filter_z.argtypes = [_ip, ctypes.c_int, _dp]
        L.or_set_threads.argtypes = [ctypes.c_int]
        L.or_get_threads.restype = ctypes.c_int
        L.or_openmp.restype = ctypes.c_int
        L.or_set_threads(1)          # one fixed summation order unless a caller asks for more
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's loops (OpenMP builds); returns the number in effect."""
    lib().or_set_threads(int(n))
    return lib().or_get_threads()


def openmp() -> bool:
    return bool(lib().or_openmp())


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class Grid:
    """Grid, time step, axial stencil and particle shape of one oracle instance.

    C: coefficients of the axial operators.  Cb (optional): separate coefficients of the
    B-side operator d- ([k]_B1: Ampere's and Gauss's laws), C then being the E-side d+
    ([k]_E1: Faraday's law); the shorter set is padded with zeros."""

    def __init__(self, ndim, nz, nx, ny=1, dz=1.0, dx=1.0, dy=1.0, dt=0.5, C=(1.0,), shape=1,
                 periodic_z=False, Cb=None):
        self.ndim, self.nz, self.nx = int(ndim), int(nz), int(nx)
        self.ny = int(ny) if ndim == 3 else 1
        self.dz, self.dx, self.dy, self.dt = float(dz), float(dx), float(dy), float(dt)
        C = np.asarray(C, dtype=np.float64)
        Cb = None if Cb is None else np.asarray(Cb, dtype=np.float64)
        M = max(len(C), len(Cb) if Cb is not None else 0)
        self.C = np.ascontiguousarray(np.pad(C, (0, M - len(C))))
        self.Cb = None if Cb is None else np.ascontiguousarray(np.pad(Cb, (0, M - len(Cb))))
        # what the C routines receive: C, followed by Cb when the operators are split
        self.Cpar = self.C if self.Cb is None else np.ascontiguousarray(np.concatenate([self.C, self.Cb]))
        self.shape = int(shape)
        self.periodic_z = bool(periodic_z)
        self.ip = (ctypes.c_int * 8)(self.ndim, self.nz, self.nx, self.ny, M, self.shape,
                                     int(self.periodic_z), int(self.Cb is not None))
        self.dpar = (ctypes.c_double * 4)(self.dz, self.dx, self.dy, self.dt)

    @property
    def fshape(self):
        return (3, self.ny, self.nx, self.nz)

    def zeros(self):
        return np.zeros(self.fshape, dtype=np.float64)

    def cell_volume(self):
        return self.dz * self.dx * (self.dy if self.ndim == 3 else 1.0)


def field_advance(g: Grid, E, B, J):
    lib().or_field_advance(g.ip, g.dpar, _d(g.Cpar), _d(E), _d(B), _d(J))


def faraday_half(g: Grid, E, B):
    lib().or_faraday_half(g.ip, g.dpar, _d(g.Cpar), _d(E), _d(B))


def ampere(g: Grid, E, B, J):
    lib().or_ampere(g.ip, g.dpar, _d(g.Cpar), _d(E), _d(B), _d(J))


def correct_j1(g: Grid, h, J):
    h = np.ascontiguousarray(h, dtype=np.float64)
    lib().or_correct_j1(g.ip, _d(h), (len(h) - 1) // 2, _d(J))


def gather(g: Grid, E, B, xi):
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    out = np.zeros((len(xi), 6))
    lib().or_gather(g.ip, g.dpar, _d(E), _d(B), len(xi), _d(xi), _d(out))
    return out


def boris(eb, u, eps):
    lib().or_boris(len(u), _d(np.ascontiguousarray(eb)), _d(u), float(eps))


def move(g: Grid, xi0, u):
    xi1 = np.zeros_like(xi0)
    lib().or_move(g.ip, g.dpar, len(xi0), _d(xi0), _d(u), _d(xi1))
    return xi1


def deposit(g: Grid, xi0, xi1, u, Q, J):
    lib().or_deposit(g.ip, g.dpar, len(xi0), _d(xi0), _d(xi1), _d(u), float(Q), _d(J))


def rho(g: Grid, xi, Q, out=None):
    if out is None:
        out = np.zeros(g.fshape[1:])
    lib().or_rho(g.ip, g.dpar, len(xi), _d(np.ascontiguousarray(xi)), float(Q), _d(out))
    return out


def gauss(g: Grid, E, rho_nodes):
    G = np.zeros(g.fshape[1:])
    lib().or_gauss(g.ip, g.dpar, _d(g.Cpar), _d(E), _d(np.ascontiguousarray(rho_nodes)), _d(G))
    return G


def shift_z(g: Grid, F):
    lib().or_shift_z(g.ip, F.shape[0], _d(F))


def filter_z(g: Grid, F):
    """The 5-pass current filter along z, in place, on every leading component of F
    (F of shape (ncomp, ny, nx, nz) or a single (ny, nx, nz) array)."""
    ncomp = F.shape[0] if F.ndim == 4 else 1
    lib().or_filter_z(g.ip, ncomp, _d(F))


class Species:
    """Macro-particles of one species: positions xi (n,3) in cell units, momenta u = gamma v (n,3)."""

    def __init__(self, xi, u, q, m, w, ids=None):
        self.xi = np.ascontiguousarray(xi, dtype=np.float64)
        self.u = np.ascontiguousarray(u, dtype=np.float64)
        self.q, self.m, self.w = float(q), float(m), float(w)
        self.ids = np.arange(len(self.xi), dtype=np.int64) if ids is None else np.asarray(ids, dtype=np.int64)

    @property
    def Q(self):
        return self.q * self.w

    def keep(self, mask):
        self.xi = np.ascontiguousarray(self.xi[mask])
        self.u = np.ascontiguousarray(self.u[mask])
        self.ids = self.ids[mask]


class Sim:
    """Plain FP64 PIC loop over the C oracle routines (one grid, several species)."""

    def __init__(self, g: Grid, species, h=None, moving_window=False, inject=None, filt=False, kspace=None):
        self.g = g
        # kspace: None (finite differences, Eq. 1) or the kind of oracle.spectral's k-space advance
        # ("spectral", "kt"), which carries its own form of the Sec. 3 correction
        self.kspace = kspace
        self.filt = bool(filt)
        self.E = g.zeros()
        self.B = g.zeros()
        self.J = g.zeros()
        self.species = list(species)
        self.h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        self.moving_window = bool(moving_window)
        # inject = dict(species=index, ppc=(pz, px[, py]), next_id=int)
        self.inject = inject
        self.n = 0
        self.shifts = 0

    def step(self):
        g = self.g
        self.J[:] = 0.0
        for sp in self.species:
            eb = gather(g, self.E, self.B, sp.xi)
            boris(eb, sp.u, sp.q * g.dt / (2.0 * sp.m))
            xi1 = move(g, sp.xi, sp.u)
            deposit(g, sp.xi, xi1, sp.u, sp.Q, self.J)
            sp.xi = xi1
        if self.filt:
            filter_z(g, self.J)
        if self.kspace is not None:
            from . import spectral
            spectral.advance(g, self.E, self.B, self.J, self.kspace)
        else:
            if self.h is not None:
                correct_j1(g, self.h, self.J)
            field_advance(g, self.E, self.B, self.J)
        for sp in self.species:
            sp.xi[:, 1] = np.mod(sp.xi[:, 1], g.nx)
            if g.ndim == 3:
                sp.xi[:, 2] = np.mod(sp.xi[:, 2], g.ny)
            sp.keep((sp.xi[:, 0] >= 0.0) & (sp.xi[:, 0] < g.nz))
        self.n += 1
        if self.moving_window and window_due(self.n, g.dt, g.dz, self.shifts):
            self.shift()

    def shift(self):
        g = self.g
        shift_z(g, self.E)
        shift_z(g, self.B)
        for sp in self.species:
            sp.xi[:, 0] -= 1.0
            sp.keep(sp.xi[:, 0] >= 0.0)
        if self.inject is not None:
            self._inject()
        self.shifts += 1

    def _inject(self):
        g, inj = self.g, self.inject
        sp = self.species[inj["species"]]
        xi = injection_positions(g, inj["ppc"])
        ids = inj["next_id"] + np.arange(len(xi), dtype=np.int64)
        inj["next_id"] += len(xi)
        sp.xi = np.ascontiguousarray(np.concatenate([sp.xi, xi]))
        sp.u = np.ascontiguousarray(np.concatenate([sp.u, np.zeros_like(xi)]))
        sp.ids = np.concatenate([sp.ids, ids])

    def rho(self):
        r = np.zeros(self.g.fshape[1:])
        for sp in self.species:
            rho(self.g, sp.xi, sp.Q, r)
        return r

    def gauss(self):
        # with the current filter the field advance keeps Gauss's law for the filtered charge
        r = self.rho()
        if self.filt:
            filter_z(self.g, r)
        return gauss(self.g, self.E, r)

    def field_energy(self):
        return 0.5 * (np.sum(self.E ** 2) + np.sum(self.B ** 2)) * self.g.cell_volume()

    def kinetic_energy(self):
        e = 0.0
        for sp in self.species:
            gam = np.sqrt(1.0 + np.sum(sp.u ** 2, axis=1))
            e += sp.w * sp.m * np.sum(gam - 1.0)
        return e


def window_due(n_done: int, dt: float, dz: float, shifts_done: int) -> bool:
    """A moving window at c has moved floor(n dt / dz) cells after n steps."""
    return math.floor(n_done * dt / dz + 1e-9) > shifts_done


def injection_positions(g: Grid, ppc):
    """Cold quiet-start plasma in the front column nz-1: sub-cell centres, order (k, j, a, b, c)."""
    pz, px = int(ppc[0]), int(ppc[1])
    py = int(ppc[2]) if g.ndim == 3 else 1
    out = []
    for k in range(g.ny if g.ndim == 3 else 1):
        for j in range(g.nx):
            for a in range(pz):
                for b in range(px):
                    for c in range(py):
                        out.append((g.nz - 1 + (a + 0.5) / pz, j + (b + 0.5) / px,
                                    (k + (c + 0.5) / py) if g.ndim == 3 else 0.0))
    return np.array(out, dtype=np.float64).reshape(-1, 3)
