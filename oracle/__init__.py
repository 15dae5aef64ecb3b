"""FP64 CPU oracle of the stabilized Lattice Boltzmann-Enskog DD-TR step.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow reference that the
CUDA library is checked against.  It may be imported by the test suite, by the
smoke check of ``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``;
the library (``paper_1202_3842_gb300``) never imports it and shares no code,
table or header with it.

The arithmetic lives in ``lbe_oracle.c`` (plain C loops, double precision, no
floating-point contraction); this module only marshals numpy arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIBS = {}

_c_int_p = ctypes.POINTER(ctypes.c_int)
_c_dbl_p = ctypes.POINTER(ctypes.c_double)
_c_u8_p = ctypes.POINTER(ctypes.c_uint8)
_c_u32_p = ctypes.POINTER(ctypes.c_uint32)
_c_long_p = ctypes.POINTER(ctypes.c_long)


def lib(openmp=False):
    """Load (building first if needed) the oracle shared library: the single-threaded parity build, or with
    openmp=True the OpenMP build of the same source used to time the CPU baseline on all host cores."""
    key = bool(openmp)
    if key not in _LIBS:
        path = _build.build(openmp=key)
        L = ctypes.CDLL(path)
        L.or_lattice.argtypes = [_c_int_p, _c_dbl_p, _c_int_p]
        L.or_shell.argtypes = [ctypes.c_double, _c_int_p, ctypes.c_int]
        L.or_shell.restype = ctypes.c_int
        L.or_shell_weight.argtypes = [ctypes.c_double]
        L.or_shell_weight.restype = ctypes.c_double
        L.or_ball.argtypes = [ctypes.c_double, _c_int_p, ctypes.c_int]
        L.or_ball.restype = ctypes.c_int
        L.or_bmcsl.argtypes = [ctypes.c_double] * 4
        L.or_bmcsl.restype = ctypes.c_double
        L.or_link_mask.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_u8_p, _c_u32_p]
        L.or_contact_values.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_u8_p, ctypes.c_int, _c_dbl_p,
                                                              _c_dbl_p, _c_dbl_p]
        L.or_shell_force.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_u8_p, ctypes.c_int, _c_dbl_p,
                                                          _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.or_force_field.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.or_visc_force.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_u8_p, ctypes.c_int, _c_dbl_p, _c_dbl_p,
                                                         _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.or_set_visc.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_set_visc.restype = ctypes.c_int
        L.or_quasipressure.argtypes = [ctypes.c_int] * 3 + [_c_int_p, _c_u8_p, ctypes.c_int, _c_dbl_p, _c_dbl_p,
                                                            _c_dbl_p, _c_dbl_p, _c_dbl_p]
        L.or_create.argtypes = [ctypes.c_int] * 7
        L.or_create.restype = ctypes.c_void_p
        L.or_destroy.argtypes = [ctypes.c_void_p]
        L.or_set_solid.argtypes = [ctypes.c_void_p, _c_u8_p]
        L.or_set_species.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.or_set_potential.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p]
        L.or_set_wall_potential.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_dbl_p]
        L.or_set_body_force.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p]
        L.or_set_consistent_moments.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_set_scheme.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_set_flux_plane.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        L.or_init_density.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p]
        L.or_set_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p, _c_dbl_p]
        L.or_get_populations.argtypes = [ctypes.c_void_p, ctypes.c_int, _c_dbl_p, _c_dbl_p]
        L.or_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.or_observe.argtypes = [ctypes.c_void_p] + [_c_dbl_p] * 6
        L.or_get_flux.argtypes = [ctypes.c_void_p, _c_dbl_p, _c_long_p]
        L.or_steps_done.argtypes = [ctypes.c_void_p]
        L.or_steps_done.restype = ctypes.c_long
        _LIBS[key] = L
    return _LIBS[key]


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dbl(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    """D3Q19 velocities c [19,3], weights w [19], opposite index [19]."""
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    o = np.zeros(19, dtype=np.int32)
    lib().or_lattice(_p(c, ctypes.c_int), _p(w, ctypes.c_double), _p(o, ctypes.c_int))
    return c, w, o


def shell(sigma):
    """Contact shell K_sigma as an int array [k,3] in the oracle's list order."""
    k = lib().or_shell(float(sigma), None, 0)
    e = np.zeros((max(k, 1), 3), dtype=np.int32)
    lib().or_shell(float(sigma), _p(e, ctypes.c_int), k)
    return e[:k]


def shell_weight(sigma):
    return lib().or_shell_weight(float(sigma))


def ball(radius):
    k = lib().or_ball(float(radius), None, 0)
    d = np.zeros((max(k, 1), 3), dtype=np.int32)
    lib().or_ball(float(radius), _p(d, ctypes.c_int), k)
    return d[:k]


def bmcsl(sa, sb, xi2, xi3):
    return lib().or_bmcsl(float(sa), float(sb), float(xi2), float(xi3))


def _per(periodic):
    return np.ascontiguousarray(periodic, dtype=np.int32)


def _solid(solid, N):
    if solid is None:
        return np.zeros(N, dtype=np.uint8)
    return np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)


def link_mask(shape, periodic, solid=None):
    """Per-node 19-bit blocked-link mask, shape (nz, ny, nx) order of indices x fastest."""
    nx, ny, nz = shape
    N = nx * ny * nz
    s = _solid(solid, N)
    m = np.zeros(N, dtype=np.uint32)
    lib().or_link_mask(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(s, ctypes.c_uint8),
                       _p(m, ctypes.c_uint32))
    return m


def contact_values(shape, periodic, sigma, n, solid=None):
    """g_ab for n of shape [M, N]; returns [M, M, N]."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = _dbl(n).reshape(-1, N)
    M = n.shape[0]
    sig = _dbl(sigma)
    out = np.zeros((M, M, N))
    s = _solid(solid, N)
    lib().or_contact_values(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(s, ctypes.c_uint8), M,
                            _p(sig, ctypes.c_double), _p(n, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def shell_force(shape, periodic, sigma, n, gpair, solid=None):
    """C^{a,mf} [M, 3, N] from n [M, N] and g_ab [M, M, N]."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = _dbl(n).reshape(-1, N)
    M = n.shape[0]
    gp = _dbl(gpair).reshape(M, M, N)
    sig = _dbl(sigma)
    out = np.zeros((M, 3, N))
    s = _solid(solid, N)
    lib().or_shell_force(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(s, ctypes.c_uint8), M,
                         _p(sig, ctypes.c_double), _p(n, ctypes.c_double), _p(gp, ctypes.c_double),
                         _p(out, ctypes.c_double))
    return out


def force_field(shape, periodic, V=None, gbody=(0.0, 0.0, 0.0)):
    nx, ny, nz = shape
    N = nx * ny * nz
    Vp = None if V is None else _dbl(V).reshape(N)
    g = _dbl(gbody)
    F = np.zeros((3, N))
    lib().or_force_field(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(Vp, ctypes.c_double),
                         _p(g, ctypes.c_double), _p(F, ctypes.c_double))
    return F


def visc_force(shape, periodic, sigma, n, u, gpair, solid=None):
    """C^{a,visc} [M, 3, N] from n [M, N], velocities u [M, 3, N] and g_ab [M, M, N]."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = _dbl(n).reshape(-1, N)
    M = n.shape[0]
    uu = _dbl(u).reshape(M, 3, N)
    gp = _dbl(gpair).reshape(M, M, N)
    sig = _dbl(sigma)
    out = np.zeros((M, 3, N))
    s = _solid(solid, N)
    lib().or_visc_force(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(s, ctypes.c_uint8), M,
                        _p(sig, ctypes.c_double), _p(n, ctypes.c_double), _p(uu, ctypes.c_double),
                        _p(gp, ctypes.c_double), _p(out, ctypes.c_double))
    return out


def quasipressure(shape, periodic, sigma, n, V, gbody, solid=None):
    """Pi^a = n^a - beta * trapezoidal path integral of C^{a,mf} + n^a F^a (x, then y, then z from the
    origin); n and V [M, N] (V the full potential of each species), gbody [M, 3].  Returns [M, N]."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = _dbl(n).reshape(-1, N)
    M = n.shape[0]
    Vp = _dbl(V).reshape(M, N)
    gb = _dbl(gbody).reshape(M, 3)
    sig = _dbl(sigma)
    out = np.zeros((M, N))
    s = _solid(solid, N)
    lib().or_quasipressure(nx, ny, nz, _p(_per(periodic), ctypes.c_int), _p(s, ctypes.c_uint8), M,
                           _p(sig, ctypes.c_double), _p(n, ctypes.c_double), _p(Vp, ctypes.c_double),
                           _p(gb, ctypes.c_double), _p(out, ctypes.c_double))
    return out


class Sim:
    """Oracle simulation: the same sequence of set-up calls as the library."""

    def __init__(self, shape, periodic=(1, 1, 1), nspecies=1, openmp=False):
        self._L = lib(openmp)
        self.shape = tuple(int(v) for v in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.M = int(nspecies)
        per = [int(bool(v)) for v in periodic]
        self._h = self._L.or_create(*self.shape, *per, self.M)
        if not self._h:
            raise ValueError("oracle: bad sizes")

    def close(self):
        if self._h:
            self._L.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, solid):
        s = _solid(solid, self.N)
        self._L.or_set_solid(self._h, _p(s, ctypes.c_uint8))

    def set_species(self, s, sigma, tau):
        if self._L.or_set_species(self._h, s, float(sigma), float(tau)) != 0:
            raise ValueError("oracle: bad species parameters")

    def set_potential(self, s, V):
        V = _dbl(V).reshape(self.N)
        self._L.or_set_potential(self._h, s, _p(V, ctypes.c_double))

    def set_wall_potential(self, phi, amp):
        phi = _dbl(phi).reshape(self.N)
        amp = _dbl(amp).reshape(self.N)
        self._L.or_set_wall_potential(self._h, _p(phi, ctypes.c_double), _p(amp, ctypes.c_double))

    def set_body_force(self, s, g):
        g = _dbl(g)
        self._L.or_set_body_force(self._h, s, _p(g, ctypes.c_double))

    def set_consistent_moments(self, on):
        """0 (or False): the moments as printed; 1 (or True): the map g = g~ + Omega/2 applied to the printed S_g;
        2: that map with the d Pi/d n term of S_g added (Sec. "Stabilization")."""
        if self._L.or_set_consistent_moments(self._h, int(on)) != 0:
            raise ValueError("consistent_moments must be 0, 1 or 2")

    def set_visc(self, on):
        if self._L.or_set_visc(self._h, int(bool(on))) != 0:
            raise ValueError("C^visc needs the DD-TR scheme")

    def set_scheme(self, scheme):
        """0 DD-TR (default), 1 SD-TR, 2 SD-EU, 3 DD-EU (Sec. "Results": single or double distribution,
        Euler or trapezoidal integration)."""
        if self._L.or_set_scheme(self._h, int(scheme)) != 0:
            raise ValueError("unknown scheme %r" % (scheme,))

    def set_flux_plane(self, axis, plane):
        self._L.or_set_flux_plane(self._h, int(axis), int(plane))

    def init_density(self, s, n):
        n = _dbl(n).reshape(self.N)
        self._L.or_init_density(self._h, s, _p(n, ctypes.c_double))

    def set_populations(self, s, f, g):
        f = _dbl(f).reshape(19, self.N)
        g = _dbl(g).reshape(19, self.N)
        self._L.or_set_populations(self._h, s, _p(f, ctypes.c_double), _p(g, ctypes.c_double))

    def get_populations(self, s):
        f = np.zeros((19, self.N))
        g = np.zeros((19, self.N))
        self._L.or_get_populations(self._h, s, _p(f, ctypes.c_double), _p(g, ctypes.c_double))
        return f, g

    def step(self, nsteps=1):
        self._L.or_step(self._h, int(nsteps))

    def observe(self):
        """dict of n [M,N], J [M,3,N], C [M,3,N], Pi [M,N], F [M,3,N], g [M,M,N] of the current state."""
        M, N = self.M, self.N
        out = dict(n=np.zeros((M, N)), J=np.zeros((M, 3, N)), C=np.zeros((M, 3, N)), Pi=np.zeros((M, N)),
                   F=np.zeros((M, 3, N)), g=np.zeros((M, M, N)))
        self._L.or_observe(self._h, *[_p(out[k], ctypes.c_double) for k in ("n", "J", "C", "Pi", "F", "g")])
        return out

    def flux(self):
        """(per-species running flux sum [M], number of steps accumulated)."""
        s = np.zeros(self.M)
        c = ctypes.c_long(0)
        self._L.or_get_flux(self._h, _p(s, ctypes.c_double), ctypes.byref(c))
        return s, c.value

    def steps_done(self):
        return self._L.or_steps_done(self._h)
