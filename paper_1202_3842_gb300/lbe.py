"""Thin ctypes binding of the C ABI in ``include/lbe.h``.

Every function here has the name of its C counterpart and only marshals
arguments (numpy arrays in and out, status codes to exceptions).  All compute
runs in the CUDA library ``liblbe.so``; there is no CPU fallback: if the
library is missing or the device is not sm_103a, the calls raise.

PyTorch supplies device memory (its caching allocator, through the
``lbe_allocator`` callbacks) and the CUDA stream.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbe.so")

LBE_FP64, LBE_FP32, LBE_BF16_SHIFTED, LBE_FP16_SHIFTED = 0, 1, 2, 3
LBE_DD_TR, LBE_SD_TR, LBE_SD_EU, LBE_DD_EU = 0, 1, 2, 3
PRECISIONS = {"fp64": LBE_FP64, "fp32": LBE_FP32, "bf16": LBE_BF16_SHIFTED, "fp16": LBE_FP16_SHIFTED}
(LBE_OK, LBE_ERR_INVALID_ARG, LBE_ERR_UNSUPPORTED, LBE_ERR_OOM, LBE_ERR_CUDA, LBE_ERR_DIVERGED, LBE_ERR_TIMEOUT,
 LBE_ERR_STATE) = range(8)
STATUS = {0: "LBE_OK", 1: "LBE_ERR_INVALID_ARG", 2: "LBE_ERR_UNSUPPORTED", 3: "LBE_ERR_OOM", 4: "LBE_ERR_CUDA",
          5: "LBE_ERR_DIVERGED", 6: "LBE_ERR_TIMEOUT", 7: "LBE_ERR_STATE"}


class LbeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class lbe_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3), ("nspecies", ctypes.c_int), ("precision", ctypes.c_int),
                ("scheme", ctypes.c_int), ("enable_visc", ctypes.c_int), ("consistent_moments", ctypes.c_int),
                ("check_every", ctypes.c_int)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class lbe_allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


_L = None
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_P = ctypes.c_void_p


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblbe.so is not built (run paper_1202_3842_gb300/build.py); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "lbe_create": [ctypes.POINTER(lbe_config), ctypes.POINTER(lbe_allocator), _P, ctypes.POINTER(_P)],
            "lbe_set_geometry": [_P, ctypes.POINTER(ctypes.c_uint8)],
            "lbe_set_species": [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double],
            "lbe_set_potential": [_P, ctypes.c_int, _D],
            "lbe_set_wall_potential": [_P, _D, _D],
            "lbe_set_body_force": [_P, ctypes.c_int, _D],
            "lbe_init_density": [_P, ctypes.c_int, _D],
            "lbe_step": [_P, ctypes.c_int],
            "lbe_get_density": [_P, ctypes.c_int, _D],
            "lbe_get_velocity": [_P, ctypes.c_int, _D],
            "lbe_get_momentum": [_P, ctypes.c_int, _D],
            "lbe_get_force": [_P, ctypes.c_int, _D],
            "lbe_get_contact": [_P, ctypes.c_int, ctypes.c_int, _D],
            "lbe_set_flux_plane": [_P, ctypes.c_int, ctypes.c_int],
            "lbe_get_flux": [_P, ctypes.c_int, _D, _D],
            "lbe_reset_flux_average": [_P],
            "lbe_get_totals": [_P, _D, _D, _D],
            "lbe_get_populations": [_P, ctypes.c_int, _D, _D],
            "lbe_set_populations": [_P, ctypes.c_int, _D, _D],
            "lbe_get_step_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
            "lbe_get_link_mask": [_P, ctypes.POINTER(ctypes.c_uint32)],
            "lbe_shell": [ctypes.c_double, _I, ctypes.c_int, _I],
            "lbe_get_launch_count": [_P, ctypes.POINTER(ctypes.c_longlong)],
            "lbe_probe_wait_timeout": [_P, ctypes.c_int],
            "lbe_set_stage_timing": [_P, ctypes.c_int],
            "lbe_get_stage_times": [_P, _D, ctypes.POINTER(ctypes.c_longlong)],
            "lbe_get_mass_noalloc": [_P, _D],
            "lbe_adjoint_flux_gradient": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D, _D],
            "lbe_save_state": [_P, _P, ctypes.POINTER(ctypes.c_size_t)],
            "lbe_load_state": [_P, _P, ctypes.c_size_t],
            "lbe_get_residual": [_P, _D],
            "lbe_get_divergence": [_P, ctypes.c_int, _D],
            "lbe_set_shell_method": [_P, ctypes.c_int],
            "lbe_init_density_quasipressure": [_P, _D],
            "lbe_get_shell_method": [_P, _I],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.lbe_destroy.argtypes = [_P]
        L.lbe_destroy.restype = None
        L.lbe_status_string.argtypes = [ctypes.c_int]
        L.lbe_status_string.restype = ctypes.c_char_p
        L.lbe_last_error.argtypes = [_P]
        L.lbe_last_error.restype = ctypes.c_char_p
        _L = L
    return _L


def declared_symbols():
    """Names of the functions declared in include/lbe.h (parsed from the header text)."""
    import re
    hdr = open(os.path.join(os.path.dirname(HERE), "include", "lbe.h")).read()
    return sorted(set(re.findall(r"\b(lbe_[a-z_0-9]+)\s*\(", hdr)))


def _check(status, ctx=None):
    if status != 0:
        msg = lib().lbe_last_error(ctx).decode(errors="replace")
        raise LbeError(status, msg)


def _dp(a):
    return a.ctypes.data_as(_D)


def _din(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


# --------------------------------------------------------------------------
# PyTorch plumbing: caching allocator and current stream
# --------------------------------------------------------------------------
class TorchAllocator:
    """lbe_allocator backed by torch.cuda's caching allocator."""

    def __init__(self, device=None):
        import torch
        self.torch = torch
        self.device = torch.cuda.current_device() if device is None else device

        def _alloc(nbytes, stream, user):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
            except Exception:
                return None

        def _free(ptr, nbytes, stream, user):
            try:
                self.torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self._a = _ALLOC_FN(_alloc)
        self._f = _FREE_FN(_free)
        self.struct = lbe_allocator(self._a, self._f, None)


def current_stream_handle():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# --------------------------------------------------------------------------
# C ABI, one function each
# --------------------------------------------------------------------------
SCHEMES = {"dd_tr": LBE_DD_TR, "sd_tr": LBE_SD_TR, "sd_eu": LBE_SD_EU, "dd_eu": LBE_DD_EU}


def lbe_create(shape, periodic=(1, 1, 1), nspecies=1, precision="fp32", consistent_moments=0, check_every=0,
               allocator=None, stream=None, scheme="dd_tr", visc=False):
    cfg = lbe_config()
    cfg.nx, cfg.ny, cfg.nz = [int(v) for v in shape]
    for k in range(3):
        cfg.periodic[k] = int(bool(periodic[k]))
    cfg.nspecies = int(nspecies)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.scheme = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    cfg.enable_visc = int(bool(visc))
    cfg.consistent_moments = int(bool(consistent_moments))
    cfg.check_every = int(check_every)
    out = ctypes.c_void_p()
    ap = ctypes.byref(allocator.struct) if allocator is not None else None
    st = stream if stream is not None else ctypes.c_void_p(0)
    _check(lib().lbe_create(ctypes.byref(cfg), ap, st, ctypes.byref(out)))
    return out


def lbe_destroy(ctx):
    lib().lbe_destroy(ctx)


def lbe_set_geometry(ctx, N, solid):
    s = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
    if s.size != N:
        raise ValueError("solid mask has %d entries, expected %d" % (s.size, N))
    _check(lib().lbe_set_geometry(ctx, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))), ctx)


def lbe_set_species(ctx, s, sigma, mass, tau):
    _check(lib().lbe_set_species(ctx, int(s), float(sigma), float(mass), float(tau)), ctx)


def lbe_set_potential(ctx, N, s, V):
    V = _din(V, N)
    _check(lib().lbe_set_potential(ctx, int(s), _dp(V)), ctx)


def lbe_set_wall_potential(ctx, N, phi, amp):
    phi = _din(phi, N)
    amp = _din(amp, N)
    _check(lib().lbe_set_wall_potential(ctx, _dp(phi), _dp(amp)), ctx)


def lbe_set_body_force(ctx, s, g):
    g = _din(g, 3)
    _check(lib().lbe_set_body_force(ctx, int(s), _dp(g)), ctx)


def lbe_init_density(ctx, N, s, n):
    n = _din(n, N)
    _check(lib().lbe_init_density(ctx, int(s), _dp(n)), ctx)


def lbe_step(ctx, nsteps):
    _check(lib().lbe_step(ctx, int(nsteps)), ctx)


def lbe_get_density(ctx, N, s, out=None):
    out = np.empty(N) if out is None else out
    _check(lib().lbe_get_density(ctx, int(s), _dp(out)), ctx)
    return out


def lbe_get_velocity(ctx, N, s):
    out = np.empty(3 * N)
    _check(lib().lbe_get_velocity(ctx, int(s), _dp(out)), ctx)
    return out.reshape(3, N)


def lbe_get_momentum(ctx, N, s):
    out = np.empty(3 * N)
    _check(lib().lbe_get_momentum(ctx, int(s), _dp(out)), ctx)
    return out.reshape(3, N)


def lbe_get_force(ctx, N, s):
    out = np.empty(3 * N)
    _check(lib().lbe_get_force(ctx, int(s), _dp(out)), ctx)
    return out.reshape(3, N)


def lbe_get_contact(ctx, N, a, b):
    out = np.empty(N)
    _check(lib().lbe_get_contact(ctx, int(a), int(b), _dp(out)), ctx)
    return out


def lbe_set_flux_plane(ctx, axis, plane):
    _check(lib().lbe_set_flux_plane(ctx, int(axis), int(plane)), ctx)


def lbe_get_flux(ctx, s=-1):
    inst = ctypes.c_double(0.0)
    avg = ctypes.c_double(0.0)
    _check(lib().lbe_get_flux(ctx, int(s), ctypes.byref(inst), ctypes.byref(avg)), ctx)
    return inst.value, avg.value


def lbe_reset_flux_average(ctx):
    _check(lib().lbe_reset_flux_average(ctx), ctx)


def lbe_get_totals(ctx, M):
    mass = np.zeros(M)
    mom = np.zeros(3)
    mu = ctypes.c_double(0.0)
    _check(lib().lbe_get_totals(ctx, _dp(mass), _dp(mom), ctypes.byref(mu)), ctx)
    return mass, mom, mu.value


def lbe_get_populations(ctx, N, s):
    f = np.empty(19 * N)
    g = np.empty(19 * N)
    _check(lib().lbe_get_populations(ctx, int(s), _dp(f), _dp(g)), ctx)
    return f.reshape(19, N), g.reshape(19, N)


def lbe_set_populations(ctx, N, s, f, g):
    f = _din(f, 19 * N)
    g = _din(g, 19 * N)
    _check(lib().lbe_set_populations(ctx, int(s), _dp(f), _dp(g)), ctx)


def lbe_get_step_count(ctx):
    v = ctypes.c_longlong(0)
    _check(lib().lbe_get_step_count(ctx, ctypes.byref(v)), ctx)
    return v.value


def lbe_save_state(ctx):
    """The state as bytes (populations as stored, n0, step count, flux plane and accumulators)."""
    n = ctypes.c_size_t(0)
    _check(lib().lbe_save_state(ctx, None, ctypes.byref(n)), ctx)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().lbe_save_state(ctx, ctypes.cast(buf, _P), ctypes.byref(n)), ctx)
    return buf.raw[:n.value]


def lbe_load_state(ctx, state):
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    _check(lib().lbe_load_state(ctx, ctypes.cast(buf, _P), len(state)), ctx)


def lbe_get_residual(ctx):
    v = ctypes.c_double(0.0)
    _check(lib().lbe_get_residual(ctx, ctypes.byref(v)), ctx)
    return v.value


def lbe_get_divergence(ctx, N, s=-1):
    out = np.empty(N)
    _check(lib().lbe_get_divergence(ctx, int(s), _dp(out)), ctx)
    return out


def lbe_get_link_mask(ctx, N):
    out = np.empty(N, dtype=np.uint32)
    _check(lib().lbe_get_link_mask(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), ctx)
    return out


def lbe_shell(sigma):
    cnt = ctypes.c_int(0)
    _check(lib().lbe_shell(float(sigma), None, 0, ctypes.byref(cnt)))
    e = np.zeros((max(cnt.value, 1), 3), dtype=np.int32)
    _check(lib().lbe_shell(float(sigma), e.ctypes.data_as(_I), cnt.value, ctypes.byref(cnt)))
    return e[:cnt.value]


def lbe_get_launch_count(ctx):
    v = ctypes.c_longlong(0)
    _check(lib().lbe_get_launch_count(ctx, ctypes.byref(v)), ctx)
    return v.value


def lbe_probe_wait_timeout(ctx, polls):
    _check(lib().lbe_probe_wait_timeout(ctx, int(polls)), ctx)


def lbe_init_density_quasipressure(ctx, M, N, n):
    """Rest populations with g from the quasi-pressure path integral; n is [M][N] (FP64)."""
    a = np.ascontiguousarray(np.asarray(n, dtype=np.float64).reshape(M, N))
    _check(lib().lbe_init_density_quasipressure(ctx, _dp(a)), ctx)


SHELL_METHODS = {"auto": 0, "direct": 1, "spectral": 2}


def lbe_set_shell_method(ctx, method):
    """K3 method: "auto", "direct" (stencil sum) or "spectral" (FFT convolution)."""
    m = SHELL_METHODS[method] if isinstance(method, str) else int(method)
    _check(lib().lbe_set_shell_method(ctx, m), ctx)


def lbe_get_shell_method(ctx):
    """The K3 method the next step uses: "direct" or "spectral"."""
    v = (ctypes.c_int * 1)()
    _check(lib().lbe_get_shell_method(ctx, v), ctx)
    return {1: "direct", 2: "spectral"}[v[0]]


STAGES = ("density", "contact", "shell", "collide", "flux")


def lbe_set_stage_timing(ctx, on):
    _check(lib().lbe_set_stage_timing(ctx, int(bool(on))), ctx)


def lbe_get_stage_times(ctx):
    ms = np.zeros(5)
    n = (ctypes.c_longlong * 5)()
    _check(lib().lbe_get_stage_times(ctx, _dp(ms), n), ctx)
    return {STAGES[k]: (float(ms[k]), int(n[k])) for k in range(5)}


def lbe_get_mass_noalloc(ctx, M):
    """Species masses of the current state through the entry point that allocates no device memory
    (for callers that cannot allocate at the time of the call; see include/lbe.h)."""
    mass = np.zeros(M)
    _check(lib().lbe_get_mass_noalloc(ctx, _dp(mass)), ctx)
    return mass


def lbe_adjoint_flux_gradient(ctx, N, nsteps, ckpt_every, axis, plane):
    """(Phi, dPhi/damp [N], dPhi/dg [3]) of the flux averaged over the next nsteps steps (state unchanged)."""
    dA = np.zeros(N)
    dg = np.zeros(3)
    phi = ctypes.c_double(0.0)
    _check(lib().lbe_adjoint_flux_gradient(ctx, int(nsteps), int(ckpt_every), int(axis), int(plane), _dp(dA),
                                           _dp(dg), ctypes.byref(phi)), ctx)
    return phi.value, dA, dg


def lbe_status_string(status):
    return lib().lbe_status_string(int(status)).decode()


def lbe_last_error(ctx=None):
    return lib().lbe_last_error(ctx).decode(errors="replace")


# --------------------------------------------------------------------------
# Convenience wrapper (same calls, fewer arguments)
# --------------------------------------------------------------------------
class Simulation:
    """One lattice on the current CUDA device; every method is one C ABI call."""

    def __init__(self, shape, periodic=(1, 1, 1), nspecies=1, precision="fp32", consistent_moments=False,
                 check_every=0, use_torch_allocator=True, stream=None, scheme="dd_tr", visc=False):
        self.shape = tuple(int(v) for v in shape)
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        self.M = int(nspecies)
        self.precision = precision
        self._alloc = None
        if use_torch_allocator:
            self._alloc = TorchAllocator()
        if stream is None and use_torch_allocator:
            stream = current_stream_handle()
        self._h = lbe_create(self.shape, periodic, nspecies, precision, consistent_moments, check_every,
                             self._alloc, stream, scheme, visc)

    def close(self):
        if getattr(self, "_h", None):
            lbe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, solid):
        lbe_set_geometry(self._h, self.N, solid)

    def set_species(self, s, sigma, tau, mass=1.0):
        lbe_set_species(self._h, s, sigma, mass, tau)

    def set_potential(self, s, V):
        lbe_set_potential(self._h, self.N, s, V)

    def set_wall_potential(self, phi, amp):
        lbe_set_wall_potential(self._h, self.N, phi, amp)

    def set_body_force(self, s, g):
        lbe_set_body_force(self._h, s, g)

    def init_density(self, s, n):
        lbe_init_density(self._h, self.N, s, n)

    def step(self, nsteps=1):
        lbe_step(self._h, nsteps)

    def density(self, s):
        return lbe_get_density(self._h, self.N, s)

    def velocity(self, s=-1):
        return lbe_get_velocity(self._h, self.N, s)

    def momentum(self, s):
        return lbe_get_momentum(self._h, self.N, s)

    def force(self, s):
        return lbe_get_force(self._h, self.N, s)

    def contact(self, a, b):
        return lbe_get_contact(self._h, self.N, a, b)

    def set_flux_plane(self, axis, plane):
        lbe_set_flux_plane(self._h, axis, plane)

    def flux(self, s=-1):
        return lbe_get_flux(self._h, s)

    def reset_flux_average(self):
        lbe_reset_flux_average(self._h)

    def totals(self):
        return lbe_get_totals(self._h, self.M)

    def populations(self, s):
        return lbe_get_populations(self._h, self.N, s)

    def set_populations(self, s, f, g):
        lbe_set_populations(self._h, self.N, s, f, g)

    def step_count(self):
        return lbe_get_step_count(self._h)

    def link_mask(self):
        return lbe_get_link_mask(self._h, self.N)

    def save_state(self):
        return lbe_save_state(self._h)

    def load_state(self, state):
        lbe_load_state(self._h, state)

    def divergence(self, s=-1):
        """div u [N] of species s (-1: barycentric), isotropic D3Q19 gradient."""
        return lbe_get_divergence(self._h, self.N, s)

    def residual(self):
        """max |n(t) - n(t0)| / ((t - t0) n0) since the previous call (-1 on the first call)."""
        return lbe_get_residual(self._h)

    def launch_count(self):
        return lbe_get_launch_count(self._h)

    def adjoint_flux_gradient(self, nsteps, ckpt_every, axis, plane):
        return lbe_adjoint_flux_gradient(self._h, self.N, nsteps, ckpt_every, axis, plane)

    def init_density_quasipressure(self, n):
        lbe_init_density_quasipressure(self._h, self.M, self.N, n)

    def set_shell_method(self, method):
        lbe_set_shell_method(self._h, method)

    def shell_method(self):
        return lbe_get_shell_method(self._h)

    def set_stage_timing(self, on):
        lbe_set_stage_timing(self._h, on)

    def stage_times(self):
        """{stage: (device ms, launches)} since timing was enabled."""
        return lbe_get_stage_times(self._h)
