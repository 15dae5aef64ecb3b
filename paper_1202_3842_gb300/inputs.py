"""Seeded synthetic inputs: density noise, potential wells, channel geometry.

This module builds input arrays only (it holds none of the method's
arithmetic), so the CUDA library and the CPU oracle can be fed bit-identical
inputs.  Every generator is deterministic: the random numbers come from the
SplitMix64 generator (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) applied to ``seed XOR node_index``.

Units are lattice units (h = 1, dx = 1, m = 1); k_B T = v_T^2 = 1/3, so a
potential of ``D`` k_B T is ``D / 3``.  Arrays are flat with x fastest:
``i = x + nx * (y + ny * z)``.
"""
import math

import numpy as np

KT = 1.0 / 3.0
_M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output for state words ``x`` (uint64 numpy array)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(n, seed):
    """``n`` uniforms in [0, 1): SplitMix64(seed XOR i) / 2**64 for i = 0..n-1."""
    idx = np.arange(n, dtype=np.uint64)
    z = splitmix64(np.uint64(seed) ^ idx)
    # top 53 bits -> exactly representable double in [0, 1)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def packing_to_density(eta, sigma):
    """Number density of hard spheres of diameter sigma at packing fraction eta = (pi/6) n sigma^3."""
    return 6.0 * eta / (math.pi * sigma ** 3)


def noisy_density(shape, n0, amplitude=0.01, seed=1202, solid=None):
    """n(r) = n0 (1 + amplitude (2U - 1)) on fluid nodes, 0 on solid nodes."""
    nx, ny, nz = shape
    N = nx * ny * nz
    n = n0 * (1.0 + amplitude * (2.0 * uniform01(N, seed) - 1.0))
    if solid is not None:
        n = np.where(np.asarray(solid).reshape(-1) != 0, 0.0, n)
    return n


def uniform_density(shape, n0, solid=None):
    nx, ny, nz = shape
    n = np.full(nx * ny * nz, float(n0))
    if solid is not None:
        n = np.where(np.asarray(solid).reshape(-1) != 0, 0.0, n)
    return n


def _coords(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.reshape(-1).astype(np.float64), y.reshape(-1).astype(np.float64), z.reshape(-1).astype(np.float64)


def _min_image(d, L, periodic):
    if periodic:
        return d - L * np.round(d / L)
    return d


def radial_distance(shape, centre, periodic=(1, 1, 1)):
    x, y, z = _coords(shape)
    dx = _min_image(x - centre[0], shape[0], periodic[0])
    dy = _min_image(y - centre[1], shape[1], periodic[1])
    dz = _min_image(z - centre[2], shape[2], periodic[2])
    return np.sqrt(dx * dx + dy * dy + dz * dz)


def gaussian_well(shape, depth_kT, radius, centre=None, periodic=(1, 1, 1)):
    """V(r) = -D k_B T exp(-|r - r_c|^2 / (2 R^2)) with the minimum-image distance on periodic axes."""
    if centre is None:
        centre = tuple(s // 2 for s in shape)
    r = radial_distance(shape, centre, periodic)
    return -depth_kT * KT * np.exp(-(r * r) / (2.0 * radius * radius))


def cosine_well(shape, eps_kT, xi, centre=None, periodic=(1, 1, 1)):
    """Central well of the paper's ideal-fluid test: U = -eps (1 + cos(pi r / xi)) for r < xi, else 0."""
    if centre is None:
        centre = tuple(s // 2 for s in shape)
    r = radial_distance(shape, centre, periodic)
    return np.where(r < xi, -eps_kT * KT * (1.0 + np.cos(np.pi * r / xi)), 0.0)


def channel_mask(shape, width, length, walls=True):
    """Bottleneck channel: solid layers at y, z in {0, n-1}; a slit constriction narrowing y only.

    Solid where x in [xc - length/2, xc + length/2) and |y - (ny-1)/2| > width/2, xc = nx/2.
    Returns uint8 [N] (1 = solid)."""
    nx, ny, nz = shape
    x, y, z = _coords(shape)
    solid = np.zeros(nx * ny * nz, dtype=np.uint8)
    if walls:
        solid |= ((y == 0) | (y == ny - 1) | (z == 0) | (z == nz - 1)).astype(np.uint8)
    if length > 0:
        xc = nx // 2
        x0 = xc - length // 2
        x1 = xc + (length - length // 2)
        in_x = (x >= x0) & (x < x1)
        out_y = np.abs(y - (ny - 1) / 2.0) > width / 2.0
        solid |= (in_x & out_y).astype(np.uint8)
    return solid


def wall_distance(shape, solid, periodic, dmax=3):
    """Euclidean distance (in lattice units) from each fluid node to the nearest solid node within dmax,
    found by brute force over the (2 dmax + 1)^3 neighbourhood; +inf when none is that close."""
    nx, ny, nz = shape
    s = np.asarray(solid).reshape(nz, ny, nx).astype(bool)
    best = np.full((nz, ny, nx), np.inf)
    for dz in range(-dmax, dmax + 1):
        for dy in range(-dmax, dmax + 1):
            for dx in range(-dmax, dmax + 1):
                d = math.sqrt(dx * dx + dy * dy + dz * dz)
                if d > dmax:
                    continue
                sh = _shift(s, dx, dy, dz, periodic)
                best = np.where(sh & (d < best), d, best)
    best[s] = 0.0
    return best.reshape(-1)


def _shift(a, dx, dy, dz, periodic):
    """b[z,y,x] = a[z+dz, y+dy, x+dx], False outside non-periodic axes."""
    out = a
    for axis, d, per in ((2, dx, periodic[0]), (1, dy, periodic[1]), (0, dz, periodic[2])):
        if d == 0:
            continue
        out = np.roll(out, -d, axis=axis)
        if not per:
            idx = [slice(None)] * 3
            n = a.shape[axis]
            if d > 0:
                idx[axis] = slice(n - d, n)
            else:
                idx[axis] = slice(0, -d)
            out = out.copy()
            out[tuple(idx)] = False
    return out


def wall_shape(shape, solid, periodic, dmax=3):
    """phi(r) = exp(-d_wall(r)) for fluid nodes with d_wall <= dmax, else 0 (shape of the wall potential)."""
    d = wall_distance(shape, solid, periodic, dmax)
    s = np.asarray(solid).reshape(-1) != 0
    return np.where((~s) & np.isfinite(d), np.exp(-d), 0.0)


# ---------------------------------------------------------------------------
# Workloads.  Each is a plain description; ``build_workload`` turns it into arrays.
# ---------------------------------------------------------------------------

def well_workload(shape, sigma, eta, tau, depth_kT, radius, seed=1202, noise=0.01):
    shape = tuple(shape)
    n0 = packing_to_density(eta, sigma)
    return dict(kind="well", shape=shape, periodic=(1, 1, 1), sigma=[sigma], tau=[tau], n0=[n0],
                depth_kT=depth_kT, radius=radius, seed=seed, noise=noise, body=[(0.0, 0.0, 0.0)])


def channel_workload(shape, sigmas, eta_total, taus, width, length, body=1e-6, wall_amp_kT=0.0):
    shape = tuple(shape)
    sig = list(sigmas)
    # equal mole fraction: (pi/6) n sum sigma^3 = eta_total
    n = 6.0 * eta_total / (math.pi * sum(s ** 3 for s in sig))
    return dict(kind="channel", shape=shape, periodic=(1, 0, 0), sigma=sig, tau=list(taus), n0=[n] * len(sig),
                width=width, length=length, body=[(body, 0.0, 0.0)] * len(sig), wall_amp_kT=wall_amp_kT)


WORKLOADS = {
    # one-component spherical well, 24^3 periodic, sigma = 3, eta = 0.2, Gaussian well 1 kT / R = 5, tau = 1
    "well24": lambda: well_workload((24, 24, 24), 3.0, 0.2, 1.0, 1.0, 5.0),
    # one-component spherical well at production size: 256^3, sigma = 6, eta = 0.3, 2 kT / R = 24, tau = 0.8
    "well256": lambda: well_workload((256, 256, 256), 6.0, 0.3, 0.8, 2.0, 24.0),
    # same well at 160^3 (radius scaled to 15): the small case of the profiler captures
    "well160": lambda: well_workload((160, 160, 160), 6.0, 0.3, 0.8, 2.0, 15.0),
    # two-component bottleneck channel 512x128x128, sigma 4/6, eta 0.25, width 16, length 64, g = 1e-6
    "channel512": lambda: channel_workload((512, 128, 128), (4.0, 6.0), 0.25, (1.0, 1.0), 16, 64),
    # same channel at 128x32x32 (same absolute width and diameters)
    "channel128": lambda: channel_workload((128, 32, 32), (4.0, 6.0), 0.25, (1.0, 1.0), 16, 64),
    # adjoint channel 256x64x64, width 12, length 32, wall potential amplitude 1 kT
    "channel256adj": lambda: channel_workload((256, 64, 64), (4.0, 6.0), 0.25, (1.0, 1.0), 12, 32,
                                              wall_amp_kT=1.0),
    # adjoint oracle case 32x16x16, width 6, length 8
    "channel32adj": lambda: channel_workload((32, 16, 16), (4.0, 6.0), 0.25, (1.0, 1.0), 6, 8, wall_amp_kT=1.0),
}


def build_workload(w):
    """Arrays for a workload: solid [N] uint8, V [M][N], n_init [M][N], phi [N], amp [N]."""
    shape = w["shape"]
    N = shape[0] * shape[1] * shape[2]
    M = len(w["sigma"])
    if w["kind"] == "well":
        solid = np.zeros(N, dtype=np.uint8)
        V1 = gaussian_well(shape, w["depth_kT"], w["radius"], periodic=w["periodic"])
        V = np.stack([V1] * M)
        n = np.stack([noisy_density(shape, w["n0"][a], w["noise"], w["seed"] + a) for a in range(M)])
        phi = np.zeros(N)
        amp = np.zeros(N)
    else:
        solid = channel_mask(shape, w["width"], w["length"])
        V = np.zeros((M, N))
        n = np.stack([uniform_density(shape, w["n0"][a], solid) for a in range(M)])
        if w.get("wall_amp_kT", 0.0) > 0.0:
            phi = wall_shape(shape, solid, w["periodic"])
            amp = np.full(N, w["wall_amp_kT"] * KT)
        else:
            phi = np.zeros(N)
            amp = np.zeros(N)
    return dict(solid=solid, V=V, n=n, phi=phi, amp=amp)
