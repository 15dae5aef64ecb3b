"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances:
  FP64 path   densities  ||dn||_inf / max n <= 1e-12;
              velocities ||du||_inf <= 1e-12 * max(||u_oracle||_inf, 1e-6 v_T)
              (near-zero spurious currents are compared against a floor);
              contact values, forces and the flux to 1e-12 relative.
  FP32 path   density <= 1e-5 relative; spurious-current magnitude max|u| and
              the channel flux <= 1e-3 relative.
  16-bit      shifted BF16/FP16 storage: errors are measured and bounded
              loosely (density <= 1e-2 / 1e-3 relative after 50 steps).
Integer work (link mask, shell tables) is bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from lbe_cases import (CS, barycentric, case_channel, case_well, rel_err, setup_gpu, setup_oracle,
                       velocity_from)
from paper_1202_3842_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _u_tol(u_ref):
    return 1e-12 * max(np.abs(u_ref).max(), 1e-6 * CS)


def gpu_state(sim, M):
    n = np.stack([sim.density(a) for a in range(M)])
    J = np.stack([sim.momentum(a) for a in range(M)])
    return n, J


# ---------------------------------------------------------------------------
# integer work
# ---------------------------------------------------------------------------

def test_link_mask_bit_exact():
    w, arr = case_channel((40, 22, 18), (2.0, 4.0), 0.2, (1.0, 1.0), 8, 10)
    sim = setup_gpu(w, arr, "fp64")
    m = sim.link_mask()
    ref = oracle.link_mask(w["shape"], w["periodic"], arr["solid"])
    np.testing.assert_array_equal(m & ~np.uint32(1), ref)
    np.testing.assert_array_equal(m & np.uint32(1), arr["solid"].astype(np.uint32))


def test_populations_roundtrip_exact():
    w, arr = case_channel((20, 12, 10), (2.0,), 0.1, (1.0,), 4, 4)
    sim = setup_gpu(w, arr, "fp64")
    rng = np.random.default_rng(4)
    N = sim.N
    fl = arr["solid"] == 0
    f = np.where(fl[None, :], rng.random((19, N)) * 1e-3, 0.0)
    g = np.where(fl[None, :], rng.random((19, N)) * 1e-3, 0.0)
    sim.set_populations(0, f, g)
    f2, g2 = sim.populations(0)
    np.testing.assert_array_equal(f2, f)
    np.testing.assert_array_equal(g2, g)


# ---------------------------------------------------------------------------
# stage parity: contact values and shell force of a given state
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shell", ["direct", "spectral"])
@pytest.mark.parametrize("shape,sig", [((40, 22, 18), (2.0, 4.0)), ((37, 19, 35), (4.0, 6.0)),
                                       ((24, 24, 24), (3.0,))])
def test_stage_parity_fp64(shape, sig, shell):
    w, arr = case_channel(shape, sig, 0.25, (1.0,) * len(sig), 8, 10)
    rng = np.random.default_rng(8)
    fl = arr["solid"] == 0
    arr["n"] = arr["n"] * (1.0 + 0.2 * (rng.random(arr["n"].shape) - 0.5)) * fl[None, :]
    g = setup_gpu(w, arr, "fp64", shell=shell)
    assert g.shell_method() == shell
    o = setup_oracle(w, arr)
    obs = o.observe()
    M = len(sig)
    for a in range(M):
        np.testing.assert_allclose(g.density(a), obs["n"][a], rtol=1e-14, atol=0)
        for b in range(M):
            np.testing.assert_allclose(g.contact(a, b), obs["g"][a, b], rtol=1e-13)
        C = g.force(a)
        assert rel_err(C, obs["C"][a]) <= 1e-12


@pytest.mark.parametrize("shell", ["direct", "spectral"])
@pytest.mark.parametrize("sig,shape", [((1.0,), (40, 22, 20)), ((2.0, 4.0), (40, 22, 20)), ((4.0, 6.0), (40, 22, 20)),
                                       ((6.0, 8.0), (40, 22, 20)), ((8.0,), (40, 22, 20)), ((3.0, 5.0), (40, 22, 20)),
                                       ((4.0, 6.0), (70, 37, 41))])
def test_stage_parity_fp32_every_pair_diameter(sig, shape, shell):
    """K1-K3 of one FP32 state against the oracle for pair diameters 1 to 8 and both contact paths
    (compile-time balls for sigma 4/6, runtime rows otherwise, up to ball radius 4).  The FP32 shell
    tiles: two rows along y and three planes along z per thread for diameters 4 to 6 (32 x 16 outputs
    per plane, 18 planes per thread block); three outputs along z for 1 to 3, two at 7, one at 8.  Both
    lattices end in a partial tile along x, y and z; 70 x 37 x 41 spans three tiles along y and three
    z-blocks.  Tolerance: 1e-5 of the largest value of each field (FP32 sums over up to 762 shell
    points)."""
    w, arr = case_channel(shape, sig, 0.2, (1.0,) * len(sig), 10, 8)
    rng = np.random.default_rng(9)
    fl = arr["solid"] == 0
    arr["n"] = arr["n"] * (1.0 + 0.2 * (rng.random(arr["n"].shape) - 0.5)) * fl[None, :]
    g = setup_gpu(w, arr, "fp32", shell=shell)
    assert g.shell_method() == shell
    o = setup_oracle(w, arr)
    obs = o.observe()
    M = len(sig)
    for a in range(M):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-6
        for b in range(M):
            assert rel_err(g.contact(a, b), obs["g"][a, b]) <= 1e-5
        assert rel_err(g.force(a), obs["C"][a]) <= 1e-5


# ---------------------------------------------------------------------------
# FP64 dynamics
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shell", ["direct", "spectral"])
def test_fp64_parity_well24_200_steps(shell):
    """One-component spherical well, 24^3 periodic, sigma 3, eta 0.2, Gaussian well 1 kT / R 5, tau 1."""
    w, arr = case_well((24, 24, 24), 3.0, 0.2, 1.0, 1.0, 5.0)
    g = setup_gpu(w, arr, "fp64", shell=shell)
    o = setup_oracle(w, arr)
    g.step(200)
    o.step(200)
    obs = o.observe()
    n, J = gpu_state(g, 1)
    assert rel_err(n[0], obs["n"][0]) <= 1e-12
    u_ref = velocity_from(obs["n"][0], obs["J"][0])
    u = g.velocity(0)
    assert np.abs(u - u_ref).max() <= _u_tol(u_ref)
    assert np.abs(u_ref).max() / CS < 0.1  # spurious current stays small


@pytest.mark.parametrize("shell", ["direct", "spectral"])
def test_fp64_parity_channel_mixture_with_flux(shell):
    w, arr = case_channel((48, 24, 20), (4.0, 6.0), 0.25, (1.0, 0.8), 10, 12, body=1e-5)
    g = setup_gpu(w, arr, "fp64", shell=shell)
    o = setup_oracle(w, arr)
    g.set_flux_plane(0, 24)
    o.set_flux_plane(0, 24)
    g.step(40)
    o.step(40)
    obs = o.observe()
    n, J = gpu_state(g, 2)
    for a in range(2):
        assert rel_err(n[a], obs["n"][a]) <= 1e-12
        u_ref = velocity_from(obs["n"][a], obs["J"][a])
        assert np.abs(velocity_from(n[a], J[a]) - u_ref).max() <= _u_tol(u_ref)
    fs, cnt = o.flux()
    inst, avg = g.flux(-1)
    assert cnt == 40
    assert abs(avg - fs.sum() / cnt) <= 1e-12 * abs(fs.sum() / cnt)
    assert avg != 0.0


def test_fp64_parity_ideal_gas_and_consistent_moments():
    w, arr = case_well((20, 18, 16), 3.0, 0.1, 0.9, 1.0, 3.0)
    w["sigma"] = [0.0]  # ideal gas: no mean-field force
    arr["n"] = arr["n"] * 0 + 0.01
    g = setup_gpu(w, arr, "fp64")
    o = setup_oracle(w, arr)
    g.step(30)
    o.step(30)
    assert rel_err(g.density(0), o.observe()["n"][0]) <= 1e-12
    w, arr = case_well((20, 18, 16), 3.0, 0.1, 1.0, 0.3, 3.0)
    g = setup_gpu(w, arr, "fp64", consistent=True)
    o = setup_oracle(w, arr, consistent=True)
    g.step(20)
    o.step(20)
    obs = o.observe()
    assert rel_err(g.density(0), obs["n"][0]) <= 1e-12
    u_ref = velocity_from(obs["n"][0], obs["J"][0])
    assert np.abs(g.velocity(0) - u_ref).max() <= _u_tol(u_ref)


def test_mass_conservation_gpu_fp64():
    w, arr = case_channel((40, 20, 16), (4.0, 6.0), 0.25, (1.0, 1.0), 8, 10, body=1e-5)
    g = setup_gpu(w, arr, "fp64")
    m0, _, _ = g.totals()
    g.step(60)
    m1, P, umax = g.totals()
    np.testing.assert_allclose(m1, m0, rtol=1e-13)
    assert P[0] > 0 and umax > 0


# ---------------------------------------------------------------------------
# FP32 and shifted 16-bit storage against the FP64 oracle
# ---------------------------------------------------------------------------

def test_fp32_well24_against_oracle():
    w, arr = case_well((24, 24, 24), 3.0, 0.2, 1.0, 1.0, 5.0)
    g = setup_gpu(w, arr, "fp32")
    o = setup_oracle(w, arr)
    g.step(200)
    o.step(200)
    obs = o.observe()
    n = g.density(0)
    assert rel_err(n, obs["n"][0]) <= 1e-5
    u_ref = velocity_from(obs["n"][0], obs["J"][0])
    umax_ref = np.sqrt((u_ref ** 2).sum(0)).max()
    umax = np.sqrt((g.velocity(0) ** 2).sum(0)).max()
    assert abs(umax - umax_ref) <= 1e-3 * umax_ref


def test_fp32_channel_flux_against_oracle():
    w, arr = case_channel((64, 24, 20), (4.0, 6.0), 0.25, (1.0, 1.0), 10, 16, body=1e-5)
    g = setup_gpu(w, arr, "fp32")
    o = setup_oracle(w, arr)
    g.set_flux_plane(0, 32)
    o.set_flux_plane(0, 32)
    g.step(60)
    o.step(60)
    fs, cnt = o.flux()
    ref = fs.sum() / cnt
    _, avg = g.flux(-1)
    assert abs(avg - ref) <= 1e-3 * abs(ref)
    obs = o.observe()
    for a in range(2):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-5


@pytest.mark.parametrize("prec,tol", [("bf16", 1e-2), ("fp16", 1e-3)])
@pytest.mark.parametrize("shell", ["direct", "spectral"])
def test_shifted_16bit_against_oracle(prec, tol, shell):
    w, arr = case_channel((64, 24, 20), (4.0, 6.0), 0.25, (1.0, 1.0), 10, 16, body=1e-5)
    g = setup_gpu(w, arr, prec, shell=shell)
    o = setup_oracle(w, arr)
    g.set_flux_plane(0, 32)
    o.set_flux_plane(0, 32)
    g.step(50)
    o.step(50)
    obs = o.observe()
    for a in range(2):
        assert rel_err(g.density(a), obs["n"][a]) <= tol
    fs, cnt = o.flux()
    _, avg = g.flux(-1)
    assert abs(avg - fs.sum() / cnt) <= 0.2 * abs(fs.sum() / cnt)


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------

def test_invalid_arguments_and_divergence_flag():
    from paper_1202_3842_gb300 import lbe
    w, arr = case_well((16, 16, 16), 3.0, 0.2, 1.0, 1.0, 4.0)
    g = setup_gpu(w, arr, "fp32")
    with pytest.raises(lbe.LbeError) as e:
        g.set_species(0, 3.0, 0.5)
    assert e.value.status == 1
    with pytest.raises(lbe.LbeError) as e:
        g.set_species(0, 3.0, 1.0, mass=2.0)
    assert e.value.status == 2
    with pytest.raises(lbe.LbeError) as e:
        g.set_species(0, 3.5, 1.0)
        g.step(1)
    assert e.value.status == 2
    g.set_species(0, 3.0, 1.0)
    f, gq = g.populations(0)
    f[:, 100] = np.nan
    g.set_populations(0, f, gq)
    g.step(2)
    with pytest.raises(lbe.LbeError) as e:
        g.density(0)
    assert e.value.status == 5


def test_check_every_reports_divergence_from_step():
    from paper_1202_3842_gb300 import lbe
    w, arr = case_well((16, 16, 16), 3.0, 0.2, 1.0, 1.0, 4.0)
    g = setup_gpu(w, arr, "fp32", check_every=1)
    f, gq = g.populations(0)
    f[:, 7] = -1.0
    g.set_populations(0, f, gq)
    with pytest.raises(lbe.LbeError) as e:
        g.step(1)
    assert e.value.status == 5


# ---------------------------------------------------------------------------
# full size (256^3, sigma 6, the benchmark launch configuration): sampled
# nodes against oracle runs on periodic sub-boxes around each sample
# ---------------------------------------------------------------------------

def _subbox(field, shape, centre, R):
    nx, ny, nz = shape
    f = field.reshape(nz, ny, nx)
    xs = [(centre[0] + d) % nx for d in range(-R, R + 1)]
    ys = [(centre[1] + d) % ny for d in range(-R, R + 1)]
    zs = [(centre[2] + d) % nz for d in range(-R, R + 1)]
    return f[np.ix_(zs, ys, xs)].reshape(-1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_well256_sampled(prec):
    w = inputs.WORKLOADS["well256"]()
    arr = inputs.build_workload(w)
    g = setup_gpu(w, arr, prec)
    g.step(1)
    n = g.density(0)
    J = g.momentum(0)
    shape = w["shape"]
    R = 20  # the density and momentum after one step depend on n(0) within 1 + 6 + 3 + 6 + 3 = 19
    L = 2 * R + 1
    rng = np.random.default_rng(0)
    samples = [(128, 128, 128), (128 + 24, 128, 128), (0, 0, 0), (255, 3, 130)]
    samples += [tuple(int(v) for v in rng.integers(0, 256, 3)) for _ in range(3)]
    tol_n = 1e-12 if prec == "fp64" else 1e-5
    for (x, y, z) in samples:
        sub_n = _subbox(arr["n"][0], shape, (x, y, z), R)
        sub_V = _subbox(arr["V"][0], shape, (x, y, z), R)
        o = oracle.Sim((L, L, L), (1, 1, 1), 1)
        o.set_species(0, w["sigma"][0], w["tau"][0])
        o.set_potential(0, sub_V)
        o.init_density(0, sub_n)
        o.step(1)
        obs = o.observe()
        c = R + L * (R + L * R)
        i = x + shape[0] * (y + shape[1] * z)
        assert abs(n[i] - obs["n"][0][c]) <= tol_n * obs["n"][0][c]
        Jref = obs["J"][0][:, c]
        Jscale = max(np.abs(Jref).max(), 1e-6 * CS * w["n0"][0])
        assert np.abs(J[:, i] - Jref).max() <= (1e-12 if prec == "fp64" else 1e-3) * Jscale
    # a property that holds at any size: the mass is unchanged by the step
    m0 = arr["n"][0].sum()
    assert abs(n.sum() - m0) <= (1e-12 if prec == "fp64" else 1e-6) * m0


def _subbox_channel(field, shape, centre, R, fill):
    """Sub-box of a channel field: periodic along x, `fill` beyond the closed y and z axes."""
    nx, ny, nz = shape
    f = field.reshape(nz, ny, nx)
    xs = [(centre[0] + d) % nx for d in range(-R, R + 1)]
    out = np.full((2 * R + 1, 2 * R + 1, 2 * R + 1), fill, dtype=field.dtype)
    for kz, z in enumerate(range(centre[2] - R, centre[2] + R + 1)):
        if not 0 <= z < nz:
            continue
        for ky, y in enumerate(range(centre[1] - R, centre[1] + R + 1)):
            if 0 <= y < ny:
                out[kz, ky, :] = f[z, y, xs]
    return out.reshape(-1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_full_size_channel512_sampled(prec):
    """The two-component bottleneck channel at its benchmark size and launch configuration: after one
    step, n and J of both species at sampled nodes (bulk, near the walls, at the constriction's corners
    and in its slit) equal the oracle's step of the sub-box around each sample.  Nodes beyond the closed
    axes are solid in the sub-box (the walls already shield them; solid and outside both read as no
    fluid).  One step of n and J depends on the initial state within 1 + 6 + 3 + 6 + 3 = 19 nodes.

    Tolerances: n as in the other parity tests.  After one step from rest under g = 1e-6 the momentum is
    about 1e-6 of the populations' momentum scale n0 v_T, while J is a sum of populations of that scale:
    its absolute round-off is a few eps n0 v_T (FP32: 4e-11 against J = 2.6e-9 in the bulk), and its
    components that vanish by symmetry carry only round-off.  The J check is therefore 1e-12 (FP64) or
    1e-3 (FP32) of |J| plus a round-off floor of 1e3 eps n0 v_T (FP64) or 4 eps n0 v_T (FP32)."""
    w = inputs.WORKLOADS["channel512"]()
    arr = inputs.build_workload(w)
    g = setup_gpu(w, arr, prec)
    g.step(1)
    n = np.stack([g.density(a) for a in range(2)])
    J = np.stack([g.momentum(a) for a in range(2)])
    shape = w["shape"]
    R = 20
    L = 2 * R + 1
    # bulk; the slit's centre; fluid at the corners before, at the entry of, at the exit of and after the
    # constriction; the slit next to a z wall; a y-z corner; the periodic x seam by a wall; one solid node
    samples = [(100, 64, 64), (256, 64, 64), (223, 55, 64), (224, 56, 64), (287, 71, 30), (288, 72, 30),
               (256, 57, 2), (5, 1, 126), (511, 126, 64), (230, 100, 100)]
    tol_n = 1e-12 if prec == "fp64" else 1e-5
    for (x, y, z) in samples:
        o = oracle.Sim((L, L, L), (0, 0, 0), 2)
        o.set_geometry(_subbox_channel(arr["solid"], shape, (x, y, z), R, 1))
        for a in range(2):
            o.set_species(a, w["sigma"][a], w["tau"][a])
            o.set_body_force(a, w["body"][a])
            o.init_density(a, _subbox_channel(arr["n"][a], shape, (x, y, z), R, 0.0))
        o.step(1)
        obs = o.observe()
        c = R + L * (R + L * R)
        i = x + shape[0] * (y + shape[1] * z)
        for a in range(2):
            nref = obs["n"][a][c]
            assert abs(n[a, i] - nref) <= tol_n * max(nref, w["n0"][a]), (x, y, z, a, n[a, i], nref)
            Jref = obs["J"][a][:, c]
            floor = (1e3 * np.finfo(np.float64).eps if prec == "fp64" else 4 * np.finfo(np.float32).eps) \
                * w["n0"][a] * CS
            tolJ = (1e-12 if prec == "fp64" else 1e-3) * np.abs(Jref).max() + floor
            assert np.abs(J[a, :, i] - Jref).max() <= tolJ, (x, y, z, a, J[a, :, i], Jref)
    # a property that holds at any size: the step conserves the mass of each species
    for a in range(2):
        m0 = arr["n"][a].sum()
        assert abs(n[a].sum() - m0) <= (1e-12 if prec == "fp64" else 1e-6) * m0
    g.close()
