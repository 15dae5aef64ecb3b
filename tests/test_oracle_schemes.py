"""Pins of the oracle's scheme ablations (Sec. "Results": single (SD) or double (DD) distribution, Euler (EU)
or trapezoidal (TR) integration).

- Without the mean-field functional (sigma = 0) and with g~ = f~ at the start, the single- and double-
  distribution forms of the same integrator coincide exactly: SD-TR = DD-TR and SD-EU = DD-EU, bit for bit.
- With C = 0 the Euler update is the textbook BGK step with the second-order Hermite force term and no
  velocity shift, relaxing at 1/tau (an independent numpy restatement).
- Every scheme conserves the mass of every species; in a periodic box without external force every scheme
  conserves the total momentum (the SD forms because the mean-field forces cancel pairwise, the DD forms
  because S_g carries no first moment of C).
- A uniform body force adds exactly n g per step to the momentum in every scheme.
"""
import numpy as np
import pytest

import oracle
from paper_1202_3842_gb300 import inputs

CS2 = 1.0 / 3.0
DD_TR, SD_TR, SD_EU, DD_EU = 0, 1, 2, 3


def _ideal_well(scheme, shape=(8, 7, 6), tau=0.9, seed=2):
    N = int(np.prod(shape))
    sim = oracle.Sim(shape, (1, 1, 1), 1)
    sim.set_scheme(scheme)
    sim.set_species(0, 0.0, tau)
    V = inputs.gaussian_well(shape, 1.0, 2.0)
    sim.set_potential(0, V)
    sim.set_body_force(0, (1e-4, -2e-4, 0.0))
    c, w, _ = oracle.lattice()
    rng = np.random.default_rng(seed)
    n = 0.01 * (1 + 0.2 * (rng.random(N) - 0.5))
    u = 0.03 * (rng.random((3, N)) - 0.5)
    f0 = w[:, None] * n * (1 + (c @ u) / CS2)
    sim.set_populations(0, f0, f0)
    return sim, V, f0


@pytest.mark.parametrize("sd, dd", [(SD_TR, DD_TR), (SD_EU, DD_EU)])
def test_single_and_double_distribution_coincide_without_mean_field(sd, dd):
    a, _, _ = _ideal_well(sd)
    b, _, _ = _ideal_well(dd)
    a.step(6)
    b.step(6)
    fa, ga = a.get_populations(0)
    fb, gb = b.get_populations(0)
    assert np.array_equal(fa, fb)
    assert np.array_equal(ga, gb)
    assert np.array_equal(ga, fa)  # SD keeps g = f
    oa, ob = a.observe(), b.observe()
    assert np.array_equal(oa["J"], ob["J"])


def _euler_textbook_step(f, shape, Fext, tau):
    """D3Q19 BGK step with the second-order Hermite force term, Euler form (no velocity shift, force
    applied with weight h = 1), pull streaming on a periodic grid."""
    c, w, _ = oracle.lattice()
    c = c.astype(float)
    nx, ny, nz = shape
    n = f.sum(0)
    Fd = n[None, :] * Fext
    u = (c.T @ f) / n
    cu = c @ u
    uu = (u * u).sum(0)
    feq = w[:, None] * n * (1 + cu / CS2 + cu * cu / (2 * CS2 ** 2) - uu / (2 * CS2))
    cF = c @ Fd
    uF = (u * Fd).sum(0)
    Fp = w[:, None] * (cF / CS2 - uF / CS2 + cu * cF / CS2 ** 2)
    post = f - (f - feq) / tau + Fp
    out = np.empty_like(post)
    P = post.reshape(19, nz, ny, nx)
    for p in range(19):
        out[p] = np.roll(P[p], shift=(c[p, 2].astype(int), c[p, 1].astype(int), c[p, 0].astype(int)),
                         axis=(0, 1, 2)).reshape(-1)
    return out


@pytest.mark.parametrize("scheme", [SD_EU, DD_EU])
def test_ideal_gas_euler_step_is_textbook_forcing(scheme):
    shape, tau = (8, 7, 6), 0.9
    sim, V, f0 = _ideal_well(scheme, shape, tau)
    Fext = oracle.force_field(shape, (1, 1, 1), V, (1e-4, -2e-4, 0.0))
    f = f0.copy()
    for _ in range(3):
        sim.step(1)
        f = _euler_textbook_step(f, shape, Fext, tau)
        fo, go = sim.get_populations(0)
        np.testing.assert_allclose(fo, f, rtol=1e-13, atol=1e-19)
        np.testing.assert_allclose(go, f, rtol=1e-13, atol=1e-19)


def _hard_sphere_box(scheme, shape=(10, 9, 8), taus=(0.8, 0.8)):
    N = int(np.prod(shape))
    sim = oracle.Sim(shape, (1, 1, 1), 2)
    sim.set_scheme(scheme)
    sim.set_species(0, 3.0, taus[0])
    sim.set_species(1, 2.0, taus[1])
    c, w, _ = oracle.lattice()
    rng = np.random.default_rng(1)
    for a, n0 in enumerate((0.012, 0.006)):
        n = n0 * (1 + 0.1 * (rng.random(N) - 0.5))
        u = 0.02 * (rng.random((3, N)) - 0.5)
        f = w[:, None] * n[None, :] * (1 + (c @ u) / CS2)
        sim.set_populations(a, f, f)
    return sim


@pytest.mark.parametrize("scheme", [SD_TR, SD_EU, DD_EU])
def test_mass_and_momentum_conserved_hard_spheres(scheme):
    sim = _hard_sphere_box(scheme)
    o0 = sim.observe()
    m0, P0 = o0["n"].sum(axis=1), o0["J"].sum(axis=(0, 2))
    assert np.abs(o0["C"]).max() > 1e-6  # the mean field is active
    sim.step(12)
    o1 = sim.observe()
    np.testing.assert_allclose(o1["n"].sum(axis=1), m0, rtol=1e-13)
    assert np.abs(P0).max() > 1e-4
    np.testing.assert_allclose(o1["J"].sum(axis=(0, 2)), P0, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("scheme", [SD_TR, SD_EU])
def test_single_distribution_momentum_conserved_with_unequal_tau(scheme):
    # each species' momentum changes by exactly its C per step, whatever tau; the pair forces cancel
    sim = _hard_sphere_box(scheme, taus=(0.8, 1.3))
    P0 = sim.observe()["J"].sum(axis=(0, 2))
    sim.step(10)
    np.testing.assert_allclose(sim.observe()["J"].sum(axis=(0, 2)), P0, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("scheme", [DD_TR, SD_TR, SD_EU, DD_EU])
def test_body_force_adds_n_g_per_step(scheme):
    shape = (6, 5, 4)
    N = int(np.prod(shape))
    gb = np.array([2e-4, -1e-4, 5e-5])
    sim = oracle.Sim(shape, (1, 1, 1), 1)
    sim.set_scheme(scheme)
    sim.set_species(0, 0.0, 0.7)
    sim.set_body_force(0, gb)
    n0 = 0.02
    sim.init_density(0, np.full(N, n0))
    P0 = sim.observe()["J"].sum(axis=(0, 2))
    k = 9
    sim.step(k)
    P1 = sim.observe()["J"].sum(axis=(0, 2))
    np.testing.assert_allclose(P1 - P0, k * N * n0 * gb, rtol=1e-11)
