"""Pins of the oracle's three readings of the DD-TR moment recovery (Sec. "Hard sphere fluid mixture in a
potential well", moment equations and S_g; Sec. "Stabilization", the evolution equation of g):

  0  as printed:      J = J~ + (C^mf + nF)/2,  Pi = Pi~ - C^mf.u^a/2   (the library's default)
  1  map-consistent:  the map g = g~ + Omega/2 applied to the printed S_g: J = J~ + nF/2,
                      Pi = Pi~ + beta C^mf.u^a/2
  2  as 1, with the d Pi/d n term of the continuum S_g that the discrete S_g drops

Each test checks a reading against something the mathematics fixes: the moments that one collision
adds (derived from the BGK relaxation and the source moments, not from the recovery formulas), the
long-wave sound speed (Carnahan-Starling for the hard-sphere fluid, v_T for the ideal gas), and the
rest state in a planar well (it cannot depend on the relaxation time and must satisfy the
chemical-potential balance c_s^2 grad n = C^mf + n F).  Where a reading fails one of them, the test
asserts the measured failure, so that any change of it shows.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1202_3842_gb300 import inputs

KT = 1.0 / 3.0
CS2 = 1.0 / 3.0
BETA = 3.0


def _planar_well(reading, tau, steps, eta=0.1, sigma=3.0, L=64, depth_kT=0.3, R=8.0):
    """Rest state of one species in a planar Gaussian well on an L x 1 x 1 periodic lattice, from a
    uniform start: (density contrast (max - min)/n0, max|u|/v_T, chemical-potential balance residual
    max|c_s^2 grad n - C - n F| over the scale max|C| + max|n F|)."""
    sim = oracle.Sim((L, 1, 1), (1, 1, 1), 1)
    sim.set_species(0, sigma, tau)
    sim.set_consistent_moments(reading)
    x = np.arange(L, dtype=float)
    sim.set_potential(0, -depth_kT * KT * np.exp(-((x - L / 2) ** 2) / (2 * R * R)))
    n0 = inputs.packing_to_density(eta, sigma)
    sim.init_density(0, np.full(L, n0))
    sim.step(steps)
    o = sim.observe()
    sim.close()
    n, J, C, F = o["n"][0], o["J"][0, 0], o["C"][0, 0], o["F"][0, 0]
    if not np.all(np.isfinite(n)):
        return float("nan"), float("nan"), float("nan")
    grad = (np.roll(n, -1) - np.roll(n, 1)) / 2.0  # the isotropic D3Q19 gradient of a field of x only
    resid = np.abs(CS2 * grad - C - n * F).max() / (np.abs(C).max() + np.abs(n * F).max())
    return (n.max() - n.min()) / n0, np.abs(J / n).max() / math.sqrt(CS2), resid


# ---------------------------------------------------------------------------
# one collision: moments added to f~ and g~
# ---------------------------------------------------------------------------

def _one_collision(reading):
    """A periodic two-species state with hard spheres and a potential, stepped once.  Streaming on a
    periodic lattice without walls is a permutation, so the post-collision populations are the streamed
    ones shifted back.  Returns the pre-collision moments and fields and the post-collision moments."""
    shape = (8, 7, 6)
    N = shape[0] * shape[1] * shape[2]
    c, w, _ = oracle.lattice()
    sig, taus = (2.0, 3.0), (0.8, 1.3)
    sim = oracle.Sim(shape, (1, 1, 1), 2)
    sim.set_consistent_moments(reading)
    x, y, z = (np.arange(N) % shape[0], (np.arange(N) // shape[0]) % shape[1], np.arange(N) // (shape[0] * shape[1]))
    pre = {}
    for a in range(2):
        sim.set_species(a, sig[a], taus[a])
        sim.set_potential(a, 0.05 * KT * (np.sin(2 * np.pi * x / shape[0]) + np.cos(2 * np.pi * y / shape[1])))
        n0 = inputs.packing_to_density(0.08, sig[a])
        n = inputs.noisy_density(shape, n0, 0.05, 7 + a) * (1 + 0.1 * np.sin(2 * np.pi * z / shape[2]))
        u = 0.02 * np.stack([np.cos(2 * np.pi * y / shape[1]), np.sin(2 * np.pi * x / shape[0]), 0 * x])
        f = np.array([w[p] * n * (1 + (c[p] @ u) / CS2) for p in range(19)])
        g = f * (1 + 0.03 * (a + 1))
        sim.set_populations(a, f, g)
        pre[a] = (f, g)
    o = sim.observe()
    sim.step(1)
    post = {}
    for a in range(2):
        fs, gs = sim.get_populations(a)
        fp, gp = np.empty_like(fs), np.empty_like(gs)
        for p in range(19):
            # f~(r, t+1)_p = f~*(r - c_p): shift back by -c_p
            for arr, out in ((fs, fp), (gs, gp)):
                v = arr[p].reshape(shape[2], shape[1], shape[0])
                v = np.roll(v, (-c[p, 2], -c[p, 1], -c[p, 0]), axis=(0, 1, 2))
                out[p] = v.reshape(-1)
        post[a] = (fp, gp)
    sim.close()
    return c.astype(float), taus, pre, post, o


@pytest.mark.parametrize("reading", [0, 1, 2])
def test_one_collision_adds_the_moments_of_the_reading(reading):
    """One TR collision adds h [omega (M_eq - M~) + M_S]/(1 + omega h/2) to each moment M~, with M_eq and
    M_S the moments of the equilibrium and of the source.  The mass of f and the momentum of g are
    relaxed to their own values (f_eq has zeroth moment n, g_eq has first moment J), so:
      f: zeroth moment unchanged;
      g: first moment + nF + (C^mf/2)(omega/(1 + omega/2)) = nF + C^mf/(2 tau) under the printed J
         (g_eq's momentum J then exceeds J~ by (C^mf + nF)/2), and + nF under the map-consistent J;
      g: zeroth moment + beta C^mf.u^a (the zeroth moment of S_g) under the map-consistent Pi, and
         + (beta - omega/2) C^mf.u^a/(1 + omega/2) under the printed Pi = Pi~ - C^mf.u^a/2
         (reading 2 adds its d Pi/d n term there and is not checked on that moment).
    A slip of sign, of 1/2 or of beta in the C^mf terms of the recovery or of S_g breaks one of these."""
    c, taus, pre, post, o = _one_collision(reading)
    for a in range(2):
        omega = 1.0 / (taus[a] - 0.5)
        f, g = pre[a]
        fp, gp = post[a]
        n, C, F = o["n"][a], o["C"][a], o["F"][a]
        nF = n * F
        scale = np.abs(g).sum(0).max()
        np.testing.assert_allclose(fp.sum(0), f.sum(0), rtol=0, atol=1e-14 * scale)
        dJ = np.einsum("pi,pn->in", c, gp - g)
        expect = nF + (C / (2.0 * taus[a]) if reading == 0 else 0.0)
        assert np.abs(C).max() > 1e-3 * np.abs(nF).max()  # the hard-sphere force is not negligible here
        np.testing.assert_allclose(dJ, expect, rtol=0, atol=1e-13 * scale)
        if reading == 2:
            continue
        ua = o["J"][a] / n
        Cu = (C * ua).sum(0)
        dPi = (gp - g).sum(0)
        expect0 = BETA * Cu if reading == 1 else (BETA - omega / 2.0) * Cu / (1.0 + omega / 2.0)
        np.testing.assert_allclose(dPi, expect0, rtol=0, atol=1e-13 * scale)
        assert np.abs(expect0).max() > 1e6 * 1e-13 * scale  # far above the round-off of the population sums


# ---------------------------------------------------------------------------
# long-wave sound speed
# ---------------------------------------------------------------------------

def _sound_speed(reading, eta, sigma=2.0, tau=1.0, L=128, steps=400, u0=1e-4):
    """Speed of a standing wave of wavelength L along x from a uniform density with the velocity profile
    u0 sin(kx): twice the time between the first two zero crossings of the momentum mode is the period."""
    c, w, _ = oracle.lattice()
    sim = oracle.Sim((L, 1, 1), (1, 1, 1), 1)
    sim.set_species(0, sigma, tau)
    sim.set_consistent_moments(reading)
    x = np.arange(L)
    k = 2 * np.pi / L
    n0 = inputs.packing_to_density(eta, sigma)
    u = u0 * np.sin(k * x)
    f = np.array([w[p] * n0 * (1 + c[p, 0] * u / CS2) for p in range(19)])
    sim.set_populations(0, f, f)
    b = []
    for _ in range(steps):
        b.append(float((sim.observe()["J"][0, 0] * np.sin(k * x)).sum()))
        sim.step(1)
    sim.close()
    z = [t + b[t] / (b[t] - b[t + 1]) for t in range(len(b) - 1) if b[t] * b[t + 1] < 0]
    return L / (2.0 * (z[1] - z[0])) / math.sqrt(CS2)


def _cs_speed(eta):
    """Carnahan-Starling sound speed over v_T: c^2 = dp/dn = v_T^2 (1 + 4 eta + 4 eta^2 - 4 eta^3 + eta^4)/(1 - eta)^4."""
    return math.sqrt((1 + 4 * eta + 4 * eta ** 2 - 4 * eta ** 3 + eta ** 4) / (1 - eta) ** 4)


@pytest.mark.parametrize("eta", [0.05, 0.1])
def test_sound_speed_of_each_reading(eta):
    """With the d Pi/d n term, Pi follows the quasi-pressure n + beta p_ex(n) as the density changes, so
    the g-momentum feels the hard-sphere pressure and a long sound wave runs at the Carnahan-Starling
    speed (the local limit of the BMCSL contact value, Sec. "Stabilization").  Without it Pi carries
    only the ideal-gas pressure and the g-system runs at v_T; the printed recovery, which feeds part of
    C^mf into the g-momentum directly (C^mf/(2 tau) per step), runs in between.  A wrong factor in
    d Pi/d n (its contact-value term or its derivative term, the latter 12% of it at packing 0.1)
    moves the first speed by more than the tolerance."""
    cs = _cs_speed(eta)
    c2 = _sound_speed(2, eta)
    c1 = _sound_speed(1, eta)
    c0 = _sound_speed(0, eta)
    assert abs(c2 / cs - 1.0) < 2e-3, (c2, cs)
    assert abs(c1 - 1.0) < 1e-3, c1
    assert 1.0 + 0.05 < c0 < cs - 0.05, (c0, cs)


# ---------------------------------------------------------------------------
# rest state in a planar well
# ---------------------------------------------------------------------------

def test_printed_recovery_rest_state_depends_on_the_relaxation_time():
    """A static equilibrium cannot depend on the relaxation time, yet under the printed recovery the
    g-momentum gains C^mf/(2 tau) per collision (test above), so the hard-sphere force enters the rest
    state with a tau-dependent weight and leaves a steady current.  This pins the measured behaviour of
    the library's default reading: on the planar well (sigma 3, packing 0.1, 0.3 k_B T) the density
    contrast rises from 0.0995 at tau 0.7 to 0.1084 at tau 1.0 (8.5%), the chemical-potential balance
    misses by 15-20% of the force scale, and the current stays near 1e-3 v_T."""
    res = {tau: _planar_well(0, tau, 12000) for tau in (0.7, 1.0)}
    c07, c10 = res[0.7][0], res[1.0][0]
    assert abs(c07 - 0.0995) < 1e-3 and abs(c10 - 0.1084) < 1e-3, res
    assert 0.07 < (c10 - c07) / c10 < 0.10, res
    for tau, (_, u, resid) in res.items():
        assert 0.1 < resid < 0.25, res
        assert 5e-4 < u < 3e-3, res


def test_dpi_dn_rest_state_is_tau_independent_and_balanced():
    """With the d Pi/d n term (reading 2) the rest state in the planar well is the same at every relaxation
    time, satisfies the chemical-potential balance to the lattice's discretisation error (0.27% of the
    force scale at this resolution), and the current decays to round-off.  The map-consistent reading has
    the same rest state (its equations differ only away from rest), reached by 8000 steps."""
    res = {tau: _planar_well(2, tau, 12000) for tau in (0.9, 1.0, 1.2)}
    ref = res[1.0][0]
    for tau, (contrast, u, resid) in res.items():
        assert abs(contrast / ref - 1.0) < 1e-6, res
        assert resid < 3e-3, res
        assert u < 1e-7, res
    c1, u1, r1 = _planar_well(1, 1.0, 8000)
    assert abs(c1 / ref - 1.0) < 1e-4 and r1 < 3e-3, (c1, ref, r1)
    # the hard-sphere fluid is less compressible than the ideal gas in the same well: its contrast lies
    # below the barometric one, exp(beta V) over its mean
    x = np.arange(64, dtype=float)
    V = -0.3 * KT * np.exp(-((x - 32) ** 2) / (2 * 64.0))
    nid = np.exp(-BETA * V)
    assert ref < (nid.max() - nid.min()) / nid.mean()


def test_map_consistent_rest_state_is_not_stationary():
    """The map-consistent reading reaches the balanced rest state (8000 steps: current 6e-6 v_T), but
    nothing restores Pi once it drifts from the quasi-pressure, and on this well the current grows again:
    by 12000 steps it is above 1e-2 v_T at tau 1.0, and the run at tau 0.7 has diverged."""
    _, u8, r8 = _planar_well(1, 1.0, 8000)
    assert u8 < 1e-5 and r8 < 3e-3, (u8, r8)
    _, u12, _ = _planar_well(1, 1.0, 12000)
    assert not (u12 < 1e-2), u12
    c07, _, _ = _planar_well(1, 0.7, 12000)
    assert not np.isfinite(c07)


def test_dpi_dn_term_is_unstable_at_the_benchmark_packing():
    """The d Pi/d n term gives the g-system the hard-sphere sound speed, which at packing 0.2 (the 24^3
    well) is 2.17 v_T = 1.25 lattice units per step, faster than the lattice links carry.  The planar well
    at packing 0.2 diverges under it within 4000 steps at every relaxation time tried, which is why the
    library keeps the printed recovery as its default."""
    for tau in (0.9, 1.0, 1.5):
        c, _, _ = _planar_well(2, tau, 4000, eta=0.2)
        assert not np.isfinite(c), (tau, c)
    assert _cs_speed(0.2) * math.sqrt(CS2) > 1.0
