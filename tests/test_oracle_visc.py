"""Pins of the oracle's viscous Enskog force C^{a,visc} (Appendix: the shell integral of
k^ g n_b k^.(u_b(r + sigma k^) - u_b(r)) with 2 sigma^2 sqrt(m k_B T / pi)).

- The paper's uniform-fluid limit: for a shear wave u_x = A cos(k y) the force is n eta lap(u_x) with
  eta = (4 pi / 15) sigma^4 sqrt(m k_B T / pi) g n, and for a compressional wave u_x = A cos(k x) it is
  n (eta + eta_b + eta / 3) lap(u_x) = 3 n eta lap(u_x) with the paper's eta_b = 5 eta / 3.  The lattice
  shell reproduces both within its isotropy error (5%); a wrong power of sigma, a dropped factor or a
  sign error fails them.  The transverse components vanish.
- A uniform velocity gives no force.
- One species: the force is antisymmetric across each pair of nodes, so it adds no total momentum.
"""
import numpy as np
import pytest

import oracle

KT = 1.0 / 3.0


def _wave(sig, L, mode):
    shape = (L, L, L)
    N = L ** 3
    i = np.arange(N)
    x, y = i % L, (i // L) % L
    k = 2 * np.pi / L
    A = 1e-3
    n0 = 6 * 0.2 / (np.pi * sig ** 3)
    n = np.full((1, N), n0)
    u = np.zeros((1, 3, N))
    arg = k * (y if mode == "shear" else x)
    u[0, 0] = A * np.cos(arg)
    g = oracle.contact_values(shape, (1, 1, 1), [sig], n)
    V = oracle.visc_force(shape, (1, 1, 1), [sig], n, u, g)
    eta = (4 * np.pi / 15) * sig ** 4 * np.sqrt(KT / np.pi) * g[0, 0, 0] * n0
    pred = n0 * (1.0 if mode == "shear" else 3.0) * eta * (-k * k * A * np.cos(arg))
    return V[0], pred


@pytest.mark.parametrize("sig", [4.0, 6.0])
@pytest.mark.parametrize("mode", ["shear", "compression"])
def test_uniform_fluid_viscosity_limits(sig, mode):
    V, pred = _wave(sig, 48, mode)
    m = np.abs(pred) > 0.5 * np.abs(pred).max()
    ratio = V[0][m] / pred[m]
    assert abs(ratio.mean() - 1.0) < 0.05, ratio.mean()
    assert ratio.std() < 1e-10
    assert np.abs(V[1:]).max() <= 1e-12 * np.abs(V[0]).max()


def test_uniform_velocity_gives_no_force_and_one_species_conserves_momentum():
    shape = (14, 12, 10)
    N = 14 * 12 * 10
    rng = np.random.default_rng(3)
    n = 0.01 * (1.0 + 0.2 * rng.random((1, N)))
    g = oracle.contact_values(shape, (1, 1, 1), [3.0], n)
    u = np.zeros((1, 3, N))
    u[0] += np.array([1e-3, -2e-3, 5e-4])[:, None]
    V = oracle.visc_force(shape, (1, 1, 1), [3.0], n, u, g)
    assert np.abs(V).max() <= 1e-18
    u = 1e-3 * (rng.random((1, 3, N)) - 0.5)
    V = oracle.visc_force(shape, (1, 1, 1), [3.0], n, u, g)
    assert np.abs(V).max() > 0
    assert np.abs(V[0].sum(axis=1)).max() <= 1e-12 * np.abs(V).sum()
