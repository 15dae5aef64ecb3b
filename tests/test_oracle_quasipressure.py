"""Pins of the oracle's quasi-pressure Pi^a = n^a - beta * path integral of C^{a,mf} + n^a F^a (Sec.
"Stabilization", the equation for Pi^alpha; trapezoidal rule along x, then y, then z from the origin).

- Uniform density under a constant body force g: Pi(r) = n0 - beta n0 g . r exactly (the trapezoidal
  rule is exact for a constant integrand), with and without hard spheres (the mean-field force of a
  uniform periodic fluid vanishes by the symmetry of the shell).
- Ideal gas at equilibrium in a smooth potential, n = n0 exp(-beta V): in the continuum n F = grad n /
  beta, so Pi is constant; on the lattice its spread falls with the square of the resolution (the
  isotropic gradient and the trapezoidal rule are both second order).  A sign error on beta or a
  dropped half in the rule leaves a spread of order one.
- Values given on solid nodes do not enter (solid nodes carry n = 0).
"""
import numpy as np

import oracle


def _xyz(shape):
    nx, ny, nz = shape
    i = np.arange(nx * ny * nz)
    return i % nx, (i // nx) % ny, i // (nx * ny)


def test_constant_body_force_closed_form():
    shape = (7, 5, 6)
    N = 7 * 5 * 6
    x, y, z = _xyz(shape)
    g = np.array([1e-3, -2e-3, 5e-4])
    for sigma in (0.0, 3.0):
        n0 = 0.02
        Pi = oracle.quasipressure(shape, (1, 1, 1), [sigma], np.full((1, N), n0), np.zeros((1, N)), g[None])
        ref = n0 - 3.0 * n0 * (g[0] * x + g[1] * y + g[2] * z)
        assert np.abs(Pi[0] - ref).max() <= 1e-13 * n0


def test_ideal_gas_equilibrium_is_flat_to_second_order():
    spreads = []
    for L in (8, 16, 32):
        shape = (L, L, L)
        x, y, z = _xyz(shape)
        k = 2 * np.pi / L
        V = (1.0 / 3.0) * 0.5 * (np.cos(k * x) * np.cos(k * y) + 0.5 * np.sin(k * z))
        n = 0.01 * np.exp(-3.0 * V)
        Pi = oracle.quasipressure(shape, (1, 1, 1), [0.0], n[None], V[None], np.zeros((1, 3)))[0]
        assert Pi[0] == n[0]  # the path starts at the origin
        spreads.append(np.abs(Pi - Pi[0]).max() / (n.max() - n.min()))
    assert spreads[2] < 0.02
    assert spreads[0] / spreads[1] > 3.5 and spreads[1] / spreads[2] > 3.5


def test_solid_node_values_do_not_enter():
    from paper_1202_3842_gb300 import inputs
    w = inputs.channel_workload((20, 12, 10), (2.0, 4.0), 0.2, (1.0, 1.0), 6, 6, body=1e-4)
    arr = inputs.build_workload(w)
    solid = arr["solid"]
    V = arr["V"] + arr["amp"] * arr["phi"]
    gb = np.array(w["body"])
    a = oracle.quasipressure(w["shape"], w["periodic"], w["sigma"], arr["n"], V, gb, solid)
    n2 = arr["n"].copy()
    n2[:, solid == 1] = 7.0
    b = oracle.quasipressure(w["shape"], w["periodic"], w["sigma"], n2, V, gb, solid)
    fl = solid == 0
    np.testing.assert_array_equal(a[:, fl], b[:, fl])
    assert np.abs(a[:, fl] - arr["n"][:, fl]).max() > 0  # the mean field and the force do enter
