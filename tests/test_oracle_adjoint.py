"""Pins of the FP64 reference gradient (oracle/torch_adjoint.py): its forward pass equals the C oracle, and
its gradient of the time-averaged flux w.r.t. the wall-potential amplitude and the body force equals
central finite differences of the C oracle and passes a Taylor test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import torch_adjoint
from paper_1202_3842_gb300 import inputs

KT = 1.0 / 3.0


def _case(shape=(16, 12, 10), sig=(2.0, 4.0), taus=(1.0, 0.9), width=6, length=4, body=2e-4):
    w = inputs.channel_workload(shape, sig, 0.2, taus, width, length, body=body, wall_amp_kT=1.0)
    arr = inputs.build_workload(w)
    rng = np.random.default_rng(21)
    N = int(np.prod(shape))
    arr["amp"] = arr["amp"] * (1.0 + 0.3 * (rng.random(N) - 0.5))
    return w, arr


def _c_phi(w, arr, amp, gshift, nsteps, axis, plane):
    M = len(w["sigma"])
    sim = oracle.Sim(w["shape"], w["periodic"], M)
    sim.set_geometry(arr["solid"])
    for a in range(M):
        sim.set_species(a, w["sigma"][a], w["tau"][a])
        sim.set_potential(a, arr["V"][a])
        sim.set_body_force(a, np.asarray(w["body"][a]) + gshift)
    sim.set_wall_potential(arr["phi"], amp)
    for a in range(M):
        sim.init_density(a, arr["n"][a])
    sim.set_flux_plane(axis, plane)
    sim.step(nsteps)
    s, cnt = sim.flux()
    return s.sum() / cnt, sim


def test_torch_forward_equals_c_oracle():
    w, arr = _case()
    T, axis, plane = 8, 0, 8
    phi_t, f, g = torch_adjoint.forward_only(w["shape"], w["periodic"], w["sigma"], w["tau"], arr["solid"],
                                             arr["phi"], arr["V"], w["body"], arr["n"], arr["amp"], T, axis, plane)
    phi_c, sim = _c_phi(w, arr, arr["amp"], np.zeros(3), T, axis, plane)
    assert abs(phi_t - phi_c) <= 1e-12 * abs(phi_c)
    for a in range(2):
        fc, gc = sim.get_populations(a)
        np.testing.assert_allclose(f[a], fc, rtol=0, atol=1e-13 * np.abs(fc).max())
        np.testing.assert_allclose(g[a], gc, rtol=0, atol=1e-13 * np.abs(gc).max())


def test_reference_gradient_matches_central_differences():
    w, arr = _case()
    T, axis, plane = 8, 0, 8
    Phi, gA, gG = torch_adjoint.reference_gradient(w["shape"], w["periodic"], w["sigma"], w["tau"], arr["solid"],
                                                   arr["phi"], arr["V"], w["body"], arr["n"], arr["amp"], T, axis,
                                                   plane)
    phi_c, _ = _c_phi(w, arr, arr["amp"], np.zeros(3), T, axis, plane)
    assert abs(Phi - phi_c) <= 1e-12 * abs(phi_c)
    rng = np.random.default_rng(5)
    N = arr["amp"].size
    wall = np.flatnonzero(arr["phi"] > 0)
    dirs = [rng.standard_normal(N) * (arr["phi"] > 0)]
    for node in wall[[0, len(wall) // 2, -1]]:
        d = np.zeros(N)
        d[node] = 1.0
        dirs.append(d)
    h = 1e-4 * KT
    for d in dirs:
        fp, _ = _c_phi(w, arr, arr["amp"] + h * d, np.zeros(3), T, axis, plane)
        fm, _ = _c_phi(w, arr, arr["amp"] - h * d, np.zeros(3), T, axis, plane)
        fd = (fp - fm) / (2 * h)
        ad = float(gA @ d)
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gA).max() * np.abs(d).sum()), (ad, fd)
    hg = 1e-4 * 2e-4
    for c in range(3):
        e = np.zeros(3)
        e[c] = hg
        fp, _ = _c_phi(w, arr, arr["amp"], e, T, axis, plane)
        fm, _ = _c_phi(w, arr, arr["amp"], -e, T, axis, plane)
        fd = (fp - fm) / (2 * hg)
        assert abs(gG[c] - fd) <= 1e-6 * max(abs(fd), 1e-3 * abs(gG[0])), (c, gG[c], fd)


def test_reference_gradient_taylor_slope_two():
    w, arr = _case()
    T, axis, plane = 6, 0, 8
    Phi, gA, gG = torch_adjoint.reference_gradient(w["shape"], w["periodic"], w["sigma"], w["tau"], arr["solid"],
                                                   arr["phi"], arr["V"], w["body"], arr["n"], arr["amp"], T, axis,
                                                   plane)
    rng = np.random.default_rng(8)
    d = rng.standard_normal(arr["amp"].size) * (arr["phi"] > 0) * KT
    rem = []
    for eps in (4e-2, 2e-2, 1e-2):
        fp, _ = _c_phi(w, arr, arr["amp"] + eps * d, np.zeros(3), T, axis, plane)
        rem.append(abs(fp - Phi - eps * float(gA @ d)))
    slopes = [np.log2(rem[k] / rem[k + 1]) for k in range(2)]
    assert all(1.8 < s < 2.2 for s in slopes), (rem, slopes)
