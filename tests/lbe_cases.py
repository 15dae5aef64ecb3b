"""Test helpers: feed one seeded input set to both the CUDA library and the oracle."""
import numpy as np

import oracle
from paper_1202_3842_gb300 import inputs

CS = np.sqrt(1.0 / 3.0)


def case_well(shape, sigma, eta, tau, depth_kT, radius, seed=1202, noise=0.01):
    w = inputs.well_workload(shape, sigma, eta, tau, depth_kT, radius, seed=seed, noise=noise)
    return w, inputs.build_workload(w)


def case_channel(shape, sigmas, eta, taus, width, length, body=1e-6, wall_amp_kT=0.0):
    w = inputs.channel_workload(shape, sigmas, eta, taus, width, length, body=body, wall_amp_kT=wall_amp_kT)
    return w, inputs.build_workload(w)


SCHEME_IDS = {"dd_tr": 0, "sd_tr": 1, "sd_eu": 2, "dd_eu": 3}


def setup_gpu(w, arrays, precision, consistent=False, check_every=0, scheme="dd_tr", shell="auto", visc=False):
    from paper_1202_3842_gb300 import lbe
    M = len(w["sigma"])
    sim = lbe.Simulation(w["shape"], w["periodic"], M, precision, consistent_moments=consistent,
                         check_every=check_every, scheme=scheme, visc=visc)
    if shell != "auto":
        sim.set_shell_method(shell)
    sim.set_geometry(arrays["solid"])
    for a in range(M):
        sim.set_species(a, w["sigma"][a], w["tau"][a])
        sim.set_potential(a, arrays["V"][a])
        sim.set_body_force(a, w["body"][a])
    sim.set_wall_potential(arrays["phi"], arrays["amp"])
    for a in range(M):
        sim.init_density(a, arrays["n"][a])
    return sim


def setup_oracle(w, arrays, consistent=False, scheme="dd_tr", visc=False):
    M = len(w["sigma"])
    sim = oracle.Sim(w["shape"], w["periodic"], M)
    sim.set_geometry(arrays["solid"])
    sim.set_consistent_moments(consistent)
    sim.set_scheme(SCHEME_IDS[scheme])
    sim.set_visc(visc)
    for a in range(M):
        sim.set_species(a, w["sigma"][a], w["tau"][a])
        sim.set_potential(a, arrays["V"][a])
        sim.set_body_force(a, w["body"][a])
    sim.set_wall_potential(arrays["phi"], arrays["amp"])
    for a in range(M):
        sim.init_density(a, arrays["n"][a])
    return sim


def velocity_from(n, J):
    """u [3, N] = J / n (0 where n = 0) for one species."""
    return np.where(n[None, :] > 0, J / np.where(n[None, :] > 0, n[None, :], 1.0), 0.0)


def barycentric(nM, JM):
    n = nM.sum(0)
    J = JM.sum(0)
    return velocity_from(n, J)


def rel_err(a, b, scale=None):
    scale = np.abs(b).max() if scale is None else scale
    return np.abs(a - b).max() / scale
