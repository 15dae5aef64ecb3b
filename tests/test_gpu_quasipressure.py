"""Quasi-pressure initialisation (lbe_init_density_quasipressure) against the oracle.

A two-species channel with walls, a wall potential and a body force, and a hard-sphere well:
- the streamed populations after the call, f_p = w_p n and g_p = w_p Pi, against the oracle's Pi:
  FP64 1e-12 and FP32 1e-5 of the largest population;
- 20 FP64 steps from that state of the well against the oracle stepping from the same populations
  (1e-12).  The channel is not stepped: from a uniform density its Pi reaches 3.5 n near the walls
  (the path runs in from the solid wall along z), and within ten steps the oracle itself has a
  negative density there, as the library reports.
"""
import numpy as np
import pytest

import oracle
from lbe_cases import case_channel, case_well, rel_err, setup_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _cases():
    yield case_channel((36, 20, 18), (4.0, 6.0), 0.25, (1.0, 0.9), 8, 10, body=1e-4, wall_amp_kT=0.5)
    yield case_well((20, 18, 16), 3.0, 0.2, 1.0, 1.0, 4.0)


def _oracle_pi(w, arr):
    V = arr["V"] + arr["amp"][None, :] * arr["phi"][None, :]
    return oracle.quasipressure(w["shape"], w["periodic"], w["sigma"], arr["n"], V, np.array(w["body"]),
                                arr["solid"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_populations_match_the_oracle(prec, tol):
    _, wq, _ = oracle.lattice()
    for w, arr in _cases():
        M = len(w["sigma"])
        g = setup_gpu(w, arr, prec)
        g.init_density_quasipressure(arr["n"])
        Pi = _oracle_pi(w, arr)
        fl = arr["solid"] == 0
        for a in range(M):
            f, gg = g.populations(a)
            fref = np.where(fl[None, :], wq[:, None] * arr["n"][a][None, :], 0.0)
            gref = np.where(fl[None, :], wq[:, None] * Pi[a][None, :], 0.0)
            assert rel_err(f, fref) <= tol
            assert rel_err(gg, gref) <= tol
            assert np.abs(Pi[a][fl] - arr["n"][a][fl]).max() > 1e-3 * arr["n"][a].max()


def test_steps_from_the_quasipressure_state_match_the_oracle():
    from lbe_cases import setup_oracle
    _, wq, _ = oracle.lattice()
    w, arr = list(_cases())[1]
    M = len(w["sigma"])
    g = setup_gpu(w, arr, "fp64")
    g.init_density_quasipressure(arr["n"])
    o = setup_oracle(w, arr)
    Pi = _oracle_pi(w, arr)
    fl = arr["solid"] == 0
    for a in range(M):
        o.set_populations(a, np.where(fl[None, :], wq[:, None] * arr["n"][a][None, :], 0.0),
                          np.where(fl[None, :], wq[:, None] * Pi[a][None, :], 0.0))
    g.step(20)
    o.step(20)
    obs = o.observe()
    for a in range(M):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-12
        fg, gg = g.populations(a)
        fo, go = o.get_populations(a)
        assert rel_err(gg, go) <= 1e-12
