"""Three species, and a mixture with a point species (sigma = 0, so one pair of the M^2 has no shell):
the collide for three or four species, and the spectral kernels' general forms (any species count, a
pair set that is not complete), against the FP64 oracle and the FP64 reference gradient.

Tolerances as for the DD-TR path: FP64 densities 1e-12 relative, velocities 1e-12 of max(|u|, 1e-6 v_T),
the flux average 1e-12; the adjoint 1e-10 of the largest gradient entry.
"""
import numpy as np
import pytest

from lbe_cases import CS, case_channel, rel_err, setup_gpu, setup_oracle, velocity_from

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _u_tol(u_ref):
    return 1e-12 * max(np.abs(u_ref).max(), 1e-6 * CS)


@pytest.mark.parametrize("shell", ["direct", "spectral"])
@pytest.mark.parametrize("sig", [(2.0, 4.0, 6.0), (0.0, 4.0)])
def test_fp64_mixture_parity(sig, shell):
    M = len(sig)
    w, arr = case_channel((30, 18, 16), sig, 0.2, (1.0, 0.9, 0.8)[:M], 8, 8, body=1e-5)
    g = setup_gpu(w, arr, "fp64", shell=shell)
    assert g.shell_method() == shell
    o = setup_oracle(w, arr)
    g.set_flux_plane(0, 15)
    o.set_flux_plane(0, 15)
    g.step(30)
    o.step(30)
    obs = o.observe()
    for a in range(M):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-12
        u_ref = velocity_from(obs["n"][a], obs["J"][a])
        assert np.abs(velocity_from(g.density(a), g.momentum(a)) - u_ref).max() <= _u_tol(u_ref)
        assert rel_err(g.force(a), obs["C"][a]) <= 1e-12
    fs, cnt = o.flux()
    assert abs(g.flux(-1)[1] - fs.sum() / cnt) <= 1e-12 * abs(fs.sum() / cnt)


@pytest.mark.parametrize("shell", ["direct", "spectral"])
def test_fp64_three_species_adjoint(shell):
    from oracle import torch_adjoint
    w, arr = case_channel((16, 12, 10), (2.0, 4.0, 6.0), 0.2, (1.0, 0.9, 0.8), 6, 4, body=2e-4,
                          wall_amp_kT=0.5)
    T, axis, plane = 6, 0, 8
    rPhi, rA, rG = torch_adjoint.reference_gradient(w["shape"], w["periodic"], w["sigma"], w["tau"],
                                                    arr["solid"], arr["phi"], arr["V"], w["body"], arr["n"],
                                                    arr["amp"], T, axis, plane)
    g = setup_gpu(w, arr, "fp64", shell=shell)
    Phi, dA, dG = g.adjoint_flux_gradient(T, 3, axis, plane)
    assert abs(Phi - rPhi) <= 1e-12 * abs(rPhi)
    assert np.abs(dA - rA).max() <= 1e-10 * np.abs(rA).max()
    assert np.abs(dG - rG).max() <= 1e-10 * np.abs(rG).max()
