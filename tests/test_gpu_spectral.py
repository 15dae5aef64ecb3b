"""The spectral shell force (K3 by fast Fourier transforms) on the GPU.

The parity tests of test_gpu_parity.py run both shell methods (direct stencil and spectral) against
the oracle.  Here:
- diameters that only the spectral method takes (FP64 pair diameter 8, diameter 9 in both storage
  precisions, with pair diameters 7, 8 and 9 in FP32) against the oracle: FP64 to 1e-12, FP32 to 1e-5
  of the largest value of each field;
- a short periodic axis (n < 2 S + 1), where shell points alias on the grid, against the oracle;
- the two methods against each other over 30 FP32 steps of a two-species channel (1e-5 relative);
- the automatic choice, and the errors for a method that cannot take the case; the adjoint of a
  diameter without a stencil tile, through the spectral transpose.
"""
import numpy as np
import pytest

from lbe_cases import case_channel, case_well, rel_err, setup_gpu, setup_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _perturbed_channel(shape, sig, seed):
    w, arr = case_channel(shape, sig, 0.2, (1.0,) * len(sig), 10, 8)
    rng = np.random.default_rng(seed)
    fl = arr["solid"] == 0
    arr["n"] = arr["n"] * (1.0 + 0.2 * (rng.random(arr["n"].shape) - 0.5)) * fl[None, :]
    return w, arr


@pytest.mark.parametrize("prec,sig,tol", [("fp64", (8.0,), 1e-12), ("fp64", (6.0, 8.0), 1e-12),
                                          ("fp64", (9.0,), 1e-12), ("fp32", (9.0,), 1e-5),
                                          ("fp32", (7.0, 9.0), 1e-5)])
def test_spectral_only_diameters_against_oracle(prec, sig, tol):
    w, arr = _perturbed_channel((44, 26, 24), sig, 11)
    g = setup_gpu(w, arr, prec)
    assert g.shell_method() == "spectral"
    obs = setup_oracle(w, arr).observe()
    for a in range(len(sig)):
        assert rel_err(g.force(a), obs["C"][a]) <= tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_short_periodic_axis_aliases_like_the_halo(prec, tol):
    # 10 nodes along a periodic z with pair diameter 6: shell points at z and z - 10 land on one grid
    # point, as the direct stencil reads the same periodic image twice
    w, arr = case_well((26, 22, 10), 6.0, 0.2, 1.0, 1.0, 4.0)
    rng = np.random.default_rng(5)
    arr["n"] = arr["n"] * (1.0 + 0.2 * (rng.random(arr["n"].shape) - 0.5))
    g = setup_gpu(w, arr, prec, shell="spectral")
    obs = setup_oracle(w, arr).observe()
    assert rel_err(g.force(0), obs["C"][0]) <= tol


def test_methods_agree_over_fp32_channel_steps():
    w, arr = case_channel((48, 24, 20), (4.0, 6.0), 0.25, (1.0, 0.8), 10, 12, body=1e-5)
    d = setup_gpu(w, arr, "fp32", shell="direct")
    s = setup_gpu(w, arr, "fp32", shell="spectral")
    d.set_flux_plane(0, 24)
    s.set_flux_plane(0, 24)
    d.step(30)
    s.step(30)
    for a in range(2):
        assert rel_err(s.density(a), d.density(a)) <= 1e-5
        assert rel_err(s.force(a), d.force(a)) <= 1e-4
    fd, fs = d.flux(-1)[1], s.flux(-1)[1]
    assert abs(fs - fd) <= 1e-3 * abs(fd)


def test_automatic_choice_and_errors():
    from paper_1202_3842_gb300 import lbe
    # mean shell 340 points on a grid 2.1 times the lattice: above the FP64 break-even (110 x 2.1),
    # below FP32's (320 x 2.1)
    w, arr = case_channel((30, 16, 14), (4.0, 6.0), 0.2, (1.0, 1.0), 8, 6)
    assert setup_gpu(w, arr, "fp64").shell_method() == "spectral"
    assert setup_gpu(w, arr, "fp32").shell_method() == "direct"
    # one species of diameter 6 (450 points) on a periodic lattice: above both
    ww, aw = case_well((24, 24, 24), 6.0, 0.2, 1.0, 1.0, 4.0)
    assert setup_gpu(ww, aw, "fp32").shell_method() == "spectral"
    # diameter 3 (98 points): below both
    ww, aw = case_well((24, 24, 24), 3.0, 0.2, 1.0, 1.0, 4.0)
    assert setup_gpu(ww, aw, "fp64").shell_method() == "direct"
    assert setup_gpu(w, arr, "fp64", shell="direct").shell_method() == "direct"
    w9, a9 = case_channel((30, 20, 20), (9.0,), 0.2, (1.0,), 12, 6)
    assert setup_gpu(w9, a9, "fp32").shell_method() == "spectral"
    g = setup_gpu(w9, a9, "fp32", shell="direct")
    with pytest.raises(lbe.LbeError) as e:
        g.step(1)
    assert e.value.status == lbe.LBE_ERR_UNSUPPORTED
    with pytest.raises(lbe.LbeError) as e:
        g.set_shell_method(7)
    assert e.value.status == lbe.LBE_ERR_INVALID_ARG
    # the adjoint takes the diameter through the spectral transpose (no stencil tile exists for it)
    g = setup_gpu(w9, a9, "fp32")
    Phi, dA, dG = g.adjoint_flux_gradient(2, 1, 0, 10)
    assert np.isfinite(Phi) and np.isfinite(dA).all() and np.isfinite(dG).all()
    assert abs(dG[0]) > 0  # the flux responds to the body force (no wall potential here, so dA = 0)
