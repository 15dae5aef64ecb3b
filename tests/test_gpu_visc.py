"""The viscous Enskog force (enable_visc; Appendix, C^{alpha,visc}) against the oracle.

The force enters where n F does (moment recovery, S_f, S_g), with the tilde velocities J~/n; on the
GPU it is folded into an effective force field.  Tolerances as for the DD-TR path: FP64 densities
1e-12 relative and velocities 1e-12 of max(|u|, 1e-6 v_T); FP32 densities 1e-5, the flux 1e-3.
"""
import numpy as np
import pytest

from lbe_cases import CS, case_channel, case_well, rel_err, setup_gpu, setup_oracle, velocity_from

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
def test_fp64_well_with_viscous_force(shell):
    w, arr = case_well((20, 18, 16), 3.0, 0.2, 1.0, 1.0, 3.0)
    g = setup_gpu(w, arr, "fp64", visc=True, shell=shell)
    o = setup_oracle(w, arr, visc=True)
    plain = setup_oracle(w, arr, visc=False)
    g.step(60)
    o.step(60)
    plain.step(60)
    obs = o.observe()
    assert rel_err(g.density(0), obs["n"][0]) <= 1e-12
    u_ref = velocity_from(obs["n"][0], obs["J"][0])
    assert np.abs(g.velocity(0) - u_ref).max() <= _u_tol(u_ref)
    # the force is not a no-op: the run without it differs far beyond the tolerance
    assert rel_err(plain.observe()["n"][0], obs["n"][0]) > 1e-6


def test_fp64_channel_mixture_with_viscous_force_and_flux():
    w, arr = case_channel((40, 22, 18), (4.0, 6.0), 0.25, (1.0, 0.8), 10, 12, body=1e-5)
    g = setup_gpu(w, arr, "fp64", visc=True)
    o = setup_oracle(w, arr, visc=True)
    g.set_flux_plane(0, 20)
    o.set_flux_plane(0, 20)
    g.step(30)
    o.step(30)
    obs = o.observe()
    for a in range(2):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-12
        u_ref = velocity_from(obs["n"][a], obs["J"][a])
        assert np.abs(velocity_from(g.density(a), g.momentum(a)) - u_ref).max() <= _u_tol(u_ref)
    fs, cnt = o.flux()
    assert abs(g.flux(-1)[1] - fs.sum() / cnt) <= 1e-12 * abs(fs.sum() / cnt)


def test_fp32_channel_with_viscous_force():
    w, arr = case_channel((40, 22, 18), (4.0, 6.0), 0.25, (1.0, 0.8), 10, 12, body=1e-5)
    g = setup_gpu(w, arr, "fp32", visc=True)
    o = setup_oracle(w, arr, visc=True)
    g.set_flux_plane(0, 20)
    o.set_flux_plane(0, 20)
    g.step(30)
    o.step(30)
    obs = o.observe()
    for a in range(2):
        assert rel_err(g.density(a), obs["n"][a]) <= 1e-5
    fs, cnt = o.flux()
    assert abs(g.flux(-1)[1] - fs.sum() / cnt) <= 1e-3 * abs(fs.sum() / cnt)


def test_viscous_force_is_rejected_where_it_does_not_apply():
    from paper_1202_3842_gb300 import lbe
    w, arr = case_well((12, 12, 12), 3.0, 0.2, 1.0, 1.0, 3.0)
    with pytest.raises(lbe.LbeError) as e:
        lbe.Simulation(w["shape"], w["periodic"], 1, "fp64", scheme="sd_tr", visc=True)
    assert e.value.status == lbe.LBE_ERR_UNSUPPORTED
    g = setup_gpu(w, arr, "fp64", visc=True)
    with pytest.raises(lbe.LbeError) as e:
        g.adjoint_flux_gradient(2, 1, 0, 6)
    assert e.value.status == lbe.LBE_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec,tol", [("bf16", 1e-2), ("fp16", 1e-3)])
def test_shifted_16bit_storage_with_viscous_force(prec, tol):
    """16-bit shifted populations with FP32 arithmetic, the viscous force on: the densities against the
    FP64 oracle within the bounds of the 16-bit storage test (bf16 1e-2, fp16 1e-3 after 30 steps)."""
    w, arr = case_channel((40, 22, 18), (4.0, 6.0), 0.25, (1.0, 0.8), 10, 12, body=1e-5)
    g = setup_gpu(w, arr, prec, visc=True)
    o = setup_oracle(w, arr, visc=True)
    g.step(30)
    o.step(30)
    obs = o.observe()
    for a in range(2):
        assert rel_err(g.density(a), obs["n"][a]) <= tol
