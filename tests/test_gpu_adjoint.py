"""GPU discrete adjoint of the time-averaged flux against the FP64 reference gradient (autograd through
an independent FP64 implementation of the step, itself pinned to the C oracle) and against central finite
differences of the GPU FP64 forward.

Tolerances: FP64 adjoint vs reference 1e-10 of the largest gradient entry; FP64 adjoint vs central
differences (h = 1e-4 of the parameter scale) 1e-6 relative; FP32 adjoint vs FP64 reference 1e-3 of the
largest entry."""
import numpy as np
import pytest

from lbe_cases import setup_gpu
from paper_1202_3842_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
KT = 1.0 / 3.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _case(shape=(16, 12, 10), sig=(2.0, 4.0), taus=(1.0, 0.9), width=6, length=4, body=2e-4, seed=21):
    w = inputs.channel_workload(shape, sig, 0.2, taus, width, length, body=body, wall_amp_kT=1.0)
    arr = inputs.build_workload(w)
    rng = np.random.default_rng(seed)
    arr["amp"] = arr["amp"] * (1.0 + 0.3 * (rng.random(arr["amp"].size) - 0.5))
    return w, arr


def _reference(w, arr, T, axis, plane, consistent=False):
    from oracle import torch_adjoint
    return torch_adjoint.reference_gradient(w["shape"], w["periodic"], w["sigma"], w["tau"], arr["solid"],
                                            arr["phi"], arr["V"], w["body"], arr["n"], arr["amp"], T, axis, plane,
                                            consistent=consistent)


@pytest.mark.parametrize("shell", ["direct", "spectral"])
@pytest.mark.parametrize("consistent", [False, True])
def test_fp64_adjoint_matches_reference(consistent, shell):
    """The recomputation's force stage runs with either shell method; the transposes are the stencil's."""
    w, arr = _case()
    T, axis, plane = 8, 0, 8
    g = setup_gpu(w, arr, "fp64", consistent=consistent, shell=shell)
    f0, g0 = g.populations(0)
    Phi, dA, dG = g.adjoint_flux_gradient(T, 3, axis, plane)
    rPhi, rA, rG = _reference(w, arr, T, axis, plane, consistent)
    assert abs(Phi - rPhi) <= 1e-12 * abs(rPhi)
    assert np.abs(dA - rA).max() <= 1e-10 * np.abs(rA).max()
    assert np.abs(dG - rG).max() <= 1e-10 * np.abs(rG).max()
    f1, g1 = g.populations(0)  # the state is left as it was
    np.testing.assert_array_equal(f1, f0)
    np.testing.assert_array_equal(g1, g0)


@pytest.mark.parametrize("shell", ["direct", "spectral"])
@pytest.mark.parametrize("sig,precs", [((1.0, 7.0), ("fp64", "fp32")), ((2.0, 8.0), ("fp32", "fp64"))])
def test_adjoint_every_shell_transpose_tile(sig, precs, shell):
    """The shell transpose of pair diameters 1, 4, 7 (FP64 and FP32 tiles) and 2, 5, 8 (FP32; the FP64
    stencil stops at 7, the spectral transpose takes 8) against the FP64 reference gradient: 1e-10 of the
    largest entry in FP64, 1e-3 in FP32.  Both methods: the stencil tiles, and the spectral transpose
    (lambda and g lambda transformed, multiplied by the shell spectra, transformed back)."""
    w, arr = _case(shape=(20, 18, 18), sig=sig, taus=(1.0, 0.9), width=8, length=6, seed=21)
    T, axis, plane = 6, 0, 10
    rPhi, rA, rG = _reference(w, arr, T, axis, plane)
    for prec in precs:
        if shell == "direct" and prec == "fp64" and max(sig) > 7:
            continue
        g = setup_gpu(w, arr, prec, shell=shell)
        Phi, dA, dG = g.adjoint_flux_gradient(T, 2, axis, plane)
        tol = 1e-10 if prec == "fp64" else 1e-3
        assert abs(Phi - rPhi) <= max(tol, 1e-12) * abs(rPhi), (prec, Phi, rPhi)
        assert np.abs(dA - rA).max() <= tol * np.abs(rA).max(), prec
        assert np.abs(dG - rG).max() <= tol * np.abs(rG).max(), prec
        g.close()


def _gpu_phi(w, arr, amp, gshift, T, axis, plane, prec="fp64"):
    a2 = dict(arr)
    a2["amp"] = amp
    w2 = dict(w)
    w2["body"] = [tuple(np.asarray(b) + gshift) for b in w["body"]]
    g = setup_gpu(w2, a2, prec)
    g.set_flux_plane(axis, plane)
    g.step(T)
    return g.flux(-1)[1]


def test_fp64_adjoint_matches_central_differences_of_the_gpu_forward():
    w, arr = _case(shape=(24, 14, 12), sig=(4.0, 6.0), taus=(1.0, 1.0), width=8, length=6, seed=3)
    T, axis, plane = 30, 0, 12
    g = setup_gpu(w, arr, "fp64")
    Phi, dA, dG = g.adjoint_flux_gradient(T, 7, axis, plane)
    rng = np.random.default_rng(4)
    N = arr["amp"].size
    wall = np.flatnonzero(arr["phi"] > 0)
    dirs = [rng.standard_normal(N) * (arr["phi"] > 0) for _ in range(2)]
    for node in wall[[3, len(wall) // 3, -5]]:
        d = np.zeros(N)
        d[node] = 1.0
        dirs.append(d)
    h = 1e-4 * KT
    for d in dirs:
        fp = _gpu_phi(w, arr, arr["amp"] + h * d, np.zeros(3), T, axis, plane)
        fm = _gpu_phi(w, arr, arr["amp"] - h * d, np.zeros(3), T, axis, plane)
        fd = (fp - fm) / (2 * h)
        ad = float(dA @ d)
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(dA).max()), (ad, fd)
    hg = 1e-4 * 2e-4
    e = np.array([hg, 0.0, 0.0])
    fd = (_gpu_phi(w, arr, arr["amp"], e, T, axis, plane) - _gpu_phi(w, arr, arr["amp"], -e, T, axis, plane)) / (2 * hg)
    assert abs(dG[0] - fd) <= 1e-6 * abs(fd)


def test_fp32_adjoint_against_fp64_reference_channel32():
    w = inputs.WORKLOADS["channel32adj"]()
    arr = inputs.build_workload(w)
    rng = np.random.default_rng(7)
    arr["amp"] = arr["amp"] * (1.0 + 0.3 * (rng.random(arr["amp"].size) - 0.5))
    T, axis, plane = 200, 0, 16
    g = setup_gpu(w, arr, "fp32")
    Phi, dA, dG = g.adjoint_flux_gradient(T, 20, axis, plane)
    from oracle import torch_adjoint
    rPhi, rA, rG = torch_adjoint.reference_gradient(w["shape"], w["periodic"], w["sigma"], w["tau"], arr["solid"],
                                                    arr["phi"], arr["V"], w["body"], arr["n"], arr["amp"], T, axis,
                                                    plane, ckpt_every=1)
    assert abs(Phi - rPhi) <= 1e-3 * abs(rPhi)
    assert np.abs(dA - rA).max() <= 1e-3 * np.abs(rA).max()
    assert np.abs(dG - rG).max() <= 1e-3 * np.abs(rG).max()


def test_autograd_function_returns_the_adjoint_gradient():
    from paper_1202_3842_gb300.autograd import FluxObjective
    w, arr = _case()
    T, axis, plane = 8, 0, 8
    g = setup_gpu(w, arr, "fp64")
    amp = torch.tensor(arr["amp"], dtype=torch.float64, requires_grad=True)
    gs = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    Phi = FluxObjective.apply(amp, gs, g, arr["phi"], w["body"], arr["n"], T, 4, axis, plane)
    (2.0 * Phi).backward()
    rPhi, rA, rG = _reference(w, arr, T, axis, plane)
    assert abs(float(Phi) - rPhi) <= 1e-12 * abs(rPhi)
    assert np.abs(amp.grad.numpy() - 2 * rA).max() <= 1e-10 * np.abs(rA).max()
    assert np.abs(gs.grad.numpy() - 2 * rG).max() <= 1e-10 * np.abs(rG).max()


def test_repeated_adjoint_calls_reuse_the_spectral_transpose():
    """The spectral transpose's plans and shell spectra stay in the context between calls and are rebuilt
    when the species set changes: three calls (the third after setting the species again) give the
    same gradient bit for bit."""
    w, arr = _case()
    g = setup_gpu(w, arr, "fp32", shell="spectral")
    first = g.adjoint_flux_gradient(4, 2, 0, 8)
    second = g.adjoint_flux_gradient(4, 2, 0, 8)
    for a in range(len(w["sigma"])):
        g.set_species(a, w["sigma"][a], w["tau"][a])
    third = g.adjoint_flux_gradient(4, 2, 0, 8)
    for other in (second, third):
        assert other[0] == first[0]
        np.testing.assert_array_equal(other[1], first[1])
        np.testing.assert_array_equal(other[2], first[2])
    g.close()


def _phi_fresh(w, arr, amp, gshift, T, axis, plane, prec="fp64"):
    a2 = dict(arr)
    a2["amp"] = amp
    w2 = dict(w)
    w2["body"] = [tuple(np.asarray(b) + gshift) for b in w["body"]]
    g = setup_gpu(w2, a2, prec)
    try:
        g.set_flux_plane(axis, plane)
        g.step(T)
        return g.flux(-1)[1]
    finally:
        g.close()


@pytest.fixture(scope="module")
def full_size_adjoint():
    """The adjoint channel at its full size (256x64x64, slit width 12 and length 32, sigma 4/6, packing
    0.25, wall potential of amplitude 1 k_BT with a seeded +-15% spread), over T = 200 steps with
    checkpoints every 20: the FP64 and FP32 gradients of the flux through x = 128."""
    w = inputs.WORKLOADS["channel256adj"]()
    arr = inputs.build_workload(w)
    rng = np.random.default_rng(11)
    arr["amp"] = arr["amp"] * (1.0 + 0.3 * (rng.random(arr["amp"].size) - 0.5))
    T, K, axis, plane = 200, 20, 0, 128
    out = {"w": w, "arr": arr, "T": T, "axis": axis, "plane": plane}
    for prec in ("fp64", "fp32"):
        g = setup_gpu(w, arr, prec)
        out[prec] = g.adjoint_flux_gradient(T, K, axis, plane)
        g.close()
    return out


def test_full_size_fp64_adjoint_matches_central_differences(full_size_adjoint):
    """The adjoint within 1e-4 relative of central differences (h = 1e-4 of the parameter
    scale), here on the full-size adjoint channel: four random directions over the wall nodes, four
    single wall nodes and the body force g_x, each against two FP64 forward runs of the GPU."""
    S = full_size_adjoint
    w, arr, T, axis, plane = S["w"], S["arr"], S["T"], S["axis"], S["plane"]
    Phi, dA, dG = S["fp64"]
    rng = np.random.default_rng(5)
    N = arr["amp"].size
    wall = np.flatnonzero(arr["phi"] > 0)
    dirs = [rng.standard_normal(N) * (arr["phi"] > 0) for _ in range(4)]
    # single nodes: the largest gradient entry, and three spread over the wall list
    for node in (int(np.argmax(np.abs(dA))), wall[len(wall) // 7], wall[len(wall) // 2], wall[-3]):
        d = np.zeros(N)
        d[node] = 1.0
        dirs.append(d)
    h = 1e-4 * KT
    for d in dirs:
        fd = (_phi_fresh(w, arr, arr["amp"] + h * d, np.zeros(3), T, axis, plane)
              - _phi_fresh(w, arr, arr["amp"] - h * d, np.zeros(3), T, axis, plane)) / (2 * h)
        ad = float(dA @ d)
        assert abs(ad - fd) <= 1e-4 * max(abs(fd), 1e-3 * np.abs(dA).max()), (ad, fd)
    hg = 1e-4 * w["body"][0][0]
    e = np.array([hg, 0.0, 0.0])
    fd = (_phi_fresh(w, arr, arr["amp"], e, T, axis, plane) - _phi_fresh(w, arr, arr["amp"], -e, T, axis, plane)) / (2 * hg)
    assert abs(dG[0] - fd) <= 1e-4 * abs(fd), (dG[0], fd)


def test_full_size_fp32_adjoint_against_fp64(full_size_adjoint):
    """The FP32 adjoint on the same full-size case, against the FP64 adjoint (FP32 forward and adjoint
    arithmetic over 200 steps).  Measured: Phi 1.6e-4 relative, the wall-amplitude gradient 7.7e-6 of its
    largest entry, dPhi/dg_x 2.7e-6 relative.  Held to the FP32 flux bound of 1e-3 on Phi and to
    about twice the measured errors on the gradients (2e-5 and 1e-5)."""
    Phi64, dA64, dG64 = full_size_adjoint["fp64"]
    Phi32, dA32, dG32 = full_size_adjoint["fp32"]
    err = {"Phi": abs(Phi32 - Phi64) / abs(Phi64), "dA": float(np.abs(dA32 - dA64).max() / np.abs(dA64).max()),
           "dG": abs(dG32[0] - dG64[0]) / abs(dG64[0])}
    print("full-size FP32 adjoint errors against FP64:", err)
    assert err["Phi"] <= 1e-3 and err["dA"] <= 2e-5 and err["dG"] <= 1e-5, err
