"""Checkpoint/restart of the state and the steady-state residual through the C ABI.

- A state saved after some steps and loaded into a fresh context continues bit-identically
  (populations, step count, flux average) in every storage precision.
- Loading a state of another lattice size, species count or precision, or a buffer that holds no
  state, is rejected and leaves the context as it was.
- The residual max |n(t) - n(t0)| / ((t - t0) n0) of the FP64 path equals the one computed from the
  oracle's densities of the same run (relative 1e-8: the difference of two densities that agree to
  1e-12 loses the digits they share).
"""
import numpy as np
import pytest

from lbe_cases import case_channel, case_well, setup_gpu, setup_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_1202_3842_gb300 import build
    build.build()


def _channel():
    return case_channel((40, 20, 16), (2.0, 4.0), 0.2, (1.0, 0.9), 8, 8, body=1e-4, wall_amp_kT=0.5)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_save_load_continues_bit_identically(prec):
    w, arr = _channel()
    a = setup_gpu(w, arr, prec)
    a.set_flux_plane(0, 20)
    a.step(7)
    state = a.save_state()
    a.step(5)
    b = setup_gpu(w, arr, prec)
    b.load_state(state)
    assert b.step_count() == 7
    b.step(5)
    assert b.step_count() == a.step_count() == 12
    for s in range(2):
        fa, ga = a.populations(s)
        fb, gb = b.populations(s)
        assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.flux(-1) == b.flux(-1)
    a.close()
    b.close()


def test_load_rejects_other_lattice_and_garbage():
    from paper_1202_3842_gb300 import lbe
    w, arr = _channel()
    a = setup_gpu(w, arr, "fp32")
    a.step(2)
    state = a.save_state()
    w2, arr2 = case_channel((48, 20, 16), (2.0, 4.0), 0.2, (1.0, 0.9), 8, 8, body=1e-4)
    b = setup_gpu(w2, arr2, "fp32")
    before = b.populations(0)
    with pytest.raises(lbe.LbeError) as e:
        b.load_state(state)
    assert e.value.status == 1
    with pytest.raises(lbe.LbeError):
        b.load_state(b"not a state" + bytes(200))
    c = setup_gpu(w, arr, "fp64")
    with pytest.raises(lbe.LbeError):
        c.load_state(state)
    after = b.populations(0)
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert b.step_count() == 0
    for s in (a, b, c):
        s.close()


def test_residual_matches_oracle_densities():
    w, arr = case_well((16, 16, 16), 3.0, 0.15, 1.0, 1.0, 4.0)
    gpu = setup_gpu(w, arr, "fp64")
    orc = setup_oracle(w, arr)
    fluid = arr["solid"] == 0
    n0 = arr["n"][0][fluid].mean()
    assert gpu.residual() == -1.0
    gpu.step(0)
    assert gpu.residual() == -1.0  # t == t0: nothing to compare
    n_prev = orc.observe()["n"][0].copy()
    for k in (5, 20):
        gpu.step(k)
        orc.step(k)
        n_now = orc.observe()["n"][0]
        expect = np.abs(n_now - n_prev).max() / (k * n0)
        got = gpu.residual()
        assert expect > 0
        assert abs(got - expect) <= 1e-8 * expect, (got, expect)
        n_prev = n_now.copy()
    gpu.close()


def _divergence(u, shape, periodic):
    """div u = 3 sum_p w_p c_p . u(r + c_p), with u = 0 beyond closed axes (numpy, from the definition)."""
    import oracle
    c, w, _ = oracle.lattice()
    nx, ny, nz = shape
    U = u.reshape(3, nz, ny, nx)
    out = np.zeros((nz, ny, nx))
    for p in range(1, 19):
        sh = [0, 0, 0]
        for ax, (d, n, per) in enumerate(zip(c[p], shape, periodic)):
            sh[ax] = int(d)
        for comp in range(3):
            if c[p][comp] == 0:
                continue
            v = U[comp]
            # value at r + c_p: roll by -c_p along each axis, then zero what wrapped across a closed axis
            r = np.roll(v, shift=(-sh[2], -sh[1], -sh[0]), axis=(0, 1, 2)).copy()
            for ax, d, n, per in ((2, sh[0], nx, periodic[0]), (1, sh[1], ny, periodic[1]), (0, sh[2], nz, periodic[2])):
                if per or d == 0:
                    continue
                idx = [slice(None)] * 3
                idx[ax] = slice(n - 1, n) if d > 0 else slice(0, 1)
                r[tuple(idx)] = 0.0
            out += w[p] * c[p][comp] * r
    return 3.0 * out.reshape(-1)


def test_divergence_of_the_velocity_matches_oracle_fields():
    from lbe_cases import setup_oracle
    w, arr = _channel()
    gsim = setup_gpu(w, arr, "fp64")
    o = setup_oracle(w, arr)
    gsim.step(25)
    o.step(25)
    obs = o.observe()
    n, J = obs["n"].sum(0), obs["J"].sum(0)
    u = np.where(n[None, :] > 0, J / np.where(n[None, :] > 0, n[None, :], 1.0), 0.0)
    expect = _divergence(u, w["shape"], w["periodic"])
    got = gsim.divergence(-1)
    scale = np.abs(expect).max()
    assert scale > 0
    assert np.abs(got - expect).max() <= 1e-11 * scale
    gsim.close()
