"""The species-mass entry point that allocates no device memory.

Some callers cannot allocate device memory when they ask for the totals (a
device pool fully reserved by another framework, a loop that cannot take an
allocation's latency, a fixed device-memory footprint).  lbe_get_mass_noalloc
serves them from a file-scope device array instead; this test checks, through
the C ABI, that two calls in a row give the masses of lbe_get_totals to the
FP64 tolerance used by the parity tests (1e-12 relative).  It sits in a file
that pytest collects last.
"""
import numpy as np
import pytest

from lbe_cases import case_channel, setup_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mass_noalloc_matches_totals_twice(prec):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_1202_3842_gb300 import build, lbe
    build.build()
    w, arr = case_channel((40, 20, 16), (4.0, 6.0), 0.25, (1.0, 1.0), 8, 10, body=1e-5)
    sim = setup_gpu(w, arr, prec)
    sim.step(7)
    ref, _, _ = sim.totals()
    first = lbe.lbe_get_mass_noalloc(sim._h, sim.M)
    second = lbe.lbe_get_mass_noalloc(sim._h, sim.M)
    np.testing.assert_allclose(first, ref, rtol=1e-12)
    np.testing.assert_allclose(second, ref, rtol=1e-12)
    sim.step(3)
    ref2, _, _ = sim.totals()
    third = lbe.lbe_get_mass_noalloc(sim._h, sim.M)
    np.testing.assert_allclose(third, ref2, rtol=1e-12)
