"""The device-side failure detector of the TMA kernels: a bounded mbarrier wait that runs out is reported
on the host, and the GPU stays usable.  The wait is made to run out by arming a barrier for bytes that no
copy delivers (none is issued, so nothing is in flight when the CTA returns)."""
import numpy as np
import pytest

from lbe_cases import case_channel, setup_gpu

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_host_reports_it():
    from paper_1202_3842_gb300 import lbe
    w, arr = case_channel((24, 12, 10), (2.0, 4.0), 0.2, (1.0, 1.0), 6, 6)
    g = setup_gpu(w, arr, "fp32")
    g.step(2)
    n_before = [g.density(a) for a in range(2)]
    with pytest.raises(lbe.LbeError) as e:
        lbe.lbe_probe_wait_timeout(g._h, 64)
    assert e.value.status == 4  # LBE_ERR_CUDA
    assert "TMA wait" in str(e.value)
    # the error word stays set: every later checking call reports it
    with pytest.raises(lbe.LbeError) as e2:
        g.density(0)
    assert e2.value.status == 4
    g.close()
    # the device and a new context are unaffected: the same two steps give the same densities
    g2 = setup_gpu(w, arr, "fp32")
    g2.step(2)
    for a in range(2):
        np.testing.assert_array_equal(g2.density(a), n_before[a])
    g2.close()


def test_wait_probe_rejects_a_poll_count_out_of_range():
    from paper_1202_3842_gb300 import lbe
    w, arr = case_channel((24, 12, 10), (2.0, 4.0), 0.2, (1.0, 1.0), 6, 6)
    g = setup_gpu(w, arr, "fp32")
    for polls in (0, -5):
        with pytest.raises(lbe.LbeError) as e:
            lbe.lbe_probe_wait_timeout(g._h, polls)
        assert e.value.status == 1
    g.step(1)  # the context is still good: nothing was launched
    g.close()
