"""The precision form (FP32 and the shifted 16-bit storage forms, FP32 arithmetic) against FP64 on the
128x32x32 two-component bottleneck channel (the same absolute slit as the 512x128x128 channel; sigma 4/6,
packing 0.25, tau 1/1, body force 1e-6): 1000 DD-TR steps from the uniform start, flux plane x = 64.

The reference is the FP64 oracle's run of the same case, stored in tests/golden/channel128_oracle.json by
tests/golden/make_channel128.py (oracle only): the time-averaged flux of each species and n, J at sampled
fluid nodes.  The GPU FP64 run is checked against it to round-off; the other storage forms are checked
against it and, over the whole lattice, against the GPU FP64 run.

Measured (max over species and fluid nodes, relative to the largest density or velocity; summed flux):
  FP32 (deviations f - w_p n0 stored and updated):  n 1.5e-6, u 4.9e-6, flux 3.5e-6
  BF16 shifted:                                    n 2.1e-2, u 0.12,   flux 6.6e-2
  FP16 shifted:                                    n 1.8e-3, u 1.0e-2, flux 1.6e-2
FP32 is held to 1e-5 on the density and 1e-3 on the velocities and the flux; the 16-bit forms to about
twice their measured errors."""
import json
import os

import numpy as np
import pytest

from paper_1202_3842_gb300 import studies

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "channel128_oracle.json")
# bounds: density (max |dn| / max n), per-species velocity (max |du| / max |u|), summed flux (relative)
BOUNDS = {
    "fp32": {"n": 1e-5, "u": 1e-3, "flux": 1e-3},
    "bf16": {"n": 4.5e-2, "u": 0.25, "flux": 0.15},
    "fp16": {"n": 4e-3, "u": 2.5e-2, "flux": 3.5e-2},
}


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


@pytest.fixture(scope="module")
def runs(golden):
    """The four precisions after the golden's step count, and the errors against the FP64 run."""
    return studies.precision(steps=golden["steps"], plane=golden["flux_plane_x"], keep_fields=True)


def test_fp64_matches_the_oracle_golden(golden, runs):
    ref = runs["fields"]["fp64"]
    for a in range(2):
        fl = golden["flux_time_avg"][a]
        assert abs(ref["flux"][a] - fl) <= 1e-12 * abs(fl), (a, ref["flux"][a], fl)
        idx = np.array(golden["nodes"])
        n = np.array(golden["n"][a])
        assert np.abs(ref["n"][a][idx] - n).max() <= 1e-12 * golden["max_n"][a]
        J = np.array(golden["J"][a])
        Jg = ref["J"][a][:, idx]
        assert np.abs(Jg - J).max() <= 1e-11 * np.abs(J).max() + 1e-16 * golden["max_n"][a]


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16"])
def test_storage_precision_errors(prec, golden, runs):
    e = runs[prec]
    b = BOUNDS[prec]
    assert e["n"] <= b["n"], (prec, e)
    assert e["u"] <= b["u"], (prec, e)
    assert e["flux"] <= b["flux"], (prec, e)
    # against the oracle itself: the summed flux and the sampled densities
    f = runs["fields"][prec]
    fl = sum(golden["flux_time_avg"])
    assert abs(sum(f["flux"]) - fl) <= 1.01 * b["flux"] * abs(fl)
    idx = np.array(golden["nodes"])
    for a in range(2):
        assert np.abs(f["n"][a][idx] - np.array(golden["n"][a])).max() <= 1.01 * b["n"] * golden["max_n"][a]
