"""Host logic of the scheme-comparison studies (no GPU): the lattice gradient behind the ideal-gas
current shift, scheme-name handling and the command line."""
import inspect

import numpy as np
import pytest

import oracle
from paper_1202_3842_gb300 import inputs, studies


def test_gradient_is_minus_the_oracle_force_field():
    # The force from a potential is F = -grad_h V with the isotropic D3Q19 gradient; on a periodic
    # lattice with no body force the oracle's F and the study's gradient must agree to round-off.
    shape = (12, 10, 8)
    V = inputs.cosine_well(shape, 0.3, 4.0)
    F = oracle.force_field(shape, (1, 1, 1), V)
    G = studies.gradient_periodic(V, shape)
    assert np.abs(F).max() > 1e-3
    assert np.abs(G + F).max() <= 1e-15


def test_gradient_of_a_plane_wave_is_the_lattice_derivative():
    # For V = sin(k x) the D3Q19 gradient is the central difference cos(k x) sin(k) (weights sum to
    # 1/3 along each axis, times 3): exact on any lattice, independent of the oracle.
    shape = (16, 4, 4)
    k = 2 * np.pi / 16
    x = np.arange(16.0)
    V = np.tile(np.sin(k * x), 16)
    G = studies.gradient_periodic(V, shape).reshape(3, 4, 4, 16)
    assert np.allclose(G[0], np.cos(k * x) * np.sin(k), atol=1e-15)
    assert np.abs(G[1:]).max() <= 1e-15


def test_scheme_names():
    assert studies._split("dd_tr_c") == ("dd_tr", True)
    assert studies._split("sd_eu") == ("sd_eu", False)
    with pytest.raises(ValueError):
        studies._split("dd_xx")
    with pytest.raises(ValueError):
        studies.main(["spurious", "--schemes", "dd_tr,bogus"])


def test_quick_settings_match_the_study_signatures():
    assert set(studies.QUICK) == set(studies.STUDIES)
    for name, kw in studies.QUICK.items():
        params = inspect.signature(studies.STUDIES[name]).parameters
        assert set(kw) <= set(params), name
