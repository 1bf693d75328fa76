"""The library's host evaluation of the prescribed flapping kinematics (Sec. 5.1) against the oracle's
(adaptive quadrature of G_t there, composite Gauss-Legendre in the library).  Host logic: no GPU."""

import numpy as np
import pytest

from oracle import kinematics as okin


@pytest.fixture(scope="module")
def lib():
    from paper_2103_06415_gb300 import build as b
    b.build()
    import paper_2103_06415_gb300 as p
    return p


@pytest.mark.parametrize("sigma,freq", [(3.770, 1.0), (0.628, 1.0), (2.0, 0.7)])
def test_host_kinematics_match_oracle(lib, sigma, freq):
    params = (1.4, np.pi / 4, sigma, sigma, freq)
    kin = okin.FlappingKinematics(*params)
    for t in (0.0, 1e-3, 0.05, 0.25, 0.3, 0.61, 1.0, 1.37, 2.9):
        got = lib.flapping_kinematics(params, t)
        ref = np.array(kin.state(t))
        scale = np.array([0.7, 0.7 * 2 * np.pi * freq, 0.7 * (2 * np.pi * freq) ** 2 * sigma,
                          np.pi / 4, np.pi / 4 * 2 * np.pi * freq, np.pi / 4 * (2 * np.pi * freq) ** 2 * sigma])
        assert np.all(np.abs(got - ref) <= 1e-12 * scale), (t, got - ref)


def test_host_kinematics_reject_invalid_parameters(lib):
    for bad in ((-1.0, 0.7, 1.0, 1.0, 1.0), (1.4, 0.7, 0.0, 1.0, 1.0), (1.4, 0.7, 1.0, 1.0, 0.0),
                (1.4, np.nan, 1.0, 1.0, 1.0)):
        with pytest.raises(lib.FsiError):
            lib.flapping_kinematics(bad, 0.1)
