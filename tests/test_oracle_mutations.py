"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Each mutation replaces one oracle function for the duration of the test; the
pin is then expected to raise AssertionError."""
import numpy as np
import pytest

import oracle
import oracle.prnu_oracle as po
from tests import test_oracle_pins as pins


def _wrong_sign_xcorr(X, K0, K0_spectrum=None):
    H, W = X.shape
    return np.fft.irfft2(np.fft.rfft2(X) * np.conj(np.fft.rfft2(K0)), s=(H, W))


def _transposed_matrix(lam, theta_deg):
    th = np.deg2rad(theta_deg)
    c, s = np.cos(th), np.sin(th)
    return np.array([[c, -s], [s, c]]) / lam


def _zero_padded_moments(I):
    from scipy import ndimage
    I = np.asarray(I, np.float64)
    m1 = ndimage.uniform_filter(I, 3, mode="constant")
    m2 = ndimage.uniform_filter(I * I, 3, mode="constant")
    return m1, m2 - m1 * m1


def _pce_window9(C, exclusion=9):
    return _orig_pce(C, 9)


def _no_mean_removal(K):
    return np.asarray(K, np.float64)


_orig_pce = po.pce

MUTATIONS = [
    ("xcorr", _wrong_sign_xcorr, pins.test_shift_sign_convention),
    ("warp_matrix", _transposed_matrix, lambda: pins.test_warp_reproduces_linear_ramp(1.07, 3.3)),
    ("local_moments_3x3", _zero_padded_moments, pins.test_local_moments_match_scipy_nearest),
    ("pce", _pce_window9, pins.test_pce_golden_closed_forms),
    ("fingerprint_term", _no_mean_removal, pins.test_fingerprint_term_makes_correlation_blind_to_offsets),
]


@pytest.mark.parametrize("name,mutant,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_mutation(monkeypatch, name, mutant, pin):
    monkeypatch.setattr(po, name, mutant)
    monkeypatch.setattr(oracle, name, mutant)
    with pytest.raises(AssertionError):
        pin()
