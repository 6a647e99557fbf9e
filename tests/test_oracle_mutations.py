"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin fails.

Covered: the correlation sign, the warp matrix, the moments' border, the PCE
window, the mean removal, the correction steps, Eq. 2's weighting, the wavelet
filter (a sign typo, and the filter reversed), the wavelet analysis phase, the
shrinkage window choice, the fingerprint resampling, the frame-literal warp,
the homography's angle and the Wiener noise power (a median, zero-padded
moments, the variance of the whole frame).

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
_orig_prnu_residual = po.prnu_residual


def _widening_steps(n):
    """Eq. 8's steps read literally (0.01^-n, 0.1^-n grow): the narrowing lost."""
    return po._f32(0.01 * 10.0 ** (n - 1)), po._f32(0.1 * 10.0 ** (n - 1))


def _estimate_without_intensity(frames):
    """Eq. 2 with sum W(I) in the numerator instead of sum I W(I)."""
    num = den = 0.0
    for f in frames:
        I = np.asarray(f, np.float64)
        num = num + po.wiener_residual(I)[0]
        den = den + I * I
    out = np.zeros_like(num)
    np.divide(num, den, out=out, where=den > 0)
    return out


_DB8_TYPO = po.DB8.copy()
_DB8_TYPO[3] = -_DB8_TYPO[3]


def _shrink_with_the_largest_window(c, sigma0):
    """The largest of the four window variances instead of the smallest."""
    c = np.asarray(c, np.float64)
    c2 = c * c
    s2 = None
    for Wn in (3, 5, 7, 9):
        r = Wn // 2
        P = np.pad(c2, r)
        acc = sum(P[dy:dy + c.shape[0], dx:dx + c.shape[1]] for dy in range(Wn) for dx in range(Wn))
        v = np.maximum(acc / (Wn * Wn) - sigma0 ** 2, 0.0)
        s2 = v if s2 is None else np.maximum(s2, v)
    den = s2 + sigma0 ** 2
    return np.where(den > 0, c * sigma0 ** 2 / np.where(den > 0, den, 1.0), 0.0)


def _unwidened_tent(n_in, scale, first, n_out):
    """Resampling with the tent never widened: shrinking aliases."""
    Wm = np.zeros((n_out, n_in))
    for r in range(n_out):
        u = (first + r + 0.5) / scale - 0.5
        j0 = int(np.floor(u))
        for j, t in ((j0, 1.0 - (u - j0)), (j0 + 1, u - j0)):
            Wm[r, min(max(j, 0), n_in - 1)] += t
    return Wm


def _literal_without_warp(frame, lam, theta_deg, weight_by_intensity=True):
    """The frame's own residual whatever the candidate."""
    return _orig_prnu_residual(frame, weight_by_intensity=weight_by_intensity)[0]


def _similarity_angle_flipped(Hm):
    lam, th = _orig_similarity(Hm)
    return lam, -th


_orig_similarity = po.similarity_from_homography
_orig_moments = po.local_moments_3x3


def _wiener_with(nu2_of):
    """wiener_residual with the noise power taken by nu2_of(I, var) instead of
    the mean of the replicated-border local variances."""
    def wiener(I):
        I = np.asarray(I, np.float64)
        mu, var = _orig_moments(I)
        nu2 = float(nu2_of(I, var))
        den = np.maximum(var, nu2)
        safe = np.where(den > 0, den, 1.0)
        gain = np.where(den > 0, np.maximum(var - nu2, 0.0) / safe, 1.0)
        return I - (mu + (I - mu) * gain), nu2
    return wiener


def _nu2_zero_padded(I, var):
    return _zero_padded_moments(I)[1].mean()


_DB8_REVERSED = po.DB8[::-1].copy()


def _analysis_shifted(x, axis):
    """The periodic analysis read one sample late: x[2n + k + 1]."""
    return _orig_analysis(np.roll(x, -1, axis=axis), axis)


def _synthesis_shifted(a, d, axis):
    """Its transpose (so that the shifted pair still reconstructs)."""
    return np.roll(_orig_synthesis(a, d, axis), 1, axis=axis)


_orig_analysis = po._analysis_1d
_orig_synthesis = po._synthesis_1d

MUTATIONS = [
    ("xcorr", _wrong_sign_xcorr, pins.test_shift_sign_convention),
    ("warp_matrix", _transposed_matrix, lambda: pins.test_warp_reproduces_linear_ramp(1.07, 3.3)),
    ("local_moments_3x3", _zero_padded_moments, pins.test_local_moments_match_scipy_nearest),
    ("pce", _pce_window9, pins.test_pce_golden_closed_forms),
    ("fingerprint_term", _no_mean_removal, pins.test_fingerprint_term_makes_correlation_blind_to_offsets),
    ("_corr_step", _widening_steps, pins.test_correction_nodes_are_centred_and_spaced_by_the_iteration_step),
    ("fingerprint_estimate", _estimate_without_intensity, pins.test_fingerprint_estimate_is_a_ratio_of_sums),
    ("DB8", _DB8_TYPO, pins.test_dwt2_reconstructs_and_keeps_energy),
    ("mihcak_shrink", _shrink_with_the_largest_window, pins.test_mihcak_shrink_of_an_isolated_coefficient),
    ("resize_weights", _unwidened_tent, pins.test_resize_half_is_the_1331_filter),
    ("literal_residual", _literal_without_warp, lambda: pins.test_literal_residual_commutes_with_a_quarter_turn(33)),
    ("similarity_from_homography", _similarity_angle_flipped,
     pins.test_similarity_from_homography_inverts_the_warp),
    ("wiener_residual", _wiener_with(lambda I, var: np.median(var)), pins.test_wiener_impulse_closed_form),
    ("wiener_residual", _wiener_with(_nu2_zero_padded), pins.test_wiener_impulse_closed_form),
    ("wiener_residual", _wiener_with(lambda I, var: np.var(I)), pins.test_wiener_impulse_closed_form),
    ("DB8", _DB8_REVERSED, pins.test_wavelet_analysis_of_an_impulse_closed_form),
    (("_analysis_1d", "_synthesis_1d"), (_analysis_shifted, _synthesis_shifted),
     pins.test_wavelet_analysis_of_an_impulse_closed_form),
]
MUTATION_IDS = ["xcorr", "warp_matrix", "local_moments_3x3", "pce", "fingerprint_term", "_corr_step",
                "fingerprint_estimate", "DB8", "mihcak_shrink", "resize_weights", "literal_residual",
                "similarity_from_homography", "nu2_median", "nu2_zero_padded", "nu2_frame_variance",
                "DB8_reversed", "wavelet_phase_shift"]


def test_mutants_still_reconstruct():
    """The wavelet mutants are the ones the older pins let through: the
    reversed filter and the one-sample phase shift keep the transform
    orthonormal, so reconstruction and energy hold."""
    X = np.random.default_rng(3).standard_normal((32, 48))
    for a, s in ((_analysis_shifted, _synthesis_shifted),):
        lo, hi = a(X, 1)
        np.testing.assert_allclose(s(lo, hi, 1), X, atol=1e-12)


@pytest.mark.parametrize("name,mutant,pin", MUTATIONS, ids=MUTATION_IDS)
def test_pin_catches_mutation(monkeypatch, name, mutant, pin):
    names, mutants = (name, mutant) if isinstance(name, tuple) else ((name,), (mutant,))
    for n, m in zip(names, mutants):
        monkeypatch.setattr(po, n, m)
        monkeypatch.setattr(oracle, n, m, raising=False)
    with pytest.raises(AssertionError):
        pin()
