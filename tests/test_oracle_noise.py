"""Pins of the oracle's noise term (Eq. 1's additive N(t, x)) against what the mathematics
fixes, on CPU.

The paper names the term and gives no model; the reading is spectral noise per wire: the
normalised inverse DFT over n_ft points of an amplitude spectrum A(k) times unit complex
Gaussians xi(k) (Hermitian, real at k = 0 and Nyquist).  The pins: a brute-force DFT sum on
tiny sizes (orientation, scaling, Hermitian extension, crop), Parseval's variance for a flat
spectrum, the periodogram against A^2, Gaussian marginals, independence across wires, unit
mean square of the draws, and the real DC / Nyquist terms.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S


def _geom(n_w, n_t):
    return S.Geometry(n_wires=n_w, n_imp=10, n_ticks=n_t, pitch_mm=3.0)


@pytest.mark.parametrize("n_ft,n_t", [(8, 8), (9, 9), (12, 10)])
def test_noise_is_the_brute_force_inverse_dft(n_ft, n_t):
    g = _geom(3, n_t)
    rng = np.random.default_rng(n_ft)
    amp = rng.uniform(0.5, 2.0, n_ft // 2 + 1)
    xi = O.noise_spectrum(3, n_ft, 7, 11)
    got = O.noise(g, amp, n_ft, 7, 11)
    full_a = np.array([amp[min(k, n_ft - k)] for k in range(n_ft)])
    for w in range(3):
        full_x = np.array([xi[w, k] if k <= n_ft // 2 else np.conj(xi[w, n_ft - k])
                           for k in range(n_ft)])
        for t in range(n_t):
            ref = sum(full_a[k] * full_x[k] * np.exp(2j * np.pi * k * t / n_ft)
                      for k in range(n_ft)) / n_ft
            assert abs(ref.imag) < 1e-12
            assert got[w, t] == pytest.approx(ref.real, abs=1e-12)


def test_zero_amplitude_gives_no_noise():
    g = _geom(4, 64)
    assert not O.noise(g, np.zeros(33), 64, 0, 3).any()


def test_dc_and_nyquist_draws_are_real_and_draws_have_unit_mean_square():
    xi = O.noise_spectrum(256, 64, 2, 99)
    assert not xi[:, 0].imag.any() and not xi[:, 32].imag.any()
    inner = xi[:, 1:32]
    assert np.mean(np.abs(inner) ** 2) == pytest.approx(1.0, abs=0.02)
    assert np.mean(xi[:, 0].real ** 2) == pytest.approx(1.0, abs=0.2)
    # real and imaginary parts each carry half the power and are uncorrelated
    assert np.mean(inner.real ** 2) == pytest.approx(0.5, abs=0.02)
    assert abs(np.mean(inner.real * inner.imag)) < 0.02


def test_flat_spectrum_variance_is_parseval():
    """A(k) = a for all k: E[n(t)^2] = (1/n^2) sum_k a^2 E|xi|^2 = a^2 / n."""
    n, a = 512, 3.0
    g = _geom(400, n)
    x = O.noise(g, np.full(n // 2 + 1, a), n, 1, 2024)
    assert np.mean(x ** 2) == pytest.approx(a * a / n, rel=0.02)
    assert abs(np.mean(x)) < 5 * a / n / np.sqrt(x.size)


def test_periodogram_follows_the_amplitude_spectrum():
    """|DFT of the noise|^2 / A^2 has mean 1 at every frequency (averaged over wires)."""
    n = 256
    k = np.arange(n // 2 + 1)
    amp = 5.0 / (1.0 + (k / 20.0) ** 2)            # a smooth low-pass shape
    g = _geom(600, n)
    x = O.noise(g, amp, n, 3, 77)
    ratio = np.abs(np.fft.rfft(x, axis=1)) ** 2 / amp[None, :] ** 2
    band = ratio[:, 1:-1].mean(axis=0)
    assert np.all(np.abs(band - 1.0) < 0.2)      # 600 wires: std of the mean ~ 0.04
    assert ratio[:, 1:-1].mean() == pytest.approx(1.0, abs=0.02)


def test_samples_are_gaussian_and_wires_independent():
    n = 256
    g = _geom(200, n)
    x = O.noise(g, np.full(n // 2 + 1, 1.0), n, 4, 5)
    z = x.ravel() / x.std()
    assert stats.kstest(z[::7], "norm").pvalue > 1e-3
    c = np.corrcoef(x[:50])
    off = c[~np.eye(50, dtype=bool)]
    assert np.abs(off).max() < 0.3 and abs(off.mean()) < 0.02


def test_seeds_and_planes_give_different_noise():
    g = _geom(8, 64)
    amp = np.ones(33)
    base = O.noise(g, amp, 64, 0, 1)
    assert not np.allclose(base, O.noise(g, amp, 64, 0, 2))
    assert not np.allclose(base, O.noise(g, amp, 64, 1, 1))
    assert np.array_equal(base, O.noise(g, amp, 64, 0, 1))
