"""Pins of the oracle's digitizer (M read as an ADC value) on CPU: round half up at exact
half codes, clamping at 0 and 2^bits - 1, the pedestal alone for M = 0, monotonicity, and
codes that are exact integers of g M + p when that value is an integer."""
import numpy as np

from oracle import oracle as O


def test_round_half_up_and_clamp():
    m = np.array([-1000.0, -0.25, 0.0, 0.25, 0.5, 0.75, 1.0, 1.5, 2.5, 4095.4, 4095.6, 1e9],
                 np.float32)
    got = O.digitize(m, gain=1.0, pedestal=0.0, bits=12)
    assert got.tolist() == [0, 0, 0, 0, 1, 1, 1, 2, 3, 4095, 4095, 4095]
    assert got.dtype == np.uint16


def test_pedestal_gain_and_integers():
    m = np.arange(-5, 6, dtype=np.float32) * 2.0
    got = O.digitize(m, gain=0.5, pedestal=900.0, bits=12)
    assert got.tolist() == (900 + np.arange(-5, 6)).tolist()      # g M + p is an integer
    assert O.digitize(np.zeros(3, np.float32), 3.0, 412.4, 12).tolist() == [412] * 3
    assert O.digitize(np.zeros(1, np.float32), 3.0, 412.5, 12).tolist() == [413]
    assert O.digitize(np.full(1, 1e6, np.float32), 1.0, 0.0, 14).tolist() == [16383]


def test_monotone_in_the_waveform():
    rng = np.random.default_rng(3)
    m = np.sort(rng.normal(0, 200, 5000).astype(np.float32))
    c = O.digitize(m, gain=2.5, pedestal=2048.0, bits=12).astype(np.int64)
    assert np.all(np.diff(c) >= 0)
    assert c.max() <= 4095
    # one code per 1/g of the waveform away from the clamps
    mid = (m > -500) & (m < 500)
    assert np.all(np.abs(c[mid] - (2.5 * m[mid].astype(np.float64) + 2048.0)) <= 0.5 + 1e-3)
