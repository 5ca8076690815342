"""Frames read out as ADC codes (wcsim_run_adc) vs the oracle's digitizer (needs a GB300).

The code is an integer decision taken in FP32 on the kernel's own waveform value, so it is
compared with the oracle's digitizer applied to the float frame wcsim_run writes for the same
depos (bit for bit away from rounding edges: two runs differ in the last bits of bins where
patches overlap, the float atomics adding in a run-dependent order); against the oracle's own
FP64 frame the codes agree except where the two frames (equal within the forward's
tolerance) fall on either side of a rounding edge, and there by one count.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import wcsim
    return wcsim


def plane(W, g, prm, R):
    import torch
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())


def codes(t):
    return t.cpu().numpy().view(np.uint16)


@pytest.mark.parametrize("fluct,noise", [(0, False), (1, False), (1, True)])
def test_adc_codes_match_the_oracle(W, fluct, noise):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct)
    R = S.make_response(g, kind)
    pl = plane(W, g, prm, R)
    ref = O.run(g, prm, R, d)
    gain = 2000.0 / np.abs(ref).max()                 # the frame spans ~4000 counts
    pl.set_digitizer(gain, 2048.0, 12)
    if noise:
        k = np.arange(g.n_ticks // 2 + 1)
        amp = (0.05 * np.abs(ref).max() * np.sqrt(g.n_ticks) / (1 + (k / 100.0) ** 2)).astype(np.float32)
        pl.set_noise(amp, seed=31)
        ref = ref + O.noise(g, amp.astype(np.float64), g.n_ticks, prm.plane_id, 31)
    dd = W.DeviceDepos.from_host(d)
    wave = pl.run(dd).cpu().numpy()
    adc = codes(pl.run_adc(dd))
    # against the digitizer applied to the float frame of a wcsim_run of the same depos: bit
    # for bit, except where that frame sits on a rounding edge (two runs differ in the last
    # bits, the float atomics adding overlapping patches in a run-dependent order)
    same = O.digitize(wave, gain, 2048.0, 12)
    dsame = adc.astype(np.int64) - same.astype(np.int64)
    xg = gain * wave.astype(np.float64) + 2048.0 + 0.5
    near = np.abs(xg - np.round(xg)) < 1e-5 * (1 + np.abs(xg))
    assert np.abs(dsame).max() <= 1 and np.all(near[dsame != 0])
    assert np.count_nonzero(dsame) <= 1e-3 * dsame.size
    # against the FP64 frame: one count at most, and only next to a rounding edge
    ora = O.digitize(ref.astype(np.float32), gain, 2048.0, 12)
    diff = adc.astype(np.int64) - ora.astype(np.int64)
    assert np.abs(diff).max() <= 1
    x = gain * ref + 2048.0 + 0.5
    edge = np.abs(x - np.round(x)) < 1e-3 * (1 + np.abs(x))
    assert np.all(edge[diff != 0])
    assert adc.max() <= 4095


def test_empty_frame_reads_the_pedestal_and_codes_clamp(W):
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    pl = plane(W, g, S.DriftParams(), S.make_response(g, "collection"))
    empty = S.Depos(p=np.zeros(0), t=np.zeros(0), td=np.zeros(0), q=np.zeros(0, np.float32),
                    id=np.zeros(0, np.uint32))
    dd = W.DeviceDepos.from_host(empty)
    pl.set_digitizer(1.0, 411.5, 10)
    assert np.all(codes(pl.run_adc(dd)) == 412)       # round half up
    pl.set_digitizer(1.0, 5000.0, 10)
    assert np.all(codes(pl.run_adc(dd)) == 1023)      # clamped at 2^10 - 1
    pl.set_digitizer(1.0, -3.0, 10)
    assert np.all(codes(pl.run_adc(dd)) == 0)         # clamped at 0


def test_digitizer_argument_errors(W):
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    pl = plane(W, g, S.DriftParams(), S.make_response(g, "collection"))
    d = S.make_workload("plane128-2k").planes[0][3]
    with pytest.raises(W.WcsimError) as e:
        pl.run_adc(W.DeviceDepos.from_host(d))        # no digitizer set yet
    assert e.value.status == W.EINVAL
    for bits in (0, 17):
        with pytest.raises(W.WcsimError) as e:
            pl.set_digitizer(1.0, 0.0, bits)
        assert e.value.status == W.EINVAL
