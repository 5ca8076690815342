"""Eq. 1's noise term through the C-ABI vs the FP64 oracle (needs a GB300).

The plane's noise (wcsim_plane_set_noise) is added to the wire spectra as the inverse time
FFT stages them; the oracle draws the same Philox normals in FP64 and transforms with
numpy's irfft.  Tolerances as for the forward: relative L2 <= 1e-5, max |err| <= 1e-4 x
peak.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5
MAX_PEAK = 1e-4


@pytest.fixture(scope="module")
def W():
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import wcsim
    return wcsim


def assert_close(got, ref, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.linalg.norm(got - ref)
    assert np.isfinite(got).all(), what
    assert err <= REL_L2 * np.linalg.norm(ref), "%s rel L2 %.3e" % (what, err / np.linalg.norm(ref))
    assert np.abs(got - ref).max() <= MAX_PEAK * np.abs(ref).max(), what


def amplitude(n_ft, scale):
    """A smooth low-pass amplitude spectrum (n_ft / 2 + 1 values)."""
    k = np.arange(n_ft // 2 + 1)
    return (scale / (1.0 + (k / (0.1 * n_ft)) ** 2)).astype(np.float32)


def plane(W, g, prm, R):
    import torch
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())


def noise_scale(signal, n_ft):
    """Amplitude whose noise RMS is about a tenth of the signal's."""
    return 0.1 * float(np.sqrt(np.mean(signal ** 2))) * np.sqrt(n_ft)


def test_noise_alone_matches_oracle(W):
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    prm = S.DriftParams()
    R = S.make_response(g, "induction")
    pl = plane(W, g, prm, R)
    amp = amplitude(1024, 50.0)
    pl.set_noise(amp, seed=12345)
    empty = S.Depos(p=np.zeros(0), t=np.zeros(0), td=np.zeros(0), q=np.zeros(0, np.float32),
                    id=np.zeros(0, np.uint32))
    got = pl.run(W.DeviceDepos.from_host(empty)).cpu().numpy()
    assert_close(got, O.noise(g, amp.astype(np.float64), 1024, prm.plane_id, 12345), "noise alone")


@pytest.mark.parametrize("n_fw,n_ft", [(0, 0), (150, 1200), (128, 1125)])
def test_run_with_noise_matches_oracle(W, n_fw, n_ft):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=1)
    R = S.make_response(g, kind, n_fw=n_fw or None, n_ft=n_ft or None)
    nft = R.shape[2]
    ref_sig = O.run(g, prm, R, d)
    amp = amplitude(nft, noise_scale(ref_sig, nft))
    pl = plane(W, g, prm, R)
    pl.set_noise(amp, seed=777)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    ref = ref_sig + O.noise(g, amp.astype(np.float64), nft, prm.plane_id, 777)
    assert_close(got, ref, "signal + noise (n_ft %d)" % nft)
    # turned off, the same plane gives the noiseless frame again
    pl.set_noise(None)
    assert_close(pl.run(W.DeviceDepos.from_host(d)).cpu().numpy(), ref_sig, "noise off")


def test_full_size_plane_with_noise_matches_oracle(W):
    wl = S.make_workload("plane960-100k")
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(g, kind)
    ref_sig = O.run(g, prm, R, d)
    amp = amplitude(g.n_ticks, noise_scale(ref_sig, g.n_ticks))
    pl = plane(W, g, prm, R)
    pl.set_noise(amp, seed=2021)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    ref = ref_sig + O.noise(g, amp.astype(np.float64), g.n_ticks, prm.plane_id, 2021)
    assert_close(got, ref, "960 x 6000 with noise")


def test_batched_events_take_seed_plus_event_index(W):
    import torch
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    prm = S.DriftParams(fluctuate=0)
    R = S.make_response(g, "collection")
    pl = plane(W, g, prm, R)
    amp = amplitude(1024, 20.0)
    pl.set_noise(amp, seed=900)
    rng = np.random.default_rng(5)
    events = [S.track_depos(rng, 2, 300, g.n_wires * g.pitch_mm, 0.75 * g.n_ticks * g.tick_us)
              for _ in range(3)]
    dev = [W.DeviceDepos.from_host(d) for d in events]
    got = [w.cpu().numpy() for w in W.Batch([pl] * 3, dev).run()]
    torch.cuda.synchronize()
    for e, d in enumerate(events):
        ref = O.run(g, prm, R, d) + O.noise(g, amp.astype(np.float64), 1024, prm.plane_id, 900 + e)
        assert_close(got[e], ref, "batched event %d" % e)


def test_noise_argument_errors(W):
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    pl = plane(W, g, S.DriftParams(), S.make_response(g, "collection"))
    with pytest.raises(W.WcsimError) as e:
        pl.set_noise(np.ones(100, np.float32))
    assert e.value.status == W.ESHAPE
    bad = np.ones(513, np.float32)
    bad[3] = -1.0
    with pytest.raises(W.WcsimError) as e:
        pl.set_noise(bad)
    assert e.value.status == W.EINVAL
