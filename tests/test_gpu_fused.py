"""The two forward variants against the FP64 oracle, through the C-ABI (needs a GB300): the
plain flow (rasterize into the grid, then Eq. 2) and the fused flow (depos binned by wire,
rasterized inside the time-axis transform, the grid never written).

Both must give Eq. 2 of the scatter-added patches of Sec. 2.1.1: relative L2 <= 1e-5 and
max |err| <= 1e-4 x peak against the oracle, with and without fluctuation, for even, odd
and single impact counts, depos whose rows reach over many wires (the binning's wide
bucket), windows wider than the stored tick weights, renormalisation, padded spectra, the
block-level wire pass, empty and off-grid depo sets, and a growing binning scratch; the
autotuner keeps one of them and both must agree with each other.
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
    import torch
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import wcsim
    assert torch.cuda.is_available()
    return wcsim


def assert_close(got, ref, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape and np.isfinite(got).all(), what
    nref, pk = np.linalg.norm(ref), np.abs(ref).max()
    if nref == 0.0:
        assert np.abs(got).max() == 0.0, what
        return
    rel = np.linalg.norm(got - ref) / nref
    mx = np.abs(got - ref).max() / pk
    assert rel <= REL_L2 and mx <= MAX_PEAK, "%s rel L2 %.3e max/peak %.3e" % (what, rel, mx)


def plane(W, g, prm, R, n_fw=0, n_ft=0):
    import torch
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda(),
                   n_fw=n_fw, n_ft=n_ft)


def scattered_depos(g, rng, n, td_max, border=0.05):
    """Depos spread over the plane (and a little past its borders), uniform drift times."""
    span_p = g.n_rows * g.pitch_mm / g.n_imp
    span_t = g.n_ticks * g.tick_us
    p = g.p0_mm + rng.uniform(-border * span_p, (1 + border) * span_p, n)
    t = g.t0_us + rng.uniform(-border * span_t, 0.5 * span_t, n)
    td = rng.uniform(0.0, td_max, n)
    td[: n // 20] = 0.0                                   # point depos (sigma = 0)
    q = rng.lognormal(np.log(6000), 0.3, n).astype(np.float32)
    return S.Depos(p=p, t=t, td=td, q=q, id=rng.permutation(n).astype(np.uint32))


FLOWS = [True, False]      # fused, plain


@pytest.mark.parametrize("fused", FLOWS)
@pytest.mark.parametrize("fluct", [0, 1])
def test_forward_matches_oracle(W, fused, fluct):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct)
    R = S.make_response(g, kind)
    pl = plane(W, g, prm, R)
    pl.set_forward(fused)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), "fused %d fluct %d" % (fused, fluct))
    assert pl.check_flags() == 0
    pl.close()


@pytest.mark.parametrize("fused", FLOWS)
@pytest.mark.parametrize("n_imp", [5, 1, 7, 10])
def test_forward_odd_impact_counts(W, fused, n_imp):
    g = S.Geometry(n_wires=64, n_imp=n_imp, n_ticks=640, pitch_mm=3.0, p0_mm=-4.0, t0_us=-20.0)
    prm = S.DriftParams(fluctuate=1, seed=0x1234 + n_imp, plane_id=n_imp)
    rng = np.random.default_rng(40 + n_imp)
    d = scattered_depos(g, rng, 1500, 250.0)
    R = S.make_response(g, "induction")
    pl = plane(W, g, prm, R)
    pl.set_forward(fused)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), "n_imp %d" % n_imp)
    pl.close()


@pytest.mark.parametrize("fused", FLOWS)
def test_forward_wide_depos_and_wide_tick_windows(W, fused):
    """Large D_T puts depos' rows over more than four wires (the wide bucket, read by every
    CTA); large D_L gives tick windows wider than the stored weights (formed in the
    transform); n_sigma = 5 widens both."""
    g = S.Geometry(n_wires=96, n_imp=10, n_ticks=1200, pitch_mm=3.0)
    prm = S.DriftParams(DL_cm2_s=60.0, DT_cm2_s=150.0, nsigma=5.0, fluctuate=1, seed=77)
    rng = np.random.default_rng(3)
    d = scattered_depos(g, rng, 800, 400.0)
    R = S.make_response(g, "collection")
    pl = plane(W, g, prm, R)
    w = O.windows(g, prm, d)
    ok = w[:, 0] >= 0
    wires = (w[ok, 1] // g.n_imp) - (w[ok, 0] // g.n_imp)
    tick_groups = (w[ok, 3] // 4) - (w[ok, 2] // 4) + 1
    assert (wires >= 4).sum() > 50 and (tick_groups > 6).sum() > 50   # both paths are taken
    pl.set_forward(fused)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), "wide")
    pl.close()


@pytest.mark.parametrize("fused", FLOWS)
@pytest.mark.parametrize("renorm", [0, 1])
def test_forward_renormalised_and_padded(W, fused, renorm):
    g = S.Geometry(n_wires=120, n_imp=10, n_ticks=1000, pitch_mm=4.7, p0_mm=2.0, t0_us=3.0)
    prm = S.DriftParams(fluctuate=1, renormalize=renorm, seed=5)
    rng = np.random.default_rng(11)
    d = scattered_depos(g, rng, 1200, 600.0, border=0.1)
    R = S.make_response(g, "induction", n_fw=128, n_ft=1050)
    pl = plane(W, g, prm, R)
    pl.set_forward(fused)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), "renorm %d" % renorm)
    pl.close()


@pytest.mark.parametrize("fused", FLOWS)
def test_forward_block_wire_pass(W, fused):
    """A wire count the one-warp wire pass does not take (100 = 4 x 25): every impact
    position is transformed before the block-level wire pass takes them."""
    g = S.Geometry(n_wires=100, n_imp=10, n_ticks=900, pitch_mm=3.0)
    prm = S.DriftParams(fluctuate=1, seed=9)
    d = scattered_depos(g, np.random.default_rng(12), 1000, 300.0)
    R = S.make_response(g, "collection")
    pl = plane(W, g, prm, R)
    pl.set_forward(fused)
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), "block wire pass")
    pl.close()


def test_fused_matches_plain_forward_with_fluctuation(W):
    """The two forward variants draw the same Philox numbers per bin: equal frames up to
    summation order."""
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=1)
    R = S.make_response(g, kind)
    pl = plane(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    pl.set_forward(True)
    fused = pl.run(dd).cpu().numpy()
    pl.set_forward(False)
    plain = pl.run(dd).cpu().numpy()
    assert_close(fused, plain, "fused vs plain")
    pl.close()


@pytest.mark.parametrize("fused", FLOWS)
def test_forward_empty_offgrid_and_growing_depo_sets(W, fused):
    import torch
    g = S.Geometry(n_wires=64, n_imp=10, n_ticks=512, pitch_mm=3.0)
    prm = S.DriftParams(fluctuate=1, seed=21)
    R = S.make_response(g, "collection")
    pl = plane(W, g, prm, R)
    pl.set_forward(fused)
    rng = np.random.default_rng(8)
    empty = S.Depos(p=np.zeros(0), t=np.zeros(0), td=np.zeros(0), q=np.zeros(0, np.float32),
                    id=np.zeros(0, np.uint32))
    off = scattered_depos(g, rng, 300, 100.0)
    off = dataclasses.replace(off, p=off.p + 1e4)               # every depo off the grid
    for d in (scattered_depos(g, rng, 100, 200.0), empty, off,
              scattered_depos(g, rng, 6000, 200.0), scattered_depos(g, rng, 50, 200.0)):
        out = torch.full((g.n_wires, g.n_ticks), float("nan"), device="cuda")
        got = pl.run(W.DeviceDepos.from_host(d), out=out).cpu().numpy()
        ref = O.run(g, prm, R, d) if len(d.p) else np.zeros((g.n_wires, g.n_ticks))
        assert_close(got, ref, "n %d" % len(d.p))
    pl.close()


def test_autotune_keeps_a_forward_variant_that_matches_the_oracle(W):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=1)
    R = S.make_response(g, kind)
    pl = plane(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    rep = pl.autotune(dd)
    assert rep["ms_forward_plain"] > 0 and rep["ms_forward_fused"] > 0
    assert rep["forward_fused"] == int(rep["ms_forward_fused"] < rep["ms_forward_plain"])
    assert_close(pl.run(dd).cpu().numpy(), O.run(g, prm, R, d), "autotuned")
    pl.close()
