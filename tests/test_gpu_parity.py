"""CUDA path vs FP64 oracle, element by element, through the C-ABI (needs a GB300).

Tolerances (forward waveforms, grids and spectra): relative L2 <= 1e-5 and
max |err| <= 1e-4 x peak |oracle|.  Bin windows are compared bit for bit.
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


def assert_close(got, ref, rel=REL_L2, peak=MAX_PEAK, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    assert got.shape == ref.shape
    nref = np.linalg.norm(ref)
    err = np.linalg.norm(got - ref)
    mx = np.abs(got - ref).max() if got.size else 0.0
    pk = np.abs(ref).max() if ref.size else 0.0
    assert np.isfinite(got).all(), what
    assert err <= rel * nref + 1e-30, "%s rel L2 %.3e" % (what, err / max(nref, 1e-300))
    assert mx <= peak * pk + 1e-30, "%s max/peak %.3e" % (what, mx / max(pk, 1e-300))
    return err / max(nref, 1e-300), mx / max(pk, 1e-300)


def to_dev(W, d):
    return W.DeviceDepos.from_host(d)


def plane_for(W, g, prm, R):
    import torch
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())


def edge_case_depos(g, rng, n=600):
    """Point depos, depos on exact bin edges, straddling the grid border, off-grid."""
    dp = g.pitch_mm / g.n_imp
    span_p = g.n_rows * dp
    span_t = g.n_ticks * g.tick_us
    p = rng.uniform(-0.05 * span_p, 1.05 * span_p, n)
    t = rng.uniform(-0.05 * span_t, 0.4 * span_t, n)
    td = rng.uniform(0.0, 0.6 * span_t, n)
    td[:60] = 0.0                                          # sigma = 0
    k = rng.integers(0, g.n_rows, 60)
    p[60:120] = g.p0_mm + k * dp                            # exactly on row edges
    kt = rng.integers(0, g.n_ticks, 60)
    t[120:180] = g.t0_us + kt * g.tick_us - td[120:180]     # arrival on tick edges
    p[180:200] = [-1e9, 1e9, -1e13, 1e13] * 5                # far off-grid
    td[200:210] = 1e-30                                     # tiny, not zero
    q = rng.lognormal(np.log(6000), 0.3, n).astype(np.float32)
    q[210:220] = 0.0
    return S.Depos(p=p, t=t, td=td, q=q, id=np.arange(n, dtype=np.uint32))


# ------------------------------------------------------------------ windows: bit exact
@pytest.mark.parametrize("name", ["plane128-2k", "plane960-100k"])
def test_windows_bit_exact_on_workload(W, name):
    wl = S.make_workload(name)
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(S.Geometry(8, g.n_imp, 16, g.pitch_mm), kind)  # any valid response
    pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    got = pl.windows(to_dev(W, d)).cpu().numpy()
    ref = O.windows(g, prm, d)
    assert np.array_equal(got, ref.astype(np.int32))
    assert pl.check_flags() == 0


def test_windows_bit_exact_edge_cases(W):
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=512, pitch_mm=3.0)
    rng = np.random.default_rng(31)
    d = edge_case_depos(g, rng)
    for prm in (S.DriftParams(), S.DriftParams(nsigma=1.7, DL_cm2_s=0.0, DT_cm2_s=25.0),
                S.DriftParams(nsigma=5.0, v_mm_per_us=0.9, lifetime_us=float("inf"))):
        pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
        got = pl.windows(to_dev(W, d)).cpu().numpy()
        ref = O.windows(g, prm, d)
        assert np.array_equal(got, ref.astype(np.int32))
        assert (got[:, 0] >= 0).sum() > 300


# ------------------------------------------------------------------ rasterize + scatter
@pytest.mark.parametrize("fluct", [0, 1])
def test_rasterize_grid_matches_oracle(W, fluct):
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct)
    pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
    pl.rasterize(to_dev(W, d), grid)
    ref = O.rasterize(g, prm, d)
    assert_close(grid.cpu().numpy(), ref, what="grid")
    # accumulation: a second call adds the same patches again
    pl.rasterize(to_dev(W, d), grid)
    assert_close(grid.cpu().numpy(), 2 * ref, what="grid x2")


def test_rasterize_edge_cases_match_oracle(W):
    import torch
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=512, pitch_mm=3.0)
    d = edge_case_depos(g, np.random.default_rng(32))
    for prm in (S.DriftParams(), S.DriftParams(fluctuate=1, seed=77, plane_id=3),
                S.DriftParams(nsigma=40.0, DT_cm2_s=30.0)):           # patches > 64 bins
        pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
        grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
        pl.rasterize(to_dev(W, d), grid)
        assert_close(grid.cpu().numpy(), O.rasterize(g, prm, d), what=str(prm))


def test_invalid_depos_are_flagged_and_skipped(W):
    import torch
    g = S.Geometry(n_wires=16, n_imp=10, n_ticks=256, pitch_mm=3.0)
    prm = S.DriftParams()
    d = S.make_workload("plane128-2k", n_depos=200).planes[0][3]
    d.p = d.p * (g.n_wires / 128.0)
    d.td = d.td * 0.2
    bad = d.subset(slice(None))
    bad.p[3] = np.nan
    bad.td[5] = -1.0
    bad.q[7] = -5.0
    bad.t[9] = np.inf
    pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
    pl.rasterize(to_dev(W, bad), grid)
    assert pl.check_flags() & 1
    assert pl.check_flags() == 0                 # cleared by the read
    good = d.subset(np.setdiff1d(np.arange(len(d)), [3, 5, 7, 9]))
    assert_close(grid.cpu().numpy(), O.rasterize(g, prm, good), what="skip invalid")


# ------------------------------------------------------------------ convolution
CONV_CASES = [
    # n_w, n_imp, n_t, n_fw, n_ft, hermitian response
    (128, 10, 1024, 128, 1024, True),
    (12, 3, 200, 14, 210, True),
    (7, 2, 30, 7, 30, False),
    (5, 1, 49, 5, 49, True),          # odd length 7^2
    (33, 4, 96, 35, 98, False),
    (1, 1, 64, 1, 64, True),          # single wire, single impact
    (3, 2, 13500, 3, 13500, True),    # longest supported time axis
    (960, 10, 16, 960, 16, True),     # many wires, short time axis (staged wire pass)
    (1200, 1, 32, 1200, 32, True),    # wire pass without staging, 4 columns per CTA
    (2400, 2, 16, 2400, 16, False),   # wire pass without staging, 1 column per CTA
    (8192, 1, 8, 8192, 8, True),      # widest supported wire axis
]


@pytest.mark.parametrize("case", CONV_CASES)
def test_convolve_matches_oracle(W, case):
    import torch
    n_w, n_imp, n_t, n_fw, n_ft, herm = case
    rng = np.random.default_rng(n_w * 7 + n_t)
    g = S.Geometry(n_wires=n_w, n_imp=n_imp, n_ticks=n_t, pitch_mm=3.0)
    grid = rng.normal(size=(g.n_rows, n_t)).astype(np.float32)
    grid[rng.uniform(size=grid.shape) < 0.7] = 0.0
    if herm:
        r = rng.normal(size=(n_imp, n_fw, n_ft))
        R = np.stack([np.fft.fft2(x) for x in r]).astype(np.complex64)
    else:
        R = (rng.normal(size=(n_imp, n_fw, n_ft)) + 1j * rng.normal(size=(n_imp, n_fw, n_ft))
             ).astype(np.complex64)
    pl = plane_for(W, g, S.DriftParams(), R)
    wave = pl.convolve(torch.from_numpy(grid).cuda())
    ref = O.convolve(g, R, grid.astype(np.float64))
    assert_close(wave.cpu().numpy(), ref, what=str(case))


@pytest.mark.parametrize("variant", [("", "", ""), ("staged", "", ""), ("", "block", ""),
                                     ("staged", "block", ""), ("", "", "0")])
def test_kernel_variants_match_oracle(W, variant, monkeypatch):
    """Every time-axis / wire-axis kernel variant on the 960 x 6000 plane (the time-axis
    kernels moving half spectra by TMA box copies, the default, and by per-thread loads and
    stores)."""
    import torch
    rows, wire, store = variant
    if rows:
        monkeypatch.setenv("WCSIM_ROWS_KERNEL", rows)
    if wire:
        monkeypatch.setenv("WCSIM_WIRE_KERNEL", wire)
    if store:
        monkeypatch.setenv("WCSIM_SPECTRA_TMA", store)
    rng = np.random.default_rng(41)
    g = S.Geometry(n_wires=960, n_imp=10, n_ticks=6000, pitch_mm=4.7)
    grid = np.zeros((g.n_rows, g.n_ticks), np.float32)
    idx = rng.integers(0, grid.size, 200000)
    grid.reshape(-1)[idx] = rng.normal(size=idx.size).astype(np.float32)
    R = S.make_response(g, "induction")
    pl = plane_for(W, g, S.DriftParams(), R)
    wave = pl.convolve(torch.from_numpy(grid).cuda()).cpu().numpy()
    assert_close(wave, O.convolve(g, R, grid.astype(np.float64)), what=str(variant))


def test_point_depo_gives_shifted_response(W):
    g = S.Geometry(n_wires=24, n_imp=10, n_ticks=256, pitch_mm=3.0)
    R = S.make_response(g, "induction")
    w0, j0, k0 = 7, 3, 201
    p = (w0 * g.n_imp + j0 + 0.37) * g.pitch_mm / g.n_imp
    t = (k0 + 0.81) * g.tick_us
    d = S.Depos(p=np.array([p]), t=np.array([t]), td=np.array([0.0]),
                q=np.array([3000.0], np.float32), id=np.zeros(1, np.uint32))
    pl = plane_for(W, g, S.DriftParams(), R)
    got = pl.run(to_dev(W, d)).cpu().numpy()
    rj = np.fft.ifft2(R[j0].astype(np.complex128)).real
    assert_close(got, 3000.0 * np.roll(np.roll(rj, w0, 0), k0, 1), what="point depo")


# ------------------------------------------------------------------ whole forward
@pytest.mark.parametrize("fluct", [0, 1])
def test_run_small_plane_matches_oracle(W, fluct):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    got = pl.run(to_dev(W, d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), what="plane128")


def test_run_padded_spectrum_matches_oracle(W):
    wl = S.make_workload("plane128-2k", n_depos=600)
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(g, kind, n_fw=150, n_ft=1200)
    pl = plane_for(W, g, prm, R)
    got = pl.run(to_dev(W, d)).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), what="padded")


def test_run_empty_depo_set_gives_zero_frame(W):
    g = S.Geometry(n_wires=16, n_imp=10, n_ticks=128, pitch_mm=3.0)
    pl = plane_for(W, g, S.DriftParams(), S.make_response(g))
    d = S.Depos(p=np.zeros(0), t=np.zeros(0), td=np.zeros(0), q=np.zeros(0, np.float32),
                id=np.zeros(0, np.uint32))
    import torch
    out = torch.full((g.n_wires, g.n_ticks), 7.0, device="cuda")
    pl.run(to_dev(W, d), out=out)
    assert (out.cpu().numpy() == 0).all()


@pytest.mark.parametrize("fluct", [1, 0])
def test_run_dune_plane_full_size_matches_oracle(W, fluct):
    """960 wires x 6000 ticks, 100,000 depos: the benchmark's launch configuration."""
    wl = S.make_workload("plane960-100k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    got = pl.run(to_dev(W, d)).cpu().numpy()
    ref = O.run(g, prm, R, d)
    rel, mx = assert_close(got, ref, what="plane960")
    print("plane960 fluct=%d rel L2 %.2e max/peak %.2e" % (fluct, rel, mx))
    assert pl.check_flags() == 0


def test_run_three_plane_event_matches_oracle(W):
    """The full event: 1,000,000 depos (200 tracks and 5000 short segments) projected on
    800 (U) + 800 (V) + 960 (W) wires x 6000 ticks, bipolar induction responses, fluctuation
    on.  The oracle fills bands of rows on all host threads (bit for bit its serial grid)."""
    wl = S.make_workload("event3p-1m")
    assert sum(len(d) for _, _, _, d in wl.planes) == 3 * 1000000
    for g, prm, kind, d in wl.planes:
        R = S.make_response(g, kind)
        pl = plane_for(W, g, prm, R)
        got = pl.run(to_dev(W, d)).cpu().numpy()
        rel, mx = assert_close(got, O.run(g, prm, R, d, threads=0), what="plane %d" % prm.plane_id)
        print("event3p-1m plane %d rel L2 %.2e max/peak %.2e" % (prm.plane_id, rel, mx))
        assert pl.check_flags() == 0
        pl.close()


def test_stage_timing_reports_every_stage(W):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    pl = plane_for(W, g, prm, S.make_response(g, kind))
    pl.set_timing(True)
    pl.run(to_dev(W, d))
    t = pl.stage_times()
    assert set(t) == {"prep", "rasterize", "rows_r2c", "wire_pass", "rows_c2r"}
    assert all(v >= 0 for v in t.values()) and sum(t.values()) > 0


def test_repeated_runs_leave_a_clean_grid(W):
    """wcsim_run clears its grid while transforming it; a backward pass leaves it dirty and
    the next run must reset it: every run of the same depos gives the same frame."""
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    pl = plane_for(W, g, prm, S.make_response(g, kind))
    dd = to_dev(W, d)
    ref = O.run(g, prm, S.make_response(g, kind), d)
    outs = [pl.run(dd).cpu().numpy() for _ in range(3)]
    pl.backward(dd, torch.ones((g.n_wires, g.n_ticks), device="cuda"))
    outs.append(pl.run(dd).cpu().numpy())
    for o in outs:
        assert_close(o, ref, what="repeat")


def test_copy_wait_timeout_is_reported_and_the_plane_recovers(W, monkeypatch):
    """Failure detection without a fault: with a wait limit of 0 the wire pass's waits for
    its bulk-copied response tiles run out (a copy issued just before is not complete yet),
    wcsim_plane_check reports WCSIM_ETIMEOUT, and with the normal limit restored the same
    plane gives the oracle's frame again (the context stays usable)."""
    monkeypatch.delenv("WCSIM_WIRE_KERNEL", raising=False)
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    dd = to_dev(W, d)
    ref = O.run(g, prm, R, d)
    assert pl.check_flags() == 0
    pl.set_wait_limit(0)
    pl.run(dd)
    with pytest.raises(W.WcsimError) as e:
        pl.check_flags()
    assert e.value.status == W.ETIMEOUT
    pl.set_wait_limit(2_000_000_000)
    got = pl.run(dd).cpu().numpy()
    assert pl.check_flags() == 0
    assert_close(got, ref, what="after a timed-out run")


def test_autotune_picks_variants_without_changing_results(W):
    wl = S.make_workload("plane960-100k", n_depos=20000)
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    dd = to_dev(W, d)
    rep = pl.autotune(dd)
    prod = 1
    for r in rep["time_radix"]:
        prod *= r
    assert prod == g.n_ticks and rep["depos_per_block"] in (32, 64, 128)
    assert rep["candidates_timed"] >= 6 and rep["ms_rows"] > 0
    got = pl.run(dd).cpu().numpy()
    assert_close(got, O.run(g, prm, R, d), what="after autotune %s" % rep)


RASTER_TILES = [(32, 8), (64, 8), (128, 8), (256, 8), (64, 16), (128, 16), (256, 16), (64, 32),
                (128, 32), (256, 32)]


@pytest.mark.parametrize("fluct", [0, 1, 2])
def test_every_rasterization_tile_matches_oracle(W, fluct):
    """Each tile (depos per CTA, lanes per depo) the autotuner may keep: the grid against
    the oracle's (the exact binomial's counts equal but at CDF steps, at most 1e-4 of the
    draws off by one), and the plain and batched rasterizers alike."""
    import torch
    g = S.Geometry(n_wires=64, n_imp=10, n_ticks=800, pitch_mm=3.0, p0_mm=-3.0, t0_us=-10.0)
    prm = S.DriftParams(fluctuate=fluct, seed=0x71E + fluct, DT_cm2_s=20.0)
    d = edge_case_depos(g, np.random.default_rng(7 + fluct), n=900)
    ref = O.rasterize(g, prm, d)
    pl = plane_for(W, g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    dd = to_dev(W, d)
    for kd, kg in RASTER_TILES:
        pl.set_raster_tile(kd, kg)
        grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
        pl.rasterize(dd, grid)
        got = grid.cpu().numpy()
        what = "tile %d x %d fluct %d" % (kd, kg, fluct)
        if fluct == 2:
            diff = got - ref
            assert np.abs(diff).max() <= 1 and np.count_nonzero(diff) <= max(2, 1e-4 * got.size), what
        else:
            assert_close(got, ref, what=what)
    with pytest.raises(W.WcsimError):
        pl.set_raster_tile(48, 8)
    pl.close()
