"""Exact binomial fluctuation (fluctuate = 2) through the C-ABI vs the FP64 oracle (needs a
GB300).

Each bin holds an integer count drawn by inversion of the Binomial(rint Q', mean / Q') CDF
at a 23-bit Philox uniform.  The kernel evaluates the CDF in FP32 (Loader's saddle-point
mass at the mode and the ratio recurrence) with p_b from its FP32 patch weights, the oracle
in FP64 from log-gamma, so the two pick the same count except where the uniform falls
within FP32 rounding of a CDF step; there they differ by one.  Counts are integers, so the
grid sums are exact and the grids are compared bin by bin: all equal but at most 1e-4 of
the draws (depo x bin), those by exactly one count, and each such bin must hold a draw of
the oracle whose uniform lies within FP32 rounding of the CDF step between the two counts:
    |u - F(x; N, p_b)| <= max over p' = p_b (1 +- 2^-20) of |F(x; N, p') - F(x; N, p_b)|
                          + 2^-21,
x the oracle's count (GPU one above) or x - 1 (GPU one below).  2^-20 bounds the relative
error of the kernel's p_b (a product of two FP32 bin masses, each a few ulp from its FP64
value: 16 ulp of FP32), and 2^-21 (4 ulp of 1) the kernel's FP32 sum of the mass function
(compensated and re-anchored).  The full-size plane (960 x 6000, 100k depos, the bench's
launch) is compared the same way on 48 sampled rows, which the oracle computes row by row.
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


def rasterize(W, g, prm, d):
    import torch
    pl = W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
    pl.rasterize(W.DeviceDepos.from_host(d), grid)
    assert pl.check_flags() == 0
    return grid.cpu().numpy().astype(np.float64)


def draws(g, prm, d):
    """Binomial draws a rasterization makes: the bins of every depo's window."""
    w = O.windows(g, prm, d)
    ok = w[:, 0] >= 0
    return int(((w[ok, 1] - w[ok, 0] + 1) * (w[ok, 3] - w[ok, 2] + 1)).sum())


P_REL = 2.0 ** -20      # relative error bound of the kernel's FP32 p_b
F_ABS = 2.0 ** -21      # error bound of the kernel's FP32 CDF sum


def _near_step(F, n, p, x, u):
    """Whether u lies within FP32 rounding (of p_b and of the CDF sum) of F(x; n, p)."""
    f = F(x, n, p)
    tol = max(abs(F(x, n, p * (1 + P_REL)) - f), abs(F(x, n, min(1.0, p * (1 - P_REL))) - f))
    return abs(u - f) <= tol + F_ABS


def assert_counts_match(got, ref, n_draws, what, g=None, prm=None, d=None, rows=None):
    """Integer counts equal bin by bin but for at most 1e-4 of the draws, each off by one at a
    CDF step of one of the bin's draws (checked through the oracle's terms of that bin when
    g, prm and d are given; rows maps the compared rows to grid rows)."""
    from scipy.stats import binom
    assert np.array_equal(got, np.round(got)), what
    diff = got - ref
    bad = np.count_nonzero(diff)
    assert np.abs(diff).max(initial=0) <= 1, what
    assert bad <= max(2, 1e-4 * n_draws), "%s: %d bins differ, %d draws" % (what, bad, n_draws)
    if g is None:
        return bad
    F = lambda x, n, p: float(binom.cdf(x, n, p))
    for i, k in np.argwhere(diff != 0):
        r = int(rows[i]) if rows is not None else int(i)
        t = O.bin_terms(g, prm, d, r, int(k))
        up = diff[i, k] > 0
        ok = False
        for n_e, p, u, x in zip(t["n_e"], t["p"], t["u"], t["val"]):
            if n_e < 0:
                continue
            step = x if up else x - 1            # the CDF step between the two counts
            if step >= 0 and _near_step(F, int(n_e), p, int(step), u):
                ok = True
                break
        assert ok, "%s: bin (%d, %d) differs by %+d, no draw at a CDF step: %s" % (
            what, r, k, diff[i, k], {kk: v.tolist() for kk, v in t.items()})
    return bad


@pytest.mark.parametrize("renorm", [0, 1])
def test_binomial_grid_matches_oracle(W, renorm):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=2, renormalize=renorm)
    got = rasterize(W, g, prm, d)
    ref = O.rasterize(g, prm, d)
    assert np.array_equal(ref, np.round(ref))
    assert_counts_match(got, ref, draws(g, prm, d), "plane128-2k renormalize %d" % renorm,
                        g, prm, d)
    # not the normal approximation, and not the mean
    assert not np.array_equal(got, rasterize(W, g, dataclasses.replace(prm, fluctuate=1), d))


def test_binomial_small_charges_and_edge_cases(W):
    """Depos of a few electrons (N of 0, 1, 2, ...), point depos, border depos."""
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=512, pitch_mm=3.0)
    rng = np.random.default_rng(71)
    n = 1500
    span_p, span_t = g.n_rows * g.pitch_mm / g.n_imp, g.n_ticks * g.tick_us
    td = rng.uniform(0.0, 0.5 * span_t, n)
    td[:100] = 0.0
    d = S.Depos(p=rng.uniform(-0.02 * span_p, 1.02 * span_p, n),
                t=rng.uniform(-0.02 * span_t, 0.45 * span_t, n), td=td,
                q=np.concatenate([rng.uniform(0.0, 4.0, 500), rng.lognormal(np.log(3000), 1.0, 1000)]).astype(np.float32),
                id=np.arange(n, dtype=np.uint32))
    prm = S.DriftParams(fluctuate=2, seed=77, plane_id=2)
    assert_counts_match(rasterize(W, g, prm, d), O.rasterize(g, prm, d), draws(g, prm, d),
                        "edge cases", g, prm, d)


def test_binomial_large_variance_bins_take_the_normal_approximation(W):
    """A depo of 3e6 electrons: bins with N p (1 - p) > 65536 follow the normal approximation
    (compared at the forward's tolerance), the rest are exact counts."""
    g = S.Geometry(n_wires=2, n_imp=10, n_ticks=32, pitch_mm=3.0)
    d = S.Depos(p=np.array([3.05]), t=np.array([-50.0]), td=np.array([60.0]),
                q=np.array([3.0e6], np.float32), id=np.array([0], np.uint32))
    prm = S.DriftParams(fluctuate=2, seed=4)
    got = rasterize(W, g, prm, d)
    ref = O.rasterize(g, prm, d)
    mean = O.rasterize(g, S.DriftParams(), d)
    qa = O.depo_weights(g, S.DriftParams(), 3.05, -50.0, 60.0, 3.0e6)[0]
    pb = mean / qa
    wide = round(qa) * pb * (1 - pb) > 65536
    assert wide.sum() >= 3
    assert np.abs(got[wide] - ref[wide]).max() <= MAX_PEAK * np.abs(ref).max()
    assert_counts_match(got[~wide], ref[~wide], draws(g, prm, d), "narrow bins")


def test_binomial_moments_over_seeds_on_the_gpu(W):
    """400 seeds of one depo: per-bin mean N p and variance N p (1 - p)."""
    import torch
    g = S.Geometry(n_wires=2, n_imp=10, n_ticks=32, pitch_mm=3.0)
    d = S.Depos(p=np.array([3.05]), t=np.array([-50.0]), td=np.array([60.0]),
                q=np.array([2000.0], np.float32), id=np.array([0], np.uint32))
    mean = O.rasterize(g, S.DriftParams(), d)
    qa = O.depo_weights(g, S.DriftParams(), 3.05, -50.0, 60.0, 2000.0)[0]
    n_e, pb = round(qa), mean / qa
    pl = W.Plane(g, S.DriftParams(fluctuate=2), np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    dd = W.DeviceDepos.from_host(d)
    grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
    n = 400
    acc = np.zeros_like(mean); acc2 = np.zeros_like(mean)
    for s in range(n):
        pl.set_params(S.DriftParams(fluctuate=2, seed=s))
        grid.zero_()
        pl.rasterize(dd, grid)
        x = grid.cpu().numpy().astype(np.float64)
        acc += x; acc2 += x * x
    m, v = acc / n, acc2 / n - (acc / n) ** 2
    var = n_e * pb * (1 - pb)
    big = mean > 5.0
    assert big.sum() >= 10
    assert np.abs((m[big] - n_e * pb[big]) / np.sqrt(var[big] / n)).max() < 4.5
    assert np.abs(v[big] / var[big] - 1).max() < 5.0 * np.sqrt(2 / n)


def test_binomial_forward_and_batch_match_oracle(W):
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=2)
    R = S.make_response(g, kind)
    pl = W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())
    got = pl.run(W.DeviceDepos.from_host(d)).cpu().numpy().astype(np.float64)
    ref = O.run(g, prm, R, d)
    err = np.linalg.norm(got - ref)
    assert err <= REL_L2 * np.linalg.norm(ref)
    assert np.abs(got - ref).max() <= MAX_PEAK * np.abs(ref).max()
    # a batch of three events: event e draws with seed + e
    rng = np.random.default_rng(9)
    events = [S.track_depos(rng, 2, 300, g.n_wires * g.pitch_mm, 0.75 * g.n_ticks * g.tick_us)
              for _ in range(3)]
    waves = [w.cpu().numpy() for w in W.Batch([pl] * 3, [W.DeviceDepos.from_host(e) for e in events]).run()]
    torch.cuda.synchronize()
    for e, de in enumerate(events):
        r = O.run(g, dataclasses.replace(prm, seed=prm.seed + e), R, de)
        assert np.linalg.norm(waves[e] - r) <= REL_L2 * np.linalg.norm(r), e


def test_fluctuate_out_of_range_is_rejected(W):
    g = S.Geometry(n_wires=8, n_imp=10, n_ticks=64, pitch_mm=3.0)
    with pytest.raises(W.WcsimError) as e:
        W.Plane(g, S.DriftParams(fluctuate=3), np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    assert e.value.status == W.EINVAL


def test_binomial_full_size_plane_bin_by_bin(W):
    """The 960 x 6000 plane with 100k depos, rasterized as the bench's forward does, against
    the oracle on 48 sampled rows (every bin of those rows): equal integer counts but at
    CDF steps, as above."""
    wl = S.make_workload("plane960-100k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=2)
    got = rasterize(W, g, prm, d)
    rows = np.sort(np.random.default_rng(2101).choice(g.n_rows, 48, replace=False))
    ref = O.rasterize_rows(g, prm, d, rows)
    w = O.windows(g, prm, d)
    ok = w[:, 0] >= 0
    in_rows = sum(((w[ok, 0] <= r) & (r <= w[ok, 1])) * (w[ok, 3] - w[ok, 2] + 1) for r in rows)
    n_draws = int(in_rows.sum())
    assert n_draws > 20000 and ref.sum() > 0
    assert_counts_match(got[rows], ref, n_draws, "full size", g, prm, d, rows)


def test_binomial_full_size_plane_properties(W):
    """The 960 x 6000 plane with 100k depos, as the bench times it: integer counts, zero
    outside the patches' windows, and a total within six standard deviations of the mean
    total (variance sum_b N p_b (1 - p_b) <= sum of the means; the oracle's FP64 mean grid)."""
    wl = S.make_workload("plane960-100k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=2)
    got = rasterize(W, g, prm, d)
    assert np.array_equal(got, np.round(got)) and got.min() >= 0
    mean = O.rasterize(g, dataclasses.replace(prm, fluctuate=0), d)
    assert np.all(got[mean == 0] == 0)
    mu = mean.sum()
    assert abs(got.sum() - mu) <= 6.0 * np.sqrt(mu) + 1e-4 * mu
    # and it is not the mean itself: per-bin deviations of the binomial's size
    live = mean > 50
    z = (got[live] - mean[live]) / np.sqrt(mean[live])
    assert 0.5 < z.std() < 1.1
