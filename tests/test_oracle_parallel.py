"""The oracle's row-restricted, per-bin and multi-threaded rasterizations reproduce its plain
serial rasterization bit for bit (CPU only).

The serial rasterization (pinned in test_oracle_pins.py against closed forms, brute force and
library routines) adds every depo's patch in depo order.  The other forms are only other
loop orders over the same per-bin values: restricted to a set of rows, term by term for one
bin, or in bands of rows on several threads, each band in depo order.  So every bin must come
out identical, and every exact binomial term must be the draw og_binomial_draw makes from its
own trial count, p_b and uniform.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S


def _edge_depos(g, rng, n=700):
    """Point depos, border and off-grid depos, wide windows, zero charge."""
    span_p = g.n_rows * g.pitch_mm / g.n_imp
    span_t = g.n_ticks * g.tick_us
    p = rng.uniform(-0.05 * span_p, 1.05 * span_p, n)
    t = rng.uniform(-0.05 * span_t, 0.45 * span_t, n)
    td = rng.uniform(0.0, 0.6 * span_t, n)
    td[:50] = 0.0
    p[50:60] = [-1e9, 1e9] * 5
    q = rng.lognormal(np.log(6000), 0.5, n).astype(np.float32)
    q[60:70] = 0.0
    q[70:120] = rng.uniform(0.0, 5.0, 50).astype(np.float32)
    return S.Depos(p=p, t=t, td=td, q=q, id=rng.permutation(n).astype(np.uint32))


CASES = [(f, r) for f in (0, 1, 2) for r in (0, 1)]


@pytest.mark.parametrize("fluct,renorm", CASES)
@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_rasterization_is_the_serial_one_bit_for_bit(fluct, renorm, threads):
    wl = S.make_workload("plane128-2k")
    g, prm, _, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct, renormalize=renorm)
    assert np.array_equal(O.rasterize(g, prm, d, threads=threads), O.rasterize(g, prm, d))
    g2 = S.Geometry(n_wires=37, n_imp=7, n_ticks=300, pitch_mm=3.0, p0_mm=-2.0, t0_us=4.0)
    d2 = _edge_depos(g2, np.random.default_rng(fluct + 10 * renorm))
    prm2 = dataclasses.replace(prm, DT_cm2_s=40.0, nsigma=4.0)
    assert np.array_equal(O.rasterize(g2, prm2, d2, threads=threads), O.rasterize(g2, prm2, d2))


@pytest.mark.parametrize("fluct,renorm", CASES)
def test_row_restricted_rasterization_is_the_full_one_bit_for_bit(fluct, renorm):
    wl = S.make_workload("plane128-2k")
    g, prm, _, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct, renormalize=renorm)
    full = O.rasterize(g, prm, d)
    rows = np.random.default_rng(3).choice(g.n_rows, 40, replace=False)
    assert np.array_equal(O.rasterize_rows(g, prm, d, rows), full[rows])
    with pytest.raises(ValueError):
        O.rasterize_rows(g, prm, d, [1, 1])


@pytest.mark.parametrize("fluct", [0, 1, 2])
def test_bin_terms_sum_to_the_grid_and_repeat_their_draws(fluct):
    wl = S.make_workload("plane128-2k")
    g, prm, _, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct, seed=0xBEEF)
    grid = O.rasterize(g, prm, d)
    rng = np.random.default_rng(4)
    nz = np.argwhere(grid > 0)
    picks = nz[rng.choice(len(nz), 60, replace=False)]
    n_terms = 0
    for r, k in picks:
        t = O.bin_terms(g, prm, d, r, k)
        assert len(t["idx"]) >= 1
        acc = 0.0
        for v in t["val"]:
            acc += v                                  # the grid's order: depo order from 0
        assert acc == grid[r, k]
        for i, v, n_e, p, u in zip(t["idx"], t["val"], t["n_e"], t["p"], t["u"]):
            if fluct == 2 and n_e >= 0:
                assert u == O.bin_uniform(r, k, int(d.id[i]), prm.plane_id, prm.seed)
                assert v == O.binomial_draw(int(n_e), p, u)
                n_terms += 1
            else:
                assert n_e == -1.0
    if fluct == 2:
        assert n_terms > 100
    # a bin no window holds has no terms
    assert len(O.bin_terms(g, prm, d, 0, g.n_ticks - 1)["idx"]) == 0 or grid[0, -1] != 0
