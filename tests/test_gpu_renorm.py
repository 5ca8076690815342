"""Renormalised patches (renormalize = 1) through the C-ABI vs the FP64 oracle (needs a GB300).

With renormalisation each axis' bin weights are divided by their sum over the truncated
window, so a patch carries Q' = Q exp(-t_d / tau) whatever the n-sigma cut removed.  The
kernels form the sum as the mass between the window's outer edges (the bin masses
telescope) and the gradients by the quotient rule; the oracle sums the bins in FP64.
Tolerances as for the forward and the adjoint: relative L2 <= 1e-5 and max |err| <= 1e-4 x
peak per output; the three global sums to 1e-5 x the sum of their terms' magnitudes
(gradcheck.py).
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S

from gradcheck import assert_globals_close

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
    got = np.asarray(got, np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref, got.dtype)
    nref = np.linalg.norm(ref)
    err = np.linalg.norm(got - ref)
    assert np.isfinite(got).all(), what
    assert err <= REL_L2 * nref, "%s rel L2 %.3e" % (what, err / nref)
    assert np.abs(got - ref).max() <= MAX_PEAK * np.abs(ref).max(), what


def plane(W, g, prm, R=None):
    import torch
    if R is None:
        return W.Plane(g, prm, np.zeros((g.n_imp, g.n_wires, g.n_ticks), np.complex64))
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())


def rasterize(W, pl, g, d):
    import torch
    grid = torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda")
    pl.rasterize(W.DeviceDepos.from_host(d), grid)
    return grid.cpu().numpy()


def border_depos(g, rng, n=800):
    """Depos near and across the grid's borders (windows clipped, means outside the grid),
    point depos (sigma = 0), and wide ones."""
    dp = g.pitch_mm / g.n_imp
    span_p, span_t = g.n_rows * dp, g.n_ticks * g.tick_us
    p = rng.uniform(-0.02 * span_p, 1.02 * span_p, n)
    td = rng.uniform(0.0, 0.5 * span_t, n)
    t = rng.uniform(-0.02 * span_t, 0.5 * span_t, n)
    p[:100] = rng.choice([-1.0, 1.0], 100) * rng.uniform(0, 2.0, 100) + rng.choice([0.0, span_p], 100)
    ta = rng.choice([0.0, span_t], 100) + rng.uniform(-2.0, 2.0, 100)
    t[100:200] = ta - td[100:200]
    td[200:260] = 0.0
    q = rng.lognormal(np.log(6000), 0.3, n).astype(np.float32)
    return S.Depos(p=p, t=t, td=td, q=q, id=np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("fluct", [0, 1])
def test_renormalised_grid_matches_oracle(W, fluct):
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=fluct, renormalize=1, nsigma=2.0)
    got = rasterize(W, plane(W, g, prm), g, d)
    ref = O.rasterize(g, prm, d)
    assert_close(got, ref, "renormalised grid (fluctuate %d)" % fluct)
    if not fluct:
        # the renormalised patches differ from the truncated ones (2-sigma windows of
        # whole bins lose a few per cent)
        plain = O.rasterize(g, dataclasses.replace(prm, renormalize=0), d)
        assert ref.sum() > 1.02 * plain.sum()


@pytest.mark.parametrize("nsigma", [1.0, 3.0, 40.0])
def test_renormalised_border_and_point_depos_match_oracle(W, nsigma):
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=512, pitch_mm=3.0)
    d = border_depos(g, np.random.default_rng(int(nsigma * 10)))
    prm = S.DriftParams(nsigma=nsigma, DT_cm2_s=30.0 if nsigma > 10 else 10.0, renormalize=1)
    got = rasterize(W, plane(W, g, prm), g, d)
    assert_close(got, O.rasterize(g, prm, d), "border depos, nsigma %g" % nsigma)


def test_renormalised_patches_inside_the_grid_carry_the_attenuated_charge(W):
    g = S.Geometry(n_wires=64, n_imp=10, n_ticks=2048, pitch_mm=3.0)
    prm = S.DriftParams(nsigma=1.5, renormalize=1)
    rng = np.random.default_rng(3)
    n = 500
    td = rng.uniform(10.0, 800.0, n)
    d = S.Depos(p=rng.uniform(20.0, 170.0, n), t=rng.uniform(10.0, 200.0, n), td=td,
                q=rng.uniform(1000.0, 9000.0, n).astype(np.float32),
                id=np.arange(n, dtype=np.uint32))
    win = O.windows(g, prm, d)
    inside = (win[:, 0] > 0) & (win[:, 1] < g.n_rows - 1) & (win[:, 2] > 0) & (win[:, 3] < g.n_ticks - 1)
    assert inside.all()
    qatt = d.q.astype(np.float64) * np.exp(-td / prm.lifetime_us)
    got = rasterize(W, plane(W, g, prm), g, d)
    assert got.sum(dtype=np.float64) == pytest.approx(qatt.sum(), rel=1e-5)


def _grads_close(got, ref, what, prm, depos):
    for k in ("q", "p", "t", "sigma_L", "sigma_T"):
        assert_close(got[k].cpu().numpy(), ref[k], "%s %s" % (what, k))
    assert_globals_close(got, ref, prm, depos, what)


def test_renormalised_rasterize_adjoint_matches_oracle(W):
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0,
                              nsigma=2.0, renormalize=1)
    dS = np.random.default_rng(82).normal(size=(g.n_rows, g.n_ticks)).astype(np.float32)
    pl = plane(W, g, prm, S.make_response(g, kind))
    got = pl.rasterize_adjoint(W.DeviceDepos.from_host(d), torch.from_numpy(dS).cuda())
    _grads_close(got, O.depo_grads(g, prm, d, dS.astype(np.float64)), "renormalised adjoint",
                 prm, d)


def test_renormalised_adjoint_on_border_depos_matches_oracle(W):
    import torch
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=512, pitch_mm=3.0)
    d = border_depos(g, np.random.default_rng(83))
    prm = S.DriftParams(DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0, renormalize=1)
    dS = np.random.default_rng(84).normal(size=(g.n_rows, g.n_ticks)).astype(np.float32)
    pl = plane(W, g, prm, S.make_response(g, "collection"))
    got = pl.rasterize_adjoint(W.DeviceDepos.from_host(d), torch.from_numpy(dS).cuda())
    _grads_close(got, O.depo_grads(g, prm, d, dS.astype(np.float64)), "border adjoint", prm, d)


@pytest.mark.parametrize("name", ["plane128-2k", "plane960-100k"])
def test_renormalised_run_and_backward_match_oracle(W, name):
    import torch
    wl = S.make_workload(name)
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0, renormalize=1)
    R = S.make_response(g, kind)
    pl = plane(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    M = pl.run(dd)
    ref = O.run(g, prm, R, d)
    assert_close(M.cpu().numpy(), ref, name + " forward")
    if name != "plane128-2k":
        return
    G = torch.from_numpy(np.random.default_rng(85).normal(size=ref.shape).astype(np.float32)).cuda()
    got = pl.backward(dd, G, want_resp=True)
    dS, dR = O.convolve_adjoint(g, R, O.rasterize(g, prm, d), G.cpu().numpy().astype(np.float64))
    _grads_close(got, O.depo_grads(g, prm, d, dS), name + " backward", prm, d)
    assert_close(got["response"].cpu().numpy(), dR, name + " dR")
