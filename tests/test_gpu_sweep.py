"""A seeded sweep of random planes through the C-ABI against the FP64 oracle (needs a GB300).

Each case draws a geometry (wires, impacts per pitch, ticks: sizes whose factors are 2, 3,
5 and 7, with ragged tails against every tile size; pitch, tick and origins), drift
parameters (speed, D_L, D_T, lifetime, n_sigma, fluctuation mode, renormalisation, seed,
plane id), a response kind and spectrum padding, and a few hundred depos on tracks that
cross the plane's borders; odd seeds take the fused forward.  The forward frame must match
the oracle at the forward's tolerance (relative L2 <= 1e-5, max |err| <= 1e-4 x peak), and
so must the depo and response gradients of the backward on every plane (one warp per time
frequency for n_fw = 32 M, the block-level adjoint otherwise), the three global gradients
to 1e-5 x the sum of their terms' magnitudes.
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


def smooth_sizes(lo, hi):
    out = []
    for a in range(0, 14):
        for b in range(0, 9):
            for c in range(0, 6):
                for e in range(0, 4):
                    n = 2 ** a * 3 ** b * 5 ** c * 7 ** e
                    if lo <= n <= hi:
                        out.append(n)
    return sorted(out)


def close(got, ref, what):
    got = np.asarray(got, np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref, got.dtype)
    nref = np.linalg.norm(ref)
    assert np.isfinite(got).all(), what
    assert np.linalg.norm(got - ref) <= REL_L2 * nref + 1e-30, what
    assert np.abs(got - ref).max(initial=0) <= MAX_PEAK * np.abs(ref).max(initial=0) + 1e-30, what


def draw_case(seed):
    rng = np.random.default_rng(1000 + seed)
    wires = smooth_sizes(1, 300)
    ticks = smooth_sizes(16, 3000)
    n_w = int(rng.choice(wires))
    if seed % 3 == 0:                                   # the one-warp wire kernels' sizes
        n_w = int(32 * rng.choice([4, 8, 15]))
    g = S.Geometry(n_wires=n_w, n_imp=int(rng.integers(1, 13)), n_ticks=int(rng.choice(ticks)),
                   pitch_mm=float(rng.uniform(2.0, 5.0)), p0_mm=float(rng.uniform(-50, 50)),
                   tick_us=float(rng.choice([0.5, 0.4, 1.0])), t0_us=float(rng.uniform(-100, 100)))
    fl = int(rng.integers(0, 3))
    prm = S.DriftParams(v_mm_per_us=float(rng.uniform(1.0, 2.0)), DL_cm2_s=float(rng.uniform(0, 10)),
                        DT_cm2_s=float(rng.uniform(0, 15)), lifetime_us=float(rng.uniform(2e3, 3e4)),
                        nsigma=float(rng.uniform(1.0, 4.0)), fluctuate=fl,
                        renormalize=int(rng.integers(0, 2)), seed=int(rng.integers(0, 2**40)),
                        plane_id=int(rng.integers(0, 3)))
    kind = str(rng.choice(["collection", "induction"]))
    pad = bool(rng.integers(0, 2)) and seed % 3 != 0
    span_p = g.n_wires * g.pitch_mm
    span_t = g.n_ticks * g.tick_us
    d = S.track_depos(rng, 3, int(rng.integers(50, 200)), span_p * 1.1, span_t * 0.7)
    d = dataclasses.replace(d, p=d.p + g.p0_mm - 0.05 * span_p, t=d.t + g.t0_us)
    return g, prm, kind, pad, d


@pytest.mark.parametrize("seed", range(24))
def test_random_plane_matches_oracle(W, seed):
    import torch
    g, prm, kind, pad, d = draw_case(seed)
    n_fw = n_ft = None
    if pad:
        sizes = smooth_sizes(g.n_wires, 2 * g.n_wires + 8)
        n_fw = sizes[0] if sizes[0] > g.n_wires else sizes[min(1, len(sizes) - 1)]
        n_ft = smooth_sizes(g.n_ticks + 1, 2 * g.n_ticks)[0]
    R = S.make_response(g, kind, n_fw=n_fw, n_ft=n_ft)
    pl = W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())
    pl.set_forward(seed % 2 == 1)                       # both forward variants
    dd = W.DeviceDepos.from_host(d)
    what = "seed %d: %s %s" % (seed, g, prm)
    M = pl.run(dd)
    assert pl.check_flags() == 0
    close(M.cpu().numpy(), O.run(g, prm, R, d), what + " forward")
    G = torch.from_numpy(np.random.default_rng(seed).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    got = pl.backward(dd, G, want_resp=True)
    mean = dataclasses.replace(prm, fluctuate=0)
    dS, dR = O.convolve_adjoint(g, R, O.rasterize(g, mean, d), G.cpu().numpy().astype(np.float64))
    ref = O.depo_grads(g, mean, d, dS)
    for k in ("q", "p", "t", "sigma_L", "sigma_T"):
        close(got[k].cpu().numpy(), ref[k], what + " d" + k)
    close(got["response"].cpu().numpy(), dR, what + " dR")
    assert_globals_close(got, ref, mean, d, what)
