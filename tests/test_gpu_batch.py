"""Batched multi-event runs (wcsim_batch_run) vs one wcsim_run per event, and vs the oracle
(needs a GB300).  Event e of a batch uses the fluctuation seed of its plane plus e."""
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


def rel(a, b):
    a = np.asarray(a, np.float64); b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max()


def small_batch(W):
    import torch
    rng = np.random.default_rng(91)
    specs = {"A": (S.Geometry(128, 10, 1024, 3.0), "collection"),   # warp wire pass (M = 4)
             "B": (S.Geometry(96, 10, 2000, 4.7), "induction"),     # no warp kernel for 96
             "C": (S.Geometry(480, 10, 960, 4.7), "collection")}    # M = 15
    prm = S.DriftParams(fluctuate=1, seed=0x5EED00AA)
    planes = {k: W.Plane(g, prm, torch.from_numpy(S.make_response(g, kind)).cuda())
              for k, (g, kind) in specs.items()}
    order = ["A", "B", "A", "C", "A", "B", "C"]
    events = []
    for k in order:
        g = specs[k][0]
        n = int(rng.integers(200, 3000))
        d = S.track_depos(rng, 3, -(-n // 3), g.n_wires * g.pitch_mm, 0.75 * g.n_ticks * g.tick_us)
        events.append((k, d))
    return specs, prm, planes, events


def test_batch_matches_individual_runs_and_oracle(W):
    specs, prm, planes, events = small_batch(W)
    dev = [W.DeviceDepos.from_host(d) for _, d in events]
    b = W.Batch([planes[k] for k, _ in events], dev)
    got = [w.cpu().numpy() for w in b.run()]
    for e, (k, d) in enumerate(events):
        pl = planes[k]
        pe = dataclasses.replace(prm, seed=prm.seed + e)
        pl.set_params(pe)
        ref = pl.run(dev[e]).cpu().numpy()
        r, m = rel(got[e], ref)
        assert r <= 1e-5 and m <= 1e-4, (e, k, r, m)
        pl.set_params(prm)
    # one event all the way to the FP64 oracle
    e, (k, d) = 3, events[3]
    g, kind = specs[k]
    ref = O.run(g, dataclasses.replace(prm, seed=prm.seed + e), S.make_response(g, kind), d)
    r, m = rel(got[e], ref)
    assert r <= 1e-5 and m <= 1e-4, (r, m)


def test_batch_replays_from_a_cuda_graph(W):
    import torch
    specs, prm, planes, events = small_batch(W)
    dev = [W.DeviceDepos.from_host(d) for _, d in events]
    b = W.Batch([planes[k] for k, _ in events], dev)
    eager = [w.clone() for w in b.run()]
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.run()
    for w in b.waves:
        w.fill_(float("nan"))
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, w in zip(eager, b.waves):
        r, m = rel(w.cpu().numpy(), a.cpu().numpy())
        assert r <= 1e-5 and m <= 1e-4


def test_batch_limits(W):
    import ctypes
    L = W.lib()
    assert L.wcsim_batch_run(W.MAX_BATCH + 1, None, None, None, None) == W.ESHAPE
    assert L.wcsim_batch_run(0, None, None, None, None) == W.OK


def test_batch_per_plane_rasterization_fallback_and_repeated_runs(W):
    """Planes with different rasterization tiles (or an exact-binomial plane among others)
    cannot share the one queued rasterization: each plane's events are rasterized in their
    own launch.  Repeated runs with other depos must start from clean grids (each grid is
    cleared as its transform reads it)."""
    specs, prm, planes, events = small_batch(W)
    planes["B"].set_raster_tile(128, 16)
    dev = [W.DeviceDepos.from_host(d) for _, d in events]
    b = W.Batch([planes[k] for k, _ in events], dev)
    for rep in range(3):
        got = [w.cpu().numpy() for w in b.run()]
        for e, (k, d) in enumerate(events):
            pl = planes[k]
            pl.set_params(dataclasses.replace(prm, seed=prm.seed + e))
            ref = pl.run(dev[e]).cpu().numpy()
            pl.set_params(prm)
            r, m = rel(got[e], ref)
            assert r <= 1e-5 and m <= 1e-4, (rep, e, k, r, m)
        # next round: other charges in place (same arrays, same batch)
        for dv in dev:
            dv.q.mul_(0.5)
    # an exact-binomial plane among normal-approximation ones
    g, kind = specs["C"]
    import torch
    binp = W.Plane(g, dataclasses.replace(prm, fluctuate=2),
                   torch.from_numpy(S.make_response(g, kind)).cuda())
    mixed = [planes["A"], binp, planes["A"]]
    dsets = [dev[0], dev[3], dev[2]]
    got = [w.cpu().numpy() for w in W.Batch(mixed, dsets).run()]
    for e, (pl, dv) in enumerate(zip(mixed, dsets)):
        p0 = pl.params
        pl.set_params(dataclasses.replace(p0, seed=p0.seed + e))
        ref = pl.run(dv).cpu().numpy()
        pl.set_params(p0)
        r, m = rel(got[e], ref)
        assert r <= 1e-5 and m <= 1e-4, ("mixed", e, r, m)
