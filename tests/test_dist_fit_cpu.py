"""The fit over events sharded by rank, on two gloo ranks (CPU, no GPU).

The loss of a fit over many events is a sum over events, so its gradients with respect to
the global parameters (D_L, D_T, lifetime, the response spectrum) are sums of per-event
gradients: sharding events over ranks and all-reducing the per-rank sums must give exactly
the gradient a single process gets over all events.  On CPU the per-event backward is the
FP64 oracle's adjoint (Eq. 2's adjoint, then the per-depo chain rule), which stands in for
the library's wcsim_run_backward; the sharding, the seeding (event e keeps seed + e), the
packing and the all-reduce are the product's (paper_2104_08265_gb300.fit).
"""
import dataclasses
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_EVENTS = 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _events():
    """Five small events on one plane: seeded depos, targets from D_L = 6, D_T = 10 cm^2/s
    and a lifetime of 8 ms (fluctuation off)."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2104_08265_gb300 import synth as S
    g = S.Geometry(n_wires=12, n_imp=4, n_ticks=96, pitch_mm=3.0)
    R = S.make_response(g, "induction", span_wires=3, span_ticks=40)
    rng = np.random.default_rng(77)
    events = [S.track_depos(rng, 2, 15, g.n_wires * g.pitch_mm, 30.0) for _ in range(N_EVENTS)]
    truth = S.DriftParams(DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0, seed=100)
    targets = [O.run(g, truth, R, d) for d in events]
    return g, R, events, targets


def _oracle_grad(g, d, target):
    from oracle import oracle as O
    import torch

    def fn(state, prm_e):
        prm = dataclasses.replace(prm_e, DL_cm2_s=state.DL, DT_cm2_s=state.DT,
                                  lifetime_us=state.lifetime, fluctuate=0)
        R = state.response.numpy().astype(np.complex128)
        grid = O.rasterize(g, prm, d)
        G = O.convolve(g, R, grid) - target
        dS, dR = O.convolve_adjoint(g, R, grid, G)
        gr = O.depo_grads(g, prm, d, dS)
        return (0.5 * float((G * G).sum()),
                {"DL": gr["DL"], "DT": gr["DT"], "lifetime": gr["lifetime"],
                 "response": torch.from_numpy(dR.astype(np.complex64))})
    return fn


def _state(R):
    import torch
    from paper_2104_08265_gb300.fit import FitState
    return FitState(DL=4.0, DT=8.8, lifetime=10000.0,
                    response=torch.from_numpy(np.ascontiguousarray(R, np.complex64)))


LR = {"DL": 2e-6, "DT": 2e-6, "lifetime": 1e-3, "response": 1e-7}


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from paper_2104_08265_gb300 import fit
    from paper_2104_08265_gb300 import synth as S
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        g, R, events, targets = _events()
        mine = fit.shard(N_EVENTS, ws, rank)
        base = S.DriftParams(seed=100)
        f = fit.ShardedFit(N_EVENTS, base, _state(R),
                           [_oracle_grad(g, events[e], targets[e]) for e in mine], LR)
        loss, grads = f.gradient()
        seeds = [fit.event_params(base, e).seed for e in f.events]
        loss0 = f.step()
        loss1, _ = f.gradient()
        st = f.state
        q.put((rank, f.events, seeds, loss, {k: grads[k] for k in fit.GLOBALS},
               grads["response"].numpy(), loss0, loss1,
               (st.DL, st.DT, st.lifetime, st.response.numpy())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_gradient_of_the_whole_loss():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in procs:
            r = q.get(timeout=300)
            out[r[0]] = r[1:]
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    # the shards partition the events; each event keeps its own seed
    assert out[0][0] == [0, 2, 4] and out[1][0] == [1, 3]
    assert out[0][1] == [100, 102, 104] and out[1][1] == [101, 103]
    # single process over every event: the same loss and gradients
    sys.path.insert(0, ROOT)
    from paper_2104_08265_gb300 import fit
    from paper_2104_08265_gb300 import synth as S
    g, R, events, targets = _events()
    ref = fit.ShardedFit(N_EVENTS, S.DriftParams(seed=100), _state(R),
                         [_oracle_grad(g, events[e], targets[e]) for e in range(N_EVENTS)], LR)
    assert ref.world == 1 and ref.events == list(range(N_EVENTS))
    loss, grads = ref.gradient()
    for rank in (0, 1):
        _, _, l, gg, gr, loss0, loss1, st = out[rank]
        assert l == pytest.approx(loss, rel=1e-12)
        for k in fit.GLOBALS:
            assert gg[k] == pytest.approx(grads[k], rel=1e-12, abs=1e-300)
        dr = grads["response"].numpy()
        assert np.abs(gr - dr).max() <= 1e-6 * np.abs(dr).max()
        assert loss1 < loss0                          # the step lowered the loss
    # every rank applied the same update
    s0, s1 = out[0][-1], out[1][-1]
    assert s0[:3] == s1[:3]
    assert np.array_equal(s0[3], s1[3])
    ref.step()
    assert ref.state.DL == pytest.approx(s0[0], rel=1e-12)
    assert ref.state.lifetime == pytest.approx(s0[2], rel=1e-12)


def test_shard_is_a_partition():
    sys.path.insert(0, ROOT)
    from paper_2104_08265_gb300 import fit
    for n in (0, 1, 7, 64):
        for w in (1, 2, 3, 8):
            got = sorted(e for r in range(w) for e in fit.shard(n, w, r))
            assert got == list(range(n))
    with pytest.raises(ValueError):
        fit.shard(4, 2, 2)
