"""The fit over events (paper_2104_08265_gb300.fit) with the library's backward, on one GPU
(needs a GB300).

A single process runs every event: the gradients of the summed loss with respect to D_L,
D_T, the lifetime and the response are the sums of the events' wcsim_run_backward
gradients, and must match the FP64 oracle's sums (the response per output at relative
L2 <= 1e-5 and max |err| <= 1e-4 x peak; the three globals to 1e-5 x the sum of their
per-depo terms' magnitudes over all events), for the dL/dM = M - T the library saw; a step
lowers the loss.
"""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as O
from paper_2104_08265_gb300 import synth as S

from gradcheck import TERM_REL, global_terms

pytestmark = pytest.mark.gpu


def test_single_process_fit_matches_the_oracle_sum_over_events():
    import torch
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import fit, wcsim
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    R = S.make_response(g, "collection")
    rng = np.random.default_rng(5)
    events = [S.track_depos(rng, 3, 200, g.n_wires * g.pitch_mm, 500.0) for _ in range(3)]
    truth = S.DriftParams(DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0, seed=40)
    targets = [O.run(g, truth, R, d) for d in events]
    base = S.DriftParams(seed=40)
    plane = wcsim.Plane(g, base, torch.from_numpy(R).cuda())
    fns = [fit.gpu_event_gradient(plane, wcsim.DeviceDepos.from_host(d),
                                  torch.from_numpy(t.astype(np.float32)).cuda())
           for d, t in zip(events, targets)]
    state = fit.FitState(DL=4.0, DT=8.8, lifetime=10000.0, response=torch.from_numpy(R).cuda())
    f = fit.ShardedFit(len(events), base, state, fns,
                       {"DL": 1e-7, "DT": 1e-7, "lifetime": 1e-5, "response": 1e-9})
    loss, grads = f.gradient()
    # the oracle's per-event gradients for the same dL/dM the library saw (the GPU frame less
    # the FP32 target), summed
    ref = {k: 0.0 for k in fit.GLOBALS}
    mag = {k: 0.0 for k in fit.GLOBALS}
    dR = np.zeros(R.shape, np.complex128)
    ref_loss, loss_bound = 0.0, 0.0
    for e, (d, t) in enumerate(zip(events, targets)):
        prm = dataclasses.replace(fit.event_params(base, e), DL_cm2_s=4.0, DT_cm2_s=8.8,
                                  lifetime_us=10000.0)
        plane.set_params(prm)
        M = plane.run(wcsim.DeviceDepos.from_host(d)).cpu().numpy()
        G = (M - t.astype(np.float32)).astype(np.float64)       # the FP32 difference the fit forms
        ref_loss += 0.5 * float((G * G).sum())
        # two runs of a frame differ in the order of the FP32 atomic sums: L = 1/2 |G|^2 moves
        # by about G . dG, |dG| <= 1e-5 |M| (the forward's tolerance)
        loss_bound += 2.0 * np.linalg.norm(G) * 1e-5 * np.linalg.norm(M)
        dS, dRe = O.convolve_adjoint(g, R, O.rasterize(g, prm, d), G)
        gr = O.depo_grads(g, prm, d, dS)
        terms = global_terms(prm, d, gr)
        for k in fit.GLOBALS:
            ref[k] += gr[k]
            mag[k] += float(np.abs(terms[k]).sum())
        dR += dRe
    assert abs(loss - ref_loss) <= loss_bound, (loss, ref_loss, loss_bound)
    for k in fit.GLOBALS:
        assert abs(grads[k] - ref[k]) <= TERM_REL * mag[k], (k, grads[k], ref[k])
    got = grads["response"].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - dR) <= 1e-5 * np.linalg.norm(dR)
    assert np.abs(got - dR).max() <= 1e-4 * np.abs(dR).max()
    loss0 = f.step()
    loss1, _ = f.gradient()
    assert loss1 < loss0
    plane.close()
