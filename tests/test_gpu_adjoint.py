"""Adjoint (backward) CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

The oracle's adjoint is pinned on CPU (finite differences, dot-product identity, torch
autograd); here the GPU gradients must match it per output with relative L2 <= 1e-5 and
max |err| <= 1e-4 x peak.  The three global sums (dL/dD_L, dL/dD_T, dL/dtau) add up
terms of both signs over every depo: each is held to 1e-5 x the sum of its terms' magnitudes
(1e-5 per term, times the sum's condition number; see gradcheck.py).
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


def assert_close(got, ref, rel=REL_L2, peak=MAX_PEAK, what=""):
    got = np.asarray(got, np.complex128 if np.iscomplexobj(got) else np.float64)
    ref = np.asarray(ref, got.dtype)
    nref = np.linalg.norm(ref)
    err = np.linalg.norm(got - ref)
    mx = np.abs(got - ref).max()
    pk = np.abs(ref).max()
    assert np.isfinite(got).all(), what
    assert err <= rel * nref, "%s rel L2 %.3e" % (what, err / nref)
    assert mx <= peak * pk, "%s max/peak %.3e" % (what, mx / pk)
    return err / nref, mx / pk


def plane_for(W, g, prm, R):
    import torch
    return W.Plane(g, prm, torch.from_numpy(np.ascontiguousarray(R, np.complex64)).cuda())


@pytest.mark.parametrize("shape", [(128, 10, 1024, 128, 1024), (250, 4, 1000, 256, 1024),
                                   (960, 10, 6000, 960, 6000), (960, 10, 6000, 960, 6000, "0"),
                                   (33, 3, 13500, 64, 13500)])
def test_convolve_adjoint_matches_oracle(W, shape, monkeypatch):
    """The adjoint of Eq. 2 against the oracle's, the time-axis kernels moving half spectra
    by TMA box copies (the default) and, with a trailing "0", by per-thread loads and stores;
    the last shape takes the runtime 13500-point plan with an odd wire count."""
    import torch
    if len(shape) > 5:
        monkeypatch.setenv("WCSIM_SPECTRA_TMA", shape[5])
        shape = shape[:5]
    n_w, n_imp, n_t, n_fw, n_ft = shape
    rng = np.random.default_rng(n_w + n_t)
    g = S.Geometry(n_wires=n_w, n_imp=n_imp, n_ticks=n_t, pitch_mm=3.0)
    grid = np.zeros((g.n_rows, n_t), np.float32)
    idx = rng.integers(0, grid.size, grid.size // 20)
    grid.reshape(-1)[idx] = rng.normal(size=idx.size).astype(np.float32)
    G = rng.normal(size=(n_w, n_t)).astype(np.float32)
    R = S.make_response(g, "induction", n_fw=n_fw, n_ft=n_ft)
    pl = plane_for(W, g, S.DriftParams(), R)
    dS, dR = pl.convolve_adjoint(torch.from_numpy(G).cuda(), torch.from_numpy(grid).cuda(),
                                 want_resp=True)
    rdS, rdR = O.convolve_adjoint(g, R, grid.astype(np.float64), G.astype(np.float64))
    assert_close(dS.cpu().numpy(), rdS, what="dS %s" % (shape,))
    assert_close(dR.cpu().numpy(), rdR, what="dR %s" % (shape,))


def _grads_close(got, ref, what, prm, depos):
    for k in ("q", "p", "t", "sigma_L", "sigma_T"):
        assert_close(got[k].cpu().numpy(), ref[k], what="%s %s" % (what, k))
    assert_globals_close(got, ref, prm, depos, what)


def test_rasterize_adjoint_matches_oracle(W):
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0)
    rng = np.random.default_rng(81)
    dS = rng.normal(size=(g.n_rows, g.n_ticks)).astype(np.float32)
    pl = plane_for(W, g, prm, S.make_response(g, kind))
    got = pl.rasterize_adjoint(W.DeviceDepos.from_host(d), torch.from_numpy(dS).cuda())
    ref = O.depo_grads(g, prm, d, dS.astype(np.float64))
    _grads_close(got, ref, "rasterize_adjoint", prm, d)


def _oracle_backward(g, prm, R, d, G):
    mean = dataclasses.replace(prm, fluctuate=0)
    grid = O.rasterize(g, mean, d)
    dS, dR = O.convolve_adjoint(g, R, grid, G)
    return O.depo_grads(g, mean, d, dS), dR


@pytest.mark.parametrize("name", ["plane128-2k", "fit960-100k"])
def test_run_backward_matches_oracle(W, name):
    """Loss 1/2 |M - M_target|^2, target from D_L = 6, D_T = 10 cm^2/s, tau = 8 ms."""
    import torch
    wl = S.make_workload(name)
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0)
    R = S.make_response(g, kind)
    target = dataclasses.replace(prm, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0)
    pl = plane_for(W, g, target, R)
    dd = W.DeviceDepos.from_host(d)
    M_target = pl.run(dd).clone()
    pl.set_params(prm)
    M = pl.run(dd)
    G = (M - M_target).contiguous()
    got = pl.backward(dd, G, want_resp=True)
    ref, rdR = _oracle_backward(g, prm, R, d, G.cpu().numpy().astype(np.float64))
    _grads_close(got, ref, name, prm, d)
    assert_close(got["response"].cpu().numpy(), rdR, what=name + " dR")


def test_autograd_function_gradients_and_a_fit_step(W):
    """The autograd wrapper returns the library's gradients, and a gradient step on
    (D_L, D_T, tau) toward a target frame lowers the loss."""
    import torch
    from paper_2104_08265_gb300.autograd import simulate
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    R = torch.from_numpy(S.make_response(g, kind)).cuda()
    pl = W.Plane(g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    t64 = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    with torch.no_grad():
        target = simulate(pl, dd, t64(6.0), t64(10.0), t64(8000.0)).clone()
    DL, DT, tau = (t64(4.0).requires_grad_(), t64(8.8).requires_grad_(),
                   t64(10000.0).requires_grad_())
    q = dd.q.clone().requires_grad_()
    resp = R.clone().requires_grad_()
    wave = simulate(pl, W.DeviceDepos(dd.p, dd.t, dd.td, q, dd.id), DL, DT, tau, resp)
    loss = 0.5 * ((wave - target) ** 2).sum()
    loss.backward()
    ref = pl.backward(dd, (wave - target).detach().contiguous(), want_resp=True)
    # two backward runs differ only by the summation order of the atomic scatter-add
    for a, b in ((q.grad, ref["q"]), (resp.grad, ref["response"])):
        assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 1e-6
    for x, k in ((DL, "DL"), (DT, "DT"), (tau, "lifetime")):
        assert float(x.grad) == pytest.approx(float(ref[k]), rel=1e-5)
    # one small step along -grad lowers the loss
    with torch.no_grad():
        step = [DL, DT, tau]
        gnorm = sum(float(x.grad) ** 2 for x in step) ** 0.5
        scale = [4.0, 8.8, 10000.0]
        new = [x - 0.02 * s * x.grad / gnorm for x, s in zip(step, scale)]
        loss2 = 0.5 * ((simulate(pl, dd, *new) - target) ** 2).sum()
    assert float(loss2) < float(loss.detach())


@pytest.mark.parametrize("keep2d", [False, True])
def test_backward_reusing_the_forward_spectra_matches_oracle(W, keep2d):
    """set_reuse_forward: the backward after a mean-path run on the same depos takes the
    run's spectra (keep2d: and the 2D spectra of S its wire pass kept, from which dL/dR
    streams); gradients as the oracle's and as the recomputing backward's."""
    import torch
    wl = S.make_workload("fit960-100k")
    g, prm, kind, d = wl.planes[0]
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    G = torch.from_numpy(np.random.default_rng(91).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    plain = pl.backward(dd, G, want_resp=True)
    pl.set_reuse_forward(True, keep_wire_spectra=keep2d)
    pl.run(dd)
    got = pl.backward(dd, G, want_resp=True)
    ref, rdR = _oracle_backward(g, prm, R, d, G.cpu().numpy().astype(np.float64))
    _grads_close(got, ref, "reused spectra", prm, d)
    assert_close(got["response"].cpu().numpy(), rdR, what="reused spectra dR")
    for k in ("q", "p", "t", "sigma_L", "sigma_T", "response"):
        assert_close(got[k].cpu().numpy(), plain[k].cpu().numpy(), what="reuse vs recompute " + k)


def test_reuse_is_dropped_when_the_forward_does_not_apply(W):
    """Changed parameters, a fluctuating forward, another call in between, other depo arrays:
    each backward recomputes, and its gradients are the oracle's for its own inputs."""
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=8000.0)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    pl.set_reuse_forward(True)
    dd = W.DeviceDepos.from_host(d)
    G = torch.from_numpy(np.random.default_rng(92).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    Gh = G.cpu().numpy().astype(np.float64)
    other = dataclasses.replace(prm, DT_cm2_s=4.0)
    # 1. parameters changed after the run
    pl.run(dd)
    pl.set_params(other)
    _grads_close(pl.backward(dd, G), _oracle_backward(g, other, R, d, Gh)[0], "params changed",
                 other, d)
    # 2. a fluctuating forward: the backward stays on the mean path
    pl.set_params(dataclasses.replace(prm, fluctuate=1))
    pl.run(dd)
    _grads_close(pl.backward(dd, G), _oracle_backward(g, prm, R, d, Gh)[0], "fluctuating run",
                 prm, d)
    # 3. another compute call in between
    pl.set_params(prm)
    pl.run(dd)
    pl.convolve(torch.zeros((g.n_rows, g.n_ticks), dtype=torch.float32, device="cuda"))
    _grads_close(pl.backward(dd, G), _oracle_backward(g, prm, R, d, Gh)[0], "call in between",
                 prm, d)
    # 4. other depo arrays (a copy holding other values)
    d2 = dataclasses.replace(d, q=(d.q * 0.5).astype(np.float32))
    pl.run(dd)
    _grads_close(pl.backward(W.DeviceDepos.from_host(d2), G),
                 _oracle_backward(g, prm, R, d2, Gh)[0], "other depos", prm, d2)


def test_autograd_backward_uses_its_own_forward_parameters(W):
    """Two forwards on one plane with different (D_L, D_T, tau) and one loss over both: each
    backward runs with its own forward's parameters (autograd runs the second's first)."""
    import torch
    from paper_2104_08265_gb300.autograd import simulate
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0)
    R = torch.from_numpy(S.make_response(g, kind)).cuda()
    pl = W.Plane(g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    t64 = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda", requires_grad=True)
    sets = [(4.0, 8.8, 10000.0), (6.0, 10.0, 8000.0)]
    rng = np.random.default_rng(93)
    Gs = [torch.from_numpy(rng.normal(size=(g.n_wires, g.n_ticks)).astype(np.float32)).cuda()
          for _ in sets]
    leaves, loss = [], 0.0
    for (a, b, c), G in zip(sets, Gs):
        q = dd.q.clone().requires_grad_()
        x = [t64(a), t64(b), t64(c)]
        wave = simulate(pl, W.DeviceDepos(dd.p, dd.t, dd.td, q, dd.id), *x)
        loss = loss + (wave * G).sum()
        leaves.append((q, x))
    loss.backward()
    for ((a, b, c), G, (q, x)) in zip(sets, Gs, leaves):
        pl.set_params(dataclasses.replace(prm, DL_cm2_s=a, DT_cm2_s=b, lifetime_us=c))
        ref = pl.backward(dd, G)
        rel = float(torch.linalg.vector_norm(q.grad - ref["q"]) / torch.linalg.vector_norm(ref["q"]))
        assert rel < 1e-6, (a, b, c, rel)
        for xx, k in zip(x, ("DL", "DT", "lifetime")):
            assert float(xx.grad) == pytest.approx(float(ref[k]), rel=1e-5), (a, b, c, k)
    # with the plane's spectra reused, the same gradients
    pl.set_params(prm)
    pl.set_reuse_forward(True)
    q = dd.q.clone().requires_grad_()
    x = [t64(4.0), t64(8.8), t64(10000.0)]
    (simulate(pl, W.DeviceDepos(dd.p, dd.t, dd.td, q, dd.id), *x) * Gs[0]).sum().backward()
    q0, x0 = leaves[0]
    assert float(torch.linalg.vector_norm(q.grad - q0.grad) / torch.linalg.vector_norm(q0.grad)) < 1e-5
    for a_, b_ in zip(x, x0):
        assert float(a_.grad) == pytest.approx(float(b_.grad), rel=1e-4)


def test_autograd_drift_time_gradient_and_sigma_sink(W):
    """WcsimFn gives the drift time a gradient (dL/dt + dL/dsigma_L sigma_L / (2 t_d) +
    dL/dsigma_T sigma_T / (2 t_d) - dL/dQ Q / lifetime, the chain rule pinned on CPU against
    finite differences) and hands the per-depo sigma_L / sigma_T gradients out through its
    sink; both against the oracle's per-depo gradients."""
    import torch
    from paper_2104_08265_gb300.autograd import WcsimFn
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0, DL_cm2_s=6.0, DT_cm2_s=10.0, lifetime_us=800.0)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    td = dd.td.clone().requires_grad_(True)
    t64 = lambda x: torch.tensor(x, dtype=torch.float64, device="cuda")
    sink = {}
    M = WcsimFn.apply(pl, dd.q, dd.p, dd.t, td, dd.id, t64(6.0), t64(10.0), t64(800.0), None, sink)
    G = torch.from_numpy(np.random.default_rng(93).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    (M * G).sum().backward()
    dS, _ = O.convolve_adjoint(g, R, O.rasterize(g, prm, d), G.cpu().numpy().astype(np.float64))
    ref = O.depo_grads(g, prm, d, dS)
    tdh = np.asarray(d.td, np.float64)
    live = tdh > 0
    f_l = np.where(live, np.sqrt(2e-4 * 6.0 * np.where(live, tdh, 1)) / (2 * np.where(live, tdh, 1)), 0)
    f_t = np.where(live, np.sqrt(2e-4 * 10.0 * np.where(live, tdh, 1)) / (2 * np.where(live, tdh, 1)), 0)
    ref_td = (ref["t"] + ref["sigma_L"] * f_l + ref["sigma_T"] * f_t
              - ref["q"] * np.asarray(d.q, np.float64) / 800.0)
    assert_close(td.grad.cpu().numpy(), ref_td, what="dL/dt_d")
    assert_close(sink["sigma_L"].cpu().numpy(), ref["sigma_L"], what="sink sigma_L")
    assert_close(sink["sigma_T"].cpu().numpy(), ref["sigma_T"], what="sink sigma_T")
    pl.close()


def test_reuse_is_dropped_for_other_depos_at_the_same_addresses(W):
    """The forward's depo tensors are freed and a new depo set with other charges lands at
    the same addresses (the caching allocator reuses them): the backward of the new set must
    not take the first set's spectra."""
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    pl.set_reuse_forward(True)
    a = W.DeviceDepos.from_host(d)
    pl.run(a)
    ptrs = (a.p.data_ptr(), a.q.data_ptr())
    del a
    d2 = dataclasses.replace(d, q=(d.q * 0.25).astype(np.float32))
    b = W.DeviceDepos.from_host(d2)
    G = torch.from_numpy(np.random.default_rng(94).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    got = pl.backward(b, G)
    ref, _ = _oracle_backward(g, prm, R, d2, G.cpu().numpy().astype(np.float64))
    _grads_close(got, ref, "reallocated depos", prm, d2)
    print("same addresses reused:", ptrs == (b.p.data_ptr(), b.q.data_ptr()))
    pl.close()


@pytest.mark.parametrize("n_w,n_fw", [(128, 128), (20, 24)])
def test_kept_wire_spectra_across_runs_and_sizes(W, n_w, n_fw):
    """Mode 2 over repeated fit steps with changing parameters and response (each backward's
    dL/dR the oracle's for its own forward), a backward without dL/dR in between, and a wire
    axis the one-warp pass does not take (n_fw = 24: mode 2 acts as mode 1)."""
    import torch
    g = S.Geometry(n_wires=n_w, n_imp=10, n_ticks=1000, pitch_mm=3.0)
    prm = S.DriftParams(fluctuate=0)
    rng = np.random.default_rng(n_w + n_fw)
    d = S.track_depos(rng, 3, 400, g.n_wires * g.pitch_mm, 0.6 * g.n_ticks * g.tick_us)
    dd = W.DeviceDepos.from_host(d)
    R = S.make_response(g, "induction", n_fw=n_fw, n_ft=1024)
    pl = plane_for(W, g, prm, R)
    pl.set_reuse_forward(True, keep_wire_spectra=True)
    Gh = rng.normal(size=(g.n_wires, g.n_ticks))
    G = torch.from_numpy(Gh.astype(np.float32)).cuda()
    for step in range(3):
        prm_s = dataclasses.replace(prm, DT_cm2_s=prm.DT_cm2_s * (1.0 + 0.2 * step))
        R_s = (R * (1.0 + 0.1 * step)).astype(np.complex64)
        pl.set_params(prm_s)
        pl.set_response(torch.from_numpy(R_s).cuda())
        pl.run(dd)
        got = pl.backward(dd, G, want_resp=(step != 1))
        ref, rdR = _oracle_backward(g, prm_s, R_s, d, Gh)
        _grads_close(got, ref, "kept 2D spectra, step %d" % step, prm_s, d)
        if step != 1:
            assert_close(got["response"].cpu().numpy(), rdR, what="kept 2D spectra dR %d" % step)


def test_run_residual_matches_run_and_oracle(W):
    """wcsim_run_residual: M - T and L = 1/2 |M - T|^2 in one forward, against run() and
    the oracle's frame; then a backward from the residual, its dL/dR the oracle's."""
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    dd = W.DeviceDepos.from_host(d)
    T = torch.from_numpy(np.random.default_rng(95).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    M = pl.run(dd).clone()
    res, loss = pl.run_residual(dd, T)
    ref = O.run(g, prm, R, d) - T.cpu().numpy().astype(np.float64)
    assert_close(res.cpu().numpy(), ref, what="residual vs oracle")
    assert_close(res.cpu().numpy(), (M - T).cpu().numpy(), rel=1e-6, peak=1e-6,
                 what="residual vs run")
    r64 = res.double()
    assert float(loss) == pytest.approx(0.5 * float((r64 * r64).sum()), rel=1e-5)
    pl.set_reuse_forward(True, keep_wire_spectra=True)
    res, loss = pl.run_residual(dd, T, out=res, loss=loss)
    got = pl.backward(dd, res, want_resp=True)
    refg, rdR = _oracle_backward(g, prm, R, d, res.cpu().numpy().astype(np.float64))
    _grads_close(got, refg, "from the residual", prm, d)
    assert_close(got["response"].cpu().numpy(), rdR, what="from the residual dR")


@pytest.mark.parametrize("case", ["noise", "padded"])
def test_run_residual_with_noise_and_padded_spectra(W, case):
    """The residual of a plane with Eq. 1's noise (M includes it) and of padded spectra
    (n_ft > n_ticks, n_fw > n_wires: M is cropped before T is subtracted), against run()."""
    import torch
    g = S.Geometry(n_wires=40, n_imp=10, n_ticks=600, pitch_mm=3.0)
    prm = S.DriftParams(fluctuate=1, seed=11)
    rng = np.random.default_rng(96)
    d = S.track_depos(rng, 2, 300, g.n_wires * g.pitch_mm, 0.5 * g.n_ticks * g.tick_us)
    n_fw, n_ft = (64, 640) if case == "padded" else (None, None)
    R = S.make_response(g, "induction", n_fw=n_fw, n_ft=n_ft)
    pl = plane_for(W, g, prm, R)
    if case == "noise":
        nh = g.n_ticks // 2 + 1
        pl.set_noise(np.full(nh, 3.0, np.float32), seed=4321)
    dd = W.DeviceDepos.from_host(d)
    T = torch.from_numpy(rng.normal(size=(g.n_wires, g.n_ticks)).astype(np.float32)).cuda()
    M = pl.run(dd).clone()
    res, loss = pl.run_residual(dd, T)
    assert_close(res.cpu().numpy(), (M - T).cpu().numpy(), rel=1e-6, peak=1e-6, what=case)
    r64 = res.double()
    assert float(loss) == pytest.approx(0.5 * float((r64 * r64).sum()), rel=1e-5)


def test_kept_wire_spectra_after_the_fused_forward(W):
    """Mode 2 after the fused forward (rasterization inside the time-axis transform): the
    wire pass keeps the 2D spectra all the same, and dL/dR and the depo gradients are the
    oracle's."""
    import torch
    wl = S.make_workload("plane128-2k")
    g, prm, kind, d = wl.planes[0]
    prm = dataclasses.replace(prm, fluctuate=0)
    R = S.make_response(g, kind)
    pl = plane_for(W, g, prm, R)
    pl.set_forward(True)
    pl.set_reuse_forward(True, keep_wire_spectra=True)
    dd = W.DeviceDepos.from_host(d)
    T = torch.from_numpy(np.random.default_rng(97).normal(size=(g.n_wires, g.n_ticks))
                         .astype(np.float32)).cuda()
    res, loss = pl.run_residual(dd, T)
    got = pl.backward(dd, res, want_resp=True)
    ref, rdR = _oracle_backward(g, prm, R, d, res.cpu().numpy().astype(np.float64))
    _grads_close(got, ref, "fused forward, kept spectra", prm, d)
    assert_close(got["response"].cpu().numpy(), rdR, what="fused forward, kept spectra dR")


@pytest.mark.parametrize("split", ["1", "2", "4"])
def test_adjoint_impact_split_matches_oracle(W, split, monkeypatch):
    """The one-warp wire adjoint with the impacts of a frequency block split over 1, 2 and 4
    CTAs (WCSIM_ADJ_SPLIT; the automatic choice takes 3 on these planes): dL/dS and dL/dR
    against the oracle."""
    import torch
    monkeypatch.setenv("WCSIM_ADJ_SPLIT", split)
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    rng = np.random.default_rng(98)
    grid = np.zeros((g.n_rows, g.n_ticks), np.float32)
    idx = rng.integers(0, grid.size, grid.size // 20)
    grid.reshape(-1)[idx] = rng.normal(size=idx.size).astype(np.float32)
    G = rng.normal(size=(g.n_wires, g.n_ticks)).astype(np.float32)
    R = S.make_response(g, "induction")
    pl = plane_for(W, g, S.DriftParams(), R)
    dS, dR = pl.convolve_adjoint(torch.from_numpy(G).cuda(), torch.from_numpy(grid).cuda(),
                                 want_resp=True)
    rdS, rdR = O.convolve_adjoint(g, R, grid.astype(np.float64), G.astype(np.float64))
    assert_close(dS.cpu().numpy(), rdS, what="dS split %s" % split)
    assert_close(dR.cpu().numpy(), rdR, what="dR split %s" % split)
