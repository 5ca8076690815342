"""wcsim_convolve_noalloc against wcsim_convolve (needs a GB300).

The no-allocation entry point serves callers that may not allocate device memory; it keeps
its scratch in a static device array shared by every call.  This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2104_08265_gb300 import synth as S

pytestmark = pytest.mark.gpu


def _rel_and_peak(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return (np.linalg.norm(got - ref) / np.linalg.norm(ref),
            np.abs(got - ref).max() / np.abs(ref).max())


def test_noalloc_matches_plane_convolve_on_two_calls_in_a_row():
    import torch
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import wcsim
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    R = torch.from_numpy(S.make_response(g, "induction")).cuda()
    plane = wcsim.Plane(g, S.DriftParams(), R)
    rng = np.random.default_rng(71)
    for call in range(2):                     # different grids: no state may leak across calls
        grid = np.zeros((g.n_rows, g.n_ticks), np.float32)
        idx = rng.integers(0, grid.size, 20000)
        grid.reshape(-1)[idx] = rng.normal(size=idx.size).astype(np.float32)
        gd = torch.from_numpy(grid).cuda()
        ref = plane.convolve(gd).cpu().numpy()
        out = torch.full((g.n_wires, g.n_ticks), float("nan"), device="cuda")
        got = wcsim.convolve_noalloc(g, R, gd, out=out).cpu().numpy()
        rel, peak = _rel_and_peak(got, ref)
        assert np.isfinite(got).all()
        assert rel <= 1e-5 and peak <= 1e-4, (call, rel, peak)
    plane.close()


def test_noalloc_rejects_frames_beyond_its_scratch():
    import torch
    from paper_2104_08265_gb300 import wcsim
    g = S.Geometry(n_wires=960, n_imp=10, n_ticks=6000, pitch_mm=4.7)
    R = torch.zeros((g.n_imp, g.n_wires, g.n_ticks), dtype=torch.complex64, device="cuda")
    grid = torch.zeros((g.n_rows, g.n_ticks), device="cuda")
    with pytest.raises(wcsim.WcsimError) as ei:
        wcsim.convolve_noalloc(g, R, grid)
    assert ei.value.status == wcsim.ESHAPE and "scratch" in str(ei.value)
