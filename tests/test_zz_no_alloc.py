"""wcsim_convolve_noalloc against wcsim_convolve and the FP64 oracle (needs a GB300).

The no-allocation entry point serves callers that may not allocate device memory (code
running under an allocator it does not own, or a process that forbids allocation after
start-up); it keeps its scratch in a static device array shared by every call, and
wcsim_convolve_noalloc_check reads back the flag word of the last call.  This file is
collected last so that a run stopping at the first failure has already run every other test.
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


def _sparse_grid(g, rng, n):
    grid = np.zeros((g.n_rows, g.n_ticks), np.float32)
    idx = rng.integers(0, grid.size, n)
    grid.reshape(-1)[idx] = rng.normal(size=idx.size).astype(np.float32)
    return grid


# (wires, ticks, n_fw, n_ft): the one-warp wire pass (n_fw = 32 M); the block-level wire pass
# (n_fw = 100, not 32 M); a padded spectrum on both axes
CASES = [(128, 1024, 0, 0), (100, 1024, 0, 0), (120, 1000, 128, 1050)]


@pytest.mark.parametrize("n_wires,n_ticks,n_fw,n_ft", CASES)
def test_noalloc_matches_plane_convolve_and_oracle_on_two_calls_in_a_row(n_wires, n_ticks,
                                                                          n_fw, n_ft):
    import torch
    from oracle import oracle as O
    from paper_2104_08265_gb300 import _build
    _build.build()
    from paper_2104_08265_gb300 import wcsim
    g = S.Geometry(n_wires=n_wires, n_imp=10, n_ticks=n_ticks, pitch_mm=3.0)
    R_h = S.make_response(g, "induction", n_fw=n_fw or n_wires, n_ft=n_ft or n_ticks)
    R = torch.from_numpy(R_h).cuda()
    plane = wcsim.Plane(g, S.DriftParams(), R)
    rng = np.random.default_rng(71 + n_wires)
    for call in range(2):                     # different grids: no state may leak across calls
        grid = _sparse_grid(g, rng, 20000)
        gd = torch.from_numpy(grid).cuda()
        ref = plane.convolve(gd).cpu().numpy()
        out = torch.full((g.n_wires, g.n_ticks), float("nan"), device="cuda")
        got = wcsim.convolve_noalloc(g, R, gd, out=out, n_fw=n_fw, n_ft=n_ft)
        assert wcsim.convolve_noalloc_check() == 0
        got = got.cpu().numpy()
        assert np.isfinite(got).all()
        rel, peak = _rel_and_peak(got, ref)
        assert rel <= 1e-5 and peak <= 1e-4, (call, rel, peak)
        rel, peak = _rel_and_peak(got, O.convolve(g, R_h, grid))
        assert rel <= 1e-5 and peak <= 1e-4, ("oracle", call, rel, peak)
    plane.close()


def test_noalloc_allocates_no_device_memory():
    """After the first call (which looks up the static array's address), a call leaves the
    device's free memory unchanged."""
    import torch
    from paper_2104_08265_gb300 import wcsim
    g = S.Geometry(n_wires=128, n_imp=10, n_ticks=1024, pitch_mm=3.0)
    R = torch.from_numpy(S.make_response(g, "collection")).cuda()
    gd = torch.from_numpy(_sparse_grid(g, np.random.default_rng(5), 5000)).cuda()
    out = torch.empty((g.n_wires, g.n_ticks), device="cuda")
    wcsim.convolve_noalloc(g, R, gd, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    wcsim.convolve_noalloc(g, R, gd, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert wcsim.convolve_noalloc_check() == 0


def test_noalloc_rejects_frames_beyond_its_scratch():
    import torch
    from paper_2104_08265_gb300 import wcsim
    g = S.Geometry(n_wires=960, n_imp=10, n_ticks=6000, pitch_mm=4.7)
    R = torch.zeros((g.n_imp, g.n_wires, g.n_ticks), dtype=torch.complex64, device="cuda")
    grid = torch.zeros((g.n_rows, g.n_ticks), device="cuda")
    with pytest.raises(wcsim.WcsimError) as ei:
        wcsim.convolve_noalloc(g, R, grid)
    assert ei.value.status == wcsim.ESHAPE and "scratch" in str(ei.value)
