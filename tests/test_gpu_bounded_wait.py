"""The transform kernels' waits on TMA transfers are bounded: a kernel that
polls an mbarrier nothing completes must give up after its poll cap, raise
the timeout flag and leave the GPU usable (a box solve right after still
matches the oracle)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from oracle import boxsolve  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402


def test_capped_wait_times_out_and_context_survives():
    for polls in (16, 256):
        timed_out, ms = K.selftest_bounded_wait(polls)
        print(f"{polls} polls of an incomplete mbarrier: timed out {timed_out}, {ms:.3f} ms")
        assert timed_out
        assert ms < 5000.0
    geom, grid = G.sphere3(0.3, 4), C.Grid(3, 32)
    g = K.KFBI(geom, grid)
    r = np.random.default_rng(9).standard_normal(grid.shape)
    v = torch.empty(grid.shape, dtype=torch.float64, device="cuda:0")
    g.box_solve(torch.tensor(r, device="cuda:0"), v, 40.0)
    ref = boxsolve.solve(r, 40.0, grid)
    assert np.abs(v.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    g.close()
