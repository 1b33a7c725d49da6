"""The allocation-free box solve (kfbi_box_solve_noalloc) must give the same
result as the handle-based kfbi_box_solve, within the 1e-12 relative bound
the box-solve parity tests use, on two calls in a row (the static scratch
keeps the previous call's contents, so the second call checks that nothing
stale leaks into it).

It exists for callers that cannot allocate device memory -- code running
inside a memory pool or arena that owns the device's memory, or under a rule
that forbids allocation after start-up -- so it takes no handle and uses a
fixed static device array instead of a workspace.

Kept in a file of its own, collected last, so that a failure here does not
hide the other GPU tests in a run that stops at the first failure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from kfbi_workloads import configs as C, geometry as G  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("dim,N", [(3, 32), (3, 64), (2, 128), (2, 512)])
def test_noalloc_matches_handle_solve_twice(dim, N):
    geom = G.sphere3(0.45, 4) if dim == 3 else G.disk2(0.5, 64)
    grid = C.Grid(dim, N)
    h = K.KFBI(geom, grid)
    rng = np.random.default_rng(100 + N)
    for call, lam in enumerate((60.0, 3.5)):
        r = torch.tensor(rng.standard_normal(grid.shape), device=DEV)
        ref = torch.empty_like(r)
        out = torch.full_like(r, float("nan"))
        h.box_solve(r, ref, lam, precision=K.FP64)
        K.box_solve_noalloc(r, out, lam, dim, N)
        torch.cuda.synchronize()
        assert _rel(out, ref) < 1e-12, (call, _rel(out, ref))
    h.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    r = torch.zeros((127, 127, 127), dtype=torch.float64, device=DEV)
    with pytest.raises(K.KFBIError) as e:
        K.box_solve_noalloc(r, r, 1.0, 3, 128)
    assert e.value.code == K.ERR_ARG
