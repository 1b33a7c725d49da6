"""Checkpoint / resume of a Strang run through the C ABI: a run stopped after
k steps, saved to disk (state V, w plus the density history psi^n, psi^{n-1},
g^n that seeds the next GMRES solve), and resumed in a fresh handle must
repeat the uninterrupted run bit for bit on the deterministic paths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from kfbi_workloads import configs as C  # noqa: E402
from paper_2104_05024_gb300 import kfbi as K  # noqa: E402

DEV = "cuda:0"


def _cuda(a):
    return torch.tensor(a, dtype=torch.float64, device=DEV)


def _case(name):
    if name == "ellipse128":
        geom, grid, cfg, V0, w0 = C.config0()
    else:
        geom, grid, cfg, V0, w0 = C.config2(N=64, steps=4)
    return geom, grid, V0, w0


@pytest.mark.parametrize("name", ["ellipse128", "shell64"])
@pytest.mark.parametrize("precision,warm", [(K.FP64, K.WARM_PREVIOUS), (K.MIXED, K.WARM_PREVIOUS),
                                            (K.FP64, K.WARM_PROJECTION), (K.MIXED, K.WARM_PROJECTION)])
def test_resume_bit_identical(tmp_path, name, precision, warm):
    geom, grid, V0, w0 = _case(name)
    total, split = 12, 9     # the split falls after the history ring has wrapped
    kw = dict(sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-10, precision=precision, warm=warm)

    h = K.KFBI(geom, grid, **kw)
    Va, wa = _cuda(V0), _cuda(w0)
    h.bidomain_step(C.FHN_CONFIG, Va, wa, None, nsteps=total)
    h.close()

    h = K.KFBI(geom, grid, **kw)
    Vb, wb = _cuda(V0), _cuda(w0)
    h.bidomain_step(C.FHN_CONFIG, Vb, wb, None, nsteps=split)
    ck = h.checkpoint(Vb, wb)
    assert ck["n_solves"] == split
    h.close()
    path = tmp_path / "ck.npz"
    np.savez(path, **ck)

    h = K.KFBI(geom, grid, **kw)
    Vc, wc = h.restore(dict(np.load(path)), DEV)
    stats = h.bidomain_step(C.FHN_CONFIG, Vc, wc, None, nsteps=total - split)
    h.close()
    assert all(s["rel_res"] <= 1e-10 for s in stats)
    assert torch.equal(Vc, Va) and torch.equal(wc, wa)


def test_resume_without_history():
    """Dropping the history (n_solves = 0) restarts GMRES from a zero density:
    the same answer to the tolerance (the midpoint update makes successive
    densities alternate, so the previous density is no better a start than
    zero and the iteration counts stay close)."""
    geom, grid, V0, w0 = _case("ellipse128")
    kw = dict(sigma_i=1.0, sigma_e=2.0, dt=0.05, tol=1e-12, precision=K.FP64)
    h = K.KFBI(geom, grid, **kw)
    V, w = _cuda(V0), _cuda(w0)
    h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=2)
    ck = h.checkpoint(V, w)
    ref = h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=1)
    h.close()

    cold = dict(ck, n_solves=0)
    h = K.KFBI(geom, grid, **kw)
    V2, w2 = h.restore(cold, DEV)
    st = h.bidomain_step(C.FHN_CONFIG, V2, w2, None, nsteps=1)
    h.close()
    print(f"first resumed solve: {st[0]['iters']} iterations cold, {ref[0]['iters']} with the history")
    assert st[0]["rel_res"] <= 1e-12 and abs(st[0]["iters"] - ref[0]["iters"]) <= 5
    err = (V2 - V).abs().max().item() / V.abs().max().item()
    assert err < 1e-9
