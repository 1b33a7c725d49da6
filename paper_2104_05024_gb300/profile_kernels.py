"""Launch the hot-path kernels of one workload a few times each, for ncu.

    python -m paper_2104_05024_gb300.profile_kernels [--N 256] [--precision fp64|mixed] [--reps 3] [--passes-only]
        [--box neumann] [--mesh] [--coupled]

Sets up the prolate-shell workload (configs 2/3 geometry), then runs each
transform pass of the box solver, one irregular-node correction and one
interface-limit gather `reps` times on the library's stream, and with
--strang one Strang step of the bidomain model (reactions, refinement
residuals, GMRES).  --box neumann runs `reps` float64 box solves of the
Neumann box (all (N+1)^3 nodes) instead; --mesh hands the shell over as a
bare triangle mesh, so the handle's creation runs the mesh setup kernels;
--coupled runs `reps` Strang steps of the anisotropic coupled system (the
paper's conductivities, Example 3's sphere) in the given precision with the
history projection.  No timing is reported: this only gives a profiler a short, representative
launch list.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    from kfbi_workloads import configs as C
    from paper_2104_05024_gb300 import kfbi as K

    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--strang", action="store_true")
    ap.add_argument("--passes-only", action="store_true", help="only the four transform passes (no A psi)")
    ap.add_argument("--box", default="dirichlet", choices=["dirichlet", "neumann"])
    ap.add_argument("--mesh", action="store_true", help="the shell as a bare triangle mesh")
    ap.add_argument("--coupled", action="store_true", help="coupled Strang steps on the sphere")
    a = ap.parse_args()
    if a.coupled:
        from kfbi_workloads import geometry as G
        geom, grid = G.sphere3(0.9, C.surface_res(a.N)), C.Grid(3, a.N)
        h = K.KFBI(geom, grid, D_i=(30.0, 5.0, 5.0), D_e=(20.0, 10.0, 10.0), dt=0.05, tol=1e-8,
                   precision=K.FP64 if a.precision == "fp64" else K.MIXED, warm=K.WARM_PROJECTION)
        dev = torch.device("cuda:0")
        V = torch.tensor(C.ball_stimulus(grid, (0.8, 0.0, 0.0), 0.1), device=dev)
        w = torch.zeros_like(V)
        h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=a.reps)
        torch.cuda.synchronize()
        print("ok")
        return
    prec = K.FP64 if a.precision == "fp64" else K.MIXED
    geom, grid, cfg, V0, w0 = C.config2(N=a.N, bc=a.box)
    if a.mesh:
        from kfbi_workloads import geometry as G
        geom = G.as_mesh(geom)
    h = K.KFBI(geom, grid, tol=cfg.tol)
    lam = h.info["lambda"]
    dev = torch.device("cuda:0")
    if a.box == "neumann":
        r = torch.ones(grid.shape, dtype=torch.float64, device=dev)
        v = torch.empty_like(r)
        for _ in range(a.reps):
            h.box_solve(r, v, lam, precision=K.FP64)
        torch.cuda.synchronize()
        print("ok")
        return
    psi = torch.ones(geom.M, dtype=torch.float64, device=dev)
    out = torch.empty(geom.M, dtype=torch.float64, device=dev)
    for _ in range(a.reps):
        for p in (0, 1, 2, 3):
            h.transform_pass(p, lam, prec)
        if not a.passes_only:
            h.apply_A(psi, out, lam, prec)
    if a.strang:
        V = torch.tensor(V0, device=dev)
        w = torch.tensor(w0, device=dev)
        h.bidomain_step(C.FHN_CONFIG, V, w, None, nsteps=1, precision=prec)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
