"""Python binding of the KFBI C ABI (include/kfbi.h): argument marshalling only.

Every numeric step runs in the CUDA kernels of libkfbi.so; this module only
converts torch CUDA tensors and numpy geometry arrays into the C structs and
pointers the library expects.  Importing it without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkfbi.so")

OK, ERR_ARG, ERR_GEOMETRY, ERR_NOT_CONVERGED, ERR_NAN, ERR_CUDA, ERR_OOM, ERR_NEWTON = range(8)
ELLIPSE2, ELLIPSOID3, STAR3, SHELL3, MESH3 = 1, 2, 3, 4, 5
FP64, MIXED, MIXED_LEARNED, FP32 = 0, 1, 2, 3
GMRES, RICHARDSON = 0, 1
WARM_PREVIOUS, WARM_PROJECTION = 0, 1
BOX_DIRICHLET, BOX_NEUMANN = 0, 1
HISTORY = 8
MAX_COMP = 4


class Geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("kind", C.c_int), ("params", C.c_double * 16), ("n_nodes", C.c_int),
                ("nodes", C.POINTER(C.c_double)), ("n_tri", C.c_int), ("tri", C.POINTER(C.c_int32)),
                ("cube_n", C.c_int), ("cube_t", C.POINTER(C.c_double)), ("n_comp", C.c_int),
                ("comp_map", C.c_int * MAX_COMP), ("comp_axes", (C.c_double * 3) * MAX_COMP),
                ("comp_vert_offset", C.c_int * MAX_COMP), ("comp_n_vert", C.c_int * MAX_COMP),
                ("comp_tri_offset", C.c_int * MAX_COMP)]


class GridStruct(C.Structure):
    _fields_ = [("dim", C.c_int), ("N", C.c_int), ("lo", C.c_double), ("hi", C.c_double), ("box", C.c_int)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("solver", C.c_int), ("tol", C.c_double), ("restart", C.c_int),
                ("max_iter", C.c_int), ("gamma", C.c_double), ("stream", C.c_void_p), ("warm", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("warmstart", C.c_int), ("rel_res", C.c_double),
                ("true_rel_res", C.c_double),
                ("init_rel_res", C.c_double), ("ms", C.c_double), ("react_ms", C.c_double),
                ("rhs_ms", C.c_double), ("warm_ms", C.c_double), ("solve_ms", C.c_double),
                ("assemble_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FHNStruct(C.Structure):
    _fields_ = [("H", C.c_double), ("theta", C.c_double), ("alpha", C.c_double), ("zeta", C.c_double),
                ("Cm", C.c_double), ("beta", C.c_double)]


class Info(C.Structure):
    _fields_ = [("M", C.c_int), ("n_irregular", C.c_int), ("n_crossings", C.c_int), ("n_inside", C.c_int),
                ("device_bytes", C.c_size_t), ("lambda", C.c_double), ("xy_fused", C.c_int)]


EXPORTS = [
    "kfbi_last_error", "kfbi_create", "kfbi_destroy", "kfbi_query", "kfbi_set_opts", "kfbi_solve_neumann",
    "bidomain_step", "kfbi_export_setup", "kfbi_box_solve", "kfbi_correction", "kfbi_interface_limit",
    "kfbi_apply_A", "kfbi_rhs_g", "kfbi_solve_bie", "kfbi_react_fe", "kfbi_react_be", "kfbi_export_tables",
    "kfbi_transform_pass", "kfbi_launch_count", "kfbi_box_solve_noalloc", "kfbi_mlp_num_params",
    "kfbi_mlp_create", "kfbi_mlp_destroy", "kfbi_mlp_get", "kfbi_mlp_forward", "kfbi_mlp_grad",
    "kfbi_mlp_train_step", "kfbi_set_warmstart", "kfbi_get_densities", "kfbi_set_densities",
    "kfbi_get_history", "kfbi_set_history", "kfbi_get_projection", "kfbi_bidomain_step_stim",
    "kfbi_selftest_bounded_wait", "kfbi_get_warm_guess", "kfbi_training_rows", "kfbi_mlp_fit_norm",
    "kfbi_mlp_layers", "kfbi_create_coupled", "kfbi_solve_coupled", "kfbi_box_solve_coupled",
    "kfbi_apply_A_coupled",
]


class MLP:
    """Device copy of the warm-start network (float32 masters, bf16 copies)."""

    def __init__(self, params, norm, max_batch):
        lib = load()
        self.params = np.ascontiguousarray(params, dtype=np.float32)
        self.norm = np.ascontiguousarray(norm, dtype=np.float32)   # the normalisation vector (host copy)
        if self.params.size != lib.kfbi_mlp_num_params() or self.norm.size != 20:
            raise ValueError("parameter or normalisation vector has the wrong size")
        h = C.c_void_p()
        _check(lib.kfbi_mlp_create(self.params.ctypes.data_as(C.POINTER(C.c_float)),
                                   self.norm.ctypes.data_as(C.POINTER(C.c_float)), int(max_batch), _stream(),
                                   C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().kfbi_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        out = np.empty(load().kfbi_mlp_num_params(), np.float32)
        _check(load().kfbi_mlp_get(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    @staticmethod
    def fit_norm(F, T):
        """Normalisation vector [mean[9], std[9], target mean, target std] of
        training rows F [n, 9] and raw targets T [n] (CUDA float32)."""
        out = np.empty(20, np.float32)
        _check(load().kfbi_mlp_fit_norm(_ptr(F, "float32"), _ptr(T, "float32"), F.shape[0], _stream(),
                                        out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def forward(self, F, o):
        _check(load().kfbi_mlp_forward(self._h, _ptr(F, "float32"), F.shape[0], _ptr(o, "float32")))

    def layers(self, F, T=None):
        """Hidden pre-activations z [4, B, 128], output o [B] and, with raw
        targets T, the deltas dL/dz of the hidden layers [4, B, 128] (order
        l = 3..0) and dL/do [B] of the training path (device float32)."""
        import torch
        B = F.shape[0]
        z = torch.empty((4, B, 128), dtype=torch.float32, device=F.device)
        o = torch.empty(B, dtype=torch.float32, device=F.device)
        d = torch.empty_like(z) if T is not None else None
        d4 = torch.empty_like(o) if T is not None else None
        _check(load().kfbi_mlp_layers(self._h, _ptr(F, "float32"), _ptr(T, "float32"), B, _ptr(z, "float32"),
                                      _ptr(o, "float32"), _ptr(d, "float32"), _ptr(d4, "float32")))
        return z, o, d, d4

    def grad(self, F, t):
        """Loss and gradient for raw features F [B, 9] and raw targets t [B]."""
        g = np.empty(load().kfbi_mlp_num_params(), np.float32)
        loss = C.c_float()
        _check(load().kfbi_mlp_grad(self._h, _ptr(F, "float32"), _ptr(t, "float32"), F.shape[0], C.byref(loss),
                                    g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def train_step(self, F, t, lr):
        loss = C.c_float()
        _check(load().kfbi_mlp_train_step(self._h, _ptr(F, "float32"), _ptr(t, "float32"), F.shape[0], lr,
                                          C.byref(loss)))
        return loss.value


def box_solve_noalloc(r, v, lam, dim, N, lo=-1.0, hi=1.0):
    """Box solve through the allocation-free entry point (static scratch)."""
    _check(load().kfbi_box_solve_noalloc(dim, N, lo, hi, lam, _ptr(r), _ptr(v), _stream()))


def selftest_bounded_wait(polls):
    """(timed_out, ms) of a capped wait on an mbarrier that never completes."""
    t, ms = C.c_int(), C.c_double()
    _check(load().kfbi_selftest_bounded_wait(int(polls), C.byref(t), C.byref(ms)))
    return bool(t.value), ms.value


def launch_count() -> int:
    return int(load().kfbi_launch_count())

_lib = None


def load(path: str = LIB_PATH):
    """Load libkfbi.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libkfbi.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.c_int
    lib.kfbi_last_error.restype = C.c_char_p
    lib.kfbi_create.argtypes = [C.POINTER(Geometry), C.POINTER(GridStruct), C.c_double, C.c_double, C.c_double,
                                C.POINTER(Opts), C.POINTER(vp)]
    lib.kfbi_destroy.argtypes = [vp]
    lib.kfbi_destroy.restype = None
    lib.kfbi_query.argtypes = [vp, C.POINTER(Info)]
    lib.kfbi_set_opts.argtypes = [vp, C.POINTER(Opts)]
    lib.kfbi_solve_neumann.argtypes = [vp, C.c_double, vp, vp, vp, vp, C.POINTER(Stats)]
    lib.bidomain_step.argtypes = [vp, C.POINTER(FHNStruct), vp, vp, vp, ip, C.POINTER(Stats)]
    lib.kfbi_export_setup.argtypes = [vp] + [vp] * 7
    lib.kfbi_export_tables.argtypes = [vp] + [vp] * 8
    lib.kfbi_box_solve.argtypes = [vp, ip, C.c_double, vp, vp]
    lib.kfbi_correction.argtypes = [vp, vp, vp]
    lib.kfbi_interface_limit.argtypes = [vp, vp, vp, vp]
    lib.kfbi_apply_A.argtypes = [vp, ip, C.c_double, vp, vp]
    lib.kfbi_rhs_g.argtypes = [vp, C.c_double, vp, vp, vp]
    lib.kfbi_solve_bie.argtypes = [vp, C.c_double, vp, vp, C.POINTER(Stats)]
    lib.kfbi_react_fe.argtypes = [C.POINTER(FHNStruct), C.c_double, vp, vp, C.c_int64, vp]
    lib.kfbi_react_be.argtypes = [C.POINTER(FHNStruct), C.c_double, vp, vp, C.c_int64, vp]
    lib.kfbi_transform_pass.argtypes = [vp, ip, ip, C.c_double]
    lib.kfbi_box_solve_noalloc.argtypes = [ip, ip, C.c_double, C.c_double, C.c_double, vp, vp, vp]
    fp = C.POINTER(C.c_float)
    lib.kfbi_mlp_num_params.argtypes = []
    lib.kfbi_mlp_create.argtypes = [fp, fp, ip, vp, C.POINTER(vp)]
    lib.kfbi_mlp_destroy.argtypes = [vp]
    lib.kfbi_mlp_destroy.restype = None
    lib.kfbi_mlp_get.argtypes = [vp, fp]
    lib.kfbi_mlp_forward.argtypes = [vp, vp, ip, vp]
    lib.kfbi_mlp_grad.argtypes = [vp, vp, vp, ip, fp, fp]
    lib.kfbi_mlp_train_step.argtypes = [vp, vp, vp, ip, C.c_float, fp]
    lib.kfbi_set_warmstart.argtypes = [vp, vp]
    lib.kfbi_get_densities.argtypes = [vp, vp, vp, vp]
    lib.kfbi_set_densities.argtypes = [vp, vp, vp, vp, ip]
    lib.kfbi_get_history.argtypes = [vp, vp, vp, C.POINTER(C.c_int)]
    lib.kfbi_set_history.argtypes = [vp, vp, vp, ip]
    lib.kfbi_get_projection.argtypes = [vp, vp, vp]
    lib.kfbi_bidomain_step_stim.argtypes = [vp, C.POINTER(FHNStruct), vp, vp, vp, vp, ip, C.POINTER(Stats)]
    lib.kfbi_selftest_bounded_wait.argtypes = [ip, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    lib.kfbi_get_warm_guess.argtypes = [vp, vp]
    lib.kfbi_training_rows.argtypes = [vp, vp, vp]
    lib.kfbi_mlp_fit_norm.argtypes = [vp, vp, ip, vp, fp]
    lib.kfbi_mlp_layers.argtypes = [vp, vp, vp, ip, vp, vp, vp, vp]
    lib.kfbi_create_coupled.argtypes = [C.POINTER(Geometry), C.POINTER(GridStruct), dp, dp, C.c_double,
                                        C.POINTER(Opts), C.POINTER(vp)]
    lib.kfbi_solve_coupled.argtypes = [vp, C.c_double, vp, vp, vp, vp, vp, vp, vp, C.POINTER(Stats)]
    lib.kfbi_box_solve_coupled.argtypes = [vp, C.c_double, vp, vp, vp, vp]
    lib.kfbi_apply_A_coupled.argtypes = [vp, C.c_double, vp, vp]
    for name in EXPORTS:
        if name not in ("kfbi_last_error", "kfbi_destroy", "kfbi_launch_count", "kfbi_mlp_destroy"):
            getattr(lib, name).restype = C.c_int
    lib.kfbi_launch_count.restype = C.c_int64
    lib.kfbi_launch_count.argtypes = []
    _lib = lib
    return lib


class KFBIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"KFBI error {code}: {msg}")
        self.code = code


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise KFBIError(rc, load().kfbi_last_error().decode())
    return rc


def _ptr(t, dtype_name="float64"):
    """Device pointer of a contiguous CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch." + dtype_name:
        raise ValueError(f"expected a contiguous CUDA {dtype_name} tensor, got {t.dtype} on {t.device}")
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def fhn_struct(p) -> FHNStruct:
    return FHNStruct(p.H, p.theta, p.alpha, p.zeta, p.Cm, p.beta)


class KFBI:
    """Handle over one geometry, grid and conductivity/time-step setting.

    geom: any object with dim, kind, params, nodes [M, dim] and, in 3-D, tri,
    cube_n, cube_t and components (map_type, axes, vert_offset, n_vert,
    tri_offset) -- e.g. kfbi_workloads.geometry.Geometry; kind MESH3 needs
    only nodes and tri (a closed, outward-wound triangle mesh).
    grid: dim, N, lo, hi and optionally bc ("dirichlet" or "neumann": the box
    condition; Neumann-box fields hold all (N+1)^dim nodes)."""

    def __init__(self, geom, grid, sigma_i=1.0, sigma_e=2.0, dt=0.05, precision=FP64, solver=GMRES, tol=1e-10,
                 restart=50, max_iter=500, gamma=0.8, lo=-1.0, hi=1.0, warm=WARM_PREVIOUS, D_i=None, D_e=None):
        """D_i, D_e (sequences of dim conductivities): the anisotropic coupled
        system (kfbi_create_coupled) instead of the isotropic decoupled one."""
        lib = load()
        self._keep = []
        g = Geometry()
        g.dim, g.kind = int(geom.dim), int(geom.kind)
        for i, v in enumerate(np.asarray(geom.params, dtype=np.float64)[:16]):
            g.params[i] = float(v)
        nodes = np.ascontiguousarray(geom.nodes, dtype=np.float64)
        self._keep.append(nodes)
        g.n_nodes = nodes.shape[0]
        g.nodes = nodes.ctypes.data_as(C.POINTER(C.c_double))
        if g.dim == 3:
            tri = np.ascontiguousarray(geom.tri, dtype=np.int32)
            self._keep.append(tri)
            g.n_tri = tri.shape[0]
            g.tri = tri.ctypes.data_as(C.POINTER(C.c_int32))
            if geom.cube_t is not None:         # cube-sphere tables (not for bare meshes)
                ct = np.ascontiguousarray(geom.cube_t, dtype=np.float64)
                self._keep.append(ct)
                g.cube_n = int(geom.cube_n)
                g.cube_t = ct.ctypes.data_as(C.POINTER(C.c_double))
            g.n_comp = len(geom.components)
            for c, comp in enumerate(geom.components):
                g.comp_map[c] = int(comp.map_type)
                for k in range(3):
                    g.comp_axes[c][k] = float(comp.axes[k])
                g.comp_vert_offset[c] = int(comp.vert_offset)
                g.comp_n_vert[c] = int(comp.n_vert)
                g.comp_tri_offset[c] = int(comp.tri_offset)
        else:
            g.n_comp = 1
        self.dim, self.N = int(grid.dim), int(grid.N)
        box = BOX_NEUMANN if getattr(grid, "bc", "dirichlet") == "neumann" else BOX_DIRICHLET
        gs = GridStruct(self.dim, self.N, float(getattr(grid, "lo", lo)), float(getattr(grid, "hi", hi)), box)
        self.opts = Opts(precision, solver, tol, restart, max_iter, gamma, _stream(), warm)
        h = C.c_void_p()
        self.coupled = D_i is not None
        if self.coupled:
            di = (C.c_double * 3)(*[float(x) for x in list(D_i)[:3]] + [1.0] * (3 - len(list(D_i)[:3])))
            de = (C.c_double * 3)(*[float(x) for x in list(D_e)[:3]] + [1.0] * (3 - len(list(D_e)[:3])))
            _check(lib.kfbi_create_coupled(C.byref(g), C.byref(gs), di, de, dt, C.byref(self.opts), C.byref(h)))
        else:
            _check(lib.kfbi_create(C.byref(g), C.byref(gs), sigma_i, sigma_e, dt, C.byref(self.opts), C.byref(h)))
        self._h = h
        self.M = g.n_nodes
        info = Info()
        _check(lib.kfbi_query(h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in info._fields_}

    # ------------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().kfbi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_opts(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, v)
        self.opts.stream = _stream()
        _check(load().kfbi_set_opts(self._h, C.byref(self.opts)))

    @property
    def grid_shape(self):
        return (self.N - 1,) * self.dim

    def export_setup(self):
        n1 = self.N - 1
        i = self.info
        inside = np.empty((n1,) * self.dim, dtype=np.uint8)
        irr = np.empty(i["n_irregular"], dtype=np.int32)
        ax = np.empty(i["n_crossings"], dtype=np.int32)
        lo = np.empty(i["n_crossings"], dtype=np.int32)
        z = np.empty(i["n_crossings"], dtype=np.float64)
        cen = np.empty((self.M, self.dim), dtype=np.int32)
        sg = np.empty((self.M, self.dim), dtype=np.int8)
        p = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
        _check(load().kfbi_export_setup(self._h, p(inside), p(irr), p(ax), p(lo), p(z), p(cen), p(sg)))
        return {"inside": inside.astype(bool), "irregular": irr, "axis": ax, "lo": lo, "z": z, "center": cen,
                "sign": sg}

    def export_tables(self):
        M, NI, P = self.M, self.info["n_crossings"], 6 if self.dim == 2 else 10
        out = {"node_wn": np.empty((M, P)), "node_cnt": np.empty(M, np.int32), "node_pid": np.empty((M, 17), np.int32),
               "node_w": np.empty((M, 17)), "cross_cnt": np.empty(NI, np.int32),
               "cross_pid": np.empty((NI, 16), np.int32), "cross_wlo": np.empty((NI, 16)),
               "cross_whi": np.empty((NI, 16))}
        p = lambda a: C.c_void_p(a.ctypes.data)  # noqa: E731
        _check(load().kfbi_export_tables(self._h, *[p(out[k]) for k in out]))
        return out

    def set_warmstart(self, mlp):
        self._warm = mlp
        _check(load().kfbi_set_warmstart(self._h, None if mlp is None else mlp._h))

    def get_densities(self, psi=None, psi_prev=None, g=None):
        self.set_opts()
        _check(load().kfbi_get_densities(self._h, _ptr(psi), _ptr(psi_prev), _ptr(g)))

    def set_densities(self, psi, psi_prev, g, n_solves):
        self.set_opts()
        _check(load().kfbi_set_densities(self._h, _ptr(psi), _ptr(psi_prev), _ptr(g), int(n_solves)))

    def get_history(self, psi_hist, g_hist):
        n = C.c_int()
        self.set_opts()
        _check(load().kfbi_get_history(self._h, _ptr(psi_hist), _ptr(g_hist), C.byref(n)))
        return n.value

    def set_history(self, psi_hist, g_hist, n_solves):
        self.set_opts()
        _check(load().kfbi_set_history(self._h, _ptr(psi_hist), _ptr(g_hist), int(n_solves)))

    def get_projection(self, psiF, rF):
        self.set_opts()
        _check(load().kfbi_get_projection(self._h, _ptr(psiF), _ptr(rF)))

    def get_warm_guess(self, psi0):
        self.set_opts()
        _check(load().kfbi_get_warm_guess(self._h, _ptr(psi0)))

    def training_rows(self, F, T):
        """Rows F [M, 9] and raw targets T [M] (CUDA float32) of the last step."""
        self.set_opts()
        _check(load().kfbi_training_rows(self._h, _ptr(F, "float32"), _ptr(T, "float32")))

    def checkpoint(self, V, w):
        """Host copy of everything a resumed run needs: the state (V, w) and
        the density history with its solve count (the caller stores it, e.g.
        with numpy.savez)."""
        import torch
        shape = (HISTORY, self.M)
        ph = torch.empty(shape, dtype=torch.float64, device=V.device)
        gh = torch.empty_like(ph)
        n = self.get_history(ph, gh)
        torch.cuda.synchronize(V.device)
        return {"V": V.cpu().numpy(), "w": w.cpu().numpy(), "psi_hist": ph.cpu().numpy(), "g_hist": gh.cpu().numpy(),
                "n_solves": n}

    def restore(self, ck, device):
        """Inverse of checkpoint(): returns (V, w) on the device."""
        import torch
        t = {k: torch.tensor(ck[k], dtype=torch.float64, device=device) for k in ("V", "w", "psi_hist", "g_hist")}
        self.set_history(t["psi_hist"], t["g_hist"], int(ck["n_solves"]))
        return t["V"], t["w"]

    def transform_pass(self, pass_id, lam=0.0, precision=FP64):
        _check(load().kfbi_transform_pass(self._h, precision, pass_id, lam))

    def box_solve(self, r, v, lam, precision=FP64):
        self.set_opts()
        _check(load().kfbi_box_solve(self._h, precision, lam, _ptr(r), _ptr(v)))

    def correction(self, psi, rhs):
        self.set_opts()
        _check(load().kfbi_correction(self._h, _ptr(psi), _ptr(rhs)))

    def interface_limit(self, v, psi, out):
        self.set_opts()
        _check(load().kfbi_interface_limit(self._h, _ptr(v), _ptr(psi), _ptr(out)))

    def apply_A(self, psi, out, lam, precision=FP64):
        self.set_opts()
        _check(load().kfbi_apply_A(self._h, precision, lam, _ptr(psi), _ptr(out)))

    def rhs_g(self, f, gN, g, lam):
        self.set_opts()
        _check(load().kfbi_rhs_g(self._h, lam, _ptr(f), _ptr(gN), _ptr(g)))

    def solve_coupled(self, fi, fe, gNi, gNe, phi_i, phi_e, psi, kappa, **opts):
        """The coupled Neumann problem (psi: 2M density pair, in/out)."""
        self.set_opts(**opts)
        st = Stats()
        _check(load().kfbi_solve_coupled(self._h, kappa, _ptr(fi), _ptr(fe), _ptr(gNi), _ptr(gNe), _ptr(phi_i),
                                         _ptr(phi_e), _ptr(psi), C.byref(st)), allow=(ERR_NOT_CONVERGED,))
        return st.as_dict()

    def box_solve_coupled(self, ri, re, vi, ve, kappa):
        self.set_opts()
        _check(load().kfbi_box_solve_coupled(self._h, kappa, _ptr(ri), _ptr(re), _ptr(vi), _ptr(ve)))

    def apply_A_coupled(self, psi, out, kappa):
        self.set_opts()
        _check(load().kfbi_apply_A_coupled(self._h, kappa, _ptr(psi), _ptr(out)))

    def solve_bie(self, g, psi, lam, **opts):
        self.set_opts(**opts)
        st = Stats()
        _check(load().kfbi_solve_bie(self._h, lam, _ptr(g), _ptr(psi), C.byref(st)), allow=(ERR_NOT_CONVERGED,))
        return st.as_dict()

    def solve_neumann(self, f, gN, u, psi, lam, **opts):
        self.set_opts(**opts)
        st = Stats()
        _check(load().kfbi_solve_neumann(self._h, lam, _ptr(f), _ptr(gN), _ptr(u), _ptr(psi), C.byref(st)),
               allow=(ERR_NOT_CONVERGED,))
        return st.as_dict()

    def bidomain_step(self, fhn, V, w, ue=None, nsteps=1, istim=None, log=None, **opts):
        """Strang steps; istim (device field) adds the virtual-electrode
        stimulus.  Returns one stats dict per step; log (a path or a text
        file) receives them as JSON lines, numbered across calls."""
        self.set_opts(**opts)
        stats = (Stats * max(1, nsteps))()
        if istim is None:
            _check(load().bidomain_step(self._h, C.byref(fhn_struct(fhn)), _ptr(V), _ptr(w), _ptr(ue), nsteps, stats),
                   allow=(ERR_NOT_CONVERGED,))
        else:
            _check(load().kfbi_bidomain_step_stim(self._h, C.byref(fhn_struct(fhn)), _ptr(istim), _ptr(V), _ptr(w),
                                                  _ptr(ue), nsteps, stats), allow=(ERR_NOT_CONVERGED,))
        out = [stats[i].as_dict() for i in range(nsteps)]
        first = getattr(self, "_steps_done", 0)
        self._steps_done = first + nsteps
        if log is not None:
            write_step_log(log, out, first)
        return out


def write_step_log(log, stats, first=0):
    """One JSON line per Strang step: GMRES iterations, outer refinements,
    the warm start kept, initial / final / true relative residuals, and the
    phase times (device, ms)."""
    import json
    lines = "".join(json.dumps(dict({"step": first + i + 1}, **st)) + "\n" for i, st in enumerate(stats))
    if hasattr(log, "write"):
        log.write(lines)
        log.flush()
    else:
        with open(log, "a") as f:
            f.write(lines)


def react_fe(fhn, k, V, w):
    _check(load().kfbi_react_fe(C.byref(fhn_struct(fhn)), k, _ptr(V), _ptr(w), V.numel(), _stream()))


def react_be(fhn, k, V, w):
    _check(load().kfbi_react_be(C.byref(fhn_struct(fhn)), k, _ptr(V), _ptr(w), V.numel(), _stream()))
