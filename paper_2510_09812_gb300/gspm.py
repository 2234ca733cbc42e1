"""Thin ctypes binding of ``libgspm.so`` (declared in ``include/gspm.h``).

Argument marshalling only: every step of the GSPM path runs in the library's CUDA kernels.
Arrays may be NumPy (host, float64) or CUDA torch tensors (device, float64, contiguous); the
binding passes ``GSPM_HOST`` or ``GSPM_DEVICE`` accordingly.  Importing this module fails loudly
when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgspm.so")

OK, EINVAL, EMESH, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ESTATE, ENUMERIC = range(9)
HOST, DEVICE = 0, 1
PREC_F64, PREC_MIXED = 0, 1
ORDER_NONE, ORDER_RCM, ORDER_AGGREGATE = 0, 1, 2
FLAG_HOST_ONLY, FLAG_ROW2_PRINTED, FLAG_NO_AUTOTUNE, FLAG_GRAPH, FLAG_PINNED_CG = 1, 2, 4, 8, 16
FLAG_RESOLVE_AT_MSTAR, FLAG_PLAIN_CG = 32, 64
(EXPORT_UNIQUE_OF_STORED, EXPORT_ROWPTR, EXPORT_COLS, EXPORT_PERM, EXPORT_NODE_MAGNETIC,
 EXPORT_LUMPED_MASS, EXPORT_AGGREGATES, EXPORT_COARSE_K_MS, EXPORT_COARSE_K_MECH,
 EXPORT_COARSE_INV_MS, EXPORT_COARSE_INV_MECH, EXPORT_COARSE_STORED_MS,
 EXPORT_COARSE_STORED_MECH) = range(13)
FIELD_M, FIELD_U, FIELD_DISP, FIELD_HD, FIELD_STRAIN, FIELD_H, FIELD_DISP_PREV = range(7)
X0_PREV, X0_ZERO, X0_EXTRAPOLATE, X0_LEARNED = range(4)
MPNN_PARAMS = 26051
MPNN_KEYS = [("W_in", (16, 64)), ("b_in", (64,)), ("W1", (128, 64)), ("b1", (64,)),
             ("W2", (128, 64)), ("b2", (64,)), ("W3", (128, 64)), ("b3", (64,)),
             ("W_out", (64, 3)), ("b_out", (3,))]
OP_K_MS, OP_A_EPS, OP_A_AEPS, OP_M, OP_K_MECH, OP_DIV, OP_GRAD = range(7)
KCLASS_NAMES = ["spmv_mech", "spmv_gs", "spmv_ms", "cg_vec", "cg_init", "rhs_ms", "pointwise",
                "learned", "grad_ms", "rhs_mech", "strain"]
KCLASS = {name: k for k, name in enumerate(KCLASS_NAMES)}
FIELD_NCOMP = {FIELD_M: 3, FIELD_U: 1, FIELD_DISP: 3, FIELD_HD: 3, FIELD_STRAIN: 6, FIELD_H: 3,
               FIELD_DISP_PREV: 3}

_dp = C.POINTER(C.c_double)


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("coords", _dp), ("n_tets", C.c_int64),
                ("tets", C.POINTER(C.c_int32)), ("elem_magnetic", C.POINTER(C.c_uint8)),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3), ("wrap_tol", C.c_double),
                ("nodes_per_elem", C.c_int32)]


class Material(C.Structure):
    _fields_ = [("Ms", C.c_double), ("A", C.c_double), ("K1", C.c_double),
                ("lambda100", C.c_double), ("lambda111", C.c_double), ("C11", C.c_double),
                ("C12", C.c_double), ("C44", C.c_double), ("Nd", C.c_double * 9),
                ("sigma_ext", C.c_double * 6), ("gamma0", C.c_double), ("mu0", C.c_double),
                ("l_d", C.c_double), ("R", C.c_double * 9)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("ordering", C.c_int), ("dt", C.c_double),
                ("alpha", C.c_double), ("rtol_gs", C.c_double), ("rtol_ms", C.c_double),
                ("rtol_mech", C.c_double), ("max_iter", C.c_int), ("flags", C.c_uint),
                ("coarse_nodes", C.c_int64),
                ("stream", C.c_void_p)]


class MeshInfo(C.Structure):
    _fields_ = [("n_stored", C.c_int64), ("n_unique", C.c_int64), ("n_tets", C.c_int64),
                ("n_magnetic_nodes", C.c_int64), ("n_magnetic_tets", C.c_int64),
                ("nnz", C.c_int64), ("sell_entries", C.c_int64), ("volume", C.c_double),
                ("volume_magnetic", C.c_double), ("eps", C.c_double), ("dtau", C.c_double),
                ("device_bytes", C.c_int64), ("n_segments", C.c_int), ("item_slices", C.c_int),
                ("spmv_schedule_block", C.c_int),
                ("spmv_schedule_scalar", C.c_int), ("spmv_ms_block", C.c_double * 4),
                ("spmv_ms_scalar", C.c_double * 4), ("n_aggregates", C.c_int64),
                ("coarse_shift_ms", C.c_double), ("coarse_shift_mech", C.c_double),
                ("spmv_schedule_gs", C.c_int), ("spmv_ms_gs", C.c_double * 4)]


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("it_ms", C.c_int64), ("it_mech", C.c_int64),
                ("it_gs", C.c_int64), ("it_ms_last", C.c_int), ("it_mech_last", C.c_int),
                ("it_gs_last", C.c_int * 8), ("res_ms_last", C.c_double),
                ("res_mech_last", C.c_double), ("dm_last", C.c_double),
                ("m_bar", C.c_double * 3), ("noconv", C.c_int),
                ("true_res_ms_last", C.c_double), ("true_res_mech_last", C.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libgspm.so is not built ({_LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(_LIB_PATH)
    vp = C.c_void_p
    sig = {
        "gspm_mesh_load": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(Material),
                                     C.POINTER(Options), C.POINTER(vp)]),
        "gspm_destroy": (None, [vp]),
        "gspm_last_error": (C.c_char_p, []),
        "gspm_mesh_info_get": (C.c_int, [vp, C.POINTER(MeshInfo)]),
        "gspm_mesh_export": (C.c_int, [vp, C.c_int, vp, C.c_int64]),
        "gspm_set_field": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "gspm_get_field": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "gspm_step": (C.c_int, [vp, C.c_int, _dp, vp]),
        "gspm_solve_elastic": (C.c_int, [vp, vp, vp, C.c_int, C.c_int, vp, C.c_double,
                                         C.POINTER(C.c_int), _dp]),
        "gspm_volume_avg": (C.c_int, [vp, vp, C.c_int, C.c_int, _dp]),
        "gspm_apply": (C.c_int, [vp, C.c_int, vp, vp, C.c_int]),
        "gspm_launch_count": (C.c_int64, [vp]),
        "gspm_profile_enable": (C.c_int, [vp, C.c_uint]),
        "gspm_profile_read": (C.c_int, [vp, C.c_int, _dp, C.POINTER(C.c_int64)]),
        "gspm_volume_avg_noalloc": (C.c_int, [vp, vp, C.c_int64, C.c_int, vp, vp]),
        "gspm_set_x0_mode": (C.c_int, [vp, C.c_int]),
        "gspm_set_graph": (C.c_int, [vp, C.c_int]),
        "gspm_set_true_residual": (C.c_int, [vp, C.c_int]),
        "gspm_set_rtol": (C.c_int, [vp, C.c_double, C.c_double, C.c_double]),
        "gspm_coarse_round": (C.c_int, [_dp, C.c_int64, C.c_int, _dp, _dp]),
        "gspm_batch_load": (C.c_int, [C.POINTER(MeshDesc), C.c_int, C.POINTER(Material),
                                      C.POINTER(Options), C.POINTER(vp)]),
        "gspm_batch_segment": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64)]),
        "gspm_batch_step": (C.c_int, [vp, C.c_int, _dp, vp]),
        "gspm_mpnn_set_params": (C.c_int, [vp, C.POINTER(C.c_float), C.c_int64]),
        "gspm_mpnn_get_params": (C.c_int, [vp, C.POINTER(C.c_float), C.c_int64]),
        "gspm_mpnn_predict": (C.c_int, [vp, vp, vp, vp, vp, C.c_int, C.c_int]),
        "gspm_mpnn_dataset_reserve": (C.c_int, [vp, C.c_int]),
        "gspm_mpnn_dataset_add": (C.c_int, [vp, vp, vp, vp, vp, C.c_int, C.POINTER(C.c_int)]),
        "gspm_mpnn_loss_grad": (C.c_int, [vp, C.c_int, _dp, C.POINTER(C.c_float)]),
        "gspm_mpnn_train": (C.c_int, [vp, C.c_int, C.c_double, C.c_uint64, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class GSPMError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: status {code}: {lib.gspm_last_error().decode()}")


def _check(code, where, allow=()):
    if code != OK and code not in allow:
        raise GSPMError(code, where)
    return code


def _is_device(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _ptr(a, nvals=None):
    """(pointer, where, keepalive) for a float64 NumPy array or CUDA torch tensor."""
    if _is_device(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("device arrays must be contiguous float64 tensors")
        if nvals is not None and a.numel() != nvals:
            raise ValueError(f"expected {nvals} values, got {a.numel()}")
        return C.c_void_p(a.data_ptr()), DEVICE, a
    if hasattr(a, "data_ptr"):                       # CPU torch tensor (pinned or not)
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("host tensors must be contiguous float64")
        if nvals is not None and a.numel() != nvals:
            raise ValueError(f"expected {nvals} values, got {a.numel()}")
        return C.c_void_p(a.data_ptr()), HOST, a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if nvals is not None and arr.size != nvals:
        raise ValueError(f"expected {nvals} values, got {arr.size}")
    return C.c_void_p(arr.ctypes.data), HOST, arr


def material_struct(mat: dict) -> Material:
    m = Material()
    for k in ("Ms", "A", "K1", "lambda100", "lambda111", "C11", "C12", "C44"):
        setattr(m, k, float(mat[k]))
    m.Nd[:] = [float(v) for v in mat.get("Nd", [1 / 3, 0, 0, 0, 1 / 3, 0, 0, 0, 1 / 3])]
    m.sigma_ext[:] = [float(v) for v in mat.get("sigma_ext", [0.0] * 6)]
    m.gamma0 = float(mat.get("gamma0", 0.0))
    m.mu0 = float(mat.get("mu0", 0.0))
    m.l_d = float(mat.get("l_d", 0.0))
    m.R[:] = [float(v) for v in np.asarray(mat.get("R", np.zeros(9)), dtype=np.float64).reshape(-1)]
    return m


class Context:
    """One mesh + material + time step on the current CUDA device (``gspm_mesh_load``)."""

    def __init__(self, mesh, material: dict, dt: float, alpha: float, precision: str = "f64",
                 ordering: str = "auto", rtol_gs=1e-7, rtol_ms=1e-7, rtol_mech=1e-7,
                 max_iter=20000, row2_printed=False, host_only=False, stream=0, wrap_tol=0.0,
                 autotune=True, graph=False, pinned_cg=False, resolve_at_mstar=False,
                 plain_cg=False, coarse_nodes=0):
        """One mesh, or a batch when `mesh` is a list (gspm_batch_load).  ordering "auto":
        "aggregate" when the two-level preconditioner is on (neither plain_cg nor pinned_cg),
        which lets its restriction run fused with the CG update, else "none"."""
        if ordering == "auto":
            ordering = "none" if (plain_cg or pinned_cg) else "aggregate"
        meshes = list(mesh) if isinstance(mesh, (list, tuple)) else [mesh]
        keep = []
        descs = (MeshDesc * len(meshes))()
        for d, me in zip(descs, meshes):
            coords = np.ascontiguousarray(me.coords, dtype=np.float64)
            tets = np.ascontiguousarray(me.tets, dtype=np.int32)
            emag = np.ascontiguousarray(me.elem_magnetic, dtype=np.uint8)
            keep += [coords, tets, emag]
            d.n_nodes = coords.shape[0]
            d.coords = coords.ctypes.data_as(_dp)
            d.n_tets = tets.shape[0]
            d.tets = tets.ctypes.data_as(C.POINTER(C.c_int32))
            d.elem_magnetic = emag.ctypes.data_as(C.POINTER(C.c_uint8))
            d.box_lo[:] = [float(v) for v in me.box_lo]
            d.box_hi[:] = [float(v) for v in me.box_hi]
            d.wrap_tol = float(wrap_tol)
            d.nodes_per_elem = int(tets.shape[1])
        o = Options()
        o.precision = {"f64": PREC_F64, "mixed": PREC_MIXED}[precision]
        o.ordering = {"none": ORDER_NONE, "rcm": ORDER_RCM, "aggregate": ORDER_AGGREGATE}[ordering]
        o.dt, o.alpha = float(dt), float(alpha)
        o.rtol_gs, o.rtol_ms, o.rtol_mech = float(rtol_gs), float(rtol_ms), float(rtol_mech)
        o.max_iter = int(max_iter)
        o.flags = ((FLAG_ROW2_PRINTED if row2_printed else 0) | (FLAG_HOST_ONLY if host_only else 0)
                   | (0 if autotune else FLAG_NO_AUTOTUNE) | (FLAG_GRAPH if graph else 0)
                   | (FLAG_PINNED_CG if pinned_cg else 0)
                   | (FLAG_RESOLVE_AT_MSTAR if resolve_at_mstar else 0)
                   | (FLAG_PLAIN_CG if plain_cg else 0))
        o.coarse_nodes = int(coarse_nodes)
        o.stream = C.c_void_p(int(stream))
        h = C.c_void_p()
        mat = material_struct(material)
        if isinstance(mesh, (list, tuple)):
            _check(lib.gspm_batch_load(descs, len(meshes), C.byref(mat), C.byref(o), C.byref(h)),
                   "gspm_batch_load")
        else:
            _check(lib.gspm_mesh_load(descs, C.byref(mat), C.byref(o), C.byref(h)),
                   "gspm_mesh_load")
        self._h = h
        self.precision = precision
        inf = self.info()
        self.n = inf["n_unique"]
        self.n_segments = inf["n_segments"]

    def close(self):
        if getattr(self, "_h", None):
            lib.gspm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self) -> dict:
        i = MeshInfo()
        _check(lib.gspm_mesh_info_get(self._h, C.byref(i)), "gspm_mesh_info_get")
        out = {k: getattr(i, k) for k, _ in MeshInfo._fields_}
        out["spmv_ms_block"] = list(i.spmv_ms_block)
        out["spmv_ms_scalar"] = list(i.spmv_ms_scalar)
        out["spmv_ms_gs"] = list(i.spmv_ms_gs)
        return out

    def export(self, what: int) -> np.ndarray:
        inf = self.info()
        size, dtype = {EXPORT_UNIQUE_OF_STORED: (inf["n_stored"], np.int64),
                       EXPORT_ROWPTR: (inf["n_unique"] + 1, np.int64),
                       EXPORT_COLS: (inf["nnz"], np.int64),
                       EXPORT_PERM: (inf["n_unique"], np.int64),
                       EXPORT_NODE_MAGNETIC: (inf["n_unique"], np.uint8),
                       EXPORT_LUMPED_MASS: (inf["n_unique"], np.float64),
                       EXPORT_AGGREGATES: (inf["n_unique"], np.int32),
                       EXPORT_COARSE_K_MS: (inf["n_aggregates"] ** 2, np.float64),
                       EXPORT_COARSE_K_MECH: (9 * inf["n_aggregates"] ** 2, np.float64),
                       EXPORT_COARSE_INV_MS: (inf["n_aggregates"] ** 2, np.float64),
                       EXPORT_COARSE_INV_MECH: (9 * inf["n_aggregates"] ** 2, np.float64),
                       EXPORT_COARSE_STORED_MS: (inf["n_aggregates"] ** 2, np.float64),
                       EXPORT_COARSE_STORED_MECH: (9 * inf["n_aggregates"] ** 2, np.float64)}[what]
        out = np.empty(size, dtype=dtype)
        _check(lib.gspm_mesh_export(self._h, what, C.c_void_p(out.ctypes.data), size),
               "gspm_mesh_export")
        return out

    def set_field(self, field: int, data):
        p, where, keep = _ptr(data, self.n * FIELD_NCOMP[field])
        _check(lib.gspm_set_field(self._h, field, p, where), "gspm_set_field")

    def get_field(self, field: int, out=None):
        nc = FIELD_NCOMP[field]
        if out is None:
            out = np.empty((self.n, nc) if nc > 1 else (self.n,))
        p, where, keep = _ptr(out, self.n * nc)
        _check(lib.gspm_get_field(self._h, field, p, where), "gspm_get_field")
        return out

    def step(self, n_steps: int, H, stats: bool = True):
        Hc = (C.c_double * 3)(*[float(v) for v in H])
        S = (StepStats * self.n_segments)()
        s = S[0]
        code = _check(lib.gspm_step(self._h, int(n_steps), Hc, S if stats else None),
                      "gspm_step", allow=(ENOCONV,))
        if not stats:
            return code
        out = {k: getattr(s, k) for k, _ in StepStats._fields_}
        out["it_gs_last"] = list(s.it_gs_last)
        out["m_bar"] = list(s.m_bar)
        out["status"] = code
        return out

    def batch_step(self, n_steps: int, H_all, stats: bool = True):
        """gspm_batch_step: one applied field per mesh, H_all [n_meshes][3] (A/m)."""
        H = np.ascontiguousarray(H_all, dtype=np.float64).reshape(-1)
        if H.size != 3 * self.n_segments:
            raise ValueError("need one field per mesh")
        S = (StepStats * self.n_segments)()
        code = _check(lib.gspm_batch_step(self._h, int(n_steps), H.ctypes.data_as(_dp),
                                          S if stats else None), "gspm_batch_step",
                      allow=(ENOCONV,))
        if not stats:
            return code
        out = []
        for s in S:
            d = {k: getattr(s, k) for k, _ in StepStats._fields_}
            d["it_gs_last"] = list(s.it_gs_last)
            d["m_bar"] = list(s.m_bar)
            out.append(d)
        return out

    def segment(self, seg: int):
        """(first node, node count) of mesh `seg` in the batch numbering."""
        off, cnt = C.c_int64(), C.c_int64()
        _check(lib.gspm_batch_segment(self._h, int(seg), C.byref(off), C.byref(cnt)),
               "gspm_batch_segment")
        return off.value, cnt.value

    def solve_elastic(self, m, u_out=None, x0_mode=1, x0=None, rtol=0.0):
        pm, where, k1 = _ptr(m, 3 * self.n)
        if u_out is None:
            u_out = np.empty((self.n, 3)) if where == HOST else None
        pu, wu, k2 = _ptr(u_out, 3 * self.n) if u_out is not None else (None, where, None)
        if wu != where:
            raise ValueError("m and u must live on the same side")
        px = _ptr(x0, 3 * self.n)[0] if x0 is not None else None
        it = C.c_int()
        rel = C.c_double()
        code = _check(lib.gspm_solve_elastic(self._h, pm, pu, where, int(x0_mode), px,
                                             float(rtol), C.byref(it), C.byref(rel)),
                      "gspm_solve_elastic", allow=(ENOCONV,))
        return u_out, it.value, rel.value, code

    def volume_avg(self, field) -> np.ndarray:
        """Per-mesh volume averages: [ncomp] for one mesh, [n_meshes][ncomp] for a batch."""
        nc = int(np.prod(field.shape[1:])) if len(field.shape) > 1 else 1
        p, where, keep = _ptr(field, self.n * nc)
        out = np.empty((self.n_segments, nc)) if self.n_segments > 1 else np.empty(nc)
        _check(lib.gspm_volume_avg(self._h, p, where, nc, out.ctypes.data_as(_dp)),
               "gspm_volume_avg")
        return out

    def apply(self, op: int, x, out=None):
        nin = {OP_K_MECH: 3, OP_DIV: 3}.get(op, 1)
        nout = {OP_K_MECH: 3, OP_GRAD: 3}.get(op, 1)
        px, where, k1 = _ptr(x, self.n * nin)
        if out is None:
            if where == DEVICE:
                import torch
                out = torch.empty((self.n, nout) if nout > 1 else (self.n,), dtype=torch.float64,
                                  device=x.device)
            else:
                out = np.empty((self.n, nout) if nout > 1 else (self.n,))
        py, wy, k2 = _ptr(out, self.n * nout)
        _check(lib.gspm_apply(self._h, op, px, py, where), "gspm_apply")
        return out

    def launch_count(self) -> int:
        return int(lib.gspm_launch_count(self._h))

    # ---- learned warm start
    def set_graph(self, on: bool):
        """Replay each step as one captured CUDA graph (``gspm_set_graph``)."""
        _check(lib.gspm_set_graph(self._h, int(bool(on))), "gspm_set_graph")

    def set_true_residual(self, on: bool):
        """Report ||b - K x|| / ||b|| of the last K^ms / K^mech solves in the step stats
        (``gspm_set_true_residual``)."""
        _check(lib.gspm_set_true_residual(self._h, int(bool(on))), "gspm_set_true_residual")

    def set_rtol(self, rtol_gs=0.0, rtol_ms=0.0, rtol_mech=0.0):
        """New CG stopping tolerances for the following steps (<= 0 keeps one)."""
        _check(lib.gspm_set_rtol(self._h, float(rtol_gs), float(rtol_ms), float(rtol_mech)),
               "gspm_set_rtol")

    def set_x0_mode(self, mode: int):
        _check(lib.gspm_set_x0_mode(self._h, int(mode)), "gspm_set_x0_mode")

    def mpnn_set_params(self, params):
        flat = flatten_params(params) if isinstance(params, dict) else \
            np.ascontiguousarray(params, dtype=np.float32)
        _check(lib.gspm_mpnn_set_params(self._h, flat.ctypes.data_as(C.POINTER(C.c_float)),
                                        flat.size), "gspm_mpnn_set_params")

    def mpnn_get_params(self) -> np.ndarray:
        out = np.empty(MPNN_PARAMS, dtype=np.float32)
        _check(lib.gspm_mpnn_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)),
                                        out.size), "gspm_mpnn_get_params")
        return out

    def mpnn_predict(self, m, u_prev=None, u_prev2=None, what=0, out=None):
        pm, where, k1 = _ptr(m, 3 * self.n)
        pu = _ptr(u_prev, 3 * self.n)[0] if u_prev is not None else None
        pu2 = _ptr(u_prev2, 3 * self.n)[0] if u_prev2 is not None else None
        if out is None:
            if where == DEVICE:
                import torch
                out = torch.empty((self.n, 3), dtype=torch.float64, device=m.device)
            else:
                out = np.empty((self.n, 3))
        po, _, k2 = _ptr(out, 3 * self.n)
        _check(lib.gspm_mpnn_predict(self._h, pm, pu, pu2, po, int(what), where),
               "gspm_mpnn_predict")
        return out

    def mpnn_dataset_reserve(self, capacity: int):
        _check(lib.gspm_mpnn_dataset_reserve(self._h, int(capacity)), "gspm_mpnn_dataset_reserve")

    def mpnn_dataset_add(self, m, u_prev, u_prev2, u_star) -> int:
        pm, where, k1 = _ptr(m, 3 * self.n)
        pu = _ptr(u_prev, 3 * self.n)[0] if u_prev is not None else None
        pu2 = _ptr(u_prev2, 3 * self.n)[0] if u_prev2 is not None else None
        ps, _, k2 = _ptr(u_star, 3 * self.n)
        idx = C.c_int()
        _check(lib.gspm_mpnn_dataset_add(self._h, pm, pu, pu2, ps, where, C.byref(idx)),
               "gspm_mpnn_dataset_add")
        return idx.value

    def mpnn_loss_grad(self, pair: int):
        loss = C.c_double()
        g = np.empty(MPNN_PARAMS, dtype=np.float32)
        _check(lib.gspm_mpnn_loss_grad(self._h, int(pair), C.byref(loss),
                                       g.ctypes.data_as(C.POINTER(C.c_float))),
               "gspm_mpnn_loss_grad")
        return loss.value, g

    def mpnn_train(self, iterations: int, lr: float = 1e-3, seed: int = 0):
        l0, l1 = C.c_double(), C.c_double()
        _check(lib.gspm_mpnn_train(self._h, int(iterations), float(lr), int(seed), C.byref(l0),
                                   C.byref(l1)), "gspm_mpnn_train")
        return l0.value, l1.value

    def profile_enable(self, classes=()):
        mask = 0
        for c in classes:
            mask |= 1 << (KCLASS[c] if isinstance(c, str) else int(c))
        _check(lib.gspm_profile_enable(self._h, mask), "gspm_profile_enable")

    def profile_read(self, cls):
        ms = C.c_double()
        cnt = C.c_int64()
        k = KCLASS[cls] if isinstance(cls, str) else int(cls)
        _check(lib.gspm_profile_read(self._h, k, C.byref(ms), C.byref(cnt)), "gspm_profile_read")
        return ms.value, cnt.value


def coarse_round(A, bf16: bool):
    """gspm_coarse_round: the storage of a dense SPD matrix as the coarse inverse (host code).
    Returns (stored values as float64 [n][n], diagonal shift used)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    out = np.empty((n, n))
    sh = C.c_double()
    _check(lib.gspm_coarse_round(A.ctypes.data_as(_dp), n, int(bool(bf16)),
                                 out.ctypes.data_as(_dp), C.byref(sh)), "gspm_coarse_round")
    return out, sh.value


def flatten_params(p: dict) -> np.ndarray:
    """Oracle-style parameter dict -> flat float32 array in the library's layout."""
    return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1)
                           for k, _ in MPNN_KEYS]).astype(np.float32)


def unflatten_params(flat) -> dict:
    out, o = {}, 0
    for k, shp in MPNN_KEYS:
        size = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def volume_avg_noalloc(field, weights, out, stream=0):
    """gspm_volume_avg_noalloc on CUDA float64 tensors field [n][ncomp], weights [n], out
    [ncomp]; asynchronous on `stream`, allocates nothing."""
    for a in (field, weights, out):
        if not _is_device(a):
            raise ValueError("volume_avg_noalloc takes device tensors only")
    n = weights.numel()
    nc = field.numel() // max(n, 1)
    pf, _, _ = _ptr(field, n * nc)
    pw, _, _ = _ptr(weights, n)
    po, _, _ = _ptr(out, nc)
    _check(lib.gspm_volume_avg_noalloc(pf, pw, n, nc, po, C.c_void_p(int(stream))),
           "gspm_volume_avg_noalloc")
    return out
