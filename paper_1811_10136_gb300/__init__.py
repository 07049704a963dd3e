"""GB300-native FilterReg hot path: Python binding of libfilterreg.so.

This module is argument marshalling only.  Every step of the registration
(lattice build, splat, blur, slice, residuals, Gauss-Newton reduction,
float64 solve and SE(3) update) runs in the sm_103a kernels of
``libfilterreg.so``, reached through the C ABI of ``include/filterreg.h``.
There is no CPU fallback: if the library is missing or cannot be loaded, every
call raises.  PyTorch is used only to hold device memory and to supply the
current CUDA stream.

The low-level functions keep the C names (``fr_ctx_create``,
``fr_register_rigid``, ...); ``Context`` and ``Lattice`` wrap them for torch
tensors.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfilterreg.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_ECAPACITY, FR_ETIMEOUT, FR_ENOTSUPPORTED = range(7)
FR_PT2PT, FR_PT2PL = 0, 1
FR_FP32, FR_BF16, FR_FP16 = 0, 1, 2

# Every symbol include/filterreg.h declares (checked by the ABI tests).
EXPORTED = [
    "fr_options_default", "fr_status_string", "fr_ctx_create", "fr_ctx_destroy",
    "fr_ctx_set_stream", "fr_ctx_last_error", "fr_ctx_kernel_launches", "fr_lattice_embed",
    "fr_lattice_build", "fr_lattice_splat", "fr_lattice_blur", "fr_lattice_slice",
    "fr_lattice_vertices", "fr_lattice_info", "fr_lattice_destroy", "fr_estep",
    "fr_register_rigid", "fr_register_rigid_host", "fr_ctx_set_profiling", "fr_ctx_profile",
    "fr_ctx_set_workspace_limit", "fr_tune_get", "fr_tune_set", "fr_tune_save", "fr_tune_load",
    "fr_autotune_batch", "fr_gauss_transform",
    "fr_ctx_transfer_bytes", "fr_estep_noalloc", "fr_register_rigid_batch",
    "fr_register_rigid_batch_host", "fr_register_articulated", "fr_estep_storage",
    "fr_server_create", "fr_server_submit", "fr_server_poll", "fr_server_wait", "fr_server_release",
    "fr_server_stats", "fr_server_destroy", "fr_nodegraph_create", "fr_nodegraph_destroy",
    "fr_register_nodegraph", "fr_nodegraph_system", "fr_nodegraph_warp",
    "fr_feature_embed", "fr_estep_features", "fr_gauss_transform_features",
    "fr_rigid_normal_equations", "fr_rigid_solve_update", "fr_em_sharded", "fr_register_rigid_sharded",
    "fr_debug_fail_allocations", "fr_register_articulated_batch",
]
FR_ART_BATCH_MAX = 4096
FR_ART_CONCURRENT = 16
FR_NE_VALS = 30
# fr_ne_fn and fr_allreduce_fn of include/filterreg.h
NE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_float,
                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p)
FR_FEATURE_DMAX = 7
FR_NOALLOC_MAX_OBS = 8192
KERNEL_CLASSES = ("clear", "build", "blur", "em_iter", "convert", "ng_assemble", "ng_solve", "slice")


class FilterRegError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class fr_options(ctypes.Structure):
    _fields_ = [("residual", ctypes.c_int32), ("blur", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("sigma_start", ctypes.c_float), ("sigma_end", ctypes.c_float), ("w", ctypes.c_float),
                ("storage", ctypes.c_int32), ("kahan", ctypes.c_int32),
                ("renormalize_normals", ctypes.c_int32), ("stop_twist", ctypes.c_float),
                ("use_graph", ctypes.c_int32), ("update_sigma", ctypes.c_int32)]


class fr_report(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int32), ("degenerate_iters", ctypes.c_int32),
                ("last_inliers", ctypes.c_int64), ("last_sum_w", ctypes.c_double),
                ("last_cost", ctypes.c_double), ("last_twist_norm", ctypes.c_double),
                ("lattice_vertices", ctypes.c_int64), ("lattice_builds", ctypes.c_int32),
                ("lattice_vertices_sum", ctypes.c_int64), ("last_sigma", ctypes.c_double)]


class fr_request(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("M", ctypes.c_int64), ("Y", ctypes.c_void_p),
                ("Yn", ctypes.c_void_p), ("N", ctypes.c_int64), ("sigma_start", ctypes.c_float),
                ("sigma_end", ctypes.c_float), ("w", ctypes.c_float), ("T", ctypes.c_double * 16),
                ("host", ctypes.c_int32)]


class fr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("T", ctypes.c_double * 16), ("report", fr_report),
                ("submit_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64), ("complete_ns", ctypes.c_int64)]


class fr_kintree(ctypes.Structure):
    _fields_ = [("n_bodies", ctypes.c_int32), ("n_joints", ctypes.c_int32), ("parent", ctypes.c_void_p),
                ("offset", ctypes.c_void_p), ("joint_body", ctypes.c_void_p), ("joint_axis", ctypes.c_void_p),
                ("q_min", ctypes.c_void_p), ("q_max", ctypes.c_void_p)]


def kintree(tree):
    """fr_kintree view of a tree object with parent, offset (nb,4,4), joint_body,
    joint_axis (nj,3), q_min, q_max; returns (struct, keep-alive arrays)."""
    a = dict(parent=np.ascontiguousarray(tree.parent, dtype=np.int32),
             offset=np.ascontiguousarray(tree.offset, dtype=np.float64).reshape(-1, 16),
             joint_body=np.ascontiguousarray(tree.joint_body, dtype=np.int32),
             joint_axis=np.ascontiguousarray(tree.joint_axis, dtype=np.float64).reshape(-1, 3),
             q_min=np.ascontiguousarray(tree.q_min, dtype=np.float64),
             q_max=np.ascontiguousarray(tree.q_max, dtype=np.float64))
    st = fr_kintree(len(a["parent"]), len(a["joint_body"]), a["parent"].ctypes.data, a["offset"].ctypes.data,
                    a["joint_body"].ctypes.data, a["joint_axis"].ctypes.data, a["q_min"].ctypes.data,
                    a["q_max"].ctypes.data)
    return st, a


class fr_batch_item(ctypes.Structure):
    _fields_ = [("d_X", ctypes.c_void_p), ("M", ctypes.c_int64), ("d_Y", ctypes.c_void_p),
                ("d_Yn", ctypes.c_void_p), ("N", ctypes.c_int64), ("sigma_start", ctypes.c_float),
                ("sigma_end", ctypes.c_float), ("w", ctypes.c_float), ("T", ctypes.c_double * 16),
                ("status", ctypes.c_int)]


# fr_batch_item as a numpy record (same offsets): the items of a call are
# filled and read field by field for all items at once.
_BATCH_ITEM_DTYPE = np.dtype({
    "names": ["d_X", "M", "d_Y", "d_Yn", "N", "sigma_start", "sigma_end", "w", "T", "status"],
    "formats": ["u8", "i8", "u8", "u8", "i8", "f4", "f4", "f4", ("f8", (16,)), "i4"],
    "offsets": [getattr(fr_batch_item, f).offset for f in
                ("d_X", "M", "d_Y", "d_Yn", "N", "sigma_start", "sigma_end", "w", "T", "status")],
    "itemsize": ctypes.sizeof(fr_batch_item)})
_EYE16 = np.eye(4).ravel()


class fr_articulated_item(ctypes.Structure):
    _fields_ = [("d_Xref", ctypes.c_void_p), ("d_body", ctypes.c_void_p), ("M", ctypes.c_int64),
                ("d_Y", ctypes.c_void_p), ("d_Yn", ctypes.c_void_p), ("N", ctypes.c_int64),
                ("root_T", ctypes.c_double * 16), ("q", ctypes.POINTER(ctypes.c_double)),
                ("status", ctypes.c_int32)]


class fr_tune_params(ctypes.Structure):
    _fields_ = [("step_points_per_thread", ctypes.c_int32), ("build_points_per_thread", ctypes.c_int32),
                ("table_slots_x2", ctypes.c_int32), ("serve_points_per_thread", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


FR_TUNE_THROUGHPUT, FR_TUNE_LATENCY = 0, 1


class fr_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 8), ("total_ms", ctypes.c_double * 8)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_lib = None


def load(build_if_missing: bool = True):
    """Load libfilterreg.so (building it with nvcc first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH) and build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise FilterRegError(FR_ECUDA, f"{LIB_PATH} is missing: run paper_1811_10136_gb300.build")
    L = ctypes.CDLL(LIB_PATH)
    L.fr_options_default.argtypes = [ctypes.POINTER(fr_options)]
    L.fr_options_default.restype = None
    L.fr_status_string.argtypes = [ctypes.c_int]
    L.fr_status_string.restype = ctypes.c_char_p
    L.fr_ctx_create.argtypes = [ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    L.fr_ctx_destroy.argtypes = [_vp]
    L.fr_ctx_set_stream.argtypes = [_vp, _vp]
    L.fr_ctx_last_error.argtypes = [_vp]
    L.fr_ctx_last_error.restype = ctypes.c_char_p
    L.fr_ctx_kernel_launches.argtypes = [_vp]
    L.fr_ctx_kernel_launches.restype = _i64
    L.fr_lattice_embed.argtypes = [_vp, _vp, _i64, ctypes.c_float, _vp, _vp]
    L.fr_lattice_build.argtypes = [_vp, _vp, _i64, ctypes.c_float, _i64, ctypes.POINTER(_vp)]
    L.fr_lattice_splat.argtypes = [_vp, _vp, _vp, ctypes.c_int]
    L.fr_lattice_blur.argtypes = [_vp, _vp]
    L.fr_lattice_slice.argtypes = [_vp, _vp, _vp, _i64, _vp]
    L.fr_lattice_vertices.argtypes = [_vp, _vp, _vp, _vp, ctypes.POINTER(_i64)]
    L.fr_lattice_info.argtypes = [_vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                  ctypes.POINTER(ctypes.c_int32)]
    L.fr_lattice_destroy.argtypes = [_vp, _vp]
    L.fr_estep.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_float, ctypes.c_int, _f64p, _vp]
    L.fr_estep_storage.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_float, ctypes.c_int32,
                                   _f64p, _vp]
    L.fr_register_rigid.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.POINTER(fr_options),
                                    _f64p, ctypes.POINTER(fr_report)]
    L.fr_register_rigid_host.argtypes = L.fr_register_rigid.argtypes
    L.fr_ctx_set_profiling.argtypes = [_vp, ctypes.c_int]
    L.fr_ctx_set_workspace_limit.argtypes = [_vp, ctypes.c_size_t]
    L.fr_gauss_transform.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.c_float, _f64p, _vp]
    L.fr_tune_get.argtypes = [_vp, _i64, ctypes.POINTER(fr_tune_params)]
    L.fr_tune_set.argtypes = [_vp, _i64, ctypes.POINTER(fr_tune_params)]
    L.fr_tune_save.argtypes = [_vp, ctypes.c_char_p]
    L.fr_tune_load.argtypes = [_vp, ctypes.c_char_p]
    L.fr_autotune_batch.argtypes = [_vp, ctypes.POINTER(fr_batch_item), ctypes.c_int, ctypes.POINTER(fr_options),
                                    ctypes.c_int, ctypes.c_int, ctypes.POINTER(fr_tune_params),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.fr_ctx_profile.argtypes = [_vp, ctypes.POINTER(fr_profile), ctypes.c_int]
    L.fr_ctx_transfer_bytes.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    L.fr_register_rigid_batch.argtypes = [_vp, ctypes.POINTER(fr_batch_item), ctypes.c_int,
                                          ctypes.POINTER(fr_options), ctypes.POINTER(fr_report)]
    L.fr_register_rigid_batch_host.argtypes = L.fr_register_rigid_batch.argtypes
    L.fr_register_articulated.argtypes = [_vp, _vp, _vp, _i64, ctypes.POINTER(fr_kintree), _vp, _vp, _i64,
                                          ctypes.POINTER(fr_options), _f64p, _f64p, ctypes.POINTER(fr_report)]
    L.fr_register_articulated_batch.argtypes = [_vp, ctypes.POINTER(fr_kintree), ctypes.POINTER(fr_articulated_item),
                                                ctypes.c_int32, ctypes.POINTER(fr_options), ctypes.POINTER(fr_report)]
    L.fr_estep_noalloc.argtypes = [_vp, _i64, _vp, _vp, _i64, ctypes.c_float, _f64p, _vp, _vp]
    L.fr_server_create.argtypes = [_vp, ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(fr_options),
                                   ctypes.POINTER(_vp)]
    L.fr_server_submit.argtypes = [_vp, ctypes.POINTER(fr_request), ctypes.POINTER(ctypes.c_uint64)]
    L.fr_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(fr_result)]
    L.fr_server_wait.argtypes = [_vp, ctypes.c_uint64, _i64, ctypes.POINTER(fr_result)]
    L.fr_server_release.argtypes = [_vp, ctypes.c_uint64]
    L.fr_server_stats.argtypes = [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    L.fr_server_destroy.argtypes = [_vp]
    L.fr_nodegraph_create.argtypes = [_vp, _vp, _vp, _vp, _i64, _f64p, ctypes.c_int, _vp, ctypes.c_int,
                                      ctypes.POINTER(_vp)]
    L.fr_nodegraph_destroy.argtypes = [_vp]
    L.fr_register_nodegraph.argtypes = [_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(fr_options), ctypes.c_double,
                                        ctypes.c_int, _f64p, ctypes.POINTER(fr_report)]
    L.fr_nodegraph_system.argtypes = [_vp, _vp, _vp, _vp, _i64, ctypes.POINTER(fr_options), ctypes.c_double,
                                      _f64p, _f64p, _f64p, ctypes.POINTER(fr_report)]
    L.fr_nodegraph_warp.argtypes = [_vp, _vp, _f64p, _vp]
    L.fr_feature_embed.argtypes = [_vp, _vp, _i64, ctypes.c_int32, _f32p, _vp, _vp]
    L.fr_estep_features.argtypes = [_vp, _vp, _i64, _vp, _i64, ctypes.c_int32, _f32p, _vp, _vp, _vp,
                                    ctypes.POINTER(_i64)]
    L.fr_gauss_transform_features.argtypes = [_vp, _vp, _i64, _vp, _i64, ctypes.c_int32, _f32p, _vp, _vp, _vp]
    L.fr_debug_fail_allocations.argtypes = [ctypes.c_int32, ctypes.c_int32]
    L.fr_rigid_normal_equations.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.POINTER(fr_options), _i64,
                                            _f64p, _f64p]
    L.fr_rigid_solve_update.argtypes = [_f64p, _f64p, ctypes.POINTER(ctypes.c_double)]
    L.fr_em_sharded.argtypes = [NE_FN, _vp, ALLREDUCE_FN, _vp, ctypes.POINTER(fr_options), _f64p,
                                ctypes.POINTER(fr_report)]
    L.fr_register_rigid_sharded.argtypes = [_vp, _vp, _i64, _vp, _vp, _i64, ctypes.POINTER(fr_options), _i64,
                                            ALLREDUCE_FN, _vp, _f64p, ctypes.POINTER(fr_report)]
    for name in EXPORTED:  # every entry point must resolve (ctypes restype defaults to int)
        getattr(L, name)
    _lib = L
    return L


def options(**kw) -> fr_options:
    """fr_options with the library defaults, overridden by keyword."""
    o = fr_options()
    load().fr_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class Report:
    iters_run: int
    degenerate_iters: int
    last_inliers: int
    last_sum_w: float
    last_cost: float
    last_twist_norm: float
    lattice_vertices: int
    lattice_builds: int
    lattice_vertices_sum: int
    last_sigma: float = 0.0


def _report(r: fr_report) -> Report:
    return Report(r.iters_run, r.degenerate_iters, r.last_inliers, r.last_sum_w, r.last_cost,
                  r.last_twist_norm, r.lattice_vertices, r.lattice_builds, r.lattice_vertices_sum,
                  r.last_sigma)


def _host_ptr(a: np.ndarray) -> int:
    """Address of a contiguous host array's data (the buffer protocol's
    address is cheaper to take than ndarray.ctypes for a writable array)."""
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.ctypes.data


def _dev_ptr(t, name, rows=None, cols=4):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != cols or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 ({'n' if rows is None else rows}, {cols}) tensor")
    if rows is not None and t.shape[0] != rows:
        raise ValueError(f"{name} must have {rows} rows")
    return t.data_ptr()


# ---- sharded single registration (host-side EM loop, caller's collective) ----

class _Callbacks:
    """ctypes callbacks around Python callables; the first exception raised
    inside one is kept and re-raised after the library call returns."""

    def __init__(self, provider=None, allreduce=None):
        self.error = None
        self.ne = NE_FN(self._ne) if provider is not None else NE_FN()
        self.ar = ALLREDUCE_FN(self._ar) if allreduce is not None else ALLREDUCE_FN()
        self._provider, self._allreduce = provider, allreduce

    def _ne(self, T, sigma, ne, user):
        try:
            Tm = np.ctypeslib.as_array(T, shape=(16,)).reshape(4, 4).copy()
            out = np.asarray(self._provider(Tm, float(sigma)), dtype=np.float64).reshape(-1)
            if out.shape[0] != FR_NE_VALS:
                raise ValueError(f"a provider returns {FR_NE_VALS} values")
            np.ctypeslib.as_array(ne, shape=(FR_NE_VALS,))[:] = out
            return 0
        except BaseException as e:  # noqa: BLE001 -- re-raised after the call
            self.error = self.error or e
            return FR_EINVAL

    def _ar(self, vals, n, user):
        try:
            v = np.ctypeslib.as_array(vals, shape=(n,))
            v[:] = np.asarray(self._allreduce(v.copy()), dtype=np.float64)
            return 0
        except BaseException as e:  # noqa: BLE001
            self.error = self.error or e
            return FR_ECUDA


def torch_allreduce(group=None, device="cpu"):
    """An all-reduce for the sharded registration over torch.distributed
    (gloo with device="cpu", NCCL with a CUDA device): values -> summed values."""
    import torch
    import torch.distributed as dist

    def ar(v):
        t = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float64)).to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t.cpu().numpy()
    return ar


def rigid_solve_update(ne, T):
    """fr_rigid_solve_update: (T_new (4,4), |delta zeta|, ok) from summed normal equations."""
    ne = np.ascontiguousarray(ne, dtype=np.float64).reshape(-1)
    Tm = _pose(T)
    tn = ctypes.c_double(0.0)
    st = load().fr_rigid_solve_update(ne.ctypes.data_as(_f64p), Tm.ctypes.data_as(_f64p), ctypes.byref(tn))
    return Tm, float(tn.value), st == FR_OK


def debug_fail_allocations(after: int = 0, n: int = 0) -> None:
    """fr_debug_fail_allocations: of the library's next device allocations the
    first `after` proceed and the `n` after them fail (testing; n = 0 clears)."""
    st = load().fr_debug_fail_allocations(int(after), int(n))
    if st != FR_OK:
        raise FilterRegError(st, "fr_debug_fail_allocations: arguments must be >= 0")


def em_sharded(provider, allreduce=None, T0=None, **opts):
    """fr_em_sharded: the host EM loop with provider(T (4,4), sigma) -> 30
    normal-equation values of this rank and allreduce(values) -> summed values
    (None: one rank).  Returns (T, Report, status)."""
    cb = _Callbacks(provider, allreduce)
    o = options(**opts)
    T = _pose(T0)
    rep = fr_report()
    st = load().fr_em_sharded(cb.ne, None, cb.ar, None, ctypes.byref(o), T.ctypes.data_as(_f64p),
                              ctypes.byref(rep))
    if cb.error is not None:
        raise cb.error
    return T, _report(rep), int(st)


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(np.eye(4) if T is None else T, dtype=np.float64).reshape(4, 4).copy()
    return T


def estep_noalloc(X, Y, Yn=None, sigma=0.02, T=None, out=None, stream=None):
    """fr_estep_noalloc: the E step on the library's fixed scratch array (no
    device allocation by the library; at most FR_NOALLOC_MAX_OBS observation
    points).  X (M,4), Y (N,4), Yn (N,4) and `out` ((M,4) or (M,7) float32)
    are CUDA tensors owned by the caller; `out` is created here if omitted.
    Returns `out`."""
    import torch
    L = load()
    vd = 7 if Yn is not None else 4
    if out is None:
        out = torch.empty((X.shape[0], vd), dtype=torch.float32, device=X.device)
    _dev_ptr(out, "out", rows=X.shape[0], cols=vd)
    if stream is None:
        stream = torch.cuda.current_stream(X.device)
    Tm = _pose(T)
    st = L.fr_estep_noalloc(_dev_ptr(X, "X"), X.shape[0], _dev_ptr(Y, "Y"),
                            _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None,
                            Y.shape[0], float(sigma), Tm.ctypes.data_as(_f64p), out.data_ptr(),
                            _vp(stream.cuda_stream))
    if st != FR_OK:
        raise FilterRegError(st, f"fr_estep_noalloc: {L.fr_status_string(st).decode()}")
    return out


class Context:
    """An fr_ctx bound to a CUDA device and (by default) torch's current stream."""

    def __init__(self, device: int = 0, stream=None, tune_table: str | None = "default"):
        """tune_table: a launch-shape table (fr_tune_load) -- "default" the
        one shipped beside the library (tuning_gb300.txt), None the built-in
        defaults, or a path."""
        import torch
        L = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self._stream = stream
        h = _vp()
        st = L.fr_ctx_create(int(device), _vp(stream.cuda_stream), ctypes.byref(h))
        if st != FR_OK:
            raise FilterRegError(st, f"fr_ctx_create(device={device}) failed")
        self._h = h
        self.device = device
        if tune_table == "default":
            tune_table = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.txt")
            if not os.path.exists(tune_table):
                tune_table = None
        if tune_table:
            self.tune_load(tune_table)

    def close(self):
        if getattr(self, "_h", None):
            load().fr_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != FR_OK:
            L = load()
            raise FilterRegError(st, f"{what}: {L.fr_status_string(st).decode()}: "
                                     f"{L.fr_ctx_last_error(self._h).decode()}")

    @property
    def kernel_launches(self) -> int:
        return int(load().fr_ctx_kernel_launches(self._h))

    def transfer_bytes(self):
        """(host->device, device->host) bytes this context has copied."""
        a, b = _i64(), _i64()
        self._check(load().fr_ctx_transfer_bytes(self._h, ctypes.byref(a), ctypes.byref(b)),
                    "fr_ctx_transfer_bytes")
        return a.value, b.value

    def set_workspace_limit(self, nbytes: int):
        """Cap the lattice-table arena of batched calls at nbytes (0: none)."""
        self._check(load().fr_ctx_set_workspace_limit(self._h, int(nbytes)), "fr_ctx_set_workspace_limit")

    # ---- launch-shape tuning ----------------------------------------------
    def tune_get(self, n_points: int) -> dict:
        """Tuning parameters of the size class of n_points."""
        p = fr_tune_params()
        self._check(load().fr_tune_get(self._h, int(n_points), ctypes.byref(p)), "fr_tune_get")
        return p.as_dict()

    def tune_set(self, n_points: int, **params):
        """Set (some of) the tuning parameters of n_points' size class."""
        cur = self.tune_get(n_points)
        cur.update(params)
        p = fr_tune_params(**cur)
        self._check(load().fr_tune_set(self._h, int(n_points), ctypes.byref(p)), "fr_tune_set")

    def tune_save(self, path: str):
        self._check(load().fr_tune_save(self._h, os.fsencode(path)), "fr_tune_save")

    def tune_load(self, path: str):
        self._check(load().fr_tune_load(self._h, os.fsencode(path)), "fr_tune_load")

    def autotune_batch(self, pairs, objective=FR_TUNE_THROUGHPUT, reps=3, sigmas=None, ws=None, **opts):
        """Time candidate launch shapes on this batch (CUDA tensors, as for
        register_rigid_batch) and install the fastest; returns (params dict,
        best ms, default ms)."""
        items, _ = self._batch_items(pairs, sigmas, ws, None, False, options(**opts))
        o = options(**opts)
        best = fr_tune_params()
        b_ms, d_ms = ctypes.c_double(), ctypes.c_double()
        self._check(load().fr_autotune_batch(self._h, items, len(pairs), ctypes.byref(o), int(objective), int(reps),
                                             ctypes.byref(best), ctypes.byref(b_ms), ctypes.byref(d_ms)),
                    "fr_autotune_batch")
        return best.as_dict(), b_ms.value, d_ms.value

    def set_profiling(self, on: bool):
        self._check(load().fr_ctx_set_profiling(self._h, int(bool(on))), "fr_ctx_set_profiling")

    def profile(self, reset: bool = False) -> dict:
        """{kernel class: (launches, total ms)} accumulated while profiling was on."""
        p = fr_profile()
        self._check(load().fr_ctx_profile(self._h, ctypes.byref(p), int(bool(reset))), "fr_ctx_profile")
        return {name: (int(p.launches[i]), float(p.total_ms[i])) for i, name in enumerate(KERNEL_CLASSES)}

    # ---- registration ------------------------------------------------------
    def register_rigid(self, X, Y, Yn=None, T0=None, **opts):
        """Rigid FilterReg registration of X (M,4) to Y (N,4) (+ normals Yn for
        point-to-plane).  Returns (T (4,4) float64 numpy, Report)."""
        L = load()
        o = options(**opts)
        T = _pose(T0)
        rep = fr_report()
        pX = _dev_ptr(X, "X")
        pY = _dev_ptr(Y, "Y")
        pN = _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None
        st = L.fr_register_rigid(self._h, pX, X.shape[0], pY, pN, Y.shape[0], ctypes.byref(o),
                                 T.ctypes.data_as(_f64p), ctypes.byref(rep))
        self._check(st, "fr_register_rigid")
        return T, _report(rep)

    def rigid_normal_equations(self, X, Y, Yn=None, sigma=0.02, M_total=None, T=None, **opts):
        """fr_rigid_normal_equations: (30,) float64 -- A's upper triangle, b, sum_w, cost, inliers."""
        o = options(sigma_start=float(sigma), sigma_end=float(sigma), **opts)
        Tm = _pose(T)
        ne = np.zeros(FR_NE_VALS, np.float64)
        pN = _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None
        st = load().fr_rigid_normal_equations(self._h, _dev_ptr(X, "X"), X.shape[0], _dev_ptr(Y, "Y"), pN,
                                              Y.shape[0], ctypes.byref(o), int(M_total or X.shape[0]),
                                              Tm.ctypes.data_as(_f64p), ne.ctypes.data_as(_f64p))
        self._check(st, "fr_rigid_normal_equations")
        return ne

    def register_rigid_sharded(self, X, Y, Yn=None, M_total=None, allreduce=None, T0=None, **opts):
        """fr_register_rigid_sharded: this rank's shard X of a model of M_total
        points; allreduce(values) -> summed values over the ranks (None: one
        rank; see torch_allreduce).  Returns (T, Report)."""
        cb = _Callbacks(None, allreduce)
        o = options(**opts)
        T = _pose(T0)
        rep = fr_report()
        pN = _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None
        st = load().fr_register_rigid_sharded(self._h, _dev_ptr(X, "X"), X.shape[0], _dev_ptr(Y, "Y"), pN,
                                              Y.shape[0], ctypes.byref(o), int(M_total or X.shape[0]), cb.ar,
                                              None, T.ctypes.data_as(_f64p), ctypes.byref(rep))
        if cb.error is not None:
            raise cb.error
        self._check(st, "fr_register_rigid_sharded")
        return T, _report(rep)

    def register_rigid_host(self, X, Y, Yn=None, T0=None, **opts):
        """The same from host numpy arrays (pinned torch CPU tensors also work)."""
        L = load()
        o = options(**opts)
        T = _pose(T0)
        rep = fr_report()

        def hp(a, name):
            if a is None:
                return None, 0
            if hasattr(a, "data_ptr"):
                if a.is_cuda or a.dtype.itemsize != 4 or a.dim() != 2 or a.shape[1] != 4 or not a.is_contiguous():
                    raise TypeError(f"{name} must be a contiguous float32 (n, 4) host tensor")
                return a.data_ptr(), a.shape[0]
            a = np.ascontiguousarray(a, dtype=np.float32)
            if a.ndim != 2 or a.shape[1] != 4:
                raise TypeError(f"{name} must be a float32 (n, 4) array")
            return a.ctypes.data, a.shape[0]

        keep = [X, Y, Yn]
        pX, M = hp(X, "X")
        pY, N = hp(Y, "Y")
        pN, _ = hp(Yn, "Yn")
        st = L.fr_register_rigid_host(self._h, pX, M, pY, pN, N, ctypes.byref(o),
                                      T.ctypes.data_as(_f64p), ctypes.byref(rep))
        del keep
        self._check(st, "fr_register_rigid_host")
        return T, _report(rep)

    def register_articulated(self, Xref, body, tree, Y, Yn=None, root_T0=None, q0=None, **opts):
        """Articulated registration (Algorithm 1).  Xref (M,4) in body frames,
        body (M,) int32 CUDA tensor, tree a synth.KinTree-like object.  Returns
        (root_T (4,4), q (nj,), Report)."""
        import torch
        L = load()
        o = options(**opts)
        st, keep = kintree(tree)
        R = _pose(root_T0)
        q = np.ascontiguousarray(np.zeros(st.n_joints) if q0 is None else q0, dtype=np.float64).copy()
        if not (isinstance(body, torch.Tensor) and body.is_cuda and body.dtype == torch.int32
                and body.is_contiguous() and body.shape[0] == Xref.shape[0]):
            raise TypeError("body must be a contiguous int32 CUDA tensor with one entry per model point")
        rep = fr_report()
        qp = q.ctypes.data_as(_f64p) if q.size else None
        r = L.fr_register_articulated(self._h, _dev_ptr(Xref, "Xref"), body.data_ptr(), Xref.shape[0],
                                      ctypes.byref(st), _dev_ptr(Y, "Y"),
                                      _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None,
                                      Y.shape[0], ctypes.byref(o), R.ctypes.data_as(_f64p), qp,
                                      ctypes.byref(rep))
        del keep
        self._check(r, "fr_register_articulated")
        return R, q, _report(rep)

    def register_articulated_batch(self, items, tree, **opts):
        """fr_register_articulated_batch: several articulated registrations of
        one tree, run concurrently.  items: list of (Xref, body, Y, Yn,
        root_T0, q0) -- CUDA tensors as for register_articulated, Yn, root_T0
        and q0 may be None.  Returns a list of (root_T (4,4), q (nj,), Report,
        status) per item; raises if a call-level argument is invalid."""
        import torch
        L = load()
        o = options(**opts)
        st, keep = kintree(tree)
        n = len(items)
        arr = (fr_articulated_item * n)()
        qs = []
        reps = (fr_report * n)()
        for b, (Xref, body, Y, Yn, R0, q0) in enumerate(items):
            if not (isinstance(body, torch.Tensor) and body.is_cuda and body.dtype == torch.int32
                    and body.is_contiguous() and body.shape[0] == Xref.shape[0]):
                raise TypeError("body must be a contiguous int32 CUDA tensor with one entry per model point")
            it = arr[b]
            it.d_Xref, it.d_body, it.M = _dev_ptr(Xref, "Xref"), body.data_ptr(), Xref.shape[0]
            it.d_Y, it.N = _dev_ptr(Y, "Y"), Y.shape[0]
            it.d_Yn = _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None
            it.root_T[:] = _pose(R0).ravel().tolist()
            q = np.ascontiguousarray(np.zeros(st.n_joints) if q0 is None else q0, dtype=np.float64).copy()
            qs.append(q)
            it.q = q.ctypes.data_as(_f64p) if q.size else None
        r = L.fr_register_articulated_batch(self._h, ctypes.byref(st), arr, n, ctypes.byref(o), reps)
        del keep
        if r != FR_OK and all(arr[b].status == FR_OK for b in range(n)):
            self._check(r, "fr_register_articulated_batch")   # the call itself failed
        return [(np.array(arr[b].root_T[:], dtype=np.float64).reshape(4, 4), qs[b], _report(reps[b]),
                 int(arr[b].status)) for b in range(n)]

    def _batch_items(self, pairs, sigmas, ws, T0s, host, o):
        n = len(pairs)
        items = (fr_batch_item * n)()
        a = np.frombuffer(items, dtype=_BATCH_ITEM_DTYPE)   # the same memory, by field
        keep = []
        px, py, pn, rm, rn = [], [], [], [], []
        for X, Y, Yn in pairs:
            if host:
                arrs = [np.ascontiguousarray(a_, dtype=np.float32) if a_ is not None else None for a_ in (X, Y, Yn)]
                keep.append(arrs)
                px.append(_host_ptr(arrs[0]))
                py.append(_host_ptr(arrs[1]))
                pn.append(_host_ptr(arrs[2]) if arrs[2] is not None else 0)
                rm.append(arrs[0].shape[0])
                rn.append(arrs[1].shape[0])
            else:
                px.append(_dev_ptr(X, "X"))
                py.append(_dev_ptr(Y, "Y"))
                pn.append(_dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else 0)
                rm.append(X.shape[0])
                rn.append(Y.shape[0])
        a["d_X"], a["d_Y"], a["d_Yn"] = px, py, pn
        a["M"], a["N"] = rm, rn
        if sigmas is not None:
            sg = np.asarray(sigmas, dtype=np.float64).reshape(n, 2)
            a["sigma_start"], a["sigma_end"] = sg[:, 0], sg[:, 1]
        else:
            a["sigma_start"], a["sigma_end"] = o.sigma_start, o.sigma_end
        a["w"] = np.asarray(ws, dtype=np.float64).reshape(n) if ws is not None else o.w
        if T0s is None:
            a["T"] = _EYE16
        else:
            a["T"] = np.stack([_pose(T) for T in T0s]).reshape(n, 16)
        return items, keep

    def register_rigid_batch(self, pairs, sigmas=None, ws=None, T0s=None, host=False, **opts):
        """Register many (X, Y, Yn) pairs with one launch per EM iteration.
        pairs: list of (X, Y, Yn) -- CUDA tensors (host=False) or float32 (n, 4)
        host arrays / tensors (host=True); Yn may be None for point-to-point.
        sigmas: list of (sigma_start, sigma_end) per item (default: the
        options' schedule); ws: outlier ratios; T0s: initial poses.
        Returns a list of (T (4,4), Report, status) per item."""
        L = load()
        o = options(**opts)
        n = len(pairs)
        items, keep = self._batch_items(pairs, sigmas, ws, T0s, host, o)
        reps = (fr_report * n)()
        f = L.fr_register_rigid_batch_host if host else L.fr_register_rigid_batch
        st = f(self._h, items, n, ctypes.byref(o), reps)
        if st != FR_OK and not any(items[b].status != FR_OK for b in range(n)):
            self._check(st, "fr_register_rigid_batch")   # the call itself failed
        a = np.frombuffer(items, dtype=_BATCH_ITEM_DTYPE)
        T = a["T"].reshape(n, 4, 4).copy()
        status = a["status"].tolist()
        return [(T[b], _report(reps[b]), status[b]) for b in range(n)]

    def gauss_transform(self, X, Y, Yn=None, sigma=0.02, T=None):
        """Exact E-step sums at T X (every observation, no lattice): (M, 4)
        [M0, M1] or (M, 7) [M0, M1, Nsum] float32 CUDA tensor."""
        import torch
        L = load()
        vd = 7 if Yn is not None else 4
        out = torch.empty((X.shape[0], vd), dtype=torch.float32, device=X.device)
        Tm = _pose(T)
        st = L.fr_gauss_transform(self._h, _dev_ptr(X, "X"), X.shape[0], _dev_ptr(Y, "Y"),
                                  _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None, Y.shape[0],
                                  float(sigma), Tm.ctypes.data_as(_f64p), out.data_ptr())
        self._check(st, "fr_gauss_transform")
        return out

    def estep(self, X, Y, Yn=None, sigma=0.02, blur=False, T=None, storage=FR_FP32):
        """E-step sums at T X: (M, 4) [M0, M1] or (M, 7) [M0, M1, Nsum] float32
        CUDA tensor.  storage != FR_FP32 calls fr_estep_storage (no blur)."""
        import torch
        L = load()
        vd = 7 if Yn is not None else 4
        out = torch.empty((X.shape[0], vd), dtype=torch.float32, device=X.device)
        Tm = _pose(T)
        args = (_dev_ptr(X, "X"), X.shape[0], _dev_ptr(Y, "Y"),
                _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None, Y.shape[0],
                float(sigma))
        if storage == FR_FP32:
            st = L.fr_estep(self._h, *args, int(bool(blur)), Tm.ctypes.data_as(_f64p), out.data_ptr())
            self._check(st, "fr_estep")
        else:
            if blur:
                raise ValueError("16-bit lattice storage has no blur")
            st = L.fr_estep_storage(self._h, *args, int(storage), Tm.ctypes.data_as(_f64p),
                                    out.data_ptr())
            self._check(st, "fr_estep_storage")
        return out

    # ---- feature-space E step (d-dimensional features) ------------------
    def _features(self, F, name, d=None):
        import torch
        if not isinstance(F, torch.Tensor) or not F.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if F.dtype != torch.float32 or F.dim() != 2 or not F.is_contiguous() or \
                not 1 <= F.shape[1] <= FR_FEATURE_DMAX or (d is not None and F.shape[1] != d):
            raise TypeError(f"{name} must be a contiguous float32 (n, d) tensor, 1 <= d <= {FR_FEATURE_DMAX}")
        return F.data_ptr()

    @staticmethod
    def _sigma_f(sigma_f, d):
        sf = np.ascontiguousarray(sigma_f, dtype=np.float32).reshape(-1)
        if sf.shape[0] != d:
            raise ValueError("sigma_f needs one entry per feature channel")
        return sf

    def feature_embed(self, F, sigma_f):
        """Vertex keys (n, d+1, d+1) int32 and barycentric weights (n, d+1) of feature rows F."""
        import torch
        n, d = F.shape
        keys = torch.empty((n, d + 1, d + 1), dtype=torch.int32, device=F.device)
        bary = torch.empty((n, d + 1), dtype=torch.float32, device=F.device)
        sf = self._sigma_f(sigma_f, d)
        st = load().fr_feature_embed(self._h, self._features(F, "F"), n, d, sf.ctypes.data_as(_f32p),
                                     keys.data_ptr(), bary.data_ptr())
        self._check(st, "fr_feature_embed")
        return keys, bary

    def estep_features(self, FX, FY, sigma_f, Y, Yn=None, exact=False):
        """Feature-space E-step sums at the model features FX over the observation
        features FY (Eq. feature_estep): (M, 4) [M0, M1] or (M, 7) with normals,
        float32 CUDA tensor; the lattice unless exact.  Returns (out, vertices)
        (vertices None for the exact sums)."""
        import torch
        L = load()
        M, d = FX.shape
        N = FY.shape[0]
        vd = 7 if Yn is not None else 4
        sf = self._sigma_f(sigma_f, d)
        out = torch.empty((M, vd), dtype=torch.float32, device=FX.device)
        args = (self._features(FX, "FX"), M, self._features(FY, "FY", d), N, d, sf.ctypes.data_as(_f32p),
                _dev_ptr(Y, "Y", rows=N), _dev_ptr(Yn, "Yn", rows=N) if Yn is not None else None, out.data_ptr())
        if exact:
            self._check(L.fr_gauss_transform_features(self._h, *args), "fr_gauss_transform_features")
            return out, None
        nv = _i64(0)
        self._check(L.fr_estep_features(self._h, *args, ctypes.byref(nv)), "fr_estep_features")
        return out, int(nv.value)

    # ---- lattice primitives ----------------------------------------------
    def lattice_embed(self, P, sigma):
        import torch
        n = P.shape[0]
        keys = torch.empty((n, 4, 4), dtype=torch.int32, device=P.device)
        bary = torch.empty((n, 4), dtype=torch.float32, device=P.device)
        st = load().fr_lattice_embed(self._h, _dev_ptr(P, "P"), n, float(sigma), keys.data_ptr(),
                                     bary.data_ptr())
        self._check(st, "fr_lattice_embed")
        return keys, bary

    def lattice_build(self, P, sigma, capacity_hint=0) -> "Lattice":
        h = _vp()
        st = load().fr_lattice_build(self._h, _dev_ptr(P, "P"), P.shape[0], float(sigma),
                                     int(capacity_hint), ctypes.byref(h))
        self._check(st, "fr_lattice_build")
        return Lattice(self, h, P.shape[0])


class Lattice:
    def __init__(self, ctx: Context, h, n):
        self._ctx, self._h, self.n = ctx, h, n

    def close(self):
        if getattr(self, "_h", None):
            load().fr_lattice_destroy(self._ctx._h, self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        nv, cap, vd = _i64(), _i64(), ctypes.c_int32()
        self._ctx._check(load().fr_lattice_info(self._ctx._h, self._h, ctypes.byref(nv), ctypes.byref(cap),
                                                ctypes.byref(vd)), "fr_lattice_info")
        return nv.value, cap.value, vd.value

    def splat(self, V):
        import torch
        if not (isinstance(V, torch.Tensor) and V.is_cuda and V.dtype == torch.float32 and V.is_contiguous()
                and V.dim() == 2 and V.shape[0] == self.n):
            raise TypeError("values must be a contiguous float32 (n, val_dim) CUDA tensor")
        self._ctx._check(load().fr_lattice_splat(self._ctx._h, self._h, V.data_ptr(), V.shape[1]),
                         "fr_lattice_splat")

    def blur(self):
        self._ctx._check(load().fr_lattice_blur(self._ctx._h, self._h), "fr_lattice_blur")

    def slice(self, Q):
        import torch
        _, _, vd = self.info()
        out = torch.empty((Q.shape[0], vd), dtype=torch.float32, device=Q.device)
        self._ctx._check(load().fr_lattice_slice(self._ctx._h, self._h, _dev_ptr(Q, "Q"), Q.shape[0],
                                                 out.data_ptr()), "fr_lattice_slice")
        return out

    def vertices(self):
        import torch
        _, cap, vd = self.info()
        keys = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
        vals = torch.empty((cap, max(vd, 1)), dtype=torch.float32, device="cuda")
        nv = _i64()
        self._ctx._check(load().fr_lattice_vertices(self._ctx._h, self._h, keys.data_ptr(), vals.data_ptr(),
                                                    ctypes.byref(nv)), "fr_lattice_vertices")
        return keys[: nv.value], vals[: nv.value, :vd]


@dataclass
class ServeResult:
    status: int
    T: np.ndarray
    report: Report
    submit_ns: int
    admit_ns: int
    complete_ns: int

    @property
    def latency_ms(self) -> float:
        return (self.complete_ns - self.submit_ns) * 1e-6


class Server:
    """fr_server: continuous batching of rigid registrations on ctx's device.

    submit() borrows the given clouds (CUDA tensors, or host float32 arrays /
    tensors with host=True) until the request completes; this object keeps
    them alive until result() / wait() has returned the request."""

    def __init__(self, ctx: "Context", budget_bytes: int = 1 << 30, max_live: int = 256, **opts):
        L = load()
        self.ctx = ctx
        o = options(**opts)
        self.pt2pl = o.residual == FR_PT2PL
        h = _vp()
        st = L.fr_server_create(ctx._h, int(budget_bytes), int(max_live), ctypes.byref(o), ctypes.byref(h))
        ctx._check(st, "fr_server_create")
        self._h = h
        self._keep = {}

    def submit(self, X, Y, Yn=None, sigma_start=0.02, sigma_end=None, w=0.1, T0=None, host=False) -> int:
        L = load()
        r = fr_request()
        if host:
            arrs = [np.ascontiguousarray(a, dtype=np.float32) if a is not None else None for a in (X, Y, Yn)]
            for a, name in zip(arrs, ("X", "Y", "Yn")):
                if a is not None and (a.ndim != 2 or a.shape[1] != 4):
                    raise ValueError(f"{name} must be (n, 4) float32")
            ptr = lambda a: a.ctypes.data if a is not None else None
            r.X, r.Y, r.Yn = ptr(arrs[0]), ptr(arrs[1]), ptr(arrs[2])
            keep = arrs
        else:
            r.X, r.Y = _dev_ptr(X, "X"), _dev_ptr(Y, "Y")
            r.Yn = _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None
            keep = (X, Y, Yn)
        r.M, r.N = X.shape[0], Y.shape[0]
        r.sigma_start = float(sigma_start)
        r.sigma_end = float(sigma_start if sigma_end is None else sigma_end)
        r.w = float(w)
        T = _pose(T0)
        for i in range(16):
            r.T[i] = T.flat[i]
        r.host = 1 if host else 0
        t = ctypes.c_uint64()
        st = L.fr_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        self.ctx._check(st, "fr_server_submit")
        self._keep[t.value] = keep
        return t.value

    def _take(self, ticket, res):
        L = load()
        L.fr_server_release(self._h, ticket)
        self._keep.pop(ticket, None)
        return ServeResult(res.status, np.array(res.T[:]).reshape(4, 4), _report(res.report),
                           res.submit_ns, res.admit_ns, res.complete_ns)

    def poll(self, ticket):
        """The ServeResult once complete (the ticket is then released), else None."""
        L = load()
        done = ctypes.c_int()
        res = fr_result()
        st = L.fr_server_poll(self._h, ticket, ctypes.byref(done), ctypes.byref(res))
        self.ctx._check(st, "fr_server_poll")
        return self._take(ticket, res) if done.value else None

    def wait(self, ticket, timeout_ms: int = -1) -> ServeResult:
        L = load()
        res = fr_result()
        st = L.fr_server_wait(self._h, ticket, int(timeout_ms), ctypes.byref(res))
        self.ctx._check(st, "fr_server_wait")
        return self._take(ticket, res)

    def stats(self):
        L = load()
        a, b, c = _i64(), _i64(), _i64()
        L.fr_server_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"ticks": a.value, "completed": b.value, "kernel_launches": c.value}

    def close(self):
        if getattr(self, "_h", None):
            load().fr_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class NodeGraph:
    """fr_nodegraph: a node-graph model (Section 5.2) prepared on ctx's device.

    Xref (M,4) float32, knn (M,4) int32 and skw (M,4) float32 are CUDA
    tensors (copied by the library); node_pos (K,3) and edges (E,2) host
    arrays."""

    def __init__(self, ctx: "Context", Xref, knn, skw, node_pos, edges):
        import torch
        L = load()
        self.ctx = ctx
        for t, name, dt in ((knn, "knn", torch.int32), (skw, "skw", torch.float32)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()
                    and tuple(t.shape) == (Xref.shape[0], 4)):
                raise TypeError(f"{name} must be a contiguous (M, 4) {dt} CUDA tensor")
        self.node_pos = np.ascontiguousarray(node_pos, dtype=np.float64).reshape(-1, 3)
        self.edges = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
        self.K = self.node_pos.shape[0]
        self.M = Xref.shape[0]
        h = _vp()
        st = L.fr_nodegraph_create(ctx._h, _dev_ptr(Xref, "Xref"), knn.data_ptr(), skw.data_ptr(), self.M,
                                   self.node_pos.ctypes.data_as(_f64p), self.K,
                                   self.edges.ctypes.data if self.edges.size else None, self.edges.shape[0],
                                   ctypes.byref(h))
        ctx._check(st, "fr_nodegraph_create")
        self._h = h

    def _poses(self, node_T):
        if node_T is None:
            return np.ascontiguousarray(np.tile(np.eye(4), (self.K, 1, 1)))
        T = np.ascontiguousarray(node_T, dtype=np.float64).reshape(self.K, 4, 4).copy()
        return T

    def register(self, Y, Yn=None, node_T0=None, lam=10.0, pcg_iters=20, **opts):
        """EM registration; returns (node_T (K, 4, 4), Report)."""
        L = load()
        o = options(**opts)
        T = self._poses(node_T0)
        rep = fr_report()
        st = L.fr_register_nodegraph(self.ctx._h, self._h, _dev_ptr(Y, "Y"),
                                     _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None,
                                     Y.shape[0], ctypes.byref(o), float(lam), int(pcg_iters),
                                     T.ctypes.data_as(_f64p), ctypes.byref(rep))
        self.ctx._check(st, "fr_register_nodegraph")
        return T, _report(rep)

    def system(self, Y, Yn=None, node_T=None, lam=10.0, **opts):
        """(A (6K, 6K), g (6K), Report) of one E step at sigma_start."""
        L = load()
        o = options(**opts)
        T = self._poses(node_T)
        A = np.zeros((6 * self.K, 6 * self.K))
        g = np.zeros(6 * self.K)
        rep = fr_report()
        st = L.fr_nodegraph_system(self.ctx._h, self._h, _dev_ptr(Y, "Y"),
                                   _dev_ptr(Yn, "Yn", rows=Y.shape[0]) if Yn is not None else None,
                                   Y.shape[0], ctypes.byref(o), float(lam), T.ctypes.data_as(_f64p),
                                   A.ctypes.data_as(_f64p), g.ctypes.data_as(_f64p), ctypes.byref(rep))
        self.ctx._check(st, "fr_nodegraph_system")
        return A, g, _report(rep)

    def warp(self, node_T):
        """Warped model points (M, 4) float32 CUDA tensor (Eq. 21)."""
        import torch
        L = load()
        T = self._poses(node_T)
        out = torch.empty((self.M, 4), dtype=torch.float32, device="cuda")
        st = L.fr_nodegraph_warp(self.ctx._h, self._h, T.ctypes.data_as(_f64p), out.data_ptr())
        self.ctx._check(st, "fr_nodegraph_warp")
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().fr_nodegraph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
