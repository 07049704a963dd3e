"""FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow, single-threaded C restatement of the registration hot path
(exact Gaussian E step, reference permutohedral lattice, twist Gauss-Newton M
step, SE(3) exponential), written from the paper and kept independent of the
CUDA library: the two share no code, header, constant or helper and neither
imports the other.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
package.  The product path never calls it.

This module is argument marshalling only (numpy <-> ctypes); every number is
computed by the C sources beside it, compiled with ``-ffp-contract=off`` so
that the float lattice embedding is evaluated exactly as written.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["estep.c", "lattice.c", "se3.c", "rigid.c", "articulated.c", "nodegraph.c", "lattice_d.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_LIB_PATH = os.path.join(_HERE, "liboracle_omp.so")
_CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-function", "-Wno-unknown-pragmas"]

PT2PT, PT2PL = 0, 1
EXACT, LATTICE = 0, 1


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (idempotent): ``oracle/liboracle.so``, one
    thread, or with ``openmp`` ``oracle/liboracle_omp.so`` (-fopenmp: the same
    sources, per-point loops in parallel, bit-identical results)."""
    path = _OMP_LIB_PATH if openmp else _LIB_PATH
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(path):
        if os.path.getmtime(path) >= max(os.path.getmtime(d) for d in deps):
            return path
    tmp = path + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *_CFLAGS, *(["-fopenmp"] if openmp else []), "-o", tmp, *srcs, "-lm"], check=True)
    os.replace(tmp, path)
    return path


_libs = {}
_parallel = False


def _load(openmp: bool):
    if openmp not in _libs:
        L = ctypes.CDLL(build(openmp=openmp))
        _declare(L)
        _libs[openmp] = L
    return _libs[openmp]


def _L():
    return _load(_parallel)


def set_parallel(on: bool, threads: int | None = None) -> None:
    """Route later calls to the OpenMP build (on) or the single-thread one;
    threads > 0 sets the OpenMP build's thread count."""
    global _parallel
    _parallel = bool(on)
    if on and threads:
        _load(True).or_set_threads(int(threads))


def num_threads() -> int:
    """Threads the calls currently routed use (1 for the single-thread build)."""
    return int(_L().or_num_threads())


_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)


class _Options(ctypes.Structure):
    _fields_ = [("backend", ctypes.c_int), ("residual", ctypes.c_int), ("blur", ctypes.c_int),
                ("iters", ctypes.c_int), ("sigma_start", ctypes.c_double),
                ("sigma_end", ctypes.c_double), ("w", ctypes.c_double),
                ("renormalize_normals", ctypes.c_int), ("stop_twist", ctypes.c_double),
                ("update_sigma", ctypes.c_int)]


class _Report(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int), ("degenerate_iters", ctypes.c_int),
                ("last_inliers", ctypes.c_int64), ("last_sum_w", ctypes.c_double),
                ("last_cost", ctypes.c_double), ("last_twist_norm", ctypes.c_double),
                ("sigma_next", ctypes.c_double), ("last_sigma", ctypes.c_double)]


def _declare(L):
    L.or_estep_exact.argtypes = [_f32p, ctypes.c_int64, _f32p, _f32p, ctypes.c_int64,
                                 ctypes.c_double, _f64p, _f64p, _f64p]
    L.or_lattice_feature_scale.argtypes = [ctypes.c_float, _f32p]
    L.or_lattice_embed.argtypes = [_f32p, ctypes.c_int64, ctypes.c_float, _i32p, _f32p, _f32p, _i32p]
    L.or_lattice_embed.restype = ctypes.c_int
    L.or_lattice_build.argtypes = [_f32p, _f64p, ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                   ctypes.POINTER(ctypes.c_int)]
    L.or_lattice_build.restype = ctypes.c_void_p
    L.or_lattice_blur.argtypes = [ctypes.c_void_p]
    L.or_lattice_slice.argtypes = [ctypes.c_void_p, _f32p, ctypes.c_int64, _f64p]
    L.or_lattice_slice.restype = ctypes.c_int
    L.or_lattice_size.argtypes = [ctypes.c_void_p]
    L.or_lattice_size.restype = ctypes.c_int64
    L.or_lattice_vdim.argtypes = [ctypes.c_void_p]
    L.or_lattice_vertices.argtypes = [ctypes.c_void_p, _i32p, _f64p]
    L.or_lattice_free.argtypes = [ctypes.c_void_p]
    L.or_kernel_mass.argtypes = [ctypes.c_int, ctypes.c_int]
    L.or_kernel_mass.restype = ctypes.c_double
    L.or_sigma_schedule.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, _f32p]
    L.or_se3_exp.argtypes = [_f64p, _f64p]
    L.or_se3_log.argtypes = [_f64p, _f64p]
    L.or_cholesky_solve.argtypes = [ctypes.c_int, _f64p, _f64p, _f64p]
    L.or_cholesky_solve.restype = ctypes.c_int
    L.or_point_terms.argtypes = [_f64p, ctypes.c_double, _f64p, _f64p, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, ctypes.c_int, _f64p, _f64p, _f64p]
    L.or_point_terms.restype = ctypes.c_int
    L.or_outlier_constant.argtypes = [ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int]
    L.or_outlier_constant.restype = ctypes.c_double
    L.or_register_rigid.argtypes = [_f32p, ctypes.c_int64, _f32p, _f32p, ctypes.c_int64,
                                    ctypes.POINTER(_Options), _f64p, ctypes.POINTER(_Report)]
    L.or_register_rigid.restype = ctypes.c_int
    L.or_estep.argtypes = [_f32p, ctypes.c_int64, _f32p, _f32p, ctypes.c_int64, ctypes.c_int,
                           ctypes.c_int, ctypes.c_double, _f64p, _f64p]
    L.or_estep.restype = ctypes.c_int
    L.or_align_error.argtypes = [_f32p, ctypes.c_int64, _f64p, _f64p]
    L.or_align_error.restype = ctypes.c_double
    L.or_num_threads.argtypes = []
    L.or_num_threads.restype = ctypes.c_int
    L.or_set_threads.argtypes = [ctypes.c_int]
    L.or_set_threads.restype = None
    if hasattr(L, "or_register_articulated"):
        _declare_articulated(L)
        _declare_nodegraph(L)
    _declare_features(L)


def _pts(a) -> np.ndarray:
    """Points as a C-contiguous float32 (n, 4) array (a 4th column of zeros is added to (n, 3))."""
    a = np.asarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] not in (3, 4):
        raise ValueError("points must have shape (n, 3) or (n, 4)")
    if a.shape[1] == 3:
        a = np.concatenate([a, np.zeros((a.shape[0], 1), np.float32)], axis=1)
    return np.ascontiguousarray(a)


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class OracleError(RuntimeError):
    pass


def _check(status, what):
    if status != 0:
        raise OracleError(f"{what}: oracle status {status}")


# ---- E step -----------------------------------------------------------------

def estep_exact(X, Y, Yn=None, sigma=0.02):
    """Exact unnormalised Gaussian sums (Eq. 6, Eq. 9 numerator): M0 (M,), M1 (M,3), Ns (M,3)."""
    X, Y = _pts(X), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    M = X.shape[0]
    M0 = np.zeros(M, np.float64)
    M1 = np.zeros((M, 3), np.float64)
    Ns = np.zeros((M, 3), np.float64)
    _L().or_estep_exact(_p(X, _f32p), M, _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0], float(sigma),
                        _p(M0, _f64p), _p(M1, _f64p), _p(Ns, _f64p))
    return M0, M1, (Ns if Yn is not None else None)


def estep(X, Y, Yn=None, sigma=0.02, T=None, backend=LATTICE, blur=False):
    """E-step sums at T*X: (M, 4) [M0, M1] or (M, 7) [M0, M1, Ns] when normals are given."""
    X, Y = _pts(X), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    T = np.ascontiguousarray(np.eye(4) if T is None else T, dtype=np.float64)
    vdim = 7 if Yn is not None else 4
    out = np.zeros((X.shape[0], vdim), np.float64)
    _check(_L().or_estep(_p(X, _f32p), X.shape[0], _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0],
                         backend, int(blur), float(sigma), _p(T, _f64p), _p(out, _f64p)), "estep")
    return out


# ---- lattice ----------------------------------------------------------------

def feature_scale(sigma: float) -> np.ndarray:
    s = np.zeros(3, np.float32)
    _L().or_lattice_feature_scale(ctypes.c_float(sigma), _p(s, _f32p))
    return s


def lattice_embed(P, sigma):
    """Per point: keys (n,4,4) int32 [vertex k][coordinate j], bary (n,4), z (n,4), rank (n,4)."""
    P = _pts(P)
    n = P.shape[0]
    keys = np.zeros((n, 4, 4), np.int32)
    bary = np.zeros((n, 4), np.float32)
    z = np.zeros((n, 4), np.float32)
    rank = np.zeros((n, 4), np.int32)
    st = _L().or_lattice_embed(_p(P, _f32p), n, ctypes.c_float(sigma), _p(keys, _i32p),
                               _p(bary, _f32p), _p(z, _f32p), _p(rank, _i32p))
    return keys, bary, z, rank, st


class Lattice:
    """The reference lattice: a key-sorted vertex array with double values."""

    def __init__(self, P, V, sigma, blur=False):
        P = _pts(P)
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.ndim == 1:
            V = V[:, None].copy()
        st = ctypes.c_int(0)
        self._lib = _L()
        self._h = self._lib.or_lattice_build(_p(P, _f32p), _p(V, _f64p), P.shape[0], V.shape[1],
                                        ctypes.c_float(sigma), ctypes.byref(st))
        if not self._h:
            raise OracleError(f"lattice build failed ({st.value})")
        self.status = st.value
        self.vdim = V.shape[1]
        self.sigma = sigma
        if blur:
            self._lib.or_lattice_blur(self._h)

    def __del__(self):
        h = getattr(self, "_h", None)
        lib = getattr(self, "_lib", None)
        if h and lib is not None:
            lib.or_lattice_free(h)
            self._h = None

    def __len__(self):
        return int(self._lib.or_lattice_size(self._h))

    def slice(self, Q):
        Q = _pts(Q)
        out = np.zeros((Q.shape[0], self.vdim), np.float64)
        st = self._lib.or_lattice_slice(self._h, _p(Q, _f32p), Q.shape[0], _p(out, _f64p))
        return out, st

    def vertices(self):
        nv = len(self)
        keys = np.zeros((nv, 4), np.int32)
        vals = np.zeros((nv, self.vdim), np.float64)
        self._lib.or_lattice_vertices(self._h, _p(keys, _i32p), _p(vals, _f64p))
        return keys, vals


def kernel_mass(backend=LATTICE, blur=False) -> float:
    return float(_L().or_kernel_mass(backend, int(blur)))


def lattice_kernel_variance() -> float:
    L = _L()
    L.or_lattice_kernel_variance.argtypes = []
    L.or_lattice_kernel_variance.restype = ctypes.c_double
    return float(L.or_lattice_kernel_variance())


# ---- feature-space E step (d-dimensional lattice) ------------------------------

FEATURE_DMAX = 7


def _declare_features(L):
    L.or_feature_scale.argtypes = [ctypes.c_int, _f32p, _f32p]
    L.or_feature_scale.restype = None
    L.or_feature_embed.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _f32p, _i32p, _f32p]
    L.or_feature_embed.restype = ctypes.c_int
    L.or_flattice_build.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _f32p, _f64p, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
    L.or_flattice_build.restype = ctypes.c_void_p
    L.or_flattice_slice.argtypes = [ctypes.c_void_p, _f32p, ctypes.c_int64, _f64p]
    L.or_flattice_slice.restype = ctypes.c_int
    L.or_flattice_size.argtypes = [ctypes.c_void_p]
    L.or_flattice_size.restype = ctypes.c_int64
    L.or_flattice_vertices.argtypes = [ctypes.c_void_p, _i32p, _f64p]
    L.or_flattice_vertices.restype = None
    L.or_flattice_free.argtypes = [ctypes.c_void_p]
    L.or_flattice_free.restype = None
    L.or_estep_features.argtypes = [_f32p, ctypes.c_int64, _f32p, ctypes.c_int64, ctypes.c_int, _f32p,
                                    _f32p, _f32p, ctypes.c_int, _f64p]
    L.or_estep_features.restype = ctypes.c_int
    L.or_feature_kernel_mass.argtypes = [ctypes.c_int]
    L.or_feature_kernel_mass.restype = ctypes.c_double


def _feats(F, d=None) -> np.ndarray:
    F = np.ascontiguousarray(F, dtype=np.float32)
    if F.ndim != 2 or not 1 <= F.shape[1] <= FEATURE_DMAX or (d is not None and F.shape[1] != d):
        raise ValueError(f"features must have shape (n, d), 1 <= d <= {FEATURE_DMAX}")
    return F


def feature_scales(sigma_f) -> np.ndarray:
    """Per-axis float scale alpha / sqrt(i (i+1)) / sigma_f[i-1] of the d-dimensional elevation."""
    sf = np.ascontiguousarray(sigma_f, dtype=np.float32).reshape(-1)
    s = np.zeros(sf.shape[0], np.float32)
    _L().or_feature_scale(sf.shape[0], _p(sf, _f32p), _p(s, _f32p))
    return s


def feature_embed(F, sigma_f):
    """Per feature row: keys (n, d+1, d+1) int32 [vertex k][coordinate j] and bary (n, d+1)."""
    F = _feats(F)
    n, d = F.shape
    s = feature_scales(sigma_f)
    keys = np.zeros((n, d + 1, d + 1), np.int32)
    bary = np.zeros((n, d + 1), np.float32)
    st = _L().or_feature_embed(_p(F, _f32p), n, d, _p(s, _f32p), _p(keys, _i32p), _p(bary, _f32p))
    return keys, bary, st


class FeatureLattice:
    """The d-dimensional reference lattice: key-sorted vertices with double values."""

    def __init__(self, F, V, sigma_f):
        F = _feats(F)
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.ndim == 1:
            V = V[:, None].copy()
        self.d = F.shape[1]
        self.vdim = V.shape[1]
        s = feature_scales(sigma_f)
        st = ctypes.c_int(0)
        self._lib = _L()
        self._h = self._lib.or_flattice_build(_p(F, _f32p), F.shape[0], self.d, _p(s, _f32p), _p(V, _f64p),
                                              self.vdim, ctypes.byref(st))
        if not self._h:
            raise OracleError(f"feature lattice build failed ({st.value})")
        self.status = st.value

    def __del__(self):
        h = getattr(self, "_h", None)
        lib = getattr(self, "_lib", None)
        if h and lib is not None:
            lib.or_flattice_free(h)
            self._h = None

    def __len__(self):
        return int(self._lib.or_flattice_size(self._h))

    def slice(self, Q):
        Q = _feats(Q, self.d)
        out = np.zeros((Q.shape[0], self.vdim), np.float64)
        st = self._lib.or_flattice_slice(self._h, _p(Q, _f32p), Q.shape[0], _p(out, _f64p))
        return out, st

    def vertices(self):
        nv = len(self)
        keys = np.zeros((nv, self.d + 1), np.int32)
        vals = np.zeros((nv, self.vdim), np.float64)
        self._lib.or_flattice_vertices(self._h, _p(keys, _i32p), _p(vals, _f64p))
        return keys, vals


def estep_features(FX, FY, sigma_f, Y, Yn=None, backend=LATTICE):
    """Feature-space E-step sums at the model features FX: (M, 4) [M0, M1] or (M, 7) with normals.

    The kernel is exp(-sum_c (fx_c - fy_c)^2 / (2 sigma_c^2)) between feature rows; the values
    splatted are the observation points Y (and normals Yn)."""
    FX, FY = _feats(FX), _feats(FY)
    if FX.shape[1] != FY.shape[1]:
        raise ValueError("model and observation features differ in dimension")
    d = FX.shape[1]
    sf = np.ascontiguousarray(sigma_f, dtype=np.float32).reshape(-1)
    if sf.shape[0] != d:
        raise ValueError("sigma_f needs one entry per feature channel")
    Y = _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    if Y.shape[0] != FY.shape[0] or (Yn is not None and Yn.shape[0] != FY.shape[0]):
        raise ValueError("observation points and features differ in count")
    vdim = 7 if Yn is not None else 4
    out = np.zeros((FX.shape[0], vdim), np.float64)
    _check(_L().or_estep_features(_p(FX, _f32p), FX.shape[0], _p(FY, _f32p), FY.shape[0], d, _p(sf, _f32p),
                                  _p(Y, _f32p), _p(Yn, _f32p), backend, _p(out, _f64p)), "estep_features")
    return out


def feature_kernel_mass(d: int) -> float:
    """Integral of the unnormalised splat+slice kernel over normalised feature space."""
    return float(_L().or_feature_kernel_mass(int(d)))


def sigma_schedule(s0, s1, iters) -> np.ndarray:
    out = np.zeros(max(iters, 1), np.float32)
    _L().or_sigma_schedule(float(s0), float(s1), int(iters), _p(out, _f32p))
    return out[:iters]


# ---- M step -----------------------------------------------------------------

def se3_exp(zeta) -> np.ndarray:
    z = np.ascontiguousarray(zeta, dtype=np.float64)
    T = np.zeros((4, 4), np.float64)
    _L().or_se3_exp(_p(z, _f64p), _p(T, _f64p))
    return T


def se3_log(T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    z = np.zeros(6, np.float64)
    _L().or_se3_log(_p(T, _f64p), _p(z, _f64p))
    return z


def cholesky_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    st = _L().or_cholesky_solve(A.shape[0], _p(A, _f64p), _p(b, _f64p), _p(x, _f64p))
    return (x if st == 0 else None)


def point_terms(x, M0, M1, Ns=None, c_eff=0.0, sigma=1.0, residual=PT2PT, renormalize=False):
    """(W, r (rows,), J (rows, 6)) for one model point; rows = 3 (pt2pt), 1 (pt2pl) or 0."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    M1 = np.ascontiguousarray(M1, dtype=np.float64)
    Ns = np.ascontiguousarray(np.zeros(3) if Ns is None else Ns, dtype=np.float64)
    W = np.zeros(1)
    r = np.zeros(3)
    J = np.zeros(18)
    rows = _L().or_point_terms(_p(x, _f64p), float(M0), _p(M1, _f64p), _p(Ns, _f64p),
                               float(c_eff), float(sigma), int(residual), int(renormalize),
                               _p(W, _f64p), _p(r, _f64p), _p(J, _f64p))
    return float(W[0]), r[:rows].copy(), J[:6 * rows].reshape(rows, 6).copy()


def outlier_constant(w, N, M, sigma, backend=LATTICE, blur=False) -> float:
    return float(_L().or_outlier_constant(float(w), int(N), int(M), float(sigma), backend, int(blur)))


@dataclass
class Report:
    iters_run: int
    degenerate_iters: int
    last_inliers: int
    last_sum_w: float
    last_cost: float
    last_twist_norm: float
    sigma_next: float = 0.0   # update_sigma: the next iteration's sigma before the floor
    last_sigma: float = 0.0   # sigma of the last iteration run


def register_rigid(X, Y, Yn=None, *, sigma=0.02, sigma_end=None, w=0.1, iters=30,
                   residual=PT2PT, backend=LATTICE, blur=False, renormalize_normals=False,
                   stop_twist=0.0, T0=None, update_sigma=False):
    """Rigid EM registration; returns (T (4,4) float64, Report).  With
    update_sigma, sigma starts at `sigma` and is re-estimated each iteration
    (floor: sigma_end)."""
    X, Y = _pts(X), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    T = np.ascontiguousarray(np.eye(4) if T0 is None else T0, dtype=np.float64).copy()
    o = _Options(backend, residual, int(blur), int(iters), float(sigma),
                 float(sigma if sigma_end is None else sigma_end), float(w),
                 int(renormalize_normals), float(stop_twist), int(bool(update_sigma)))
    rep = _Report()
    st = _L().or_register_rigid(_p(X, _f32p), X.shape[0], _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0],
                                ctypes.byref(o), _p(T, _f64p), ctypes.byref(rep))
    _check(st, "register_rigid")
    return T, Report(rep.iters_run, rep.degenerate_iters, rep.last_inliers, rep.last_sum_w,
                     rep.last_cost, rep.last_twist_norm, rep.sigma_next, rep.last_sigma)


def rigid_normal_equations(X, Y, Yn=None, *, sigma, M_total=None, T=None, w=0.1, residual=PT2PT,
                           backend=LATTICE, blur=False, renormalize_normals=False) -> np.ndarray:
    """One EM iteration's normal equations of the shard X of a model of M_total
    points at pose T: (30,) = A's upper triangle row by row, b, sum_w, cost, inliers."""
    X, Y = _pts(X), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    T = np.ascontiguousarray(np.eye(4) if T is None else T, dtype=np.float64)
    o = _Options(backend, residual, int(blur), 1, float(sigma), float(sigma), float(w),
                 int(renormalize_normals), 0.0, 0)
    ne = np.zeros(30, np.float64)
    L = _L()
    L.or_rigid_normal_equations.argtypes = [_f32p, ctypes.c_int64, _f32p, _f32p, ctypes.c_int64,
                                            ctypes.POINTER(_Options), ctypes.c_int64, _f64p, _f64p]
    _check(L.or_rigid_normal_equations(_p(X, _f32p), X.shape[0], _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0],
                                       ctypes.byref(o), int(M_total or X.shape[0]), _p(T, _f64p),
                                       _p(ne, _f64p)), "rigid_normal_equations")
    return ne


def align_error(X, T, Tgt) -> float:
    """Eq. 22: mean |(T - T_gt) x_ref|."""
    X = _pts(X)
    T = np.ascontiguousarray(T, dtype=np.float64)
    Tgt = np.ascontiguousarray(Tgt, dtype=np.float64)
    return float(_L().or_align_error(_p(X, _f32p), X.shape[0], _p(T, _f64p), _p(Tgt, _f64p)))


class _Kintree(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("nj", ctypes.c_int), ("parent", _i32p), ("offset", _f64p),
                ("joint_body", _i32p), ("joint_axis", _f64p), ("q_min", _f64p), ("q_max", _f64p)]


def _declare_articulated(L):
    kp = ctypes.POINTER(_Kintree)
    L.or_fk.argtypes = [kp, _f64p, _f64p, _f64p, _f64p, _f64p]
    L.or_fk.restype = ctypes.c_int
    L.or_spatial_jacobian.argtypes = [kp, _f64p, _f64p, ctypes.c_int, _f64p]
    L.or_spatial_jacobian.restype = ctypes.c_int
    L.or_articulated_normal_equations.argtypes = [_f32p, _i32p, ctypes.c_int64, kp, _f32p, _f32p,
                                                  ctypes.c_int64, ctypes.POINTER(_Options),
                                                  ctypes.c_double, _f64p, _f64p, _f64p, _f64p]
    L.or_articulated_normal_equations.restype = ctypes.c_int
    L.or_register_articulated.argtypes = [_f32p, _i32p, ctypes.c_int64, kp, _f32p, _f32p,
                                          ctypes.c_int64, ctypes.POINTER(_Options), _f64p, _f64p,
                                          ctypes.POINTER(_Report)]
    L.or_register_articulated.restype = ctypes.c_int


def _tree(tree):
    """(struct, keep-alive arrays) from an object with parent, offset, joint_body,
    joint_axis, q_min, q_max (numpy arrays, see paper_1811_10136_gb300.synth.KinTree)."""
    arrs = dict(parent=np.ascontiguousarray(tree.parent, dtype=np.int32),
                offset=np.ascontiguousarray(tree.offset, dtype=np.float64).reshape(-1, 16),
                joint_body=np.ascontiguousarray(tree.joint_body, dtype=np.int32),
                joint_axis=np.ascontiguousarray(tree.joint_axis, dtype=np.float64).reshape(-1, 3),
                q_min=np.ascontiguousarray(tree.q_min, dtype=np.float64),
                q_max=np.ascontiguousarray(tree.q_max, dtype=np.float64))
    st = _Kintree(len(arrs["parent"]), len(arrs["joint_body"]), _p(arrs["parent"], _i32p),
                  _p(arrs["offset"], _f64p), _p(arrs["joint_body"], _i32p),
                  _p(arrs["joint_axis"], _f64p), _p(arrs["q_min"], _f64p), _p(arrs["q_max"], _f64p))
    return st, arrs


def fk(tree, root_T, q):
    """Body transforms (nb, 4, 4), joint world axes (nj, 3) and points (nj, 3)."""
    st, keep = _tree(tree)
    root_T = np.ascontiguousarray(root_T, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    T = np.zeros((st.nb, 4, 4))
    aw = np.zeros((max(st.nj, 1), 3))
    pw = np.zeros((max(st.nj, 1), 3))
    _check(_L().or_fk(ctypes.byref(st), _p(root_T, _f64p), _p(q, _f64p), _p(T, _f64p),
                      _p(aw, _f64p), _p(pw, _f64p)), "fk")
    return T, aw[: st.nj], pw[: st.nj]


def spatial_jacobian(tree, aw, pw, b):
    st, keep = _tree(tree)
    aw = np.ascontiguousarray(aw, dtype=np.float64)
    pw = np.ascontiguousarray(pw, dtype=np.float64)
    J = np.zeros((6, 6 + st.nj))
    _L().or_spatial_jacobian(ctypes.byref(st), _p(aw, _f64p), _p(pw, _f64p), int(b), _p(J, _f64p))
    return J


def _opts(sigma, sigma_end, w, iters, residual, backend, blur, renormalize_normals=False,
          stop_twist=0.0):
    return _Options(backend, residual, int(blur), int(iters), float(sigma),
                    float(sigma if sigma_end is None else sigma_end), float(w),
                    int(renormalize_normals), float(stop_twist))


def articulated_normal_equations(Xref, body, tree, Y, Yn=None, *, sigma, w=0.1, residual=PT2PT,
                                 backend=LATTICE, blur=False, root_T=None, q=None):
    """(A, g) of Algorithm 1 for one E step at (root_T, q)."""
    st, keep = _tree(tree)
    Xref, Y = _pts(Xref), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    body = np.ascontiguousarray(body, dtype=np.int32)
    root_T = np.ascontiguousarray(np.eye(4) if root_T is None else root_T, dtype=np.float64)
    q = np.ascontiguousarray(np.zeros(st.nj) if q is None else q, dtype=np.float64)
    nd = 6 + st.nj
    A = np.zeros((nd, nd))
    g = np.zeros(nd)
    o = _opts(sigma, sigma, w, 1, residual, backend, blur)
    _check(_L().or_articulated_normal_equations(_p(Xref, _f32p), _p(body, _i32p), Xref.shape[0],
                                                ctypes.byref(st), _p(Y, _f32p), _p(Yn, _f32p),
                                                Y.shape[0], ctypes.byref(o), float(sigma),
                                                _p(root_T, _f64p), _p(q, _f64p), _p(A, _f64p),
                                                _p(g, _f64p)), "articulated_normal_equations")
    return A, g


def register_articulated(Xref, body, tree, Y, Yn=None, *, sigma=0.01, sigma_end=None, w=0.1,
                         iters=15, residual=PT2PT, backend=LATTICE, blur=False, root_T0=None,
                         q0=None, stop_twist=0.0):
    """Articulated EM registration; returns (root_T (4,4), q (nj,), Report)."""
    st, keep = _tree(tree)
    Xref, Y = _pts(Xref), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    body = np.ascontiguousarray(body, dtype=np.int32)
    root_T = np.ascontiguousarray(np.eye(4) if root_T0 is None else root_T0, dtype=np.float64).copy()
    q = np.ascontiguousarray(np.zeros(st.nj) if q0 is None else q0, dtype=np.float64).copy()
    o = _opts(sigma, sigma_end, w, iters, residual, backend, blur, stop_twist=stop_twist)
    rep = _Report()
    _check(_L().or_register_articulated(_p(Xref, _f32p), _p(body, _i32p), Xref.shape[0],
                                        ctypes.byref(st), _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0],
                                        ctypes.byref(o), _p(root_T, _f64p), _p(q, _f64p),
                                        ctypes.byref(rep)), "register_articulated")
    return root_T, q, Report(rep.iters_run, rep.degenerate_iters, rep.last_inliers, rep.last_sum_w,
                             rep.last_cost, rep.last_twist_norm)


# ---- node-graph model (Section 5.2, Eq. 21) ----------------------------------

class _NodeGraph(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("node_pos", _f64p), ("E", ctypes.c_int), ("edges", _i32p),
                ("lam", ctypes.c_double), ("pcg_iters", ctypes.c_int)]


def _declare_nodegraph(L):
    gp = ctypes.POINTER(_NodeGraph)
    L.or_dq_from_T.argtypes = [_f64p, _f64p]
    L.or_T_from_dq.argtypes = [_f64p, _f64p]
    L.or_dqb.argtypes = [_f64p, _i32p, _f32p, _f64p]
    L.or_nodegraph_warp.argtypes = [_f32p, _i32p, _f32p, ctypes.c_int64, ctypes.c_int, _f64p, _f64p]
    L.or_nodegraph_warp.restype = ctypes.c_int
    L.or_nodegraph_normal_equations.argtypes = [_f32p, _i32p, _f32p, ctypes.c_int64, gp, _f32p, _f32p,
                                                ctypes.c_int64, ctypes.POINTER(_Options), ctypes.c_double,
                                                _f64p, _f64p, _f64p, ctypes.POINTER(_Report)]
    L.or_nodegraph_normal_equations.restype = ctypes.c_int
    L.or_pcg_block_jacobi.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_int, _f64p]
    L.or_pcg_block_jacobi.restype = ctypes.c_int
    L.or_register_nodegraph.argtypes = [_f32p, _i32p, _f32p, ctypes.c_int64, gp, _f32p, _f32p,
                                        ctypes.c_int64, ctypes.POINTER(_Options), _f64p,
                                        ctypes.POINTER(_Report)]
    L.or_register_nodegraph.restype = ctypes.c_int


def _graph(node_pos, edges, lam, pcg_iters):
    pos = np.ascontiguousarray(node_pos, dtype=np.float64).reshape(-1, 3)
    e = np.ascontiguousarray(edges, dtype=np.int32).reshape(-1, 2)
    g = _NodeGraph(pos.shape[0], _p(pos, _f64p), e.shape[0], _p(e, _i32p), float(lam), int(pcg_iters))
    return g, (pos, e)


def _skin(knn, skw):
    return (np.ascontiguousarray(knn, dtype=np.int32).reshape(-1, 4),
            np.ascontiguousarray(skw, dtype=np.float32).reshape(-1, 4))


def dq_from_T(T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    dq = np.zeros(8)
    _L().or_dq_from_T(_p(T, _f64p), _p(dq, _f64p))
    return dq


def T_from_dq(dq) -> np.ndarray:
    dq = np.ascontiguousarray(dq, dtype=np.float64)
    T = np.zeros((4, 4))
    _L().or_T_from_dq(_p(dq, _f64p), _p(T, _f64p))
    return T


def dqb(node_dq, knn4, w4) -> np.ndarray:
    """Dual-quaternion blend of 4 nodes' poses (node_dq: K x 8)."""
    node_dq = np.ascontiguousarray(node_dq, dtype=np.float64)
    knn4 = np.ascontiguousarray(knn4, dtype=np.int32)
    w4 = np.ascontiguousarray(w4, dtype=np.float32)
    T = np.zeros((4, 4))
    _L().or_dqb(_p(node_dq, _f64p), _p(knn4, _i32p), _p(w4, _f32p), _p(T, _f64p))
    return T


def nodegraph_warp(Xref, knn, skw, node_T) -> np.ndarray:
    Xref = _pts(Xref)
    knn, skw = _skin(knn, skw)
    node_T = np.ascontiguousarray(node_T, dtype=np.float64).reshape(-1, 16)
    X = np.zeros((Xref.shape[0], 3))
    _check(_L().or_nodegraph_warp(_p(Xref, _f32p), _p(knn, _i32p), _p(skw, _f32p), Xref.shape[0],
                                  node_T.shape[0], _p(node_T, _f64p), _p(X, _f64p)), "nodegraph_warp")
    return X


def nodegraph_normal_equations(Xref, knn, skw, node_pos, edges, Y, Yn=None, *, sigma, w=0.1, lam=10.0,
                               residual=PT2PT, backend=LATTICE, node_T=None):
    """(A (6K, 6K), g (6K), Report) of one E step at the node poses."""
    Xref, Y = _pts(Xref), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    knn, skw = _skin(knn, skw)
    g_, keep = _graph(node_pos, edges, lam, 0)
    K = g_.K
    node_T = np.ascontiguousarray(np.tile(np.eye(4), (K, 1, 1)) if node_T is None else node_T,
                                  dtype=np.float64).reshape(K, 16)
    A = np.zeros((6 * K, 6 * K))
    g = np.zeros(6 * K)
    o = _opts(sigma, sigma, w, 1, residual, backend, False)
    rep = _Report()
    _check(_L().or_nodegraph_normal_equations(_p(Xref, _f32p), _p(knn, _i32p), _p(skw, _f32p),
                                              Xref.shape[0], ctypes.byref(g_), _p(Y, _f32p), _p(Yn, _f32p),
                                              Y.shape[0], ctypes.byref(o), float(sigma), _p(node_T, _f64p),
                                              _p(A, _f64p), _p(g, _f64p), ctypes.byref(rep)),
           "nodegraph_normal_equations")
    return A, g, Report(rep.iters_run, rep.degenerate_iters, rep.last_inliers, rep.last_sum_w,
                        rep.last_cost, rep.last_twist_norm)


def pcg_block_jacobi(A, b, iters) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    _check(_L().or_pcg_block_jacobi(b.shape[0] // 6, _p(A, _f64p), _p(b, _f64p), int(iters), _p(x, _f64p)),
           "pcg_block_jacobi")
    return x


def register_nodegraph(Xref, knn, skw, node_pos, edges, Y, Yn=None, *, sigma=0.02, sigma_end=None, w=0.1,
                       lam=10.0, pcg_iters=20, iters=10, residual=PT2PT, backend=LATTICE, node_T0=None,
                       stop_twist=0.0):
    """Node-graph EM registration; returns (node_T (K, 4, 4), Report)."""
    Xref, Y = _pts(Xref), _pts(Y)
    Yn = _pts(Yn) if Yn is not None else None
    knn, skw = _skin(knn, skw)
    g_, keep = _graph(node_pos, edges, lam, pcg_iters)
    K = g_.K
    node_T = np.ascontiguousarray(np.tile(np.eye(4), (K, 1, 1)) if node_T0 is None else node_T0,
                                  dtype=np.float64).reshape(K, 16).copy()
    o = _opts(sigma, sigma_end, w, iters, residual, backend, False, stop_twist=stop_twist)
    rep = _Report()
    _check(_L().or_register_nodegraph(_p(Xref, _f32p), _p(knn, _i32p), _p(skw, _f32p), Xref.shape[0],
                                      ctypes.byref(g_), _p(Y, _f32p), _p(Yn, _f32p), Y.shape[0],
                                      ctypes.byref(o), _p(node_T, _f64p), ctypes.byref(rep)),
           "register_nodegraph")
    return node_T.reshape(K, 4, 4), Report(rep.iters_run, rep.degenerate_iters, rep.last_inliers,
                                           rep.last_sum_w, rep.last_cost, rep.last_twist_norm)
