"""Thin ctypes binding of libcert.so (include/cert.h).  Argument marshalling only:
every step of the certificate loop runs in the library's CUDA kernels.

Device buffers are torch CUDA tensors (torch is used for device memory and
streams only); results come back as zero-copy torch views of the library's
device arrays.  The library must have been built in-tree
(``python -m paper_2606_18314_b300.build``); loading fails loudly otherwise --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# CERT_LIB_VARIANT=debug loads the build with device index checks (libcert_debug.so)
LIB_PATH = os.path.join(HERE, "libcert_debug.so" if os.environ.get("CERT_LIB_VARIANT") == "debug" else "libcert.so")

CERT_OK, CERT_EINVAL, CERT_ENOMEM, CERT_ECUDA, CERT_ETIMEOUT, CERT_EBOUND, CERT_ESTATE, CERT_EINTERNAL = range(8)
STATUS_NAMES = ["CERT_OK", "CERT_EINVAL", "CERT_ENOMEM", "CERT_ECUDA", "CERT_ETIMEOUT", "CERT_EBOUND",
                "CERT_ESTATE", "CERT_EINTERNAL"]
CERT_AUTO, CERT_INCREMENTAL, CERT_REBUILD, CERT_ALLPAIRS, CERT_THRESHOLD = range(5)
STRATEGY = {"auto": CERT_AUTO, "incremental": CERT_INCREMENTAL, "rebuild": CERT_REBUILD,
            "allpairs": CERT_ALLPAIRS, "threshold": CERT_THRESHOLD}


class cert_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_scenes", ctypes.c_int32),
                ("offsets", ctypes.POINTER(ctypes.c_int64)), ("n_total", ctypes.c_int64),
                ("cell_scale", ctypes.c_float), ("policy", ctypes.c_int32),
                ("bucket_factor", ctypes.c_int32), ("cell_quantile", ctypes.c_float),
                ("frontier_rule", ctypes.c_int32), ("audit", ctypes.c_int32)]


class cert_scene_result(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("H_cand", ctypes.c_double), ("eps_t", ctypes.c_float),
                ("med_c", ctypes.c_float), ("n_frontier", ctypes.c_int32),
                ("frontier_start", ctypes.c_int32), ("n_failed", ctypes.c_int32),
                ("n_missed", ctypes.c_int32), ("n_false", ctypes.c_int32),
                ("n_searched", ctypes.c_int32), ("failed_cells", ctypes.c_int32),
                ("frontier_cells", ctypes.c_int32), ("occupied_cells", ctypes.c_int32),
                ("strategy", ctypes.c_int32), ("pred_inc", ctypes.c_float), ("pred_reb", ctypes.c_float),
                ("grid_res", ctypes.c_int32), ("search_res", ctypes.c_int32),
                ("n_rho", ctypes.c_int32), ("n_rho_hit", ctypes.c_int32), ("gyration", ctypes.c_double),
                ("compactness", ctypes.c_double), ("search_cycles", ctypes.c_uint64),
                ("refresh_cycles", ctypes.c_uint64)]


SCENE_DTYPE = np.dtype([(n, np.dtype(t).newbyteorder("=")) for n, t in [
    ("H", np.float64), ("H_cand", np.float64), ("eps_t", np.float32), ("med_c", np.float32),
    ("n_frontier", np.int32), ("frontier_start", np.int32), ("n_failed", np.int32),
    ("n_missed", np.int32), ("n_false", np.int32), ("n_searched", np.int32),
    ("failed_cells", np.int32), ("frontier_cells", np.int32), ("occupied_cells", np.int32),
    ("strategy", np.int32), ("pred_inc", np.float32), ("pred_reb", np.float32),
    ("grid_res", np.int32), ("search_res", np.int32), ("n_rho", np.int32), ("n_rho_hit", np.int32),
    ("gyration", np.float64), ("compactness", np.float64), ("search_cycles", np.uint64),
    ("refresh_cycles", np.uint64)]])
assert SCENE_DTYPE.itemsize == ctypes.sizeof(cert_scene_result)


class cert_knn_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("k", ctypes.c_int32), ("n", ctypes.c_int64),
                ("cell_scale", ctypes.c_float), ("reserved", ctypes.c_int32)]


class cert_knn_result(ctypes.Structure):
    _fields_ = [("eps_t", ctypes.c_float), ("n_frontier", ctypes.c_int32), ("n_failed", ctypes.c_int32),
                ("n_missed", ctypes.c_int32), ("n_false", ctypes.c_int32), ("n_searched", ctypes.c_int32),
                ("grid_res", ctypes.c_int32), ("strategy", ctypes.c_int32), ("grid_res_coarse", ctypes.c_int32),
                ("n_far", ctypes.c_int32)]


KNN_RESULT_FIELDS = [f for f, _ in cert_knn_result._fields_]


class cert_knn_views(ctypes.Structure):
    _fields_ = [("idx", ctypes.c_void_p), ("d2", ctypes.c_void_p), ("frontier", ctypes.c_void_p),
                ("failed", ctypes.c_void_p), ("result", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("k", ctypes.c_int32), ("dim", ctypes.c_int32)]


class cert_views(ctypes.Structure):
    _fields_ = [("nn", ctypes.c_void_p), ("d1sq", ctypes.c_void_p), ("d2sq", ctypes.c_void_p),
                ("cell", ctypes.c_void_p), ("frontier", ctypes.c_void_p), ("failed", ctypes.c_void_p),
                ("scenes", ctypes.c_void_p), ("n_total", ctypes.c_int64), ("n_scenes", ctypes.c_int32),
                ("dim", ctypes.c_int32)]


_lib = None

# every symbol include/cert.h declares (checked by the CPU tests)
EXPORTS = ["cert_knn_init", "cert_knn_step", "cert_knn_get_views", "cert_knn_sync_result", "cert_knn_destroy",
           "cert_knn_profile",
           "cert_init", "cert_step", "cert_step_host", "cert_step_host_stream", "cert_rebuild", "cert_get_views",
           "cert_sync_result", "cert_distances", "cert_allpairs", "cert_destroy", "cert_last_error",
           "cert_version", "cert_source_fingerprint", "cert_profile_begin", "cert_profile_end",
           "cert_allpairs_noalloc", "cert_set_cell_scale", "cert_set_cell_quantile", "cert_get_cell_scale", "cert_autotune",
           "cert_snapshot", "cert_restore", "cert_get_features", "cert_selector_load",
           "cert_mlp_workspace_bytes", "cert_mlp_forward", "cert_mlp_grad", "cert_mlp_adam",
           "cert_selftest_bounded_wait", "cert_set_step_path", "cert_get_step_path", "cert_set_scene_policy"]
MLP_PARAMS = 4866
CERT_FRONTIER_STEP, CERT_FRONTIER_POINT, CERT_FRONTIER_CLOCK = 0, 1, 2
FRONTIER_RULE = {"step": CERT_FRONTIER_STEP, "point": CERT_FRONTIER_POINT, "clock": CERT_FRONTIER_CLOCK}
N_PHASES = 8
PHASE_NAMES = ["clear", "prepare", "scan", "select", "scatter_refresh", "search", "finalize", "fused"]
CERT_PATH_AUTO, CERT_PATH_MULTI, CERT_PATH_FUSED = 0, 1, 2
STEP_PATH = {"auto": CERT_PATH_AUTO, "multi": CERT_PATH_MULTI, "fused": CERT_PATH_FUSED}


def lib():
    """Load libcert.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libcert.so not built ({LIB_PATH}); run python -m paper_2606_18314_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    L.cert_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(cert_config), vp, vp]
    L.cert_step.argtypes = [vp, vp, f32, i32, ctypes.POINTER(cert_views), vp]
    L.cert_step_host.argtypes = [vp, vp, f32, i32, vp, vp]
    L.cert_step_host_stream.argtypes = [vp, vp, i32, f32, i32, vp, vp]
    L.cert_step_host_stream.restype = ctypes.c_int
    L.cert_rebuild.argtypes = [vp, vp]
    L.cert_get_views.argtypes = [vp, ctypes.POINTER(cert_views)]
    L.cert_sync_result.argtypes = [vp, vp]
    L.cert_distances.argtypes = [vp, vp, vp, vp]
    L.cert_allpairs.argtypes = [vp, i64, i32, vp, i64, vp, vp, vp, vp]
    L.cert_destroy.argtypes = [vp]
    L.cert_destroy.restype = None
    L.cert_last_error.argtypes = [vp]
    L.cert_last_error.restype = ctypes.c_char_p
    L.cert_version.argtypes = []
    L.cert_version.restype = ctypes.c_char_p
    L.cert_set_cell_scale.argtypes = [vp, f32]
    L.cert_set_cell_quantile.argtypes = [vp, f32]
    L.cert_set_cell_quantile.restype = ctypes.c_int
    L.cert_get_cell_scale.argtypes = [vp]
    L.cert_get_cell_scale.restype = f32
    L.cert_autotune.argtypes = [vp, vp, i64, i32, f32, i32, vp, i32, vp, vp, vp]
    L.cert_snapshot.argtypes = [vp, vp]
    L.cert_restore.argtypes = [vp, vp]
    L.cert_get_features.argtypes = [vp, vp]
    L.cert_selector_load.argtypes = [vp, vp, vp]
    L.cert_set_scene_policy.argtypes = [vp, vp]
    L.cert_set_scene_policy.restype = ctypes.c_int
    L.cert_mlp_workspace_bytes.argtypes = [i64]
    L.cert_mlp_workspace_bytes.restype = ctypes.c_size_t
    L.cert_mlp_forward.argtypes = [vp, vp, vp, i64, vp, vp]
    L.cert_mlp_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, ctypes.c_size_t, vp]
    L.cert_mlp_adam.argtypes = [vp, vp, vp, vp, i32, f32, f32, f32, f32, vp]
    for name in ["cert_set_cell_scale", "cert_autotune", "cert_snapshot", "cert_restore", "cert_get_features",
                 "cert_selector_load", "cert_mlp_forward", "cert_mlp_grad", "cert_mlp_adam"]:
        getattr(L, name).restype = ctypes.c_int
    L.cert_profile_begin.argtypes = [vp, i32]
    L.cert_profile_end.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
    for name in ["cert_init", "cert_step", "cert_step_host", "cert_rebuild", "cert_get_views",
                 "cert_sync_result", "cert_distances", "cert_allpairs", "cert_profile_begin",
                 "cert_profile_end"]:
        getattr(L, name).restype = ctypes.c_int
    L.cert_knn_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(cert_knn_config), vp, vp]
    L.cert_knn_step.argtypes = [vp, vp, f32, i32, vp]
    L.cert_knn_get_views.argtypes = [vp, ctypes.POINTER(cert_knn_views)]
    L.cert_knn_profile.argtypes = [vp, vp, f32, i32, vp, vp]
    L.cert_knn_sync_result.argtypes = [vp, vp]
    L.cert_knn_destroy.argtypes = [vp]
    L.cert_knn_destroy.restype = None
    for name in ["cert_knn_init", "cert_knn_step", "cert_knn_get_views", "cert_knn_sync_result", "cert_knn_profile"]:
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


class CertError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code}: {msg}")
        self.code = code


def _check(code, ctx=None):
    if code != CERT_OK:
        msg = lib().cert_last_error(ctx).decode(errors="replace")
        raise CertError(code, msg)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype_name, shape_last=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if str(t.dtype) != dtype_name:
        raise TypeError(f"expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if shape_last is not None and (t.dim() != 2 or t.shape[1] != shape_last):
        raise ValueError(f"expected shape [n][{shape_last}]")
    return ctypes.c_void_p(t.data_ptr())


class _CudaArray:
    """__cuda_array_interface__ wrapper so torch can view a library buffer."""

    def __init__(self, ptr, shape, typestr, owner):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": tuple(shape),
                                         "typestr": typestr, "version": 3, "strides": None}
        self._owner = owner


def _view(ptr, shape, typestr, owner):
    import torch
    if any(s == 0 for s in shape):
        return torch.empty(shape, dtype={"<i4": torch.int32, "<f4": torch.float32, "|u1": torch.uint8}[typestr],
                           device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape, typestr, owner), device="cuda")


def cert_version() -> str:
    return lib().cert_version().decode()


def cert_source_fingerprint(unit: str):
    """Source fingerprint of one translation unit of the loaded library (None if unknown)."""
    fn = lib().cert_source_fingerprint
    fn.argtypes = [ctypes.c_char_p]
    fn.restype = ctypes.c_char_p
    r = fn(unit.encode())
    return r.decode() if r is not None else None


def cert_last_error(ctx=None) -> str:
    return lib().cert_last_error(ctx).decode(errors="replace")


def cert_allpairs(pos, queries=None, stream=None):
    """Exact top-2 of every point (or of the listed query indices) against all
    points of one set: returns (nn, d1sq, d2sq) as CUDA tensors."""
    import torch
    dim = pos.shape[1]
    pp = _dev_ptr(pos, "torch.float32", dim)
    n = pos.shape[0]
    if queries is not None:
        qp = _dev_ptr(queries, "torch.int32")
        nq = queries.shape[0]
    else:
        qp, nq = None, n
    nn = torch.empty(nq, dtype=torch.int32, device=pos.device)
    d1 = torch.empty(nq, dtype=torch.float32, device=pos.device)
    d2 = torch.empty(nq, dtype=torch.float32, device=pos.device)
    _check(lib().cert_allpairs(pp, n, dim, qp, nq, ctypes.c_void_p(nn.data_ptr()),
                               ctypes.c_void_p(d1.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                               _stream_ptr(stream)))
    return nn, d1, d2


def cert_allpairs_noalloc(pos, queries=None, nn=None, d1sq=None, d2sq=None, stream=None):
    """cert_allpairs_noalloc: the all-pairs top-2 using the library's fixed
    scratch array, so the call itself allocates nothing on the device.  For
    callers that must not allocate at all during the call, pass preallocated
    outputs (nn int32, d1sq/d2sq float32, length n or len(queries))."""
    import torch
    fn = lib().cert_allpairs_noalloc
    vp = ctypes.c_void_p
    fn.argtypes = [vp, ctypes.c_int64, ctypes.c_int32, vp, ctypes.c_int64, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    dim = pos.shape[1]
    pp = _dev_ptr(pos, "torch.float32", dim)
    n = pos.shape[0]
    if queries is not None:
        qp, nq = _dev_ptr(queries, "torch.int32"), queries.shape[0]
    else:
        qp, nq = None, n
    if nn is None:
        nn = torch.empty(nq, dtype=torch.int32, device=pos.device)
    if d1sq is None:
        d1sq = torch.empty(nq, dtype=torch.float32, device=pos.device)
    if d2sq is None:
        d2sq = torch.empty(nq, dtype=torch.float32, device=pos.device)
    _check(fn(pp, n, dim, qp, nq, vp(nn.data_ptr()), vp(d1sq.data_ptr()), vp(d2sq.data_ptr()),
              _stream_ptr(stream)))
    return nn, d1sq, d2sq


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def cert_selftest_bounded_wait(limit=1000):
    """Run the bounded-wait self-test; returns (status code, latched bits, polls)."""
    fn = lib().cert_selftest_bounded_wait
    fn.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    st, sp = ctypes.c_uint32(0), ctypes.c_uint32(0)
    rc = fn(int(limit), ctypes.byref(st), ctypes.byref(sp))
    return rc, int(st.value), int(sp.value)


def cert_mlp_workspace_bytes(n):
    return int(lib().cert_mlp_workspace_bytes(int(n)))


def cert_mlp_forward(params, norm, X, Y, stream=None):
    """Y[n][2] = selector(X[n][8]) on the device (all CUDA tensors, float32)."""
    _check(lib().cert_mlp_forward(_ptr(params), _ptr(norm), _ptr(X), X.shape[0], _ptr(Y), _stream_ptr(stream)))


def cert_mlp_grad(params, norm, X, T, grad, loss, work, stream=None):
    """grad = d mean((selector(X) - T)^2) / d params; loss -> loss[0]."""
    _check(lib().cert_mlp_grad(_ptr(params), _ptr(norm), _ptr(X), _ptr(T), X.shape[0], _ptr(grad), _ptr(loss),
                               _ptr(work), work.numel() * work.element_size(), _stream_ptr(stream)))


def cert_mlp_adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().cert_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(t), float(lr), float(beta1),
                               float(beta2), float(eps), _stream_ptr(stream)))


AUDIT = {"rho": 1, "geometry": 2, "cost": 4}    # cert_audit


def audit_flags(audit) -> int:
    """cert_audit flags from an int or names ("rho", "geometry", "cost")."""
    if isinstance(audit, (int, np.integer)):
        return int(audit)
    if isinstance(audit, str):
        audit = (audit,)
    return sum(AUDIT[a] for a in set(audit))


class Context:
    """A batch of scenes whose certificates are maintained on the GPU.

    ``Context(pos, offsets=None)`` calls ``cert_init``; ``step`` calls
    ``cert_step``; ``views`` exposes the per-point results as torch tensors
    (valid until the next call); ``sync`` calls ``cert_sync_result``.
    """

    def __init__(self, pos, offsets=None, cell_scale=0.0, policy=CERT_INCREMENTAL, stream=None,
                 bucket_factor=0, cell_quantile=0.0, frontier_rule="step", audit=(), path="auto"):
        import torch
        self.dim = int(pos.shape[1])
        self._keep = []
        cfg = cert_config()
        cfg.dim = self.dim
        if offsets is None:
            offsets = np.array([0, pos.shape[0]], np.int64)
        offsets = np.ascontiguousarray(offsets, np.int64)
        self.offsets = offsets
        cfg.n_scenes = len(offsets) - 1
        cfg.offsets = offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        cfg.n_total = int(offsets[-1])
        cfg.cell_scale = float(cell_scale)
        cfg.policy = int(policy)
        cfg.bucket_factor = int(bucket_factor)
        cfg.cell_quantile = float(cell_quantile)
        cfg.frontier_rule = FRONTIER_RULE[frontier_rule] if isinstance(frontier_rule, str) else int(frontier_rule)
        cfg.audit = audit_flags(audit)
        self.n_scenes = cfg.n_scenes
        self.n = cfg.n_total
        h = ctypes.c_void_p()
        if pos.shape[0] != cfg.n_total:
            raise ValueError("positions do not match the offsets")
        _check(lib().cert_init(ctypes.byref(h), ctypes.byref(cfg), _dev_ptr(pos, "torch.float32", self.dim),
                               _stream_ptr(stream)))
        self.h = h
        self.device = pos.device
        if path != "auto":
            self.set_step_path(path)

    def set_step_path(self, path):
        """cert_set_step_path: "auto", "multi" (one kernel per phase) or "fused" (one launch per step)."""
        fn = lib().cert_set_step_path
        fn.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        fn.restype = ctypes.c_int
        _check(fn(self.h, STEP_PATH[path] if isinstance(path, str) else int(path)), self.h)

    def step_path(self, strategy=CERT_INCREMENTAL):
        """The path ("multi" or "fused") the next step with this strategy takes."""
        fn = lib().cert_get_step_path
        fn.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        fn.restype = ctypes.c_int32
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        return {CERT_PATH_MULTI: "multi", CERT_PATH_FUSED: "fused"}[fn(self.h, int(strategy))]

    def close(self):
        if getattr(self, "h", None):
            lib().cert_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, pos_new, eps, strategy=CERT_INCREMENTAL, stream=None):
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        if pos_new.shape[0] != self.n:
            raise ValueError("positions do not match the context's point count")
        _check(lib().cert_step(self.h, _dev_ptr(pos_new, "torch.float32", self.dim), float(eps),
                               int(strategy), None, _stream_ptr(stream)), self.h)

    def step_host(self, pos_new_host: np.ndarray, eps, strategy=CERT_INCREMENTAL, stream=None):
        """cert_step_host: host positions in, per-scene scalars out (synchronous)."""
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        out = np.zeros(self.n_scenes, SCENE_DTYPE)
        a = pos_new_host
        if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous
                and a.shape == (self.n, self.dim)):
            raise ValueError("host positions must be C-contiguous float32 [n][dim]")
        _check(lib().cert_step_host(self.h, ctypes.c_void_p(a.ctypes.data), float(eps), int(strategy),
                                    ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)), self.h)
        return out

    def step_host_ptr(self, host_ptr: int, eps, strategy, out: np.ndarray, stream=None):
        """cert_step_host on a raw (pinned) host pointer; ``out`` receives the scalars."""
        _check(lib().cert_step_host(self.h, ctypes.c_void_p(host_ptr), float(eps), int(strategy),
                                    ctypes.c_void_p(out.ctypes.data), _stream_ptr(stream)), self.h)

    def step_host_stream(self, host_ptrs, eps, strategy, out: np.ndarray, stream=None):
        """cert_step_host_stream: one step per (pinned) host frame pointer in
        host_ptrs, copies pipelined against the steps; ``out``
        [len(host_ptrs) * n_scenes] receives each step's scalars."""
        n_steps = len(host_ptrs)
        if out is not None and out.size < n_steps * self.n_scenes:
            raise ValueError("out holds fewer than n_steps * n_scenes results")
        table = (ctypes.c_void_p * max(1, n_steps))(*[int(p) for p in host_ptrs])
        _check(lib().cert_step_host_stream(self.h, ctypes.cast(table, ctypes.c_void_p), int(n_steps), float(eps),
                                           int(strategy),
                                           ctypes.c_void_p(out.ctypes.data) if out is not None else None,
                                           _stream_ptr(stream)), self.h)

    def rebuild(self, stream=None):
        _check(lib().cert_rebuild(self.h, _stream_ptr(stream)), self.h)

    def views(self):
        v = cert_views()
        _check(lib().cert_get_views(self.h, ctypes.byref(v)), self.h)
        n = int(v.n_total)
        return {
            "nn": _view(v.nn, (n,), "<i4", self),
            "d1sq": _view(v.d1sq, (n,), "<f4", self),
            "d2sq": _view(v.d2sq, (n,), "<f4", self),
            "cell": _view(v.cell, (n,), "<i4", self),
            "frontier": _view(v.frontier, (n,), "<i4", self),
            "failed": _view(v.failed, (n,), "|u1", self),
        }

    def sync(self, raise_on_status=True):
        """cert_sync_result: per-scene scalars as a numpy structured array."""
        out = np.zeros(self.n_scenes, SCENE_DTYPE)
        rc = lib().cert_sync_result(self.h, ctypes.c_void_p(out.ctypes.data))
        if raise_on_status:
            _check(rc, self.h)
        return out, rc

    def distances(self, stream=None):
        import torch
        d1 = torch.empty(self.n, dtype=torch.float32, device=self.device)
        d2 = torch.empty(self.n, dtype=torch.float32, device=self.device)
        _check(lib().cert_distances(self.h, ctypes.c_void_p(d1.data_ptr()), ctypes.c_void_p(d2.data_ptr()),
                                    _stream_ptr(stream)), self.h)
        return d1, d2

    def profile_begin(self, max_steps):
        _check(lib().cert_profile_begin(self.h, int(max_steps)), self.h)
        self._prof_max = int(max_steps)

    def profile_end(self):
        """Per-step phase times in ms, shape [steps][N_PHASES]."""
        mx = getattr(self, "_prof_max", 0)
        out = np.zeros((max(mx, 1), N_PHASES), np.float32)
        n = ctypes.c_int32(0)
        _check(lib().cert_profile_end(self.h, ctypes.c_void_p(out.ctypes.data), mx, ctypes.byref(n)), self.h)
        return out[:n.value]

    # ---- tuning, snapshots, selector -------------------------------------------------
    def set_cell_scale(self, scale):
        _check(lib().cert_set_cell_scale(self.h, float(scale)), self.h)

    def set_cell_quantile(self, q):
        _check(lib().cert_set_cell_quantile(self.h, float(q)), self.h)

    def cell_scale(self):
        return float(lib().cert_get_cell_scale(self.h))

    def snapshot(self, stream=None):
        _check(lib().cert_snapshot(self.h, _stream_ptr(stream)), self.h)

    def restore(self, stream=None):
        _check(lib().cert_restore(self.h, _stream_ptr(stream)), self.h)

    def autotune(self, frames, eps, strategy=CERT_INCREMENTAL, scales=(2.0, 2.5, 3.0, 3.5, 4.0, 5.0), stream=None):
        """cert_autotune over consecutive device frames [F][n][dim]; returns (best, ms per scale)."""
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        sc = np.ascontiguousarray(scales, np.float32)
        ms = np.zeros(len(sc), np.float32)
        best = ctypes.c_float(0.0)
        stride = int(frames.shape[1] * frames.shape[2])
        _check(lib().cert_autotune(self.h, _dev_ptr(frames.reshape(-1, self.dim), "torch.float32", self.dim),
                                   stride, int(frames.shape[0]), float(eps), int(strategy),
                                   ctypes.c_void_p(sc.ctypes.data), len(sc), ctypes.c_void_p(ms.ctypes.data),
                                   ctypes.byref(best), _stream_ptr(stream)), self.h)
        return float(best.value), ms

    def features(self):
        """Selector features of the last step, [n_scenes][8] (synchronises)."""
        out = np.zeros((self.n_scenes, 8), np.float32)
        _check(lib().cert_get_features(self.h, ctypes.c_void_p(out.ctypes.data)), self.h)
        return out

    def set_scene_policy(self, policy=None):
        """cert_set_scene_policy: per-scene strategy under "auto" without a selector
        (a sequence of "incremental"/"rebuild" or CERT_* values; None clears)."""
        if policy is None:
            _check(lib().cert_set_scene_policy(self.h, None), self.h)
            return
        arr = np.ascontiguousarray([STRATEGY[p] if isinstance(p, str) else int(p) for p in policy], np.int32)
        _check(lib().cert_set_scene_policy(self.h, ctypes.c_void_p(arr.ctypes.data)), self.h)

    def load_selector(self, params, norm):
        """cert_selector_load: params[4866], norm[16] (host float32), or None to unload."""
        if params is None:
            _check(lib().cert_selector_load(self.h, None, None), self.h)
            return
        p = np.ascontiguousarray(params, np.float32)
        nm = np.ascontiguousarray(norm, np.float32)
        assert p.shape == (MLP_PARAMS,) and nm.shape == (16,)
        _check(lib().cert_selector_load(self.h, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(nm.ctypes.data)),
               self.h)


class KnnContext:
    """k-nearest-neighbour certificates of one point set (include/cert_knn.h).

    ``KnnContext(pos, k)`` calls ``cert_knn_init`` (exact k+1 nearest of every
    point); ``step`` calls ``cert_knn_step``; ``views`` gives the lists as
    torch tensors [k+1][n] (rank-major, valid until the next call) and the
    frontier / failure flags; ``sync`` returns the step's scalars as a dict.
    """

    def __init__(self, pos, k, cell_scale=0.0, stream=None):
        cfg = cert_knn_config()
        cfg.dim = int(pos.shape[1])
        cfg.k = int(k)
        cfg.n = int(pos.shape[0])
        cfg.cell_scale = float(cell_scale)
        self.dim, self.k, self.n = cfg.dim, cfg.k, cfg.n
        h = ctypes.c_void_p()
        _check(lib().cert_knn_init(ctypes.byref(h), ctypes.byref(cfg), _dev_ptr(pos, "torch.float32", self.dim),
                                   _stream_ptr(stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().cert_knn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, pos_new, eps, strategy=CERT_INCREMENTAL, stream=None):
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        if pos_new.shape[0] != self.n:
            raise ValueError("positions do not match the context's point count")
        _check(lib().cert_knn_step(self.h, _dev_ptr(pos_new, "torch.float32", self.dim), float(eps), int(strategy),
                                   _stream_ptr(stream)))

    KNN_PHASES = ("prepare", "scan", "refresh", "search", "finalize")

    def profile(self, pos_new, eps, strategy=CERT_INCREMENTAL, stream=None):
        """cert_knn_profile: one step with per-phase CUDA events (synchronises); ms per phase."""
        if isinstance(strategy, str):
            strategy = STRATEGY[strategy]
        ms = np.zeros(5, np.float32)
        _check(lib().cert_knn_profile(self.h, _dev_ptr(pos_new, "torch.float32", self.dim), float(eps),
                                      int(strategy), ctypes.c_void_p(ms.ctypes.data), _stream_ptr(stream)))
        return dict(zip(self.KNN_PHASES, [float(x) for x in ms]))

    def views(self):
        v = cert_knn_views()
        _check(lib().cert_knn_get_views(self.h, ctypes.byref(v)))
        n, k1 = int(v.n), int(v.k) + 1
        return {"idx": _view(v.idx, (k1, n), "<i4", self), "d2": _view(v.d2, (k1, n), "<f4", self),
                "frontier": _view(v.frontier, (n,), "|u1", self), "failed": _view(v.failed, (n,), "|u1", self)}

    def sync(self, raise_on_status=True):
        r = cert_knn_result()
        rc = lib().cert_knn_sync_result(self.h, ctypes.byref(r))
        if raise_on_status:
            _check(rc)
        return {f: getattr(r, f) for f in KNN_RESULT_FIELDS}, rc
