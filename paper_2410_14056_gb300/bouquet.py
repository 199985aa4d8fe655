"""ctypes binding of libbouquet (the C ABI in include/bouquet.h).

Argument marshalling only: every step of the walk path runs in the CUDA
kernels of the library.  PyTorch supplies device memory and streams (a
tensor's ``data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``).
There is no CPU fallback: if ``libbouquet.so`` is missing the first call
raises ``RuntimeError``.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbouquet.so")

OK = 0
EINVAL = -1
ENOMEM = -2
EGRAPH = -3
ENOEDGE = -4
EOVERFLOW = -5
ETIMEOUT = -6
EBUSY = -7
ECUDA = -8

HOST_PTRS = 0x0
DEVICE_PTRS = 0x1
BORROW = 0x2
SKIP_VALIDATE = 0x4
REQUIRE_CONNECTED = 0x8

MODE_NAIVE = 0
MODE_BOUQUET = 1
VISIT_START = 0x1
HOST_IO = 0x2
AESC_NAIVE = 0x4

SAMPLER_IND = 0
SAMPLER_COUPLED = 1
SAMPLER_SABA = 2  # the literal SABA word: walk batches only, for comparison

PLAN_CERTIFIED = 0
PLAN_SCHEDULED = 1


class Sampler(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("t", ctypes.c_uint32), ("width", ctypes.c_uint32)]


class Schedule(ctypes.Structure):
    _fields_ = [("tau_scale", ctypes.c_double), ("tau_add", ctypes.c_uint32),
                ("tau_max", ctypes.c_uint32), ("n_scale", ctypes.c_double),
                ("n_min", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class Tuning(ctypes.Structure):
    _fields_ = [("walk_lanes", ctypes.c_uint32), ("aggregate_visits", ctypes.c_uint32),
                ("aesc_lanes", ctypes.c_uint32), ("layout", ctypes.c_uint32),
                ("hub_slots", ctypes.c_uint32), ("l2_hints", ctypes.c_uint32),
                ("aesc_hub", ctypes.c_uint32), ("hub_cluster", ctypes.c_uint32),
                ("hub_relabel", ctypes.c_uint32), ("relabel_hub8", ctypes.c_uint32),
                ("hub8_hubs", ctypes.c_uint32), ("hub8_count_bits", ctypes.c_uint32),
                ("shared_lanes", ctypes.c_uint32), ("group_walks", ctypes.c_uint32),
                ("push_lanes", ctypes.c_uint32)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("m", ctypes.c_uint64), ("nnz", ctypes.c_uint64),
                ("min_degree", ctypes.c_uint32), ("max_degree", ctypes.c_uint32),
                ("bipartite", ctypes.c_int32), ("n_components", ctypes.c_int32),
                ("device_bytes", ctypes.c_uint64), ("has_spectrum", ctypes.c_int32),
                ("device", ctypes.c_int32), ("lambda2", ctypes.c_double),
                ("lambda_neg", ctypes.c_double), ("layout", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("hub_slots", ctypes.c_uint32),
                ("packed_bits", ctypes.c_uint32), ("relabel_hubs", ctypes.c_uint32),
                ("relabel_bits_id", ctypes.c_uint32), ("relabel_bits_off", ctypes.c_uint32),
                ("relabel_bits_deg", ctypes.c_uint32)]


class Profile(ctypes.Structure):
    _fields_ = [("walk_ms", ctypes.c_double), ("walk_launches", ctypes.c_uint64),
                ("group_ms", ctypes.c_double), ("group_launches", ctypes.c_uint64),
                ("aesc_ms", ctypes.c_double), ("aesc_launches", ctypes.c_uint64),
                ("aesc_aux_ms", ctypes.c_double), ("aesc_aux_launches", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64),
                ("walk_kernel_launches", ctypes.c_uint64 * 8)]


# indices of Profile.walk_kernel_launches (BQ_WALK_KERNEL_*)
WALK_KERNELS = ("naive", "bouquet", "hub", "cluster_hub", "relabel", "relabel8")


class AescQuery(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("edges_uv_dev", ctypes.c_void_p), ("k", ctypes.c_uint64),
                ("tau_dev", ctypes.c_void_p), ("nwalks_dev", ctypes.c_void_p),
                ("counts_dev", ctypes.c_void_p), ("sc_dev", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("max_inflight", ctypes.c_uint32),
                ("max_pending", ctypes.c_uint32), ("tasks_per_iteration", ctypes.c_uint64),
                ("tau_scale", ctypes.c_double), ("tau_add", ctypes.c_uint32),
                ("tau_max", ctypes.c_uint32), ("n_scale", ctypes.c_double),
                ("n_min", ctypes.c_uint32), ("planner_threads", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("pinned_arena_bytes", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("edges_completed", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64), ("walk_steps", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("uptime_s", ctypes.c_double), ("inflight", ctypes.c_uint32),
                ("pending", ctypes.c_uint32), ("worker_admit_s", ctypes.c_double),
                ("worker_launch_s", ctypes.c_double), ("worker_complete_s", ctypes.c_double),
                ("worker_idle_s", ctypes.c_double), ("planner_s", ctypes.c_double),
                ("planner_max_ms", ctypes.c_double), ("pinned_fallbacks", ctypes.c_uint64),
                ("pinned_fallback_s", ctypes.c_double)]


# every symbol include/bouquet.h declares
EXPORTS = (
    "bq_graph_create", "bq_graph_destroy", "bq_graph_info", "bq_graph_set_spectrum",
    "bq_walk_batch", "bq_aesc_plan", "bq_aesc_estimate", "bq_sync", "bq_strerror",
    "bq_last_error", "bq_version", "bq_get_tuning", "bq_set_tuning", "bq_profile_enable",
    "bq_profile_read", "bq_walk_batch_noalloc", "bq_batch_create", "bq_batch_run",
    "bq_batch_size", "bq_batch_destroy", "bq_autotune_walks", "bq_autotune_aesc",
    "bq_server_create", "bq_server_submit", "bq_server_wait", "bq_server_stats_get",
    "bq_server_destroy", "bq_aesc_estimate_push", "bq_graph_set_eigvecs", "bq_aesc_plan_pilot",
    "bq_aesc_estimate_shared", "bq_profile_read_bandwidth", "bq_batch_create_shared",
)

_lock = threading.Lock()
_lib = None


def load_library(path: str | None = None):
    """Load libbouquet.so (no GPU needed to load it)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"{p} is missing: build it with paper_2410_14056_gb300.build.build() "
                "(the library has no CPU fallback)")
        L = ctypes.CDLL(p)
        c = ctypes
        vp = c.c_void_p
        u32, u64, f64, i32 = c.c_uint32, c.c_uint64, c.c_double, c.c_int
        L.bq_graph_create.argtypes = [u32, vp, vp, u32, vp, c.POINTER(vp)]
        L.bq_graph_destroy.argtypes = [vp]
        L.bq_graph_info.argtypes = [vp, c.POINTER(GraphInfo)]
        L.bq_graph_set_spectrum.argtypes = [vp, f64, f64]
        L.bq_graph_set_eigvecs.argtypes = [vp, u32, vp, vp, f64]
        L.bq_walk_batch.argtypes = [vp, u64, vp, u64, u32, u32, c.POINTER(Sampler), u32, vp, vp, vp]
        L.bq_aesc_plan.argtypes = [vp, vp, u64, f64, f64, u32, c.POINTER(Schedule), vp, vp]
        L.bq_aesc_plan_pilot.argtypes = [vp, u64, vp, u64, f64, c.POINTER(Schedule), u32, f64,
                                         c.POINTER(Sampler), vp, vp, vp, vp]
        L.bq_aesc_estimate.argtypes = [vp, u64, vp, u64, vp, vp, c.POINTER(Sampler), u32, vp, vp, vp]
        L.bq_aesc_estimate_push.argtypes = [vp, u64, vp, u64, vp, vp, u32, u32, u32, vp, vp, vp, vp]
        L.bq_aesc_estimate_shared.argtypes = [vp, u64, vp, u64, vp, vp, c.POINTER(Sampler), u32, vp, vp,
                                              vp, vp]
        L.bq_sync.argtypes = [vp]
        L.bq_strerror.argtypes = [i32]
        L.bq_strerror.restype = c.c_char_p
        L.bq_last_error.argtypes = []
        L.bq_last_error.restype = c.c_char_p
        L.bq_version.restype = c.c_char_p
        L.bq_get_tuning.argtypes = [c.POINTER(Tuning)]
        L.bq_set_tuning.argtypes = [c.POINTER(Tuning)]
        L.bq_walk_batch_noalloc.argtypes = [vp, u64, vp, u64, u32, c.POINTER(Sampler), u32, vp, vp, vp]
        L.bq_batch_create.argtypes = [c.POINTER(AescQuery), u32, c.POINTER(Sampler), c.POINTER(vp)]
        L.bq_batch_create_shared.argtypes = [c.POINTER(AescQuery), u32, c.POINTER(Sampler), c.POINTER(vp)]
        L.bq_batch_run.argtypes = [vp, vp]
        L.bq_batch_size.argtypes = [vp, c.POINTER(u64)]
        L.bq_batch_destroy.argtypes = [vp]
        f32p = c.POINTER(c.c_float)
        L.bq_autotune_walks.argtypes = [vp, u64, vp, u64, u32, vp, vp, c.POINTER(u32), f32p]
        L.bq_autotune_aesc.argtypes = [c.POINTER(AescQuery), u32, c.POINTER(Sampler), vp,
                                       c.POINTER(u32), f32p]
        L.bq_server_create.argtypes = [vp, u32, c.POINTER(ServerConfig), c.POINTER(vp)]
        L.bq_server_submit.argtypes = [vp, u32, vp, u64, f64, u64, c.POINTER(u64)]
        L.bq_server_wait.argtypes = [vp, u64, f64, vp, vp, c.POINTER(f64)]
        L.bq_server_stats_get.argtypes = [vp, c.POINTER(ServerStats)]
        L.bq_server_destroy.argtypes = [vp]
        L.bq_profile_enable.argtypes = [i32]
        L.bq_profile_read.argtypes = [c.POINTER(Profile)]
        L.bq_profile_read_bandwidth.argtypes = [vp, u64, u32, vp, c.POINTER(f64)]
        for name in EXPORTS:
            if name not in ("bq_strerror", "bq_last_error", "bq_version"):
                getattr(L, name).restype = i32
        if path is None:
            _lib = L
        return L


class BouquetError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


def _check(rc: int):
    if rc != OK:
        L = load_library()
        msg = L.bq_last_error().decode() or L.bq_strerror(rc).decode()
        raise BouquetError(rc, msg)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _sampler(sampler):
    if sampler is None:
        return None
    if isinstance(sampler, Sampler):
        return ctypes.byref(sampler)
    kind, t, width = sampler
    return ctypes.byref(Sampler(int(kind), int(t), int(width)))


def _dptr(t, what, elem=4):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor")
    if t.element_size() != elem or not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous with {elem}-byte elements")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a, what, dtype):
    if a is None:
        return None
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what} must be a C-contiguous {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data)


class Graph:
    """A graph resident on the current CUDA device."""

    def __init__(self, n: int, offsets, nbrs, flags: int = HOST_PTRS, stream=None):
        L = load_library()
        self._h = ctypes.c_void_p()
        if flags & DEVICE_PTRS:
            self._keep = (offsets, nbrs)  # borrowed buffers stay alive
            po = _dptr(offsets, "offsets", 8)
            pn = _dptr(nbrs, "nbrs", 4)
        else:
            offsets = np.ascontiguousarray(offsets, dtype=np.int64)
            nbrs = np.ascontiguousarray(nbrs, dtype=np.uint32)
            if offsets.size != int(n) + 1 or (n >= 0 and nbrs.size < int(offsets[-1])):
                raise ValueError("offsets must have n + 1 entries and nbrs at least offsets[n]")
            self._keep = None
            po = _hptr(offsets, "offsets", np.int64)
            pn = _hptr(nbrs, "nbrs", np.uint32)
        _check(L.bq_graph_create(int(n), po, pn, int(flags), _stream_handle(stream),
                                 ctypes.byref(self._h)))
        self.n = int(n)

    @classmethod
    def from_csr(cls, g, flags: int = HOST_PTRS, stream=None) -> "Graph":
        """From any object with n, offsets, nbrs (e.g. workloads.Graph)."""
        return cls(g.n, g.offsets, g.nbrs, flags, stream)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("graph has been closed")
        return self._h

    def info(self) -> dict:
        gi = GraphInfo()
        _check(load_library().bq_graph_info(self.handle, ctypes.byref(gi)))
        return {name: getattr(gi, name) for name, _ in GraphInfo._fields_}

    def set_spectrum(self, lambda2: float, lambda_neg: float):
        _check(load_library().bq_graph_set_spectrum(self.handle, float(lambda2), float(lambda_neg)))

    def set_eigvecs(self, lambdas, vecs, lambda_rest: float):
        """Top eigenpairs for the certified plan: lambdas (omega,), vecs
        (n, omega) eigenvectors divided by sqrt(degree); omega = 0 clears."""
        lam = np.ascontiguousarray(lambdas, dtype=np.float64).reshape(-1)
        vv = np.ascontiguousarray(vecs, dtype=np.float64).reshape(-1)
        if lam.size and vv.size != self.n * lam.size:
            raise ValueError("vecs must have n * omega entries")
        _check(load_library().bq_graph_set_eigvecs(self.handle, lam.size, _hptr(lam, "lambdas", np.float64) if lam.size else None,
                                                   _hptr(vv, "vecs", np.float64) if lam.size else None,
                                                   float(lambda_rest)))

    def close(self):
        if getattr(self, "_h", None):
            load_library().bq_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def walk_batch(graph: Graph, seed: int, starts, n_steps: int, mode: int = MODE_BOUQUET,
               sampler=None, visit_start: bool = False, visits=None, paths=None, stream=None):
    """Enqueue a walk batch on device tensors; returns `visits` (accumulated)."""
    import torch
    L = load_library()
    n_walks = starts.numel()
    if visits is None:
        visits = torch.zeros(graph.n, dtype=torch.int32, device=starts.device)
    flags = VISIT_START if visit_start else 0
    _check(L.bq_walk_batch(graph.handle, int(seed) & (2**64 - 1), _dptr(starts, "starts"), n_walks,
                           int(n_steps), int(mode), _sampler(sampler), flags,
                           _dptr(visits, "visits"), _dptr(paths, "paths"), _stream_handle(stream)))
    return visits


def walk_batch_noalloc(graph: Graph, seed: int, starts, n_steps: int, sampler=None,
                       visit_start: bool = False, visits=None, paths=None, stream=None):
    """Bouquet walk batch that allocates nothing in the library (scratch is a
    fixed 32 MiB device array); device tensors only; returns `visits`."""
    import torch
    L = load_library()
    if visits is None:
        visits = torch.zeros(graph.n, dtype=torch.int32, device=starts.device)
    flags = VISIT_START if visit_start else 0
    _check(L.bq_walk_batch_noalloc(graph.handle, int(seed) & (2**64 - 1), _dptr(starts, "starts"),
                                   starts.numel(), int(n_steps), _sampler(sampler), flags,
                                   _dptr(visits, "visits"), _dptr(paths, "paths"),
                                   _stream_handle(stream)))
    return visits


def walk_batch_host(graph: Graph, seed: int, starts: np.ndarray, n_steps: int,
                    mode: int = MODE_BOUQUET, sampler=None, visit_start: bool = False,
                    visits: np.ndarray | None = None, paths: np.ndarray | None = None,
                    stream=None) -> np.ndarray:
    """Walk batch on host arrays (the library copies in and out and waits)."""
    L = load_library()
    starts = np.ascontiguousarray(starts, dtype=np.uint32)
    if visits is None:
        visits = np.zeros(graph.n, np.uint32)
    flags = HOST_IO | (VISIT_START if visit_start else 0)
    _check(L.bq_walk_batch(graph.handle, int(seed) & (2**64 - 1), _hptr(starts, "starts", np.uint32),
                           starts.size, int(n_steps), int(mode), _sampler(sampler), flags,
                           _hptr(visits, "visits", np.uint32), _hptr(paths, "paths", np.uint32),
                           _stream_handle(stream)))
    return visits


def aesc_plan(graph: Graph, uv: np.ndarray | None, eps: float, delta: float = 0.01,
              mode: int = PLAN_CERTIFIED, schedule: Schedule | None = None):
    """Host planner: returns (tau, nwalks) as uint32 numpy arrays."""
    L = load_library()
    if uv is None:
        k = graph.info()["m"]
        puv = None
    else:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        k = uv.shape[0]
        puv = _hptr(uv, "edges", np.uint32)
    tau = np.zeros(k, np.uint32)
    nw = np.zeros(k, np.uint32)
    _check(L.bq_aesc_plan(graph.handle, puv, k, float(eps), float(delta), int(mode),
                          ctypes.byref(schedule) if schedule is not None else None,
                          _hptr(tau, "tau", np.uint32), _hptr(nw, "nwalks", np.uint32)))
    return tau, nw


def aesc_plan_pilot(graph: Graph, seed: int, uv: np.ndarray | None, eps: float, schedule: Schedule,
                    n_pilot: int, z: float = 3.0, sampler=None, stream=None, moments: bool = True):
    """Pilot plan: tau from the schedule, N from the variance of n_pilot
    walks per side run on the GPU.  Returns (tau, nwalks, moments) as numpy
    arrays, moments uint64[k, 2, 5] (per side: sums of a, b, a^2, b^2, a b)
    or None when not asked for."""
    L = load_library()
    if uv is None:
        k = graph.info()["m"]
        puv = None
    else:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        k = uv.shape[0]
        puv = _hptr(uv, "edges", np.uint32)
    tau = np.zeros(k, np.uint32)
    nw = np.zeros(k, np.uint32)
    mo = np.zeros(10 * k, np.uint64) if moments else None
    _check(L.bq_aesc_plan_pilot(graph.handle, int(seed) & (2**64 - 1), puv, k, float(eps),
                                ctypes.byref(schedule), int(n_pilot), float(z), _sampler(sampler),
                                _hptr(tau, "tau", np.uint32), _hptr(nw, "nwalks", np.uint32),
                                _hptr(mo, "moments", np.uint64), _stream_handle(stream)))
    return tau, nw, (mo.reshape(-1, 2, 5) if moments else None)


def aesc_estimate(graph: Graph, seed: int, uv, tau, nwalks, sampler=None, counts=None,
                  sc=None, stream=None, naive: bool = False):
    """Enqueue an AESC estimate on device tensors; returns (counts, sc).
    naive=True runs the same walks one per thread (BQ_AESC_NAIVE)."""
    import torch
    L = load_library()
    k = tau.numel()
    dev = tau.device
    if counts is None:
        counts = torch.empty(4 * k, dtype=torch.int32, device=dev)
    if sc is None:
        sc = torch.empty(k, dtype=torch.float64, device=dev)
    _check(L.bq_aesc_estimate(graph.handle, int(seed) & (2**64 - 1), _dptr(uv, "edges"), k,
                              _dptr(tau, "tau"), _dptr(nwalks, "nwalks"), _sampler(sampler),
                              AESC_NAIVE if naive else 0,
                              _dptr(counts, "counts"), _dptr(sc, "sc", 8), _stream_handle(stream)))
    return counts, sc


def aesc_estimate_host(graph: Graph, seed: int, uv: np.ndarray | None, tau: np.ndarray,
                       nwalks: np.ndarray, sampler=None, stream=None, naive: bool = False):
    """AESC estimate on host arrays; returns (counts uint32[4k], sc float64[k]).
    naive=True runs the same walks one per thread (BQ_AESC_NAIVE)."""
    L = load_library()
    tau = np.ascontiguousarray(tau, dtype=np.uint32)
    nwalks = np.ascontiguousarray(nwalks, dtype=np.uint32)
    k = tau.size
    puv = None
    if uv is not None:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        puv = _hptr(uv, "edges", np.uint32)
    counts = np.zeros(4 * k, np.uint32)
    sc = np.zeros(k, np.float64)
    _check(L.bq_aesc_estimate(graph.handle, int(seed) & (2**64 - 1), puv, k,
                              _hptr(tau, "tau", np.uint32), _hptr(nwalks, "nwalks", np.uint32),
                              _sampler(sampler), HOST_IO | (AESC_NAIVE if naive else 0),
                              _hptr(counts, "counts", np.uint32),
                              _hptr(sc, "sc", np.float64), _stream_handle(stream)))
    return counts, sc


PUSH_SUPPORT_CAP = 512  # the usual support cap at push depths >= 2 (at most 512)


def aesc_estimate_push(graph: Graph, seed: int, uv, tau, nwalks, push_max: int = 1,
                       depth=None, acc=None, sc=None, stream=None, support_cap: int = PUSH_SUPPORT_CAP):
    """Push-phase AESC on device tensors (uv None = all edges); returns
    (depth, acc, sc) with acc the 4k uint64 fixed-point accumulators."""
    import torch
    L = load_library()
    k = tau.numel()
    dev = tau.device
    if depth is None:
        depth = torch.zeros(k, dtype=torch.int32, device=dev)
    if acc is None:
        acc = torch.zeros(4 * k, dtype=torch.int64, device=dev)
    if sc is None:
        sc = torch.empty(k, dtype=torch.float64, device=dev)
    _check(L.bq_aesc_estimate_push(graph.handle, int(seed) & (2**64 - 1), _dptr(uv, "uv"), k,
                                   _dptr(tau, "tau"), _dptr(nwalks, "nwalks"), int(push_max),
                                   int(support_cap), 0,
                                   _dptr(depth, "depth"), _dptr(acc, "acc", 8), _dptr(sc, "sc", 8),
                                   _stream_handle(stream)))
    return depth, acc, sc


def aesc_estimate_push_host(graph: Graph, seed: int, uv: np.ndarray | None, tau: np.ndarray,
                            nwalks: np.ndarray, push_max: int = 1, support_cap: int = PUSH_SUPPORT_CAP):
    """Push-phase AESC through host buffers (BQ_HOST_IO); synchronous."""
    L = load_library()
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    k = ta.size
    puv = None
    if uv is not None:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        puv = _hptr(uv, "edges", np.uint32)
    depth = np.zeros(k, np.uint32)
    acc = np.zeros(4 * k, np.uint64)
    sc = np.zeros(k, np.float64)
    _check(L.bq_aesc_estimate_push(graph.handle, int(seed) & (2**64 - 1), puv, k, _hptr(ta, "tau", np.uint32),
                                   _hptr(nw, "nwalks", np.uint32), int(push_max), int(support_cap), HOST_IO,
                                   _hptr(depth, "depth", np.uint32), _hptr(acc, "acc", np.uint64),
                                   _hptr(sc, "sc", np.float64), None))
    return depth, acc, sc


def aesc_estimate_shared(graph: Graph, seed: int, uv, tau, nwalks, sampler=None, counts=None,
                         nused=None, sc=None, stream=None):
    """Vertex-centric AESC (walks shared per vertex) on device tensors (uv
    None = all edges); returns (counts, nused, sc).  Waits for the stream
    once to size its histograms."""
    import torch
    L = load_library()
    k = tau.numel()
    dev = tau.device
    if counts is None:
        counts = torch.empty(4 * k, dtype=torch.int32, device=dev)
    if nused is None:
        nused = torch.empty(2 * k, dtype=torch.int32, device=dev)
    if sc is None:
        sc = torch.empty(k, dtype=torch.float64, device=dev)
    _check(L.bq_aesc_estimate_shared(graph.handle, int(seed) & (2**64 - 1), _dptr(uv, "uv"), k,
                                     _dptr(tau, "tau"), _dptr(nwalks, "nwalks"), _sampler(sampler), 0,
                                     _dptr(counts, "counts"), _dptr(nused, "nused"), _dptr(sc, "sc", 8),
                                     _stream_handle(stream)))
    return counts, nused, sc


def aesc_estimate_shared_host(graph: Graph, seed: int, uv: np.ndarray | None, tau: np.ndarray,
                              nwalks: np.ndarray, sampler=None):
    """Vertex-centric AESC through host buffers (BQ_HOST_IO); synchronous.
    Returns (counts uint32[4k], nused uint32[2k], sc float64[k])."""
    L = load_library()
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    k = ta.size
    puv = None
    if uv is not None:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        puv = _hptr(uv, "edges", np.uint32)
    counts = np.zeros(4 * k, np.uint32)
    nused = np.zeros(2 * k, np.uint32)
    sc = np.zeros(k, np.float64)
    _check(L.bq_aesc_estimate_shared(graph.handle, int(seed) & (2**64 - 1), puv, k, _hptr(ta, "tau", np.uint32),
                                     _hptr(nw, "nwalks", np.uint32), _sampler(sampler), HOST_IO,
                                     _hptr(counts, "counts", np.uint32), _hptr(nused, "nused", np.uint32),
                                     _hptr(sc, "sc", np.float64), None))
    return counts, nused, sc


def _query_array(queries):
    """bq_aesc_query array for a list of query dicts (outputs allocated when
    absent); returns (array, objects to keep alive, [(counts, sc)])."""
    import torch
    arr = (AescQuery * len(queries))()
    keep, outputs = [], []
    for i, q in enumerate(queries):
        tau, nw = q["tau"], q["nwalks"]
        k = tau.numel()
        counts = q.get("counts")
        sc = q.get("sc")
        if counts is None:
            counts = torch.empty(4 * k, dtype=torch.int32, device=tau.device)
        if sc is None:
            sc = torch.empty(k, dtype=torch.float64, device=tau.device)
        uv = q.get("uv")
        arr[i] = AescQuery(q["graph"].handle, int(q["seed"]) & (2**64 - 1),
                           _dptr(uv, "edges") if uv is not None else None, k,
                           _dptr(tau, "tau"), _dptr(nw, "nwalks"), _dptr(counts, "counts"),
                           _dptr(sc, "sc", 8))
        keep.append((q["graph"], uv, tau, nw, counts, sc))
        outputs.append((counts, sc))
    return arr, keep, outputs


def autotune_walks(graph: Graph, seed: int, starts, n_steps: int, visits=None, stream=None):
    """Time walk_lanes 1, 2, 4 on this walk batch; keep the fastest.
    Returns (best, [ms per candidate])."""
    import torch
    if visits is None:
        visits = torch.zeros(graph.n, dtype=torch.int32, device=starts.device)
    best = ctypes.c_uint32()
    ms = (ctypes.c_float * 3)()
    _check(load_library().bq_autotune_walks(graph.handle, int(seed) & (2**64 - 1), _dptr(starts, "starts"),
                                            starts.numel(), int(n_steps), _dptr(visits, "visits"),
                                            _stream_handle(stream), ctypes.byref(best), ms))
    return best.value, list(ms)


def autotune_aesc(queries, sampler=None, stream=None):
    """Time aesc_lanes 2, 4, 8 on a batch of these queries; keep the fastest.
    Returns (best, [ms per candidate])."""
    arr, keep, _ = _query_array(queries)
    best = ctypes.c_uint32()
    ms = (ctypes.c_float * 3)()
    _check(load_library().bq_autotune_aesc(arr, len(queries), _sampler(sampler), _stream_handle(stream),
                                           ctypes.byref(best), ms))
    del keep
    return best.value, list(ms)


class Batch:
    """Several AESC estimates run by one persistent counting launch.

    `queries` is a list of dicts with keys graph, seed, tau, nwalks (device
    uint32 tensors) and optionally uv (device pairs; None = all edges),
    counts, sc (outputs, allocated when absent).  shared=True estimates each
    query with walks shared per vertex (bq_batch_create_shared: the results
    of aesc_estimate_shared).  run() only launches kernels, so it may be
    captured in a CUDA graph."""

    def __init__(self, queries, sampler=None, shared: bool = False):
        L = load_library()
        arr, self._keep, self.outputs = _query_array(queries)
        self._h = ctypes.c_void_p()
        create = L.bq_batch_create_shared if shared else L.bq_batch_create
        _check(create(arr, len(queries), _sampler(sampler), ctypes.byref(self._h)))

    def run(self, stream=None):
        _check(load_library().bq_batch_run(self._h, _stream_handle(stream)))

    def size(self) -> int:
        e = ctypes.c_uint64()
        _check(load_library().bq_batch_size(self._h, ctypes.byref(e)))
        return e.value

    def close(self):
        if getattr(self, "_h", None):
            load_library().bq_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """SC queries on resident graphs, served with continuous batching.

    Requests (edge subset of one graph, eps, seed) are planned with the
    scheduled plan of `config` and counted by iterations that each launch one
    persistent kernel over tasks of every admitted request.  A request's
    estimates equal aesc_estimate() with the same plan and seed."""

    def __init__(self, graphs, config: ServerConfig | None = None, **kw):
        L = load_library()
        self._graphs = list(graphs)  # the server reads them: keep them alive
        arr = (ctypes.c_void_p * len(self._graphs))(*[g.handle.value for g in self._graphs])
        cfg = config
        if cfg is None and kw:
            cfg = ServerConfig(tau_scale=2.0, tau_add=2, tau_max=64, n_scale=9.0, n_min=32)
        if cfg is not None:
            for key, val in kw.items():
                setattr(cfg, key, val)
        self._h = ctypes.c_void_p()
        _check(L.bq_server_create(arr, len(self._graphs),
                                  ctypes.byref(cfg) if cfg is not None else None,
                                  ctypes.byref(self._h)))
        self._k = {}

    def submit(self, graph: int, uv, eps: float, seed: int) -> int:
        uv = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
        rid = ctypes.c_uint64()
        _check(load_library().bq_server_submit(self._h, int(graph), _hptr(uv, "edges", np.uint32),
                                               uv.shape[0], float(eps), int(seed), ctypes.byref(rid)))
        self._k[rid.value] = uv.shape[0]
        return rid.value

    def wait(self, request_id: int, timeout: float = 60.0, counts: bool = False):
        """(sc, counts or None, latency_ms); raises BouquetError on failure."""
        k = self._k.get(request_id, 0)
        sc = np.zeros(k, np.float64)
        cn = np.zeros(4 * k, np.uint32) if counts else None
        lat = ctypes.c_double()
        rc = load_library().bq_server_wait(self._h, int(request_id), float(timeout),
                                           _hptr(sc, "sc", np.float64),
                                           _hptr(cn, "counts", np.uint32) if counts else None,
                                           ctypes.byref(lat))
        if rc != ETIMEOUT:
            self._k.pop(request_id, None)  # each request is returned once
        _check(rc)
        return sc, (cn.reshape(-1, 4) if counts else None), lat.value

    def stats(self) -> dict:
        st = ServerStats()
        _check(load_library().bq_server_stats_get(self._h, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            load_library().bq_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sync(stream=None):
    """Wait for the stream and raise the first error its kernels recorded."""
    _check(load_library().bq_sync(_stream_handle(stream)))


def get_tuning() -> dict:
    t = Tuning()
    _check(load_library().bq_get_tuning(ctypes.byref(t)))
    return {name: int(getattr(t, name)) for name, _ in Tuning._fields_}


def set_tuning(**kw):
    cur = get_tuning()
    unknown = set(kw) - set(cur)
    if unknown:
        raise ValueError(f"unknown tuning fields {sorted(unknown)}")
    cur.update(kw)
    t = Tuning(*(int(cur[name]) for name, _ in Tuning._fields_))
    _check(load_library().bq_set_tuning(ctypes.byref(t)))


def profile_enable(on: bool = True):
    """Bracket the library's kernels with CUDA events (see bq_profile_read)."""
    _check(load_library().bq_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """Summed device time (ms) and launch counts per kernel group since the
    previous read; waits for the recorded events."""
    p = Profile()
    _check(load_library().bq_profile_read(ctypes.byref(p)))
    out = {name: getattr(p, name) for name, _ in Profile._fields_ if name != "walk_kernel_launches"}
    out["walk_kernels"] = {k: int(p.walk_kernel_launches[i]) for i, k in enumerate(WALK_KERNELS)}
    return out


def read_bandwidth(buf, reps: int = 20, stream=None) -> float:
    """GB/s of `reps` coalesced reads of the CUDA tensor `buf` in one launch
    (bq_profile_read_bandwidth): an L2 ceiling for a buffer well below the
    L2 size, an HBM one for a buffer well above it."""
    if not buf.is_cuda or not buf.is_contiguous():
        raise ValueError("buf must be a contiguous CUDA tensor")
    out = ctypes.c_double()
    _check(load_library().bq_profile_read_bandwidth(ctypes.c_void_p(buf.data_ptr()),
                                                    buf.numel() * buf.element_size(), int(reps),
                                                    _stream_handle(stream), ctypes.byref(out)))
    return out.value


def version() -> str:
    return load_library().bq_version().decode()
