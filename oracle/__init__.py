"""CPU oracle for the random-walk spanning-centrality path (test infrastructure).

Only the tests, the smoke check and the bench's CPU-baseline leg may use this
package.  The product library never imports it and shares no code with it.

Two parts:
  * ``walks.c`` (compiled here with gcc into ``_build/liboracle.so``): the
    hash-keyed walks, walk-batch visit counts, AESC counters, the planners
    (certified, scheduled, and the pilot sample's moments and walk count),
    the FP64 finalize, the push-phase and the vertex-centric (shared-walk)
    estimators, as plain single-threaded loops.
  * ``exact.py`` (numpy, FP64): exact spanning centrality by the Laplacian
    pseudoinverse and by the matrix-tree theorem, the spectrum of
    D^-1/2 A D^-1/2, the truncated walk series, and E(eta) of Sec. 5.6.

Parity status: every function here has at least one pin in
``tests/test_oracle_*.py`` (known-answer vectors, closed forms, brute force,
statistical tests); none is "parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "walks.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
EINVAL = -1
ENOEDGE = -4
EOVERFLOW = -5


def build(force: bool = False) -> str:
    """Compile walks.c with gcc (no FMA contraction) and return the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f64p = ctypes.POINTER(ctypes.c_double)
            c = ctypes
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_splitmix64_next.argtypes = [u64p]
            L.orc_splitmix64_next.restype = c.c_uint64
            L.orc_walk_key.argtypes = [c.c_uint64, c.c_uint64, c.c_uint64]
            L.orc_walk_key.restype = c.c_uint64
            L.orc_step_hash.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32]
            L.orc_step_hash.restype = c.c_uint32
            L.orc_choose.argtypes = [c.c_uint32, c.c_uint32]
            L.orc_choose.restype = c.c_uint32
            L.orc_walk_batch.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u32p, c.c_uint64, c.c_uint32,
                c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, u32p, u32p]
            L.orc_walk_batch.restype = c.c_int
            L.orc_walk_paths_by_id.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u64p, u32p, c.c_uint64, c.c_uint32,
                c.c_uint32, c.c_uint32, c.c_uint32, u32p]
            L.orc_walk_paths_by_id.restype = c.c_int
            L.orc_edge_ids.argtypes = [c.c_uint32, i64p, u32p, c.c_uint64, u32p, u64p]
            L.orc_edge_ids.restype = c.c_int
            L.orc_aesc_counts.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, c.c_uint64, u32p, u32p, u32p,
                c.c_uint32, c.c_uint32, c.c_uint32, u32p]
            L.orc_aesc_counts.restype = c.c_int
            L.orc_aesc_finalize.argtypes = [c.c_uint32, i64p, c.c_uint64, u32p, u32p, u32p, f64p]
            L.orc_aesc_finalize.restype = c.c_int
            L.orc_aesc_push_counts.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, c.c_uint64, u32p, u32p, u32p,
                c.c_uint32, c.c_uint32, u32p, u64p]
            L.orc_aesc_push_counts.restype = c.c_int
            L.orc_aesc_push_finalize.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u32p, u32p, u32p, u32p, u64p, f64p]
            L.orc_push_vector.argtypes = [c.c_uint32, i64p, u32p, c.c_uint32, c.c_uint32, u64p]
            L.orc_push_vector.restype = c.c_int
            L.orc_aesc_push_finalize.restype = c.c_int
            L.orc_trunc_bound.argtypes = [c.c_double, c.c_double, c.c_double, c.c_uint32]
            L.orc_trunc_bound.restype = c.c_double
            L.orc_plan_certified.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u32p, c.c_double, c.c_double,
                c.c_double, c.c_double, c.c_uint32, u32p, u32p]
            L.orc_plan_certified.restype = c.c_int
            L.orc_trunc_bound_omega.argtypes = [c.c_double, c.c_uint32, f64p, f64p, f64p, c.c_double,
                                                c.c_double, c.c_uint32]
            L.orc_trunc_bound_omega.restype = c.c_double
            L.orc_plan_certified_omega.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u32p, c.c_double, c.c_double, c.c_uint32, f64p, f64p,
                c.c_double, c.c_double, c.c_uint32, u32p, u32p]
            L.orc_plan_certified_omega.restype = c.c_int
            L.orc_plan_scheduled.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, u32p, c.c_double, c.c_double, c.c_uint32,
                c.c_uint32, c.c_double, c.c_uint32, u32p, u32p]
            L.orc_plan_scheduled.restype = c.c_int
            L.orc_aesc_moments.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, c.c_uint64, u32p, u32p, u32p,
                c.c_uint32, c.c_uint32, c.c_uint32, u64p]
            L.orc_aesc_moments.restype = c.c_int
            L.orc_plan_pilot_nwalks.argtypes = [
                c.c_uint32, i64p, c.c_uint64, u32p, u32p, u64p, c.c_uint32, c.c_double,
                c.c_double, c.c_uint32, u32p, f64p]
            L.orc_plan_pilot_nwalks.restype = c.c_int
            L.orc_aesc_shared_counts.argtypes = [
                c.c_uint32, i64p, u32p, c.c_uint64, c.c_uint64, u32p, u32p, u32p,
                c.c_uint32, c.c_uint32, c.c_uint32, u32p, u32p]
            L.orc_aesc_shared_counts.restype = c.c_int
            L.orc_aesc_shared_finalize.argtypes = [c.c_uint32, i64p, c.c_uint64, u32p, u32p, u32p, f64p]
            L.orc_aesc_shared_finalize.restype = c.c_int
            _lib = L
    return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


# ----------------------------------------------------------------- hashes

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                            _p(out, ctypes.c_uint32))
    return out


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    st = ctypes.c_uint64(seed)
    return [int(lib().orc_splitmix64_next(ctypes.byref(st))) for _ in range(count)]


def walk_key(seed: int, stream: int, k: int) -> int:
    return int(lib().orc_walk_key(seed, stream, k))


def step_hash(kw: int, step: int, cur: int) -> int:
    return int(lib().orc_step_hash(kw, step, cur))


def choose(r: int, d: int) -> int:
    return int(lib().orc_choose(r, d))


BATCH_STREAM = 0x4000000000000000
GROUP_BIT = 0x8000000000000000


# ------------------------------------------------------------- walk batch

def _graph_arrays(g):
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    nb = np.ascontiguousarray(g.nbrs, dtype=np.uint32)
    return off, nb


def _sampler(sampler):
    if sampler is None:
        return 0, 0, 1
    kind, t, width = sampler
    return int(kind), int(t), int(width)


def walk_batch(g, seed: int, starts: np.ndarray, n_steps: int, sampler=None,
               include_start: bool = False, visits: np.ndarray | None = None,
               want_paths: bool = False):
    """Visit counts (uint32[n]) and optionally paths (uint32[n_walks, n_steps+1])."""
    off, nb = _graph_arrays(g)
    st = np.ascontiguousarray(starts, dtype=np.uint32)
    vis = np.zeros(g.n, np.uint32) if visits is None else visits
    paths = np.zeros((st.size, n_steps + 1), np.uint32) if want_paths else None
    kind, t, width = _sampler(sampler)
    rc = lib().orc_walk_batch(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed,
        _p(st, ctypes.c_uint32), st.size, n_steps, kind, t, width,
        1 if include_start else 0, _p(vis, ctypes.c_uint32),
        _p(paths, ctypes.c_uint32) if paths is not None else None)
    _check(rc, "walk_batch")
    return (vis, paths) if want_paths else vis


def walk_paths_by_id(g, seed: int, ids: np.ndarray, starts: np.ndarray, n_steps: int,
                     sampler=None) -> np.ndarray:
    """Paths (uint32[len(ids), n_steps+1]) of the batch walks with these ids."""
    off, nb = _graph_arrays(g)
    idv = np.ascontiguousarray(ids, dtype=np.uint64)
    st = np.ascontiguousarray(starts, dtype=np.uint32)
    paths = np.zeros((idv.size, n_steps + 1), np.uint32)
    kind, t, width = _sampler(sampler)
    rc = lib().orc_walk_paths_by_id(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed, _p(idv, ctypes.c_uint64),
        _p(st, ctypes.c_uint32), idv.size, n_steps, kind, t, width, _p(paths, ctypes.c_uint32))
    _check(rc, "walk_paths_by_id")
    return paths


# ------------------------------------------------------------------- AESC

def edge_ids(g, uv: np.ndarray) -> np.ndarray:
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ids = np.zeros(q.shape[0], np.uint64)
    rc = lib().orc_edge_ids(g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32),
                            q.shape[0], _p(q, ctypes.c_uint32), _p(ids, ctypes.c_uint64))
    _check(rc, "edge_ids")
    return ids


def plan_certified(g, uv: np.ndarray, eps: float, delta: float, lambda2: float,
                   lambda_neg: float, tau_max: int = 1 << 20):
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    tau = np.zeros(q.shape[0], np.uint32)
    nw = np.zeros(q.shape[0], np.uint32)
    rc = lib().orc_plan_certified(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), q.shape[0],
        _p(q, ctypes.c_uint32), eps, delta, lambda2, lambda_neg, tau_max,
        _p(tau, ctypes.c_uint32), _p(nw, ctypes.c_uint32))
    _check(rc, "plan_certified")
    return tau, nw


def plan_scheduled(g, uv: np.ndarray, eps: float, tau_scale: float, tau_add: int, tau_max: int,
                   n_scale: float, n_min: int):
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    tau = np.zeros(q.shape[0], np.uint32)
    nw = np.zeros(q.shape[0], np.uint32)
    rc = lib().orc_plan_scheduled(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), q.shape[0],
        _p(q, ctypes.c_uint32), eps, tau_scale, tau_add, tau_max, n_scale, n_min,
        _p(tau, ctypes.c_uint32), _p(nw, ctypes.c_uint32))
    _check(rc, "plan_scheduled")
    return tau, nw


def plan_certified_omega(g, uv: np.ndarray, eps: float, delta: float, lambdas: np.ndarray,
                         vecs: np.ndarray, lambda_rest: float, lambda_neg: float, tau_max: int = 1 << 20):
    """Certified plan with omega = len(lambdas) known eigenpairs; vecs is
    (n, omega) with vecs[v, k] = psi_k(v) / sqrt(d(v))."""
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    vv = np.ascontiguousarray(vecs, dtype=np.float64).reshape(g.n, lam.size) if lam.size else np.zeros(1)
    tau = np.zeros(q.shape[0], np.uint32)
    nw = np.zeros(q.shape[0], np.uint32)
    rc = lib().orc_plan_certified_omega(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), q.shape[0], _p(q, ctypes.c_uint32),
        eps, delta, lam.size, _p(lam, ctypes.c_double), _p(vv, ctypes.c_double), lambda_rest, lambda_neg,
        tau_max, _p(tau, ctypes.c_uint32), _p(nw, ctypes.c_uint32))
    _check(rc, "plan_certified_omega")
    return tau, nw


def trunc_bound_omega(s_e: float, lambdas, cu, cv, lambda_rest: float, lambda_neg: float, tau: int) -> float:
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    a = np.ascontiguousarray(cu, dtype=np.float64)
    b = np.ascontiguousarray(cv, dtype=np.float64)
    return float(lib().orc_trunc_bound_omega(s_e, lam.size, _p(lam, ctypes.c_double), _p(a, ctypes.c_double),
                                             _p(b, ctypes.c_double), lambda_rest, lambda_neg, tau))


def trunc_bound(s_e: float, lambda2: float, lambda_neg: float, tau: int) -> float:
    return float(lib().orc_trunc_bound(s_e, lambda2, lambda_neg, tau))


def aesc_counts(g, seed: int, uv: np.ndarray, tau: np.ndarray, nwalks: np.ndarray,
                sampler=None) -> np.ndarray:
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    counts = np.zeros(4 * q.shape[0], np.uint32)
    kind, t, width = _sampler(sampler)
    rc = lib().orc_aesc_counts(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed, q.shape[0],
        _p(q, ctypes.c_uint32), _p(ta, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
        kind, t, width, _p(counts, ctypes.c_uint32))
    _check(rc, "aesc_counts")
    return counts


def aesc_finalize(g, uv: np.ndarray, nwalks: np.ndarray, counts: np.ndarray) -> np.ndarray:
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    cn = np.ascontiguousarray(counts, dtype=np.uint32)
    sc = np.zeros(q.shape[0], np.float64)
    rc = lib().orc_aesc_finalize(g.n, _p(off, ctypes.c_int64), q.shape[0],
                                 _p(q, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
                                 _p(cn, ctypes.c_uint32), _p(sc, ctypes.c_double))
    _check(rc, "aesc_finalize")
    return sc


def aesc_estimate(g, seed: int, uv: np.ndarray, tau: np.ndarray, nwalks: np.ndarray,
                  sampler=None):
    counts = aesc_counts(g, seed, uv, tau, nwalks, sampler)
    return counts, aesc_finalize(g, uv, nwalks, counts)


# ------------------------------------------------ AESC with a push phase

PUSH_Q = 1 << 30  # fixed-point scale of the pushed values


PUSH_MAX_DEPTH = 8       # deepest push
# The planner's usual support cap at push depths >= 2 (largest support per
# side and level); a parameter of aesc_push_counts, not part of TGT+'s rule.
PUSH_SUPPORT_CAP = 512


def push_vector(g, x: int, depth: int) -> np.ndarray:
    """r^depth_x as a dense uint64[n] (fixed point, about Q p_depth(y -> x))."""
    off, nb = _graph_arrays(g)
    out = np.zeros(g.n, np.uint64)
    rc = lib().orc_push_vector(g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), int(x), int(depth),
                               _p(out, ctypes.c_uint64))
    _check(rc, "push_vector")
    return out


def aesc_push_counts(g, seed: int, uv: np.ndarray, tau: np.ndarray, nwalks: np.ndarray,
                     push_max: int = 1, support_cap: int = PUSH_SUPPORT_CAP):
    """(depth uint32[k], acc uint64[4k]): push depth per edge and the
    fixed-point accumulators A_uu, A_uv, A_vu, A_vv (Alg. 1, depth <= 8).
    support_cap: largest support per side and level admitted at depths >= 2
    (a planner parameter; 0 = no cap, TGT+'s volume rule alone)."""
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    depth = np.zeros(q.shape[0], np.uint32)
    acc = np.zeros(4 * q.shape[0], np.uint64)
    rc = lib().orc_aesc_push_counts(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed, q.shape[0],
        _p(q, ctypes.c_uint32), _p(ta, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
        int(push_max), int(support_cap), _p(depth, ctypes.c_uint32), _p(acc, ctypes.c_uint64))
    _check(rc, "aesc_push_counts")
    return depth, acc


def aesc_push_finalize(g, uv, tau, nwalks, depth, acc) -> np.ndarray:
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    dp = np.ascontiguousarray(depth, dtype=np.uint32)
    ac = np.ascontiguousarray(acc, dtype=np.uint64)
    sc = np.zeros(q.shape[0], np.float64)
    rc = lib().orc_aesc_push_finalize(g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), q.shape[0],
                                      _p(q, ctypes.c_uint32),
                                      _p(ta, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
                                      _p(dp, ctypes.c_uint32), _p(ac, ctypes.c_uint64),
                                      _p(sc, ctypes.c_double))
    _check(rc, "aesc_push_finalize")
    return sc


def aesc_push_estimate(g, seed: int, uv, tau, nwalks, push_max: int = 1, support_cap: int = PUSH_SUPPORT_CAP):
    """(depth, acc, sc) of the push-phase estimator."""
    depth, acc = aesc_push_counts(g, seed, uv, tau, nwalks, push_max, support_cap)
    return depth, acc, aesc_push_finalize(g, uv, tau, nwalks, depth, acc)


# ------------------------------------------- pilot sample of the scheduled plan

def aesc_moments(g, seed: int, uv: np.ndarray, tau: np.ndarray, nwalks: np.ndarray,
                 sampler=None) -> np.ndarray:
    """uint64[k, 2, 5]: per query and side (0 from u, 1 from v) the sums of a,
    b, a^2, b^2, a b over the side's first nwalks walks, a and b being one
    walk's weighted hits of u and of v."""
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    mo = np.zeros(10 * q.shape[0], np.uint64)
    kind, t, width = _sampler(sampler)
    rc = lib().orc_aesc_moments(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed, q.shape[0],
        _p(q, ctypes.c_uint32), _p(ta, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
        kind, t, width, _p(mo, ctypes.c_uint64))
    _check(rc, "aesc_moments")
    return mo.reshape(-1, 2, 5)


def pilot_nwalks(g, uv: np.ndarray, tau: np.ndarray, moments: np.ndarray, n_pilot: int,
                 eps: float, z: float, n_min: int):
    """(nwalks uint32[k], var float64[k]): the pilot plan's walk count and
    the per-sample variance it was computed from."""
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    mo = np.ascontiguousarray(moments, dtype=np.uint64).reshape(-1)
    nw = np.zeros(q.shape[0], np.uint32)
    var = np.zeros(q.shape[0], np.float64)
    rc = lib().orc_plan_pilot_nwalks(
        g.n, _p(off, ctypes.c_int64), q.shape[0], _p(q, ctypes.c_uint32), _p(ta, ctypes.c_uint32),
        _p(mo, ctypes.c_uint64), int(n_pilot), float(eps), float(z), int(n_min),
        _p(nw, ctypes.c_uint32), _p(var, ctypes.c_double))
    _check(rc, "plan_pilot_nwalks")
    return nw, var


def plan_pilot(g, seed: int, uv: np.ndarray, eps: float, tau_scale: float, tau_add: int,
               tau_max: int, n_min: int, n_pilot: int, z: float = 3.0, sampler=None):
    """(tau, nwalks, moments, var): tau from the schedule, then n_pilot walks
    per side (the estimate's first walks) give the sample variance and N."""
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    tau, _ = plan_scheduled(g, q, eps, tau_scale, tau_add, tau_max, 0.0, 1)
    mo = aesc_moments(g, seed, q, tau, np.full(q.shape[0], n_pilot, np.uint32), sampler)
    nw, var = pilot_nwalks(g, q, tau, mo, n_pilot, eps, z, n_min)
    return tau, nw, mo, var


# ------------------------------------------- AESC with walks shared per vertex

VERTEX_STREAM = 1 << 61  # stream of vertex-centric walks: VERTEX_STREAM | x


def aesc_shared_counts(g, seed: int, uv: np.ndarray, tau: np.ndarray, nwalks: np.ndarray,
                       sampler=None):
    """(counts uint32[4k], nused uint32[2k]): C_uu, C_uv, C_vu, C_vv from the
    walks shared per vertex, and the walk counts N_u, N_v they used."""
    off, nb = _graph_arrays(g)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    ta = np.ascontiguousarray(tau, dtype=np.uint32)
    nw = np.ascontiguousarray(nwalks, dtype=np.uint32)
    counts = np.zeros(4 * q.shape[0], np.uint32)
    nused = np.zeros(2 * q.shape[0], np.uint32)
    kind, t, width = _sampler(sampler)
    rc = lib().orc_aesc_shared_counts(
        g.n, _p(off, ctypes.c_int64), _p(nb, ctypes.c_uint32), seed, q.shape[0],
        _p(q, ctypes.c_uint32), _p(ta, ctypes.c_uint32), _p(nw, ctypes.c_uint32),
        kind, t, width, _p(counts, ctypes.c_uint32), _p(nused, ctypes.c_uint32))
    _check(rc, "aesc_shared_counts")
    return counts, nused


def aesc_shared_finalize(g, uv: np.ndarray, counts: np.ndarray, nused: np.ndarray) -> np.ndarray:
    off = np.ascontiguousarray(g.offsets, dtype=np.int64)
    q = np.ascontiguousarray(uv, dtype=np.uint32).reshape(-1, 2)
    cn = np.ascontiguousarray(counts, dtype=np.uint32)
    nu = np.ascontiguousarray(nused, dtype=np.uint32)
    sc = np.zeros(q.shape[0], np.float64)
    rc = lib().orc_aesc_shared_finalize(g.n, _p(off, ctypes.c_int64), q.shape[0], _p(q, ctypes.c_uint32),
                                        _p(cn, ctypes.c_uint32), _p(nu, ctypes.c_uint32),
                                        _p(sc, ctypes.c_double))
    _check(rc, "aesc_shared_finalize")
    return sc


def aesc_shared_estimate(g, seed: int, uv, tau, nwalks, sampler=None):
    """(counts, nused, sc) of the vertex-centric (shared-walk) estimator."""
    counts, nused = aesc_shared_counts(g, seed, uv, tau, nwalks, sampler)
    return counts, nused, aesc_shared_finalize(g, uv, counts, nused)
