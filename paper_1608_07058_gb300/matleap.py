"""Thin Python binding of the C ABI in include/matleap.h (argument marshalling only).

Every function here has the name of the C entry point it wraps.  Device buffers are
torch CUDA tensors (their data pointers are passed through), streams are torch streams;
all simulation work runs in the CUDA library.  If the library has not been built, every
call raises MatleapError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmatleap.so")

ML_OK, ML_ERR_ARG, ML_ERR_OOM, ML_ERR_CUDA, ML_ERR_TIMEOUT, ML_ERR_BUSY, ML_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6
ML_ST_STEP_LIMIT, ML_ST_NEWTON_FAIL, ML_ST_REJECT_LIMIT, ML_ST_PTRS_CAP = 1, 2, 4, 8
ML_ST_BAD_INPUT, ML_ST_STAGE_TIMEOUT, ML_ST_OVERFLOW = 16, 32, 64
ML_MODE_ADAPTIVE, ML_MODE_EXPLICIT_ONLY, ML_MODE_SSA_ONLY = 0, 1, 2
ML_PREC_REF_FP64, ML_PREC_FAST_FP32 = 0, 1
ML_FORM_PLAIN, ML_FORM_PERSISTENT = 0, 1
ML_SHAPE_AUTO, ML_SHAPE_THREAD, ML_SHAPE_WARP, ML_SHAPE_THREAD_OCC, ML_SHAPE_THREAD_SEQ = 0, 1, 2, 3, 4
ML_SHAPE_THREAD_SEQ_OCC = 5
ML_SHAPE_THREAD_POOL, ML_SHAPE_THREAD_POOL_OCC = 6, 7
ML_JAC_FD, ML_JAC_ANALYTIC = 0, 1
ML_NEWTON_FP64, ML_NEWTON_FP32 = 0, 1


class MatleapError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class ml_sim_params(C.Structure):
    _fields_ = [("eps", C.c_double), ("n_c", C.c_int32), ("ssa_factor", C.c_double),
                ("n_ssa_explicit", C.c_int32), ("n_ssa_implicit", C.c_int32),
                ("pe_delta", C.c_double), ("stiff_ratio", C.c_double),
                ("newton_tol", C.c_double), ("newton_maxit", C.c_int32),
                ("fd_h", C.c_double), ("max_steps", C.c_int64), ("max_reject", C.c_int32),
                ("mode", C.c_int32), ("precision", C.c_int32), ("form", C.c_int32),
                ("shape", C.c_int32), ("block_size", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("use_graph", C.c_int32), ("jacobian", C.c_int32),
                ("newton_precision", C.c_int32), ("stage_poll_limit", C.c_int32),
                ("queue_order", C.c_void_p), ("specialize", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libmatleap.so (built in-tree by paper_1608_07058_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MatleapError(ML_ERR_UNSUPPORTED,
                               f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        P, v = C.POINTER, C.c_void_p
        L.ml_default_params.argtypes = [P(ml_sim_params)]
        L.ml_last_error.restype = C.c_char_p
        L.ml_model_create.argtypes = [C.c_int32, C.c_int32, P(C.c_int32), P(C.c_int32),
                                      P(C.c_double), P(v)]
        L.ml_model_destroy.argtypes = [v]
        L.ml_model_num_pairs.argtypes = [v]
        L.ml_model_last_launch_count.argtypes = [v]
        L.ml_model_last_launch_count.restype = C.c_int64
        sim = [v, C.c_int64, v, v, C.c_int32, v, C.c_int32, P(ml_sim_params), C.c_uint64,
               C.c_uint64, v, v, v, v, v, v]
        L.ml_simulate.argtypes = sim
        L.ml_simulate_host.argtypes = sim
        L.ml_simulate_noalloc.argtypes = sim
        L.ml_model_num_species.argtypes = [v]
        L.ml_model_num_reactions.argtypes = [v]
        L.ml_server_create.argtypes = [C.c_size_t, C.c_int32, P(ml_sim_params), P(v)]
        L.ml_server_submit.argtypes = [v, v, C.c_int64, v, v, C.c_int32, v, C.c_int32,
                                       C.c_uint64, C.c_uint64, P(v)]
        L.ml_request_wait.argtypes = [v, v, C.c_int32]
        L.ml_request_result.argtypes = [v, v, v, v, v, v, P(C.c_double), P(C.c_double)]
        L.ml_request_free.argtypes = [v, v]
        L.ml_server_stats.argtypes = [v, P(C.c_int64), P(C.c_int64), P(C.c_int64),
                                      P(C.c_size_t), P(C.c_int32)]
        L.ml_server_destroy.argtypes = [v]
        L.ml_autotune.argtypes = [v, C.c_int64, v, v, C.c_int32, v, C.c_int32,
                                  P(ml_sim_params), C.c_uint64, C.c_int64, P(ml_sim_params), v]
        L.ml_simulate_grid.argtypes = [v, C.c_int64, v, v, C.c_int32, v, C.c_int32,
                                       P(ml_sim_params), C.c_uint64, C.c_uint64, v, C.c_int32,
                                       v, v, v, v, v, v, v]
        L.ml_kl_divergence.argtypes = [C.c_int64, v, C.c_int64, v, C.c_int32, C.c_int32,
                                       C.c_int32, v, v, v]
        L.ml_measure_pipe_peaks.argtypes = [P(C.c_double), v]
        L.ml_posterior_sample.argtypes = [C.c_int64, C.c_int32, v, C.c_int32, v, C.c_int32, v, v,
                                          C.c_uint64, C.c_uint64, v, v, v]
        L.ml_resample_workspace_bytes.argtypes = [C.c_int64]
        L.ml_resample_workspace_bytes.restype = C.c_size_t
        L.ml_resample_systematic.argtypes = [C.c_int64, v, C.c_uint64, C.c_uint64, v, v,
                                             C.c_size_t, v]
        _lib = L
    return _lib


def _check(rc: int):
    if rc != ML_OK:
        raise MatleapError(rc, lib().ml_last_error().decode())


def ml_last_error() -> str:
    return lib().ml_last_error().decode()


def ml_default_params(**overrides) -> ml_sim_params:
    p = ml_sim_params()
    _check(lib().ml_default_params(C.byref(p)))
    for k, val in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, val)
    return p


class Model:
    """Owns an ml_model handle."""

    def __init__(self, handle: int, n_species: int, n_reactions: int):
        self.handle = handle
        self.N = n_species
        self.M = n_reactions

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def close(self):
        if self.handle:
            lib().ml_model_destroy(C.c_void_p(self.handle))
            self.handle = None


def ml_model_create(orders, stoich, rates) -> Model:
    """orders, stoich: (M, N) integer arrays; rates: (M,) float array (host)."""
    o = np.ascontiguousarray(orders, np.int32)
    s = np.ascontiguousarray(stoich, np.int32)
    r = np.ascontiguousarray(rates, np.float64)
    M, N = o.shape
    h = C.c_void_p()
    _check(lib().ml_model_create(N, M, o.ctypes.data_as(C.POINTER(C.c_int32)),
                                 s.ctypes.data_as(C.POINTER(C.c_int32)),
                                 r.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)))
    return Model(h.value, N, M)


def ml_model_destroy(model: Model):
    model.close()


def ml_model_num_pairs(model: Model) -> int:
    rc = lib().ml_model_num_pairs(C.c_void_p(model.handle))
    if rc < 0:
        _check(rc)
    return rc


def ml_model_last_launch_count(model: Model) -> int:
    return int(lib().ml_model_last_launch_count(C.c_void_p(model.handle)))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    import torch
    if stream is None and not torch.cuda.is_available():
        return C.c_void_p(None)  # the library reports the missing device itself
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def ml_simulate(model: Model, n_traj: int, x0, T, theta=None, params: Optional[ml_sim_params] = None,
                seed: int = 0, traj_id_base: int = 0, out: Optional[dict] = None,
                counters: bool = True, stream=None) -> dict:
    """Launch a simulation on the current stream (asynchronous).  x0: int64 CUDA tensor
    (N,) or (n_traj, N); T: float64 CUDA tensor (1,) or (n_traj,); theta: float64 CUDA
    tensor (n_traj, M) or None.  Returns dict X, r, G, status[, counters] of CUDA tensors
    (the given `out` buffers if passed)."""
    import torch
    dev = x0.device
    if out is None:
        out = {"X": torch.empty((n_traj, model.N), dtype=torch.int64, device=dev),
               "r": torch.empty((n_traj, model.M), dtype=torch.int64, device=dev),
               "G": torch.empty((n_traj, model.M), dtype=torch.float64, device=dev),
               "status": torch.empty((n_traj,), dtype=torch.int32, device=dev)}
        if counters:
            out["counters"] = torch.empty((n_traj, 4), dtype=torch.int64, device=dev)
    p = params if params is not None else ml_default_params()
    _check(lib().ml_simulate(C.c_void_p(model.handle), n_traj, _ptr(theta), _ptr(x0),
                             int(x0.dim() == 2), _ptr(T), int(T.numel() > 1), C.byref(p),
                             seed, traj_id_base, _ptr(out["X"]), _ptr(out["r"]), _ptr(out["G"]),
                             _ptr(out["status"]), _ptr(out.get("counters")),
                             _stream_handle(stream)))
    return out


def ml_simulate_grid(model: Model, n_traj: int, x0, T, t_obs, theta=None,
                     params: Optional[ml_sim_params] = None, seed: int = 0,
                     traj_id_base: int = 0, out: Optional[dict] = None, counters: bool = True,
                     stream=None) -> dict:
    """ml_simulate with time-grid output: t_obs is a float64 CUDA tensor (K,) of
    nondecreasing observation times; the result adds X_obs (n_traj, K, N) int64 with the
    state X(t_k) of every trajectory."""
    import torch
    dev = x0.device
    K = int(t_obs.numel())
    if out is None:
        out = {"X": torch.empty((n_traj, model.N), dtype=torch.int64, device=dev),
               "r": torch.empty((n_traj, model.M), dtype=torch.int64, device=dev),
               "G": torch.empty((n_traj, model.M), dtype=torch.float64, device=dev),
               "status": torch.empty((n_traj,), dtype=torch.int32, device=dev),
               "X_obs": torch.empty((n_traj, K, model.N), dtype=torch.int64, device=dev)}
        if counters:
            out["counters"] = torch.empty((n_traj, 4), dtype=torch.int64, device=dev)
    p = params if params is not None else ml_default_params()
    _check(lib().ml_simulate_grid(C.c_void_p(model.handle), n_traj, _ptr(theta), _ptr(x0),
                                  int(x0.dim() == 2), _ptr(T), int(T.numel() > 1), C.byref(p),
                                  seed, traj_id_base, _ptr(t_obs) if K else None, K,
                                  _ptr(out["X_obs"]) if K else None, _ptr(out["X"]),
                                  _ptr(out["r"]), _ptr(out["G"]), _ptr(out["status"]),
                                  _ptr(out.get("counters")), _stream_handle(stream)))
    return out


def ml_kl_divergence(X_ref, X_test, max_bins: int = 1024, kl_out=None, kl_mean=None,
                     stream=None):
    """KL of X_test's marginals from X_ref's (both int64 CUDA tensors (n, K, N)) per time
    point and species; returns (kl (K, N) float64, mean (1,) float64) CUDA tensors."""
    import torch
    _, K, N = X_ref.shape
    if kl_out is None:
        kl_out = torch.empty((K, N), dtype=torch.float64, device=X_ref.device)
    if kl_mean is None:
        kl_mean = torch.empty((1,), dtype=torch.float64, device=X_ref.device)
    _check(lib().ml_kl_divergence(X_ref.shape[0], _ptr(X_ref), X_test.shape[0], _ptr(X_test),
                                  K, N, max_bins, _ptr(kl_out), _ptr(kl_mean),
                                  _stream_handle(stream)))
    return kl_out, kl_mean


def ml_measure_pipe_peaks(stream=None) -> dict:
    """Measured FP64 FMA, FP32 FMA (flop/s) and special-function (op/s) throughput of the
    current device, for the roofline."""
    out = (C.c_double * 3)()
    _check(lib().ml_measure_pipe_peaks(out, _stream_handle(stream)))
    return {"fp64_fma_flops": out[0], "fp32_fma_flops": out[1], "mufu_lg2_ops": out[2]}


def ml_simulate_noalloc(model: Model, n_traj: int, x0, T, theta=None,
                        params: Optional[ml_sim_params] = None, seed: int = 0,
                        traj_id_base: int = 0, out: dict = None, stream=None) -> dict:
    """Allocation-free entry point: like ml_simulate with caller-allocated `out` (dict of
    CUDA tensors X, r, G, status[, counters]); the library allocates no device memory."""
    p = params if params is not None else ml_default_params()
    _check(lib().ml_simulate_noalloc(C.c_void_p(model.handle), n_traj, _ptr(theta), _ptr(x0),
                                     int(x0.dim() == 2), _ptr(T), int(T.numel() > 1),
                                     C.byref(p), seed, traj_id_base, _ptr(out["X"]),
                                     _ptr(out["r"]), _ptr(out["G"]), _ptr(out["status"]),
                                     _ptr(out.get("counters")), _stream_handle(stream)))
    return out


def ml_simulate_host(model: Model, n_traj: int, x0, T, theta=None,
                     params: Optional[ml_sim_params] = None, seed: int = 0,
                     traj_id_base: int = 0, out: Optional[dict] = None, counters: bool = True,
                     stream=None) -> dict:
    """Host-buffer variant: numpy (or pinned torch CPU) inputs and outputs; copies in,
    simulates, copies out and synchronizes inside the call."""
    def hp(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return C.c_void_p(a.data_ptr())
        return C.c_void_p(a.ctypes.data)
    x0a = x0 if hasattr(x0, "data_ptr") else np.ascontiguousarray(x0, np.int64)
    Ta = T if hasattr(T, "data_ptr") else np.ascontiguousarray(np.atleast_1d(T), np.float64)
    tha = None if theta is None else (theta if hasattr(theta, "data_ptr")
                                      else np.ascontiguousarray(theta, np.float64))
    if out is None:
        out = {"X": np.empty((n_traj, model.N), np.int64), "r": np.empty((n_traj, model.M), np.int64),
               "G": np.empty((n_traj, model.M), np.float64), "status": np.empty(n_traj, np.uint32)}
        if counters:
            out["counters"] = np.empty((n_traj, 4), np.int64)
    p = params if params is not None else ml_default_params()
    ndim = x0a.dim() if hasattr(x0a, "dim") else x0a.ndim
    nT = Ta.numel() if hasattr(Ta, "numel") else Ta.size
    stream_h = _stream_handle(stream) if stream is not None else C.c_void_p(None)
    _check(lib().ml_simulate_host(C.c_void_p(model.handle), n_traj, hp(tha), hp(x0a),
                                  int(ndim == 2), hp(Ta), int(nT > 1), C.byref(p), seed,
                                  traj_id_base, hp(out["X"]), hp(out["r"]), hp(out["G"]),
                                  hp(out["status"]), hp(out.get("counters")), stream_h))
    return out


def ml_autotune(model: Model, n_traj: int, x0, T, theta=None,
                params: Optional[ml_sim_params] = None, seed: int = 0, n_sample: int = 16384,
                stream=None) -> ml_sim_params:
    """Run the project autotuner on a sample of the given (device) inputs; returns the
    chosen parameters (also remembered by the model for block_size = 0 calls)."""
    p = params if params is not None else ml_default_params()
    best = ml_sim_params()
    _check(lib().ml_autotune(C.c_void_p(model.handle), n_traj, _ptr(theta), _ptr(x0),
                             int(x0.dim() == 2), _ptr(T), int(T.numel() > 1), C.byref(p), seed,
                             n_sample, C.byref(best), _stream_handle(stream)))
    return best


def ml_posterior_sample(alpha, beta, r, G, seed: int = 0, traj_id_base: int = 0,
                        theta_out=None, status_out=None, stream=None):
    """Posterior draws theta ~ Gamma(alpha + r, beta + G) on the device (Section 1).
    alpha, beta: float64 CUDA tensors (M,) shared or (n, M) per trajectory; r: int64 and
    G: float64 CUDA tensors (n, M).  Returns (theta (n, M) float64, status (n,) int32)."""
    import torch
    n, M = r.shape
    if theta_out is None:
        theta_out = torch.empty((n, M), dtype=torch.float64, device=r.device)
    if status_out is None:
        status_out = torch.empty((n,), dtype=torch.int32, device=r.device)
    _check(lib().ml_posterior_sample(n, M, _ptr(alpha), int(alpha.dim() == 2), _ptr(beta),
                                     int(beta.dim() == 2), _ptr(r), _ptr(G), seed, traj_id_base,
                                     _ptr(theta_out), _ptr(status_out), _stream_handle(stream)))
    return theta_out, status_out


def ml_resample_workspace_bytes(n: int) -> int:
    return int(lib().ml_resample_workspace_bytes(n))


def ml_resample_systematic(logw, seed: int = 0, id_base: int = 0, ancestors=None,
                           workspace=None, stream=None):
    """Systematic resampling of len(logw) particles (float64 CUDA tensor) into int64
    ancestor indices (all -1 when no weight is positive).  workspace: optional uint8 CUDA
    tensor of at least ml_resample_workspace_bytes(n) bytes."""
    import torch
    n = logw.numel()
    if ancestors is None:
        ancestors = torch.empty((n,), dtype=torch.int64, device=logw.device)
    need = ml_resample_workspace_bytes(n)
    if workspace is None:
        workspace = torch.empty((max(need, 1),), dtype=torch.uint8, device=logw.device)
    _check(lib().ml_resample_systematic(n, _ptr(logw), seed, id_base, _ptr(ancestors),
                                        _ptr(workspace), workspace.numel(),
                                        _stream_handle(stream)))
    return ancestors


def shard_bounds(n_total: int, rank: int, world: int) -> tuple:
    """Trajectory ids [lo, hi) of rank `rank` of `world` when n_total trajectories are
    split into contiguous, nearly equal ranges (the first n_total % world ranks take one
    more).  A rank simulates rows lo..hi-1 of the per-trajectory inputs with
    traj_id_base = lo; because every random number is keyed by the global id, the
    concatenated results equal one call over all ids, whatever the partition."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n_total >= 0")
    q, rem = divmod(n_total, world)
    lo = rank * q + min(rank, rem)
    return lo, lo + q + (1 if rank < rem else 0)


def model_from_crn(crn) -> Model:
    """Convenience: an ml_model from a workloads.CRN."""
    return ml_model_create(crn.orders, crn.stoich, crn.rates)


# ---- continuous-batching server -----------------------------------------------------

class ml_request:
    """A submitted request (owns the C handle)."""

    def __init__(self, server, handle, model, n):
        self.server, self.handle, self.model, self.n = server, handle, model, n

    def wait(self, timeout_ms: int = -1) -> bool:
        """True when finished; False on timeout; raises on a failed request."""
        rc = lib().ml_request_wait(C.c_void_p(self.server.handle), C.c_void_p(self.handle),
                                   timeout_ms)
        if rc == ML_ERR_TIMEOUT:
            return False
        _check(rc)
        return True

    def result(self) -> dict:
        N, M, n = self.model.N, self.model.M, self.n
        out = {"X": np.empty((n, N), np.int64), "r": np.empty((n, M), np.int64),
               "G": np.empty((n, M), np.float64), "status": np.empty(n, np.uint32),
               "counters": np.empty((n, 4), np.int64)}
        lat, q = C.c_double(), C.c_double()
        _check(lib().ml_request_result(C.c_void_p(self.handle), *[C.c_void_p(out[k].ctypes.data)
                                       for k in ("X", "r", "G", "status", "counters")],
                                       C.byref(lat), C.byref(q)))
        out["latency_s"], out["queue_s"] = lat.value, q.value
        return out

    def latency(self) -> tuple:
        """(latency_s, queue_s) of a finished request, without copying its results."""
        lat, q = C.c_double(), C.c_double()
        _check(lib().ml_request_result(C.c_void_p(self.handle), None, None, None, None, None,
                                       C.byref(lat), C.byref(q)))
        return lat.value, q.value

    def free(self):
        if self.handle:
            _check(lib().ml_request_free(C.c_void_p(self.server.handle) if self.server.handle else None,
                                         C.c_void_p(self.handle)))
            self.handle = None


class ml_server:
    """Continuous-batching server (ml_server_* entry points)."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 8,
                 params: Optional[ml_sim_params] = None):
        h = C.c_void_p()
        p = params if params is not None else ml_default_params()
        _check(lib().ml_server_create(hbm_budget_bytes, max_inflight, C.byref(p), C.byref(h)))
        self.handle = h.value

    def submit(self, model: Model, n_traj: int, x0, T, theta=None, seed: int = 0,
               traj_id_base: int = 0) -> ml_request:
        x0a = np.ascontiguousarray(x0, np.int64)
        Ta = np.ascontiguousarray(np.atleast_1d(T), np.float64)
        tha = None if theta is None else np.ascontiguousarray(theta, np.float64)
        h = C.c_void_p()
        _check(lib().ml_server_submit(C.c_void_p(self.handle), C.c_void_p(model.handle), n_traj,
                                      None if tha is None else C.c_void_p(tha.ctypes.data),
                                      C.c_void_p(x0a.ctypes.data), int(x0a.ndim == 2),
                                      C.c_void_p(Ta.ctypes.data), int(Ta.size > 1), seed,
                                      traj_id_base, C.byref(h)))
        return ml_request(self, h.value, model, n_traj)

    def stats(self) -> dict:
        a, c, t = C.c_int64(), C.c_int64(), C.c_int64()
        pb, pi = C.c_size_t(), C.c_int32()
        _check(lib().ml_server_stats(C.c_void_p(self.handle), C.byref(a), C.byref(c), C.byref(t),
                                     C.byref(pb), C.byref(pi)))
        return {"admitted": a.value, "completed": c.value, "trajectories": t.value,
                "peak_bytes": pb.value, "peak_inflight": pi.value}

    def close(self):
        if self.handle:
            lib().ml_server_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


ml_server_create = ml_server
