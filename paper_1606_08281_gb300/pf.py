"""Python binding of the C ABI in include/pf1606.h (argument marshalling only).

Every step of the likelihood computation runs in the CUDA library
``_build/libpf1606.so``; this module converts arrays to pointers and calls it.
There is no CPU fallback: if the library is missing, ``load()`` raises.

Host mode: pass numpy arrays; the call copies to the GPU and back.
Device mode: pass torch CUDA tensors for thetas / obs_times / y (and the
outputs are allocated as CUDA tensors); the call enqueues on the current torch
stream (or ``stream``) and returns without synchronising.
"""
from __future__ import annotations

import ctypes as ct
import threading
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libpf1606.so"
_lib = None
_lock = threading.Lock()

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_ETIMEOUT, PF_EAGAIN, PF_ENOTFOUND, PF_EBUSY = (
    0, -1, -2, -3, -4, -5, -6, -7)
PF_ST_OK, PF_ST_BUDGET, PF_ST_NONFINITE, PF_ST_INVALID_THETA, PF_ST_REJECTED = 0, 1, 2, 3, 4
PF_SCHED_AUTO, PF_SCHED_NATURAL, PF_SCHED_HEAVY_FIRST = 0, 1, 2
PF_MAX_CLUSTER_BLOCKS = 8
PF_CTX_CLUSTER_ARENA = 96 << 10


def split_fits(n_particles: int, cluster_blocks: int, n_species: int) -> bool:
    """Whether a batch request of N particles of U species can run split over
    a cluster of C blocks (pf_ctx_config.cluster_blocks in include/pf1606.h):
    every block holds a particle and its share, ceil(N/C) (12 + 8U) + 16
    bytes, fits PF_CTX_CLUSTER_ARENA less 1 KB."""
    C, N = int(cluster_blocks), int(n_particles)
    np_ = -(-N // C)
    return N - (C - 1) * np_ >= 1 and np_ * (12 + 8 * int(n_species)) + 16 + 1024 <= PF_CTX_CLUSTER_ARENA

EXPORTED = ["pf_loglik", "pf_strerror", "pf_last_error", "pf_version", "pf_philox4x32_10",
            "pf_fp64_probe", "pf_neg_log_u53", "pf_loglik_noalloc", "pf_ctx_create",
            "pf_ctx_load_problem", "pf_ctx_run_batch", "pf_submit", "pf_poll", "pf_ctx_stats",
            "pf_ctx_destroy", "pf_exp_variates", "pf_div_check", "pf_ctx_load_problem_model",
            "pf_fsp_loglik", "pf_erk_loglik", "pf_convert_check",
            "pf_ctx_create_config"]


class PfError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__(f"{where}: {detail or 'error'} (code {code})")
        self.code = code


class pf_network(ct.Structure):
    _fields_ = [("n_species", ct.c_int32), ("n_reactions", ct.c_int32),
                ("reactants", ct.c_void_p), ("products", ct.c_void_p),
                ("rate_index", ct.c_void_p)]


class pf_request(ct.Structure):
    _fields_ = [("problem_id", ct.c_int32), ("d", ct.c_int32), ("thetas", ct.c_void_p),
                ("M", ct.c_int64), ("n_particles", ct.c_int32), ("K_use", ct.c_int32),
                ("seed", ct.c_uint64), ("event_budget", ct.c_uint64),
                ("loglik_threshold", ct.c_double), ("loglik", ct.c_void_p),
                ("status", ct.c_void_p), ("theta_id_base", ct.c_uint32),
                ("cluster_blocks", ct.c_int32)]


class pf_ctx_config(ct.Structure):
    _fields_ = [("block_threads", ct.c_int32 * 4), ("cluster_blocks", ct.c_int32),
                ("grab", ct.c_int32)]


class pf_model(ct.Structure):
    _fields_ = [("rate_coef", ct.c_void_p), ("x0_hi", ct.c_void_p), ("obs_offset", ct.c_void_p),
                ("obs_var", ct.c_void_p)]


class pf_options(ct.Structure):
    _fields_ = [("event_budget", ct.c_uint64), ("device_ptrs", ct.c_int32),
                ("block_threads", ct.c_int32), ("stream", ct.c_void_p),
                ("ll_traj", ct.c_void_p), ("events", ct.c_void_p), ("digest", ct.c_void_p),
                ("final_states", ct.c_void_p), ("schedule", ct.c_int32),
                ("early_reject", ct.c_int32), ("row_order", ct.c_void_p),
                ("reject_below", ct.c_double), ("model", ct.POINTER(pf_model)),
                ("cluster_blocks", ct.c_int32), ("theta_ids", ct.c_void_p),
                ("phase_cycles", ct.c_void_p)]


class pf_fsp_options(ct.Structure):
    _fields_ = [("device_ptrs", ct.c_int32), ("stream", ct.c_void_p), ("ll_traj", ct.c_void_p),
                ("leak", ct.c_void_p), ("model", ct.POINTER(pf_model))]


class pf_ode_options(ct.Structure):
    _fields_ = [("device_ptrs", ct.c_int32), ("stream", ct.c_void_p), ("rtol", ct.c_double),
                ("atol", ct.c_double), ("max_steps", ct.c_int32), ("ll_pattern", ct.c_void_p),
                ("steps", ct.c_void_p)]


class _Model:
    """pf_model from a dict {"rate_coef": [R][d], "x0_hi": [U], "obs_offset": [P],
    "obs_var": [P][U]} (any subset); keeps the host arrays alive."""

    def __init__(self, model: dict | None):
        self.arrays = {}
        self.s = None
        if not model:
            return
        kinds = {"rate_coef": np.float64, "x0_hi": np.int32, "obs_offset": np.float64,
                 "obs_var": np.float64}
        unknown = set(model) - set(kinds)
        if unknown:
            raise ValueError(f"unknown model fields {sorted(unknown)}")
        for k, dt in kinds.items():
            if model.get(k) is not None:
                self.arrays[k] = _host(model[k], dt)
        self.s = pf_model(*[(_hptr(self.arrays[k]) if k in self.arrays else None) for k in kinds])

    def ptr(self):
        return None if self.s is None else ct.pointer(self.s)


def library_path() -> Path:
    return _LIB_PATH


def load():
    """Load libpf1606.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _LIB_PATH.exists():
                raise RuntimeError(f"{_LIB_PATH} is missing: build it with "
                                   "`python -m paper_1606_08281_gb300.build` (no CPU fallback)")
            lib = ct.CDLL(str(_LIB_PATH))
            P = ct.c_void_p
            lib.pf_loglik.argtypes = [ct.POINTER(pf_network), P, ct.c_int64, ct.c_int32, P, P,
                                      ct.c_int32, P, ct.c_int32, ct.c_int32, P, P, ct.c_int32,
                                      ct.c_uint64, P, P, ct.POINTER(pf_options)]
            lib.pf_loglik.restype = ct.c_int
            lib.pf_strerror.argtypes = [ct.c_int]
            lib.pf_strerror.restype = ct.c_char_p
            lib.pf_last_error.argtypes = []
            lib.pf_last_error.restype = ct.c_char_p
            lib.pf_version.argtypes = []
            lib.pf_version.restype = ct.c_char_p
            lib.pf_philox4x32_10.argtypes = [P, P, P, ct.c_int64]
            lib.pf_philox4x32_10.restype = ct.c_int
            lib.pf_fp64_probe.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int64,
                                          ct.POINTER(ct.c_double), ct.POINTER(ct.c_double)]
            lib.pf_fp64_probe.restype = ct.c_int
            lib.pf_neg_log_u53.argtypes = [P, P, ct.c_int64]
            lib.pf_neg_log_u53.restype = ct.c_int
            lib.pf_exp_variates.argtypes = [ct.c_uint64, ct.c_int64, P]
            lib.pf_exp_variates.restype = ct.c_int
            lib.pf_div_check.argtypes = [ct.c_uint64, ct.c_int64, ct.POINTER(ct.c_uint64)]
            lib.pf_div_check.restype = ct.c_int
            lib.pf_convert_check.argtypes = [ct.c_uint64, ct.c_int64, ct.POINTER(ct.c_uint64)]
            lib.pf_convert_check.restype = ct.c_int
            lib.pf_loglik_noalloc.argtypes = [ct.POINTER(pf_network), P, ct.c_int64, ct.c_int32,
                                              P, P, ct.c_int32, P, ct.c_int32, ct.c_int32, P, P,
                                              ct.c_int32, ct.c_uint64, P, P, ct.c_uint64, P]
            lib.pf_loglik_noalloc.restype = ct.c_int
            V = ct.c_void_p
            lib.pf_ctx_create.argtypes = [ct.POINTER(V), ct.c_size_t, ct.c_int32, ct.c_int32]
            lib.pf_ctx_create_config.argtypes = [ct.POINTER(V), ct.c_size_t, ct.c_int32, ct.c_int32,
                                                 ct.POINTER(pf_ctx_config)]
            lib.pf_ctx_load_problem.argtypes = [V, ct.POINTER(pf_network), ct.c_int32, P, P,
                                                ct.c_int32, P, ct.c_int32, ct.c_int32, P, P,
                                                ct.POINTER(ct.c_int32)]
            lib.pf_ctx_load_problem_model.argtypes = [V, ct.POINTER(pf_network), ct.c_int32, P,
                                                      P, ct.c_int32, P, ct.c_int32, ct.c_int32,
                                                      P, P, ct.POINTER(pf_model),
                                                      ct.POINTER(ct.c_int32)]
            lib.pf_ctx_load_problem_model.restype = ct.c_int
            lib.pf_fsp_loglik.argtypes = [ct.POINTER(pf_network), P, ct.c_int64, ct.c_int32, P, P,
                                          P, ct.c_int32, P, ct.c_int32, ct.c_int32, P, P, P, P,
                                          ct.POINTER(pf_fsp_options)]
            lib.pf_fsp_loglik.restype = ct.c_int
            lib.pf_erk_loglik.argtypes = [P, ct.c_int64, P, P, P, ct.c_int32, P, ct.c_int32, P, P,
                                          P, ct.POINTER(pf_ode_options)]
            lib.pf_erk_loglik.restype = ct.c_int
            lib.pf_ctx_run_batch.argtypes = [V, ct.POINTER(pf_request), ct.c_int32]
            lib.pf_submit.argtypes = [V, ct.POINTER(pf_request), ct.POINTER(ct.c_int64)]
            lib.pf_poll.argtypes = [V, ct.c_int64, ct.c_int32, ct.POINTER(ct.c_double),
                                    ct.POINTER(ct.c_double)]
            lib.pf_ctx_stats.argtypes = [V, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                         ct.POINTER(ct.c_int64)]
            lib.pf_ctx_destroy.argtypes = [V]
            for name in ("pf_ctx_create", "pf_ctx_create_config", "pf_ctx_load_problem",
                         "pf_ctx_run_batch", "pf_submit",
                         "pf_poll", "pf_ctx_stats", "pf_ctx_destroy"):
                getattr(lib, name).restype = ct.c_int
            _lib = lib
    return _lib


def _check(rc: int, where: str):
    if rc != PF_OK:
        lib = load()
        raise PfError(rc, where, lib.pf_last_error().decode())


def pf_strerror(code: int) -> str:
    return load().pf_strerror(code).decode()


def pf_last_error() -> str:
    return load().pf_last_error().decode()


def pf_version() -> str:
    return load().pf_version().decode()


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


class _Net:
    """Keeps the host arrays of a pf_network alive for the duration of a call."""

    def __init__(self, net: dict):
        self.reac = _host(net["reactants"], np.int32)
        self.prod = _host(net["products"], np.int32)
        ri = net.get("rate_index")
        self.ri = None if ri is None else _host(ri, np.int32)
        R, U = self.reac.shape
        self.s = pf_network(U, R, _hptr(self.reac), _hptr(self.prod), _hptr(self.ri))


def _is_torch_cuda(x) -> bool:
    return type(x).__module__.startswith("torch") and getattr(x, "is_cuda", False)


def pf_loglik(net: dict, thetas, x0, obs_times, y, C, sigma, n_particles: int, seed: int, *,
              event_budget: int = 0, block_threads: int = 0, stream=None,
              diagnostics: bool = False, final_states: bool = False, out=None,
              schedule: int = PF_SCHED_AUTO, row_order=None, reject_below=None,
              model: dict | None = None, cluster_blocks: int = 0, theta_ids=None,
              phase_cycles: bool = False):
    """Log-likelihood of every theta row (see pf_loglik in include/pf1606.h).

    model: optional Lac-Gfp extensions {"rate_coef", "x0_hi", "obs_offset",
    "obs_var"} (pf_model; host arrays).
    cluster_blocks: 2..8 splits each filter over a thread-block cluster of
    that many blocks (pf_options.cluster_blocks); 0 = one block per filter.
    phase_cycles: also return 'phase_cycles' [M][T][3], the SM cycles each
    filter spent in resampling + gather, simulation, weights + increment.
    theta_ids: optional [M] uint32 theta ids of the rows in the random-number
    counter (pf_options.theta_ids; default 0..M-1), in the memory space of
    `thetas` (a uint32-valued CUDA tensor of dtype int32 in device mode).

    Returns a dict with 'loglik' [M] and 'status' [M]; with diagnostics=True
    also 'll_traj', 'events', 'digest' [M][T]; with final_states=True also
    'final_states' [M][T][N][U].  Arrays are numpy (host mode) or torch CUDA
    tensors (device mode, chosen when `thetas` is a CUDA tensor).
    """
    lib = load()
    n = _Net(net)
    U = n.s.n_species
    x0h = _host(x0, np.int32)
    device = _is_torch_cuda(thetas)
    if device:
        import torch
        th = thetas.contiguous()
        assert th.dtype == torch.float64
        M, d = th.shape
        ts = _host(obs_times.cpu().numpy() if hasattr(obs_times, "cpu") else obs_times, np.float64)
        yy = y.contiguous()
        T, K, P = yy.shape
        dev = th.device
        if out is None:
            out = {"loglik": torch.empty(M, dtype=torch.float64, device=dev),
                   "status": torch.empty(M, dtype=torch.uint8, device=dev)}
            if diagnostics:
                out["ll_traj"] = torch.empty((M, T), dtype=torch.float64, device=dev)
                out["events"] = torch.empty((M, T), dtype=torch.int64, device=dev)
                out["digest"] = torch.empty((M, T), dtype=torch.int64, device=dev)
            if final_states:
                out["final_states"] = torch.empty((M, T, n_particles, U), dtype=torch.int32,
                                                  device=dev)
            if phase_cycles:
                out["phase_cycles"] = torch.empty((M, T, 3), dtype=torch.int64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        ptr = lambda k: (out[k].data_ptr() if k in out else None)  # noqa: E731
        p_th, p_ts, p_y = th.data_ptr(), _hptr(ts), yy.data_ptr()
    else:
        th = _host(thetas, np.float64)
        if th.ndim == 1:
            th = th[None, :]
        M, d = th.shape
        ts = _host(obs_times, np.float64)
        yy = _host(y, np.float64)
        T, K, P = yy.shape
        if out is None:
            out = {"loglik": np.empty(M, np.float64), "status": np.empty(M, np.uint8)}
            if diagnostics:
                out["ll_traj"] = np.empty((M, T), np.float64)
                out["events"] = np.empty((M, T), np.uint64)
                out["digest"] = np.empty((M, T), np.uint64)
            if final_states:
                out["final_states"] = np.empty((M, T, n_particles, U), np.int32)
            if phase_cycles:
                out["phase_cycles"] = np.empty((M, T, 3), np.uint64)
        ptr = lambda k: (out[k].ctypes.data if k in out else None)  # noqa: E731
        p_th, p_ts, p_y = _hptr(th), _hptr(ts), _hptr(yy)
    Ch = _host(C, np.float64).reshape(P, U)
    sg = _host(sigma, np.float64).reshape(P)
    if row_order is None:
        p_ro = None
    elif device:
        ro = row_order.contiguous()
        p_ro = ro.data_ptr()
    else:
        ro = _host(row_order, np.uint32)
        p_ro = _hptr(ro)
    if theta_ids is None:
        p_ids = None
    elif device:
        ids = theta_ids.contiguous()
        ok_types = (torch.int32, getattr(torch, "uint32", torch.int32))
        if ids.dtype not in ok_types or ids.numel() != M or not ids.is_cuda:
            raise ValueError("theta_ids must be a CUDA tensor of M 32-bit ids")
        p_ids = ids.data_ptr()
    else:
        ids = np.asarray(theta_ids)
        if ids.shape != (M,) or ids.min(initial=0) < 0 or ids.max(initial=0) >= 2**32:
            raise ValueError("theta_ids must hold M ids in 0..2^32-1")
        ids = _host(ids, np.uint32)
        p_ids = _hptr(ids)
    mdl = _Model(model)
    opt = pf_options(int(event_budget), 1 if device else 0, int(block_threads),
                     stream if device else None, ptr("ll_traj"), ptr("events"), ptr("digest"),
                     ptr("final_states"), int(schedule), 0 if reject_below is None else 1, p_ro,
                     float("nan") if reject_below is None else float(reject_below), mdl.ptr(),
                     int(cluster_blocks), p_ids, ptr("phase_cycles"))
    rc = lib.pf_loglik(ct.byref(n.s), p_th, M, d, _hptr(x0h), p_ts, K, p_y, T, P, _hptr(Ch),
                       _hptr(sg), int(n_particles), ct.c_uint64(int(seed) & (2**64 - 1)),
                       ptr("loglik"), ptr("status"), ct.byref(opt))
    _check(rc, "pf_loglik")
    return out


def pf_fsp_loglik(net: dict, thetas, x0, box_max, obs_times, y, C, sigma, *,
                  model: dict | None = None, diagnostics: bool = False, stream=None, out=None):
    """Exact (truncated) log-likelihood by the finite state projection (see
    pf_fsp_loglik in include/pf1606.h).  Returns 'loglik' [M], 'status' [M] and,
    with diagnostics=True, 'll_traj' and 'leak' [M][T]; numpy arrays (host
    mode) or torch CUDA tensors (device mode, when `thetas` is one)."""
    lib = load()
    n = _Net(net)
    U = n.s.n_species
    x0h = _host(x0, np.int32)
    box = _host(box_max, np.int32).reshape(U)
    device = _is_torch_cuda(thetas)
    if device:
        import torch
        th = thetas.contiguous()
        M, d = th.shape
        yy = y.contiguous()
        T, K, P = yy.shape
        dev = th.device
        if out is None:
            out = {"loglik": torch.empty(M, dtype=torch.float64, device=dev),
                   "status": torch.empty(M, dtype=torch.uint8, device=dev)}
            if diagnostics:
                out["ll_traj"] = torch.empty((M, T), dtype=torch.float64, device=dev)
                out["leak"] = torch.empty((M, T), dtype=torch.float64, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        ptr = lambda k: (out[k].data_ptr() if k in out else None)  # noqa: E731
        p_th, p_y = th.data_ptr(), yy.data_ptr()
    else:
        th = _host(thetas, np.float64)
        if th.ndim == 1:
            th = th[None, :]
        M, d = th.shape
        yy = _host(y, np.float64)
        T, K, P = yy.shape
        if out is None:
            out = {"loglik": np.empty(M, np.float64), "status": np.empty(M, np.uint8)}
            if diagnostics:
                out["ll_traj"] = np.empty((M, T), np.float64)
                out["leak"] = np.empty((M, T), np.float64)
        ptr = lambda k: (out[k].ctypes.data if k in out else None)  # noqa: E731
        p_th, p_y = _hptr(th), _hptr(yy)
    ts = _host(obs_times, np.float64)
    mdl = _Model(model)
    opt = pf_fsp_options(1 if device else 0, stream if device else None, ptr("ll_traj"),
                         ptr("leak"), mdl.ptr())
    rc = lib.pf_fsp_loglik(ct.byref(n.s), p_th, M, d, _hptr(x0h), _hptr(box), _hptr(ts), K, p_y, T,
                           P, _hptr(_host(C, np.float64).reshape(P, U)),
                           _hptr(_host(sigma, np.float64).reshape(P)), ptr("loglik"),
                           ptr("status"), ct.byref(opt))
    _check(rc, "pf_fsp_loglik")
    return out


def pf_erk_loglik(thetas, patterns, obs_times, y, *, rtol: float = 0.0, atol: float = 0.0,
                  max_steps: int = 0, diagnostics: bool = False, stream=None, out=None):
    """Deterministic likelihood of the Egf-Ras-Raf-Mek-Erk model (see
    pf_erk_loglik in include/pf1606.h).  patterns: list of (switch_times,
    switch_values) per input pattern; y [n_patterns][K].  Returns 'loglik' [M],
    'status' [M] and, with diagnostics=True, 'll_pattern' and 'steps'
    [M][n_patterns]; numpy (host mode) or torch CUDA tensors (device mode)."""
    lib = load()
    st = np.concatenate([np.asarray(t, np.float64) for t, _ in patterns])
    sv = np.concatenate([np.asarray(v, np.float64) for _, v in patterns])
    off = np.zeros(len(patterns) + 1, np.int32)
    off[1:] = np.cumsum([len(t) for t, _ in patterns])
    NP = len(patterns)
    ts = _host(obs_times, np.float64)
    K = len(ts)
    device = _is_torch_cuda(thetas)
    if device:
        import torch
        th = thetas.contiguous()
        M = th.shape[0]
        yy = y.contiguous()
        dev = th.device
        if out is None:
            out = {"loglik": torch.empty(M, dtype=torch.float64, device=dev),
                   "status": torch.empty(M, dtype=torch.uint8, device=dev)}
            if diagnostics:
                out["ll_pattern"] = torch.empty((M, NP), dtype=torch.float64, device=dev)
                out["steps"] = torch.empty((M, NP), dtype=torch.int32, device=dev)
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream
        ptr = lambda k: (out[k].data_ptr() if k in out else None)  # noqa: E731
        p_th, p_y = th.data_ptr(), yy.data_ptr()
    else:
        th = _host(thetas, np.float64)
        if th.ndim == 1:
            th = th[None, :]
        M = th.shape[0]
        yy = _host(y, np.float64).reshape(NP, K)
        if out is None:
            out = {"loglik": np.empty(M, np.float64), "status": np.empty(M, np.uint8)}
            if diagnostics:
                out["ll_pattern"] = np.empty((M, NP), np.float64)
                out["steps"] = np.empty((M, NP), np.uint32)
        ptr = lambda k: (out[k].ctypes.data if k in out else None)  # noqa: E731
        p_th, p_y = _hptr(th), _hptr(yy)
    if th.shape[-1] != 36:
        raise ValueError("thetas must have 36 columns")
    opt = pf_ode_options(1 if device else 0, stream if device else None, float(rtol), float(atol),
                         int(max_steps), ptr("ll_pattern"), ptr("steps"))
    rc = lib.pf_erk_loglik(p_th, M, _hptr(st), _hptr(sv), _hptr(off), NP, _hptr(ts), K, p_y,
                           ptr("loglik"), ptr("status"), ct.byref(opt))
    _check(rc, "pf_erk_loglik")
    return out


def pf_philox4x32_10(ctr, key) -> np.ndarray:
    """Device Philox4x32-10 for n (counter[4], key[2]) pairs; returns uint32 [n][4]."""
    lib = load()
    c = _host(ctr, np.uint32).reshape(-1, 4)
    k = _host(key, np.uint32).reshape(-1, 2)
    out = np.zeros_like(c)
    _check(lib.pf_philox4x32_10(_hptr(c), _hptr(k), _hptr(out), len(c)), "pf_philox4x32_10")
    return out


def pf_fp64_probe(kind: int, blocks: int, threads: int, iters: int):
    """FP64 cost probe; returns (elapsed_ms, checksum).  See include/pf1606.h."""
    lib = load()
    ms = ct.c_double()
    cs = ct.c_double()
    _check(lib.pf_fp64_probe(kind, blocks, threads, iters, ct.byref(ms), ct.byref(cs)),
           "pf_fp64_probe")
    return ms.value, cs.value


def pf_exp_variates(seed: int, n: int) -> np.ndarray:
    """n Exp(1) variates of the device generator (draw counters 0..n-1)."""
    lib = load()
    out = np.empty(int(n), np.float64)
    _check(lib.pf_exp_variates(ct.c_uint64(int(seed)), int(n), _hptr(out)), "pf_exp_variates")
    return out


def pf_div_check(seed: int, n: int) -> int:
    """Number of the kernels' waiting-time quotients differing from IEEE division."""
    lib = load()
    m = ct.c_uint64()
    _check(lib.pf_div_check(ct.c_uint64(int(seed)), int(n), ct.byref(m)), "pf_div_check")
    return int(m.value)


def pf_convert_check(seed: int, n: int) -> int:
    """Number of the kernels' count-to-double conversions differing from IEEE."""
    lib = load()
    m = ct.c_uint64()
    _check(lib.pf_convert_check(ct.c_uint64(int(seed)), int(n), ct.byref(m)), "pf_convert_check")
    return int(m.value)


def pf_neg_log_u53(v) -> np.ndarray:
    """The kernels' -log(v 2^-53), for 1 <= v <= 2^53 (device computation)."""
    lib = load()
    vv = _host(v, np.uint64).reshape(-1)
    out = np.empty(len(vv), np.float64)
    _check(lib.pf_neg_log_u53(_hptr(vv), _hptr(out), len(vv)), "pf_neg_log_u53")
    return out


def pf_loglik_noalloc(net: dict, thetas, x0, obs_times, y, C, sigma, n_particles: int,
                      seed: int, loglik, status=None, *, event_budget: int = 0, stream=None):
    """Allocation-free pf_loglik (see include/pf1606.h).  thetas [M][d], y
    [T][K][P], loglik [M] and status [M] are torch CUDA tensors the caller owns;
    the call enqueues on `stream` (default: the current torch stream).

    The tensors are checked, never copied: a temporary copy could be freed
    before the kernel that reads it runs.  Each must be a contiguous CUDA
    tensor on the current device with the right dtype (float64; status
    uint8) and enough elements, else ValueError."""
    import torch
    lib = load()
    n = _Net(net)
    U = n.s.n_species
    th = thetas
    if getattr(th, "ndim", 0) != 2 or getattr(y, "ndim", 0) != 3:
        raise ValueError("thetas must be [M][d] and y [T][K][P]")
    M, d = th.shape
    T, K, P = y.shape
    dev = torch.cuda.current_device()

    def need(name, t, dtype, numel):
        if not (type(t).__module__.startswith("torch") and t.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        if t.numel() < numel:
            raise ValueError(f"{name} has {t.numel()} elements, needs {numel}")

    need("thetas", th, torch.float64, M * d)
    need("y", y, torch.float64, T * K * P)
    need("loglik", loglik, torch.float64, M)
    if status is not None:
        need("status", status, torch.uint8, M)
    ts = _host(obs_times, np.float64)
    Ch = _host(C, np.float64).reshape(P, U)
    sg = _host(sigma, np.float64).reshape(P)
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    rc = lib.pf_loglik_noalloc(ct.byref(n.s), th.data_ptr(), M, d, _hptr(_host(x0, np.int32)),
                               _hptr(ts), K, y.data_ptr(), T, P, _hptr(Ch), _hptr(sg),
                               int(n_particles), ct.c_uint64(int(seed) & (2**64 - 1)),
                               loglik.data_ptr(), None if status is None else status.data_ptr(),
                               ct.c_uint64(int(event_budget)), stream)
    _check(rc, "pf_loglik_noalloc")


# --------------------------------------------------------------------------
# batching / serving context (pf_ctx_* in include/pf1606.h)
# --------------------------------------------------------------------------
def pf_ctx_create(mem_budget_bytes: int = 0, n_slots: int = 0, max_particles: int = 0):
    """Create a batching/serving context on the current device; returns a handle."""
    lib = load()
    h = ct.c_void_p()
    _check(lib.pf_ctx_create(ct.byref(h), int(mem_budget_bytes), int(n_slots),
                             int(max_particles)), "pf_ctx_create")
    return h


def pf_ctx_create_config(mem_budget_bytes: int = 0, n_slots: int = 0, max_particles: int = 0,
                         block_threads=(0, 0, 0, 0), cluster_blocks: int = 0, grab: int = 0):
    """pf_ctx_create with a launch shape (pf_ctx_config): threads per filter
    block for each reaction tier, the cluster size of split requests, and the
    filters a block takes from a work list at a time (0 = defaults)."""
    lib = load()
    h = ct.c_void_p()
    cfg = pf_ctx_config((ct.c_int32 * 4)(*[int(b) for b in block_threads]), int(cluster_blocks),
                        int(grab))
    _check(lib.pf_ctx_create_config(ct.byref(h), int(mem_budget_bytes), int(n_slots),
                                    int(max_particles), ct.byref(cfg)), "pf_ctx_create_config")
    return h


def pf_ctx_load_problem(ctx, net: dict, d: int, x0, obs_times, y, C, sigma,
                        model: dict | None = None) -> int:
    """Load a problem into a context; `model` as in pf_loglik (uses
    pf_ctx_load_problem_model when given)."""
    lib = load()
    n = _Net(net)
    U = n.s.n_species
    yy = _host(y, np.float64)
    T, K, P = yy.shape
    pid = ct.c_int32()
    args = (ctx, ct.byref(n.s), int(d), _hptr(_host(x0, np.int32)),
            _hptr(_host(obs_times, np.float64)), K, _hptr(yy), T, P,
            _hptr(_host(C, np.float64).reshape(P, U)), _hptr(_host(sigma, np.float64).reshape(P)))
    if model:
        return pf_ctx_load_problem_model(ctx, net, d, x0, obs_times, y, C, sigma, model)
    _check(lib.pf_ctx_load_problem(*args, ct.byref(pid)), "pf_ctx_load_problem")
    return pid.value


def pf_ctx_load_problem_model(ctx, net: dict, d: int, x0, obs_times, y, C, sigma,
                              model: dict | None) -> int:
    """pf_ctx_load_problem with the pf_model extensions (None: the basic model)."""
    lib = load()
    n = _Net(net)
    U = n.s.n_species
    yy = _host(y, np.float64)
    T, K, P = yy.shape
    pid = ct.c_int32()
    mdl = _Model(model)
    _check(lib.pf_ctx_load_problem_model(ctx, ct.byref(n.s), int(d), _hptr(_host(x0, np.int32)),
                                         _hptr(_host(obs_times, np.float64)), K, _hptr(yy), T, P,
                                         _hptr(_host(C, np.float64).reshape(P, U)),
                                         _hptr(_host(sigma, np.float64).reshape(P)), mdl.ptr(),
                                         ct.byref(pid)),
           "pf_ctx_load_problem_model")
    return pid.value


class Request:
    """Host arrays of one request, kept alive until pf_poll reports completion."""

    def __init__(self, problem_id: int, thetas, n_particles: int, seed: int, K_use: int = 0,
                 event_budget: int = 0, loglik_threshold: float = float("nan"),
                 theta_id_base: int = 0, cluster_blocks: int = 0):
        self.thetas = _host(thetas, np.float64)
        if self.thetas.ndim == 1:
            self.thetas = self.thetas[None, :]
        M, d = self.thetas.shape
        self.loglik = np.full(M, np.nan)
        self.status = np.full(M, 255, np.uint8)
        self.s = pf_request(int(problem_id), int(d), _hptr(self.thetas), int(M),
                            int(n_particles), int(K_use), int(seed) & (2**64 - 1),
                            int(event_budget), float(loglik_threshold),
                            _hptr(self.loglik), _hptr(self.status), int(theta_id_base),
                            int(cluster_blocks))
        self.id = None
        self.t_submit = self.t_done = None


def pf_ctx_run_batch(ctx, requests) -> None:
    """Evaluate the requests together (one batch) and wait."""
    lib = load()
    arr = (pf_request * len(requests))(*[r.s for r in requests])
    _check(lib.pf_ctx_run_batch(ctx, arr, len(requests)), "pf_ctx_run_batch")


def pf_submit(ctx, request: Request) -> int:
    lib = load()
    rid = ct.c_int64()
    _check(lib.pf_submit(ctx, ct.byref(request.s), ct.byref(rid)), "pf_submit")
    request.id = rid.value
    return rid.value


def pf_poll(ctx, request: Request, wait_ms: int = 0) -> bool:
    """True when finished (results are in request.loglik / request.status)."""
    lib = load()
    ts, td = ct.c_double(), ct.c_double()
    rc = lib.pf_poll(ctx, int(request.id), int(wait_ms), ct.byref(ts), ct.byref(td))
    if rc == PF_EAGAIN:
        return False
    _check(rc, "pf_poll")
    request.t_submit, request.t_done = ts.value, td.value
    return True


def pf_ctx_stats(ctx):
    lib = load()
    b, r, f = ct.c_int64(), ct.c_int64(), ct.c_int64()
    _check(lib.pf_ctx_stats(ctx, ct.byref(b), ct.byref(r), ct.byref(f)), "pf_ctx_stats")
    return {"batches": b.value, "requests": r.value, "filters": f.value}


def pf_ctx_destroy(ctx) -> None:
    _check(load().pf_ctx_destroy(ctx), "pf_ctx_destroy")
