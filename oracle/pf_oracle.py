"""ctypes front end of the C oracle ``pf_oracle.c`` (test infrastructure only).

The C file is compiled on first use with ``gcc -O2 -ffp-contract=off`` into
``oracle/_build/liboracle.so``; ``build()`` does it explicitly.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pf_oracle.c"
_TRACE_SRC = _HERE / "pf_trace.c"     # includes pf_oracle.c: the library's unit
_LIB = _HERE / "_build" / "liboracle.so"
_lock = threading.Lock()
_lib = None

OK, BUDGET, NONFINITE = 0, 1, 2
DEFAULT_BUDGET = 1 << 20


def build(force: bool = False) -> Path:
    """Compile the oracle shared library (no FMA contraction): the oracle and
    the trace instrumentation that includes it."""
    newest = max(_SRC.stat().st_mtime, _TRACE_SRC.stat().st_mtime)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < newest:
        _LIB.parent.mkdir(parents=True, exist_ok=True)
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=gnu11", "-I", str(_HERE), "-o", str(tmp), str(_TRACE_SRC),
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path: Path) -> ct.CDLL:
    lib = ct.CDLL(str(path))
    P = ct.c_void_p
    lib.orc_philox4x32_10.argtypes = [P, P, P]
    lib.orc_philox4x32_10.restype = None
    lib.orc_resample_systematic.argtypes = [P, ct.c_int32, ct.c_uint64, P]
    lib.orc_resample_systematic.restype = None
    lib.orc_pf_loglik.argtypes = [ct.c_int32, ct.c_int32, P, P, P, P, P, ct.c_int64, ct.c_int32,
                                  P, P, P, P, P, ct.c_int32, P, ct.c_int32, ct.c_int32, P, P, P,
                                  P, ct.c_int32, ct.c_uint64, ct.c_uint64, P, P, P, P, P, P]
    lib.orc_pf_loglik.restype = ct.c_int
    lib.orc_ssa_paths.argtypes = [ct.c_int32, ct.c_int32, P, P, P, P, P, ct.c_int32, P, P,
                                  ct.c_int32, ct.c_int64, ct.c_uint64, ct.c_uint64, P, P, P]
    lib.orc_ssa_paths.restype = ct.c_int
    lib.orc_exp_variates.argtypes = [ct.c_uint64, ct.c_int64, P]
    lib.orc_exp_variates.restype = None
    if hasattr(lib, "orc_pf_trace"):      # the instrumented library (not a bare variant)
        lib.orc_grid20.argtypes = [P, ct.c_int64, P]
        lib.orc_grid20.restype = None
        lib.orc_quantise_weights.argtypes = [P, ct.c_int32, ct.c_int32, P]
        lib.orc_quantise_weights.restype = None
        lib.orc_pf_trace.argtypes = [ct.c_int32, ct.c_int32, P, P, P, P, P, ct.c_int32,
                                     ct.c_int64, ct.c_int64, P, P, P, ct.c_int32, P, ct.c_int32,
                                     P, P, P, P, ct.c_int32, ct.c_uint64, ct.c_uint64,
                                     ct.c_int32, P, P, P, P, P, P, P, P, P, P]
        lib.orc_pf_trace.restype = ct.c_int
        lib.orc_ssa_replay.argtypes = [ct.c_int32, ct.c_int32, P, P, P, P, P, ct.c_int32, P,
                                       ct.c_double, ct.c_double, ct.c_uint64, ct.c_uint32,
                                       ct.c_uint32, ct.c_uint32, ct.c_uint64, ct.c_int64,
                                       ct.c_int32, P, ct.c_int64, P, P]
        lib.orc_ssa_replay.restype = ct.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def compile_variant(source_text: str, out_dir: Path) -> "Oracle":
    """Compile a modified copy of the oracle source (used by the mutation tests
    to show that the pins detect planted mistakes) and bind it, with the trace
    instrumentation built over the modified copy."""
    out_dir = Path(out_dir)
    src = out_dir / "variant.c"
    unit = out_dir / "variant_unit.c"
    so = out_dir / "libvariant.so"
    src.write_text(source_text)
    trace = _TRACE_SRC.read_text()
    assert trace.count('#include "pf_oracle.c"') == 1
    unit.write_text(trace.replace('#include "pf_oracle.c"', '#include "variant.c"'))
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11",
                           "-I", str(out_dir), "-o", str(so), str(unit), "-lm"])
    return Oracle(_bind(so))


def source_text() -> str:
    return _SRC.read_text()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Oracle:
    """The oracle's entry points bound to one compiled library."""

    def __init__(self, lib: ct.CDLL):
        self._lib = lib

    def philox4x32_10(self, ctr, key) -> np.ndarray:
        """Philox4x32-10 block for one (counter[4], key[2]) pair, as uint32[4]."""
        lib = self._lib
        c = _c(ctr, np.uint32)
        k = _c(key, np.uint32)
        out = np.zeros(4, np.uint32)
        lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
        return out


    def exp_variates(self, seed: int, n: int) -> np.ndarray:
        """n Exp(1) variates of the ziggurat generator (draw counters 0..n-1)."""
        out = np.empty(n, np.float64)
        self._lib.orc_exp_variates(ct.c_uint64(int(seed)), int(n), _ptr(out))
        return out

    def resample_systematic(self, q, r64: int) -> np.ndarray:
        """Ancestor indices of integer-weight systematic resampling."""
        lib = self._lib
        q = _c(q, np.uint64)
        anc = np.zeros(len(q), np.int32)
        lib.orc_resample_systematic(_ptr(q), len(q), ct.c_uint64(int(r64)), _ptr(anc))
        return anc


    def pf_loglik(self, net: dict, thetas, x0, obs_times, y, C, sigma, n_particles: int, seed: int,
                      budget: int = DEFAULT_BUDGET, theta_ids=None,
                      want_final_states: bool = False, model: dict | None = None,
                      traj_ids=None):
        """Filter log-likelihood of every theta row.

        theta_ids [M] / traj_ids [T] (optional): the rows' and trajectories'
        indices in the random-number counter (default 0..M-1 and 0..T-1), so
        that part of a larger problem reproduces the whole problem's values.

        net: {"reactants": [R][U], "products": [R][U], "rate_index": [R] or None}
        y: [T][K][P].  model (optional): {"rate_coef": [R][d], "x0_hi": [U],
        "obs_offset": [P], "obs_var": [P][U]}, any subset (the Lac-Gfp
        extensions).  Returns a dict with loglik[M], status[M], ll_traj[M][T],
        events[M][T], digest[M][T] and optionally final_states[M][T][N][U].
        """
        lib = self._lib
        reac = _c(net["reactants"], np.int32)
        prod = _c(net["products"], np.int32)
        R, U = reac.shape
        ri = net.get("rate_index")
        ri = None if ri is None else _c(ri, np.int32)
        th = _c(thetas, np.float64)
        if th.ndim == 1:
            th = th[None, :]
        M, d = th.shape
        ids = None if theta_ids is None else _c(theta_ids, np.int64)
        tids = None if traj_ids is None else _c(traj_ids, np.int64)
        x0 = _c(x0, np.int32)
        ts = _c(obs_times, np.float64)
        yy = _c(y, np.float64)
        T, K, P = yy.shape
        Cm = _c(C, np.float64).reshape(P, U)
        sg = _c(sigma, np.float64).reshape(P)
        N = int(n_particles)
        md = model or {}
        rc_ = md.get("rate_coef")
        rc_ = None if rc_ is None else _c(rc_, np.float64).reshape(R, d)
        xhi = md.get("x0_hi")
        xhi = None if xhi is None else _c(xhi, np.int32).reshape(U)
        off = md.get("obs_offset")
        off = None if off is None else _c(off, np.float64).reshape(P)
        ov = md.get("obs_var")
        ov = None if ov is None else _c(ov, np.float64).reshape(P, U)
        out = {
            "loglik": np.zeros(M, np.float64),
            "status": np.zeros(M, np.uint8),
            "ll_traj": np.zeros((M, T), np.float64),
            "events": np.zeros((M, T), np.uint64),
            "digest": np.zeros((M, T), np.uint64),
        }
        fs = np.zeros((M, T, N, U), np.int32) if want_final_states else None
        if tids is not None and tids.shape != (T,):
            raise ValueError("traj_ids must have one entry per trajectory")
        rc = lib.orc_pf_loglik(U, R, _ptr(reac), _ptr(prod), _ptr(ri), _ptr(rc_), _ptr(th), M, d,
                               _ptr(ids), _ptr(tids), _ptr(x0), _ptr(xhi), _ptr(ts), K, _ptr(yy), T, P,
                               _ptr(Cm), _ptr(sg), _ptr(off), _ptr(ov), N,
                               ct.c_uint64(int(seed)), ct.c_uint64(int(budget)),
                               _ptr(out["loglik"]), _ptr(out["status"]), _ptr(out["ll_traj"]),
                               _ptr(out["events"]), _ptr(out["digest"]), _ptr(fs))
        if rc != 0:
            raise ValueError(f"oracle rejected the problem (code {rc})")
        if fs is not None:
            out["final_states"] = fs
        return out


    def grid20(self, e) -> np.ndarray:
        """The log-weight rounding of the state-dependent-variance model."""
        e = _c(e, np.float64).reshape(-1)
        out = np.empty_like(e)
        self._lib.orc_grid20(_ptr(e), len(e), _ptr(out))
        return out

    def quantise_weights(self, e, svar: bool = False) -> np.ndarray:
        """The integer resampling weights of log-weights e (first maximum)."""
        e = _c(e, np.float64).reshape(-1)
        q = np.empty(len(e), np.uint64)
        self._lib.orc_quantise_weights(_ptr(e), len(e), int(bool(svar)), _ptr(q))
        return q

    def pf_trace(self, net: dict, theta, theta_id: int, traj_id: int, x0, obs_times, y_traj, C,
                 sigma, n_particles: int, seed: int, k_trace: int,
                 budget: int = DEFAULT_BUDGET, model: dict | None = None) -> dict:
        """One filter (row `theta` with id theta_id, trajectory y_traj [K][P]
        with id traj_id) over len(obs_times) intervals, recording interval
        k_trace: x_start, x_end [N][U], anc, e_prev, q_prev, fired [N], plus
        the filter's ll, status, events and digest."""
        reac = _c(net["reactants"], np.int32)
        prod = _c(net["products"], np.int32)
        R, U = reac.shape
        ri = net.get("rate_index")
        ri = None if ri is None else _c(ri, np.int32)
        th = _c(theta, np.float64).reshape(-1)
        d = len(th)
        ts = _c(obs_times, np.float64)
        yy = _c(y_traj, np.float64)
        K, P = yy.shape
        N = int(n_particles)
        md = model or {}
        arr = {k: (None if md.get(k) is None else _c(md[k], dt)) for k, dt in
               (("rate_coef", np.float64), ("x0_hi", np.int32), ("obs_offset", np.float64),
                ("obs_var", np.float64))}
        out = {"x_start": np.zeros((N, U), np.int64), "x_end": np.zeros((N, U), np.int64),
               "anc": np.zeros(N, np.int32), "e_prev": np.zeros(N), "q_prev": np.zeros(N, np.uint64),
               "fired": np.zeros(N, np.uint64)}
        ll, st = ct.c_double(), ct.c_int32()
        ev, dg = ct.c_uint64(), ct.c_uint64()
        rc = self._lib.orc_pf_trace(U, R, _ptr(reac), _ptr(prod), _ptr(ri), _ptr(arr["rate_coef"]),
                                    _ptr(th), d, int(theta_id), int(traj_id), _ptr(_c(x0, np.int32)),
                                    _ptr(arr["x0_hi"]), _ptr(ts), K, _ptr(yy), P,
                                    _ptr(_c(C, np.float64).reshape(P, U)),
                                    _ptr(_c(sigma, np.float64).reshape(P)), _ptr(arr["obs_offset"]),
                                    _ptr(arr["obs_var"]), N, ct.c_uint64(int(seed)),
                                    ct.c_uint64(int(budget)), int(k_trace), _ptr(out["x_start"]),
                                    _ptr(out["x_end"]), _ptr(out["anc"]), _ptr(out["e_prev"]),
                                    _ptr(out["q_prev"]), _ptr(out["fired"]), ct.byref(ll),
                                    ct.byref(st), ct.byref(ev), ct.byref(dg))
        if rc != 0:
            raise ValueError(f"oracle rejected the trace (code {rc})")
        out.update(ll=ll.value, status=st.value, events=ev.value, digest=dg.value)
        return out

    def ssa_replay(self, net: dict, theta, x, t0: float, t1: float, seed: int, particle: int,
                   lane: int, m: int, budget: int = DEFAULT_BUDGET, alt_draw: int = -1,
                   alt_kind: int = 0, rate_coef=None, cap: int = 1 << 20):
        """One particle's direct-method steps over (t0, t1] from state x, with
        an optional alternative decision at draw alt_draw (see pf_trace.c).
        Returns (x_end [U], fired, status, records [n][10])."""
        reac = _c(net["reactants"], np.int32)
        prod = _c(net["products"], np.int32)
        R, U = reac.shape
        ri = net.get("rate_index")
        ri = None if ri is None else _c(ri, np.int32)
        th = _c(theta, np.float64).reshape(-1)
        rcf = None if rate_coef is None else _c(rate_coef, np.float64).reshape(R, len(th))
        xx = _c(x, np.int64).reshape(U).copy()
        rec = np.zeros((cap, 10))
        n = ct.c_int64()
        fired = ct.c_uint64()
        st = self._lib.orc_ssa_replay(U, R, _ptr(reac), _ptr(prod), _ptr(ri), _ptr(rcf), _ptr(th),
                                      len(th), _ptr(xx), float(t0), float(t1),
                                      ct.c_uint64(int(seed)), int(particle) & 0xFFFFFFFF,
                                      int(lane) & 0xFFFFFFFF, int(m) & 0xFFFFFFFF,
                                      ct.c_uint64(int(budget)), int(alt_draw), int(alt_kind),
                                      _ptr(rec), cap, ct.byref(n), ct.byref(fired))
        if st < 0:
            raise ValueError(f"oracle rejected the replay (code {st})")
        return xx, int(fired.value), int(st), rec[: n.value].copy()

    def ssa_paths(self, net: dict, theta, x0, times, n_paths: int, seed: int,
                      budget: int = DEFAULT_BUDGET, rate_coef=None):
        """Independent direct-method paths; returns (states[n][K][U], fired[n], status[n]).
        rate_coef [R][d] (optional) composes the rates from theta."""
        lib = self._lib
        reac = _c(net["reactants"], np.int32)
        prod = _c(net["products"], np.int32)
        R, U = reac.shape
        ri = net.get("rate_index")
        ri = None if ri is None else _c(ri, np.int32)
        th = _c(theta, np.float64).reshape(-1)
        rcf = None if rate_coef is None else _c(rate_coef, np.float64).reshape(R, len(th))
        x0 = _c(x0, np.int32)
        ts = _c(times, np.float64)
        K = len(ts)
        states = np.zeros((n_paths, K, U), np.int32)
        fired = np.zeros(n_paths, np.uint64)
        status = np.zeros(n_paths, np.uint8)
        rc = lib.orc_ssa_paths(U, R, _ptr(reac), _ptr(prod), _ptr(ri), _ptr(rcf), _ptr(th), len(th),
                               _ptr(x0),
                               _ptr(ts), K, n_paths, ct.c_uint64(int(seed)), ct.c_uint64(int(budget)),
                               _ptr(states), _ptr(fired), _ptr(status))
        if rc != 0:
            raise ValueError(f"oracle rejected the problem (code {rc})")
        return states, fired, status


_default = None


def default() -> Oracle:
    global _default
    if _default is None:
        _default = Oracle(_load())
    return _default


def philox4x32_10(ctr, key):
    return default().philox4x32_10(ctr, key)


def resample_systematic(q, r64: int):
    return default().resample_systematic(q, r64)


def exp_variates(seed: int, n: int):
    return default().exp_variates(seed, n)


def pf_loglik(*args, **kwargs):
    return default().pf_loglik(*args, **kwargs)


def ssa_paths(*args, **kwargs):
    return default().ssa_paths(*args, **kwargs)


def grid20(e):
    return default().grid20(e)


def quantise_weights(e, svar: bool = False):
    return default().quantise_weights(e, svar)


def pf_trace(*args, **kwargs):
    return default().pf_trace(*args, **kwargs)


def ssa_replay(*args, **kwargs):
    return default().ssa_replay(*args, **kwargs)
