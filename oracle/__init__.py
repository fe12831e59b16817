"""FP64 CPU oracle for the Tensor Monte Carlo estimator -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference
leg may import this package.  It shares no code with the CUDA path: the arithmetic lives in
``tmc_oracle.c`` (plain double-precision loops), this file only compiles it and marshals
numpy arrays through ctypes.

Functions (each takes a ``paper_1806_08593_gb300.workload.Problem``):
    log_marginal(p)          log P_TMC per instance (Eq. (is) by summing out one index at a
                             time, Section 2.2 / Appendix)
    grad(p, grad_out)        analytic reparameterisation gradients of sum_b g_b log P_TMC_b
    brute_force(p)           Eq. (is) enumerated over all prod_i K_i combinations
Parity pins: all three are checked in tests/test_oracle_*.py against brute force, closed-form
Gaussian marginals, K=1, exactness under a factorising exact posterior, unbiasedness and
central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_tmc.so")
_SRC = os.path.join(_HERE, "tmc_oracle.c")
_SRC_LOOPY = os.path.join(_HERE, "tmc_oracle_loopy.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (OpenMP over parent-sample rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(_SRC_LOOPY),
            os.path.getmtime(os.path.join(_HERE, "tmc_oracle.h"))):
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-Wall", "-o", tmp, _SRC, _SRC_LOOPY, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            common = [ctypes.c_int, P, P, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                      P, P, P, P, P, P, P, P]
            lib.tmc_oracle_log_marginal.argtypes = common + [P]
            lib.tmc_oracle_grad.argtypes = common + [P, P, P, P, P, P, P, P, P]
            lib.tmc_oracle_brute_force.argtypes = common + [ctypes.c_longlong, P]
            dia = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_double, P, P, P, P, P, P, P]
            lib.tmc_oracle_diamond_log_marginal.argtypes = dia + [P]
            lib.tmc_oracle_diamond_brute_force.argtypes = dia + [ctypes.c_longlong, P]
            for f in (lib.tmc_oracle_log_marginal, lib.tmc_oracle_grad, lib.tmc_oracle_brute_force,
                      lib.tmc_oracle_diamond_log_marginal, lib.tmc_oracle_diamond_brute_force):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _common(p, overrides=None):
    o = dict(overrides or {})
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    f64 = lambda k: np.ascontiguousarray(o.get(k, getattr(p, k)), dtype=np.float64)
    # per-latent K_i and d_i (the oracle's layout); uniform problems repeat K[b], d[b]
    arrs = dict(n=i32(p.n), parent=i32(p.parent), K=i32(p.K_nodes()), d=i32(p.d_nodes()), obs=i32(p.obs),
                eps=f64("eps"), q_mean=f64("q_mean"), q_logstd=f64("q_logstd"), W=f64("W"),
                bias=f64("bias"), C=f64("C"), x=f64("x"))
    qa = o.get("q_A", p.q_A)  # coupled (non-factorised) proposal, or None
    arrs["q_A"] = None if qa is None else np.ascontiguousarray(qa, dtype=np.float64)
    args = [p.B, _ptr(arrs["n"]), _ptr(arrs["parent"]), _ptr(arrs["K"]), _ptr(arrs["d"]),
            _ptr(arrs["obs"]), int(p.shared), float(p.prior_var), float(p.obs_var),
            _ptr(arrs["eps"]), _ptr(arrs["q_mean"]), _ptr(arrs["q_logstd"]), _ptr(arrs["q_A"]),
            _ptr(arrs["W"]), _ptr(arrs["bias"]), _ptr(arrs["C"]), _ptr(arrs["x"])]
    return args, arrs


def _check(rc, what):
    if rc != 0:
        raise RuntimeError("oracle %s failed with status %d" % (what, rc))


def log_marginal(p, **overrides) -> np.ndarray:
    """log P_TMC[b] in FP64.  ``overrides`` replaces input arrays (e.g. eps=...)."""
    lib = _load()
    args, keep = _common(p, overrides)
    out = np.zeros(p.B, dtype=np.float64)
    _check(lib.tmc_oracle_log_marginal(*args, _ptr(out)), "log_marginal")
    return out


def grad(p, grad_out=None, want_dz=True, **overrides) -> dict:
    """Gradients of sum_b grad_out[b] * log P_TMC[b] (FP64), keyed like the C-ABI."""
    lib = _load()
    args, keep = _common(p, overrides)
    g = None if grad_out is None else np.ascontiguousarray(grad_out, dtype=np.float64)
    out = dict(log_phat=np.zeros(p.B), dz=np.zeros(p.eps.size) if want_dz else None,
               dq_mean=np.zeros(p.q_mean.size), dq_logstd=np.zeros(p.q_logstd.size),
               dq_A=None if keep["q_A"] is None else np.zeros(keep["q_A"].size),
               dW=np.zeros(p.W.size), dbias=np.zeros(p.bias.size), dC=np.zeros(p.C.size))
    _check(lib.tmc_oracle_grad(*args, _ptr(g), _ptr(out["log_phat"]), _ptr(out["dz"]),
                               _ptr(out["dq_mean"]), _ptr(out["dq_logstd"]), _ptr(out["dq_A"]),
                               _ptr(out["dW"]), _ptr(out["dbias"]), _ptr(out["dC"])), "grad")
    if out["dq_A"] is None:
        del out["dq_A"]
    return out


def brute_force(p, max_combos: int = 2_000_000, **overrides) -> np.ndarray:
    lib = _load()
    args, keep = _common(p, overrides)
    out = np.zeros(p.B, dtype=np.float64)
    _check(lib.tmc_oracle_brute_force(*args, ctypes.c_longlong(max_combos), _ptr(out)),
           "brute_force")
    return out


def _diamond_args(p, overrides):
    o = dict(overrides or {})
    f64 = lambda k: np.ascontiguousarray(o.get(k, getattr(p, k)), dtype=np.float64)
    keep = {k: f64(k) for k in ("eps", "q_mean", "q_logstd", "W", "bias", "C", "x")}
    args = [p.B, int(p.K), int(p.d), int(p.obs), int(p.shared), float(p.prior_var), float(p.obs_var)] + \
        [_ptr(keep[k]) for k in ("eps", "q_mean", "q_logstd", "W", "bias", "C", "x")]
    return args, keep


def diamond_log_marginal(p, **overrides) -> np.ndarray:
    """log P_TMC of the loopy graph of Fig. 1 (a workload.Diamond) by its two matrix messages."""
    lib = _load()
    args, keep = _diamond_args(p, overrides)
    out = np.zeros(p.B)
    _check(lib.tmc_oracle_diamond_log_marginal(*args, _ptr(out)), "diamond_log_marginal")
    return out


def diamond_brute_force(p, max_combos: int = 2_000_000, **overrides) -> np.ndarray:
    lib = _load()
    args, keep = _diamond_args(p, overrides)
    out = np.zeros(p.B)
    _check(lib.tmc_oracle_diamond_brute_force(*args, ctypes.c_longlong(max_combos), _ptr(out)),
           "diamond_brute_force")
    return out


def subset(p, idx):
    """The sub-batch of instances ``idx`` of problem p (same flat layout)."""
    from paper_1806_08593_gb300.workload import Problem
    idx = list(idx)
    every = p.slices_all(max(idx) + 1) if idx else []
    sl = [every[b] for b in idx]
    cat = lambda key, name: np.concatenate([getattr(p, name)[s[key][0]:s[key][1]] for s in sl])
    kw = dict(n=p.n[idx].copy(), K=p.K[idx].copy(), d=p.d[idx].copy(), obs=p.obs[idx].copy(),
              parent=cat("parent", "parent"), eps=cat("eps", "eps"), q_mean=cat("q", "q_mean"),
              q_logstd=cat("q", "q_logstd"), x=cat("x", "x"))
    if p.ragged:
        kw.update(Kn=np.concatenate([p.K_nodes()[s["parent"][0]:s["parent"][1]] for s in sl]),
                  dn=np.concatenate([p.d_nodes()[s["parent"][0]:s["parent"][1]] for s in sl]))
    if p.shared:
        kw.update(W=p.W.copy(), bias=p.bias.copy(), C=p.C.copy())
    else:
        kw.update(W=cat("W", "W"), bias=cat("bias", "bias"), C=cat("C", "C"))
    if p.q_A is not None:  # per-instance couplings, laid out like per-instance W blocks
        kw.update(q_A=np.concatenate([p.q_A[s["A"][0]:s["A"][1]] for s in sl]))
    return Problem(shared=p.shared, prior_var=p.prior_var, obs_var=p.obs_var, name=p.name, **kw)
