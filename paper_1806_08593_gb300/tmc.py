"""Python binding of the C ABI in include/tmc.h (argument marshalling only).

Every step of the TMC hot path runs in the CUDA library ``_build/libtmc_gb300.so``; this
module only passes device pointers and streams.  PyTorch provides device memory, streams
and autograd plumbing.  There is no CPU fallback: if the library or a CUDA device is
missing, the calls raise.

    plan = Plan.from_problem(problem, precision="fp32")
    t = plan.to_device(problem)                 # dict of CUDA tensors in the C-ABI layout
    logp = tmc_log_marginal(plan, **t)          # differentiable w.r.t. eps, q_mean, q_logstd, W, bias, C
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtmc_gb300.so")

PRECISIONS = {"fp32": 0, "fp16": 2, "fp32_unfused": 3}
STATUS = {0: "TMC_OK", 1: "TMC_ERR_INVALID_ARG", 2: "TMC_ERR_UNSUPPORTED", 3: "TMC_ERR_NOMEM",
          4: "TMC_ERR_CUDA", 5: "TMC_ERR_NUMERIC", 6: "TMC_ERR_TIMEOUT", 7: "TMC_ERR_STATE"}
KERNEL_CLASSES = ["sample", "project", "edge_fwd", "root", "edge_bwd", "param", "sample_grad"]
EXPORTS = ["tmc_plan_create", "tmc_log_marginal", "tmc_backward", "tmc_plan_sync_status",
           "tmc_plan_workspace_bytes", "tmc_plan_destroy", "tmc_status_string",
           "tmc_profile_enable", "tmc_profile_read", "tmc_log_marginal_noalloc",
           "tmc_plan_instance_times", "tmc_plan_set_schedule", "tmc_plan_get_schedule",
           "tmc_plan_set_wait_limit", "tmc_loopy_plan_create", "tmc_loopy_log_marginal",
           "tmc_loopy_profile", "tmc_loopy_plan_destroy", "tmc_plan_set_tuning", "tmc_plan_get_tuning",
           "tmc_loopy_plan_set_tile"]
TUNING = {"schedule": 0, "prologue_lead": 1, "grid": 2}


class TMCError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS.get(status, str(status))))


class ProblemDesc(ctypes.Structure):
    _fields_ = [("num_instances", ctypes.c_int32), ("n", ctypes.c_void_p),
                ("parent", ctypes.c_void_p), ("K", ctypes.c_void_p), ("d", ctypes.c_void_p),
                ("obs_dim", ctypes.c_void_p), ("shared_params", ctypes.c_int32),
                ("prior_var", ctypes.c_double), ("obs_var", ctypes.c_double),
                ("precision", ctypes.c_int32), ("K_node", ctypes.c_void_p), ("d_node", ctypes.c_void_p),
                ("coupled_proposal", ctypes.c_int32)]


class LoopyDesc(ctypes.Structure):
    _fields_ = [("num_instances", ctypes.c_int32), ("K", ctypes.c_int32), ("d", ctypes.c_int32),
                ("obs_dim", ctypes.c_int32), ("shared_params", ctypes.c_int32),
                ("prior_var", ctypes.c_double), ("obs_var", ctypes.c_double),
                ("message_precision", ctypes.c_int32)]


class Inputs(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("eps", "q_mean", "q_logstd", "W", "bias", "C", "x", "q_A")]


class Grads(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("dz", "dq_mean", "dq_logstd", "dW", "dbias", "dC", "deps",
                                               "dq_A")]


INPUT_NAMES = [f[0] for f in Inputs._fields_]
GRAD_NAMES = [f[0] for f in Grads._fields_]

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (built by ``paper_1806_08593_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("TMC CUDA library not built (%s); run paper_1806_08593_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    P, V = ctypes.c_void_p, ctypes.c_void_p
    lib.tmc_plan_create.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(P)]
    lib.tmc_log_marginal.argtypes = [P, ctypes.POINTER(Inputs), P, V]
    lib.tmc_backward.argtypes = [P, ctypes.POINTER(Inputs), P, ctypes.POINTER(Grads), V]
    lib.tmc_plan_sync_status.argtypes = [P, V]
    lib.tmc_plan_workspace_bytes.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
    lib.tmc_plan_destroy.argtypes = [P]
    lib.tmc_status_string.argtypes = [ctypes.c_int]
    lib.tmc_status_string.restype = ctypes.c_char_p
    lib.tmc_profile_enable.argtypes = [P, ctypes.c_int]
    lib.tmc_profile_read.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_longlong)]
    lib.tmc_log_marginal_noalloc.argtypes = [ctypes.POINTER(ProblemDesc), ctypes.POINTER(Inputs), P, V]
    lib.tmc_plan_instance_times.argtypes = [P, P, P]
    lib.tmc_plan_instance_times.restype = ctypes.c_int
    lib.tmc_plan_set_schedule.argtypes = [P, ctypes.c_int]
    lib.tmc_plan_set_schedule.restype = ctypes.c_int
    lib.tmc_plan_get_schedule.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    lib.tmc_plan_get_schedule.restype = ctypes.c_int
    lib.tmc_plan_set_wait_limit.argtypes = [P, ctypes.c_longlong]
    lib.tmc_plan_set_wait_limit.restype = ctypes.c_int
    lib.tmc_plan_set_tuning.argtypes = [P, ctypes.c_int, ctypes.c_int]
    lib.tmc_plan_get_tuning.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.tmc_loopy_plan_set_tile.argtypes = [P, ctypes.c_int]
    for f in ("tmc_plan_set_tuning", "tmc_plan_get_tuning", "tmc_loopy_plan_set_tile"):
        getattr(lib, f).restype = ctypes.c_int
    lib.tmc_loopy_plan_create.argtypes = [ctypes.POINTER(LoopyDesc), ctypes.POINTER(P)]
    lib.tmc_loopy_log_marginal.argtypes = [P, ctypes.POINTER(Inputs), P, V]
    lib.tmc_loopy_profile.argtypes = [P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.tmc_loopy_plan_destroy.argtypes = [P]
    for f in ("tmc_loopy_plan_create", "tmc_loopy_log_marginal", "tmc_loopy_profile", "tmc_loopy_plan_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    for f in ("tmc_plan_create", "tmc_log_marginal", "tmc_backward", "tmc_plan_sync_status",
              "tmc_plan_workspace_bytes", "tmc_plan_destroy", "tmc_profile_enable", "tmc_profile_read",
              "tmc_log_marginal_noalloc"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != 0:
        raise TMCError(st, where)


def _ptr(t):
    if t is None:
        return None
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """Owns a tmc_plan (topology, schedule, device workspace) for one batch shape."""

    def __init__(self, n, parent, K, d, obs, shared: bool, prior_var: float, obs_var: float,
                 precision: str = "fp32", K_node=None, d_node=None, coupled: bool = False):
        lib = load_library()
        self._keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (n, parent, K, d, obs)]
        n_, par_, K_, d_, o_ = self._keep
        per = [None if a is None else np.ascontiguousarray(a, dtype=np.int32) for a in (K_node, d_node)]
        self._keep += per
        desc = ProblemDesc(len(n_), n_.ctypes.data, par_.ctypes.data, K_.ctypes.data, d_.ctypes.data,
                           o_.ctypes.data, int(bool(shared)), float(prior_var), float(obs_var),
                           PRECISIONS[precision], *[None if a is None else a.ctypes.data for a in per],
                           int(bool(coupled)))
        self.coupled = bool(coupled)
        h = ctypes.c_void_p()
        _check(lib.tmc_plan_create(ctypes.byref(desc), ctypes.byref(h)), "tmc_plan_create")
        self._h = h
        self._lib = lib
        self.B = len(n_)
        self.precision = precision
        self.shared = bool(shared)
        self.forward_calls = 0  # identifies the forward whose state the plan holds

    @classmethod
    def from_problem(cls, p, precision: str = "fp32") -> "Plan":
        return cls(p.n, p.parent, p.K, p.d, p.obs, p.shared, p.prior_var, p.obs_var, precision,
                   K_node=p.Kn, d_node=p.dn, coupled=p.q_A is not None)

    @staticmethod
    def to_device(p, device="cuda") -> dict:
        import torch
        return {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32)).to(device)
                for k in INPUT_NAMES if getattr(p, k, None) is not None}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tmc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- raw C-ABI calls ---------------------------------------------------------------
    def _inputs(self, t: dict) -> Inputs:
        return Inputs(*[_ptr(t.get(k)) for k in INPUT_NAMES])

    def forward(self, t: dict, out=None, stream=None):
        """log P_TMC per instance (float64 CUDA tensor [B])."""
        import torch
        if out is None:
            out = torch.empty(self.B, dtype=torch.float64, device=t["eps"].device)
        inp = self._inputs(t)
        _check(self._lib.tmc_log_marginal(self._h, ctypes.byref(inp), _ptr(out), _stream(stream)),
               "tmc_log_marginal")
        self.forward_calls += 1
        return out

    def backward(self, t: dict, grad_out=None, want=("deps", "dq_mean", "dq_logstd", "dW", "dbias", "dC"),
                 out: dict | None = None, stream=None) -> dict:
        """Gradients of sum_b grad_out[b] log P_TMC_b; ``want`` selects the outputs."""
        import torch
        src = {"dz": "eps", "deps": "eps", "dq_mean": "q_mean", "dq_logstd": "q_logstd",
               "dW": "W", "dbias": "bias", "dC": "C", "dq_A": "q_A"}
        if out is None:
            out = {k: torch.empty_like(t[src[k]]) for k in want}
        g = Grads(*[_ptr(out.get(k)) for k in GRAD_NAMES])
        go = None if grad_out is None else grad_out.to(torch.float64).contiguous()
        inp = self._inputs(t)
        _check(self._lib.tmc_backward(self._h, ctypes.byref(inp), _ptr(go), ctypes.byref(g),
                                      _stream(stream)), "tmc_backward")
        return out

    def sync_status(self, stream=None):
        _check(self._lib.tmc_plan_sync_status(self._h, _stream(stream)), "tmc_plan_sync_status")

    def workspace_bytes(self) -> int:
        v = ctypes.c_size_t()
        _check(self._lib.tmc_plan_workspace_bytes(self._h, ctypes.byref(v)), "tmc_plan_workspace_bytes")
        return int(v.value)

    def set_schedule(self, schedule: int):
        _check(self._lib.tmc_plan_set_schedule(self._h, int(schedule)), "tmc_plan_set_schedule")

    def set_wait_limit(self, cycles: int):
        _check(self._lib.tmc_plan_set_wait_limit(self._h, int(cycles)), "tmc_plan_set_wait_limit")

    def set_tuning(self, knob: str, value: int):
        """One tuning knob of a tensor-core plan (TUNING: schedule, prologue_lead, grid)."""
        _check(self._lib.tmc_plan_set_tuning(self._h, TUNING[knob], int(value)), "tmc_plan_set_tuning")

    def get_tuning(self, knob: str) -> int:
        v = ctypes.c_int()
        _check(self._lib.tmc_plan_get_tuning(self._h, TUNING[knob], ctypes.byref(v)), "tmc_plan_get_tuning")
        return int(v.value)

    def get_schedule(self) -> int:
        v = ctypes.c_int()
        _check(self._lib.tmc_plan_get_schedule(self._h, ctypes.byref(v)), "tmc_plan_get_schedule")
        return int(v.value)

    def instance_times(self):
        """(fwd_us, bwd_us): per-instance completion times of the last persistent edge launches."""
        f = np.zeros(self.B)
        b = np.zeros(self.B)
        _check(self._lib.tmc_plan_instance_times(self._h, f.ctypes.data_as(ctypes.c_void_p),
                                                 b.ctypes.data_as(ctypes.c_void_p)), "tmc_plan_instance_times")
        return f, b

    def profile_enable(self, on: bool = True):
        _check(self._lib.tmc_profile_enable(self._h, int(on)), "tmc_profile_enable")

    def profile_read(self) -> dict:
        res = {}
        for i, name in enumerate(KERNEL_CLASSES):
            ms, n = ctypes.c_double(), ctypes.c_longlong()
            _check(self._lib.tmc_profile_read(self._h, i, ctypes.byref(ms), ctypes.byref(n)),
                   "tmc_profile_read")
            res[name] = (ms.value, n.value)
        return res


class LoopyPlan:
    """Owns a tmc_loopy_plan: log P_TMC of the loopy graph of Fig. 1 (two matrix messages)."""

    MESSAGE_PRECISIONS = {"bf16x2": 0, "bf16": 1}

    def __init__(self, B: int, K: int, d: int, obs: int, shared: bool, prior_var: float, obs_var: float,
                 message_precision: str = "bf16x2"):
        lib = load_library()
        desc = LoopyDesc(int(B), int(K), int(d), int(obs), int(bool(shared)), float(prior_var), float(obs_var),
                         self.MESSAGE_PRECISIONS[message_precision])
        h = ctypes.c_void_p()
        _check(lib.tmc_loopy_plan_create(ctypes.byref(desc), ctypes.byref(h)), "tmc_loopy_plan_create")
        self._h, self._lib, self.B = h, lib, int(B)

    @classmethod
    def from_problem(cls, p, message_precision: str = "bf16x2") -> "LoopyPlan":
        return cls(p.B, p.K, p.d, p.obs, p.shared, p.prior_var, p.obs_var, message_precision)

    @staticmethod
    def to_device(p, device="cuda") -> dict:
        import torch
        return {k: torch.from_numpy(np.ascontiguousarray(getattr(p, k), dtype=np.float32)).to(device)
                for k in ("eps", "q_mean", "q_logstd", "W", "bias", "C", "x")}

    def forward(self, t: dict, out=None, stream=None):
        """log P_TMC per instance (float64 CUDA tensor [B])."""
        import torch
        if out is None:
            out = torch.empty(self.B, dtype=torch.float64, device=t["eps"].device)
        inp = Inputs(*[_ptr(t.get(k)) for k in INPUT_NAMES])
        _check(self._lib.tmc_loopy_log_marginal(self._h, ctypes.byref(inp), _ptr(out), _stream(stream)),
               "tmc_loopy_log_marginal")
        return out

    STAGES = ["prep", "factor", "exp", "message", "final"]

    def set_tile(self, n_tile: int):
        """N tile of the message products: 128, 256, or 0 (automatic)."""
        _check(self._lib.tmc_loopy_plan_set_tile(self._h, int(n_tile)), "tmc_loopy_plan_set_tile")

    def profile(self, enable: bool = True) -> dict:
        """Summed stage times since the last call (ms, keyed by STAGES), the forward calls timed
        and the number of exactly recomputed message entries; then timing on / off."""
        st = np.zeros(len(self.STAGES))
        n, e = ctypes.c_longlong(), ctypes.c_int()
        _check(self._lib.tmc_loopy_profile(self._h, int(enable), st.ctypes.data_as(ctypes.c_void_p),
                                           ctypes.byref(n), ctypes.byref(e)), "tmc_loopy_profile")
        return dict(stage_ms=dict(zip(self.STAGES, st.tolist())), calls=n.value, exact_entries=e.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.tmc_loopy_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def log_marginal_noalloc(p, t: dict, out=None, stream=None):
    """log P_TMC (FP32 path, forward only) through tmc_log_marginal_noalloc: for callers that
    cannot allocate device memory.  ``p`` supplies the description (a workload.Problem or
    anything with n, parent, K, d, obs, shared, prior_var, obs_var); ``t`` the CUDA inputs.
    ``out`` must be preallocated by such callers; if omitted, torch allocates it here."""
    import torch
    lib = load_library()
    keep = [np.ascontiguousarray(a, dtype=np.int32) for a in (p.n, p.parent, p.K, p.d, p.obs)]
    desc = ProblemDesc(len(keep[0]), *[a.ctypes.data for a in keep], int(bool(p.shared)),
                       float(p.prior_var), float(p.obs_var), PRECISIONS["fp32"], None, None)
    if out is None:
        out = torch.empty(len(keep[0]), dtype=torch.float64, device=t["eps"].device)
    inp = Inputs(*[_ptr(t.get(k)) for k in INPUT_NAMES])
    _check(lib.tmc_log_marginal_noalloc(ctypes.byref(desc), ctypes.byref(inp), _ptr(out), _stream(stream)),
           "tmc_log_marginal_noalloc")
    return out


def _autograd():
    import torch

    class TMCLogMarginal(torch.autograd.Function):
        """log P_TMC per instance; backward runs the library's fused adjoint."""

        @staticmethod
        def forward(ctx, plan, eps, q_mean, q_logstd, W, bias, C, x, q_A=None):
            t = dict(eps=eps.contiguous(), q_mean=q_mean.contiguous(), q_logstd=q_logstd.contiguous(),
                     W=W.contiguous(), bias=bias.contiguous(), C=C.contiguous(), x=x.contiguous())
            if q_A is not None:
                t["q_A"] = q_A.contiguous()
            out = plan.forward(t)
            ctx.plan = plan
            ctx.t = t
            ctx.call = plan.forward_calls
            return out

        @staticmethod
        def backward(ctx, grad_out):
            plan, t = ctx.plan, ctx.t
            names = ["deps", "dq_mean", "dq_logstd", "dW", "dbias", "dC", None, "dq_A"]
            flags = ctx.needs_input_grad[1:9]
            want = [n for n, f in zip(names, flags) if f and n]
            if not want:
                return (None,) * 9
            # the adjoint reads the state saved by the matching forward; redo it if another
            # forward ran on this plan in between
            if plan.forward_calls != ctx.call:
                plan.forward(t)
            g = plan.backward(t, grad_out=grad_out.contiguous(), want=want)
            return (None,) + tuple(g.get(n) if n else None for n in names)

    return TMCLogMarginal


_TMC = None


def tmc_log_marginal(plan: Plan, eps, q_mean, q_logstd, W, bias, C, x, q_A=None):
    """Differentiable log P_TMC[b] (float64, [B]) through the CUDA library (q_A: the coupling
    matrices of a coupled-proposal plan)."""
    global _TMC
    if _TMC is None:
        _TMC = _autograd()
    return _TMC.apply(plan, eps, q_mean, q_logstd, W, bias, C, x, q_A)
