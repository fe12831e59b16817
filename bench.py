"""TMC hot-path benchmark: forward + backward factor entries per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload chain_n16_K1024_d128_B64] [--precision fp32|fp16]

A step is one full pass of the hot path over one batch of synthetic linear-Gaussian
instances: samples and node terms, conditional means, the fused pairwise-factor +
log-sum-exp messages from the leaves to the root, the FP64 root reduction, the fused
adjoint, and the gradients w.r.t. the proposal (m, logs) and the model (W, bias, C).
Unit of work: B*n*K^2 factor entries per step (summed over instances).

Prints ONE JSON line (rank 0).  Under torchrun each rank runs an independent replica of
the workload on its own GPU (no data-path collective; the path has no exchange step
because instances are independent), so scaling is weak and `value` sums all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "chain_n16_K1024_d128_B64"
# A training step needs the gradients of every parameter of the model and the proposal.
GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")
GRAD_SRC = {"dq_mean": "q_mean", "dq_logstd": "q_logstd", "dW": "W", "dbias": "bias", "dC": "C",
            "dq_A": "q_A"}


def step_grads(p):
    """The gradients of a training step: every model and proposal parameter (with a coupled
    proposal its couplings A_i as well)."""
    return GRADS + (("dq_A",) if p.q_A is not None else ())


FP32_LANES_PER_SM = 128
NUM_SMS = 152
SM_MAX_MHZ = 2070.0


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def make_workload(name):
    """A named workload, 'chain:n=..,K=..,d=..,obs=..,B=..' (same generator, seed 1), or
    'star:N=..,K=..,d=..,B=..' (one latent with N observed children)."""
    from paper_1806_08593_gb300 import workload as wl
    if name in wl.CHAIN_CONFIGS:
        return wl.chain_config(name)
    if name.startswith("trees"):
        return wl.tree_batch()
    if name.startswith("star:"):  # the Section 3.1 toy at scale: N children of one latent
        kv = dict(x.split("=") for x in name[5:].split(","))
        c = {k: int(v) for k, v in kv.items()}
        p = wl.star(c["N"], c["K"], c.get("d", 1), c.get("obs"), c.get("B", 1))
        p.name = name
        return p
    if name.startswith("layered:"):  # the paper's five-layer widths 4/8/16/32/64 (per-latent d_i)
        kv = dict(x.split("=") for x in name[8:].split(",") if x)
        c = {k: int(v) for k, v in kv.items()}
        p = wl.layered_chain([4, 8, 16, 32, 64], c.get("K", 20), c.get("obs", 96), c.get("B", 16384), seed=1)
        p.name = name
        return p
    if name.startswith("coupled:"):  # the prior as a coupled (non-factorised) proposal
        p = wl.couple_proposal(make_workload(name[8:]), "prior")
        p.name = name
        return p
    if name.startswith("chain:"):
        kv = dict(x.split("=") for x in name[6:].split(","))
        c = {k: int(v) for k, v in kv.items()}
        p = wl.make_chain(c["n"], c["K"], c["d"], c.get("obs", 2 * c["d"]), c["B"], seed=1)
        p.name = name
        return p
    raise SystemExit("unknown workload %s" % name)


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 20 ms with host timestamps; summary()
    keeps the samples taken inside the timed window (mark_start / mark_end)."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            deadline = time.time() + 10.0  # the timed window opens once sampling runs
            while not self.lines and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        if self.t0 is not None and self.t1 is not None:
            inside = [x for x in lines if self.t0 <= x[0] <= self.t1 + 0.02]
            lines = inside if inside else sorted(lines, key=lambda x: abs(x[0] - self.t1))[:1]
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# multi-rank helpers (replicas only)
# ---------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of instances
# ---------------------------------------------------------------------------------------
def oracle_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def gpu_local_cpus(dev):
    """The CPUs the system lists as local to the GPU (sysfs), intersected with the ones this
    process may use; None when either is unknown or they coincide."""
    import torch
    try:
        pr = torch.cuda.get_device_properties(dev)
        bus = "%04x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        txt = open("/sys/bus/pci/devices/%s/local_cpulist" % bus).read().strip()
        cpus = set()
        for part in txt.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        allowed = os.sched_getaffinity(0)
        use = cpus & allowed
        return use if use and use != allowed else None
    except Exception:
        return None


def time_oracle_sample(p, target_s=15.0, max_inst=None):
    import oracle
    oracle.build()
    entries_per_inst = p.entries() / p.B
    n_inst, elapsed, done = 1, 0.0, 0
    t_all = wall = 0.0
    logp = []
    while True:
        idx = list(range(done, min(p.B, done + n_inst)))
        if not idx:
            break
        t_sub = time.perf_counter()
        sub = oracle.subset(p, idx)
        t0 = time.perf_counter()
        g = oracle.grad(sub)
        dt = time.perf_counter() - t0
        logp.extend(g["log_phat"].tolist())
        t_all += dt
        wall += time.perf_counter() - t_sub
        done += len(idx)
        # the budget bounds the wall time as well: cutting a sample out of a large batch
        # can cost more than the oracle itself on small instances
        if t_all >= target_s or wall >= 2 * target_s or done >= p.B or (max_inst and done >= max_inst):
            break
        n_inst = max(1, int(len(idx) * min(4.0, (target_s - t_all) / max(dt, 1e-3))))
    return entries_per_inst * done / t_all, done, t_all, np.array(logp)


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    p = make_workload(args.workload)
    vals = []
    # bounded steps: one instance per step keeps K+W steps within minutes
    import oracle
    oracle.build()
    sub = oracle.subset(p, [0])
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.grad(sub)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            vals.append(dt)
    t = float(np.mean(vals))
    value = sub.entries() / t
    line = {
        "impl": "reference", "metric": "tmc_fwd_bwd_factor_entries_per_s", "value": value,
        "unit": "entries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": "1 instance of %d per step" % p.B},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": oracle_cores(),
                         "kind": "oracle", "sample": "instance 0 of the workload, fwd+bwd, FP64"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------
# kernel launches of one step, counted by the CUDA profiler (every kernel of the process:
# the library's, and torch's if any ran)
# ---------------------------------------------------------------------------------------
def count_kernel_launches(fn, dev):
    import torch
    from torch.profiler import ProfilerActivity, profile
    torch.cuda.synchronize(dev)
    for _ in range(2):  # the first session of a process can come back empty: keep the second
        with profile(activities=[ProfilerActivity.CUDA]) as pr:
            fn()
            torch.cuda.synchronize(dev)
    names = [e.name for e in pr.events()
             if str(getattr(e, "device_type", "")).endswith("CUDA") and "Memset" not in e.name
             and "Memcpy" not in e.name]
    return len(names), sorted(set(names))


# ---------------------------------------------------------------------------------------
# the loopy graph of Fig. 1 (two matrix messages): forward log P per instance
# ---------------------------------------------------------------------------------------
LOOPY = dict(K=4096, d=128, obs=128, B=4)
# DRAM bytes (read + write) of one message launch per instance, single bf16 operands, from an
# ncu capture of k_gemm_split<1,256> at K=4096, d=128, B=1 (scaled by instances)
LOOPY_MSG_TRAFFIC_PER_INSTANCE = {(4096, 128): 280.3e6}


def loopy_config(spec):
    """'diamond:K=..,d=..,obs=..,B=..' (missing keys from LOOPY), or None for LOOPY."""
    c = dict(LOOPY)
    if spec:
        if not spec.startswith("diamond:"):
            raise SystemExit("unknown loopy workload %s" % spec)
        c.update({k: int(v) for k, v in (x.split("=") for x in spec[8:].split(","))})
    return c


def loopy_leg(args, dev):
    """The Fig. 1 graph at K=4096, d=128: log P_TMC of B instances per step.  Unit: message
    terms, 2 K^3 per instance (the (k2, k3, k4) and (k2, k3, k1) terms the two matrix messages
    sum).  Both message precisions are timed; single bf16 is the headline (its |delta log P|
    bound, 7.8e-3, is within the 2e-2 reduced-precision tolerance)."""
    import torch
    from paper_1806_08593_gb300 import workload as wl
    from paper_1806_08593_gb300.tmc import LoopyPlan
    c = loopy_config(args.loopy_workload)
    p = wl.make_diamond(c["K"], c["d"], c["obs"], c["B"], seed=1, shared=True)
    terms = 2.0 * p.K ** 3 * p.B
    msg_flops = 4.0 * p.K ** 3 * p.B          # two K x K x K products per instance
    fac_flops = 10.0 * p.K ** 2 * p.d * p.B   # five K x K x d products per instance
    stream = torch.cuda.current_stream(dev)
    res = {}
    for mp in ("bf16", "bf16x2"):
        plan = LoopyPlan.from_problem(p, mp)
        t = plan.to_device(p, dev)
        out = torch.empty(p.B, dtype=torch.float64, device=dev)
        tuned = None
        if args.autotune:
            from paper_1806_08593_gb300.autotune import autotune_loopy
            tuned = autotune_loopy(plan, p, t, cache_path=None)
        for _ in range(3):
            plan.forward(t, out=out)
        torch.cuda.synchronize(dev)
        steps = max(3, args.steps // 5)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            plan.forward(t, out=out)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms = ev0.elapsed_time(ev1) / steps
        plan.profile(True)
        for _ in range(steps):
            plan.forward(t, out=out)
        pr = plan.profile(False)
        st = {k: v / pr["calls"] for k, v in pr["stage_ms"].items()}
        launches, _ = count_kernel_launches(lambda: plan.forward(t, out=out), dev)
        res[mp] = {"ms_per_step": ms, "value": terms / (ms * 1e-3), "stage_ms": st,
                   "exact_entries_per_step": pr["exact_entries"] / max(1, pr["calls"]),
                   "message_tflops": msg_flops / (st["message"] * 1e-3) / 1e12,
                   "factor_tflops": fac_flops / (st["factor"] * 1e-3) / 1e12,
                   "gpu_launches_per_step": launches, "logp": out.cpu().numpy().tolist(),
                   "autotune": tuned}
        plan.close()
        del t
    peaks, src = load_peaks()
    head = res["bf16"]
    peak = peaks["bf16_tflops"]
    line = {"workload": "diamond_K%d_d%d_obs%d_B%d" % (p.K, p.d, p.obs, p.B),
            "metric": "loopy_message_terms_per_s", "unit": "terms/s", "value": head["value"],
            "ms_per_step": head["ms_per_step"], "message_precision": "bf16",
            "max_abs_dlogp_bf16_vs_bf16x2": float(np.max(np.abs(np.array(head["logp"]) -
                                                                np.array(res["bf16x2"]["logp"])))),
            "roofline": {"bound": "tensor", "kernel": "k_gemm_split<1,256> (both messages)",
                         "achieved": head["message_tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": head["message_tflops"] / peak,
                         "traffic": LOOPY_MSG_TRAFFIC_PER_INSTANCE.get((p.K, p.d)) and
                         LOOPY_MSG_TRAFFIC_PER_INSTANCE[(p.K, p.d)] * p.B,
                         "peak_source": "bf16_tflops (%s)" % src,
                         "flops_per_launch": msg_flops},
            "split": res["bf16x2"], "single": res["bf16"]}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        Ks = 256
        q = wl.make_diamond(Ks, c["d"], c["obs"], 1, seed=1, shared=True)
        t0 = time.perf_counter()
        n = 0
        while True:
            oracle.diamond_log_marginal(q)
            n += 1
            if time.perf_counter() - t0 >= min(10.0, args.cpu_seconds):
                break
        dt = (time.perf_counter() - t0) / n
        line["cpu_baseline"] = {"value": 2.0 * Ks ** 3 / dt, "unit": "terms/s", "cores": oracle_cores(),
                                "kind": "oracle",
                                "sample": "1 instance at K=%d (d=%d, obs=%d), %d runs, FP64" % (Ks, c["d"], c["obs"], n)}
    return line


# ---------------------------------------------------------------------------------------
# the other workloads of the hot path, one short timing each
# ---------------------------------------------------------------------------------------
WIDENING = (
    ("trees", "512 uneven trees, per-instance models (config 5)"),
    ("layered:B=16384,K=20", "five-layer chain, widths 4/8/16/32/64, K=20 (per-latent d_i)"),
    ("coupled:chain_n16_K1024_d128_B64", "the bench chain with the prior as a coupled proposal"),
    ("star:N=10000,K=128,d=1", "one root with 10^4 children (Section 3.1 toy at scale)"),
)


def widening_leg(args, dev):
    """Each workload once: device time per training step (log P and every parameter gradient,
    plain launches, default work order, CUDA events over 10 steps after 3 warm-up steps) and
    |delta log P| to the oracle on its first and last instance."""
    import oracle
    oracle.build()
    res = {}
    for name, what in WIDENING:
        p = make_workload(name)
        ms, lp = time_plan_steps(p, args.precision, dev, steps=10, warmup=3)
        idx = sorted({0, p.B - 1})
        ref = oracle.log_marginal(oracle.subset(p, idx))
        res[name] = {"what": what, "ms_per_step": ms, "value": p.entries() / (ms * 1e-3),
                     "unit": "entries/s", "B": int(p.B), "entries_per_step": int(p.entries()),
                     "grads": list(step_grads(p)),
                     "max_abs_dlogp_vs_oracle": float(np.max(np.abs(lp[idx] - ref))),
                     "instances_checked": idx}
        del p
    # config 2's materialised-factor baseline: the FP32 forward with and without the factors
    # written to memory and read back
    p = make_workload("chain_n8_K128_d32_B256")
    ms_f, lp_f = time_forward(p, "fp32", dev, steps=10, warmup=3)
    ms_u, lp_u = time_forward(p, "fp32_unfused", dev, steps=10, warmup=3)
    ms_t, _ = time_forward(p, "fp16", dev, steps=10, warmup=3)
    res["unfused:chain_n8_K128_d32_B256"] = {
        "what": "forward only: fused FP32 kernels against the materialised-factor baseline",
        "fused_fp32_fwd_ms": ms_f, "unfused_fp32_fwd_ms": ms_u, "fused_speedup": ms_u / ms_f,
        "fp16_fwd_ms": ms_t, "factor_bytes_written": 4 * p.edge_entries(),
        "max_abs_dlogp_unfused_vs_fused": float(np.max(np.abs(lp_u - lp_f)))}
    return res


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def algorithmic_flops(p, precision):
    """Algorithmic FLOPs of the edge kernels per step, per edge p -> i: forward 2*K_p*K_i*d_i
    (S = mu~ z~^T); adjoint 2*K_p*K_i*(d_i + d_p) (S recomputed, V = P z~_p), i.e. 4*K^2*d for
    uniform sizes.  The split-fp16 tensor-core path executes each S product as 3 MMAs; those
    extra MMAs are not counted."""
    Kn, dn = p.K_nodes().astype(np.int64), p.d_nodes().astype(np.int64)
    fwd = bwd = 0.0
    off = 0
    for b in range(p.B):
        par = p.parents_of(b)
        for i in range(1, len(par)):
            kk = float(Kn[off + par[i]] * Kn[off + i])
            fwd += 2.0 * kk * dn[off + i]
            bwd += 2.0 * kk * (dn[off + i] + dn[off + par[i]])
        off += len(par)
    return {"edge_fwd": fwd, "edge_bwd": bwd}


def time_forward(p, precision, dev, steps, warmup):
    """Device time per forward pass of a plan (log P only)."""
    import torch
    from paper_1806_08593_gb300.tmc import Plan
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p, dev)
    out = torch.empty(p.B, dtype=torch.float64, device=dev)
    for _ in range(warmup):
        plan.forward(t, out=out)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.forward(t, out=out)
    e1.record()
    torch.cuda.synchronize(dev)
    plan.sync_status()
    ms = e0.elapsed_time(e1) / steps
    lp = out.cpu().numpy()
    plan.close()
    del t
    torch.cuda.empty_cache()
    return ms, lp


def time_plan_steps(p, precision, dev, steps, warmup):
    """Device time per fwd+bwd step of a plan at the given precision (for the comparison)."""
    import torch
    from paper_1806_08593_gb300.tmc import Plan
    plan = Plan.from_problem(p, precision)
    t = plan.to_device(p, dev)
    out = torch.empty(p.B, dtype=torch.float64, device=dev)
    want = step_grads(p)
    g = {k: torch.empty_like(t[GRAD_SRC[k]]) for k in want}
    for _ in range(warmup):
        plan.forward(t, out=out)
        plan.backward(t, out=g, want=want)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.forward(t, out=out)
        plan.backward(t, out=g, want=want)
    e1.record()
    torch.cuda.synchronize(dev)
    plan.sync_status()
    ms = e0.elapsed_time(e1) / steps
    lp = out.cpu().numpy()
    plan.close()
    del t, g
    torch.cuda.empty_cache()
    return ms, lp


# DRAM bytes per 128-row edge tile of the persistent edge kernels, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum) of chain n=3, K=1024, d=128, obs=256, B=64:
# 1024 tiles per launch, forward 113.2 MB, adjoint 126.2 MB.  Scaled by the tiles of a launch;
# only quoted for that K and d, and only while the kernels are the captured ones.
TRAFFIC_PER_TILE = {("edge_fwd", 1024, 128): 123.1e6 / 1024, ("edge_bwd", 1024, 128): 134.2e6 / 1024}


def edge_tiles(p):
    return int(sum((p.n[b] - 1) * ((int(p.K[b]) + 127) // 128) for b in range(p.B)))


def traffic_per_launch(p, kernel):
    ks, ds = set(int(k) for k in p.K), set(int(d) for d in p.d)
    if len(ks) != 1 or len(ds) != 1:
        return None
    per = TRAFFIC_PER_TILE.get((kernel, ks.pop(), ds.pop()))
    return None if per is None else per * edge_tiles(p)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1806_08593_gb300.build import build
    if rank == 0 or ws == 1:
        build()
    barrier()
    from paper_1806_08593_gb300.tmc import Plan

    p = make_workload(args.workload)
    plan = Plan.from_problem(p, args.precision)
    t = plan.to_device(p, dev)
    out_lp = torch.empty(p.B, dtype=torch.float64, device=dev)
    GR = step_grads(p)
    grads = {k: torch.empty_like(t[GRAD_SRC[k]]) for k in GR}
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.forward(t, out=out_lp)
        plan.backward(t, out=grads, want=GR)

    tuned = None
    if args.autotune and args.precision == "fp16":
        from paper_1806_08593_gb300.autotune import autotune
        tuned = autotune(plan, p, t, cache_path=None)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    plan.sync_status()

    # ---- device-resident timed region (CUDA events on the launch stream) ---------------
    graph = None
    if args.graph:
        # the whole step (all launches, memsets) captured once and replayed
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            step()
        stream.wait_stream(side)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        torch.cuda.synchronize(dev)
        graph.replay()
        torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local if ws > 1 else 0) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        clk.mark_start()
        ev0.record(stream)
        for _ in range(args.steps):
            if graph is not None:
                graph.replay()
            else:
                step()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
        barrier()
    ms = ev0.elapsed_time(ev1)
    # kernel-class times from a separate pass (the library's profiling events stay out of the
    # timed region)
    plan.profile_enable(True)
    for _ in range(args.steps):
        step()
    prof = plan.profile_read()
    plan.profile_enable(False)
    plan.sync_status()
    latency = None
    if args.precision == "fp16":
        step()
        f_us, b_us = plan.instance_times()
        latency = {"unit": "us", "fwd_p50": float(np.percentile(f_us, 50)), "fwd_p99": float(np.percentile(f_us, 99)),
                   "bwd_p50": float(np.percentile(b_us, 50)), "bwd_p99": float(np.percentile(b_us, 99)),
                   "definition": "time from the first edge tile of the persistent edge launch to the "
                                 "instance's last tile, per direction"}
    ms_max = max_over_ranks(ms, dev)
    ms_step = ms_max / args.steps
    entries = p.entries()
    value = entries * ws / (ms_step * 1e-3)

    # ---- end to end through host buffers ---------------------------------------------
    # Every step copies its inputs from pinned host memory and reads its results back inside
    # the timed region.  The uploads run on a copy stream into one of two device input sets,
    # so step i + 1's upload overlaps step i's kernels (as a serving loop would run them).
    # pinned host buffers are placed while the process runs on the GPU's own CPUs (when the
    # system reports them), so the uploads do not cross a socket link
    numa = gpu_local_cpus(dev)
    prev_aff = os.sched_getaffinity(0) if numa else None
    if numa:
        os.sched_setaffinity(0, numa)
    host_in = {k: v.cpu().pin_memory() for k, v in t.items()}
    dev_in = [{k: torch.empty_like(v) for k, v in t.items()} for _ in range(2)]
    host_out = {k: torch.empty(grads[k].shape, dtype=grads[k].dtype).pin_memory() for k in GR}
    host_lp = torch.empty(p.B, dtype=torch.float64).pin_memory()
    if numa:
        os.sched_setaffinity(0, prev_aff)
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = host_lp.numel() * 8 + sum(v.numel() * v.element_size() for v in host_out.values())
    copy_stream = torch.cuda.Stream(device=dev)
    uploaded = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    copy_ms = []  # duration of each upload of the timed run (diagnostic: host link bandwidth)

    def upload(i):
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(consumed[i % 2])  # the step that last read this set is done
            c0 = torch.cuda.Event(enable_timing=True)
            c0.record(copy_stream)
            for k, v in dev_in[i % 2].items():
                v.copy_(host_in[k], non_blocking=True)
            uploaded[i % 2].record(copy_stream)
            copy_ms.append((c0, uploaded[i % 2]))

    def e2e_run(nsteps):
        for i in range(2):
            consumed[i].record(stream)
        upload(0)
        for i in range(nsteps):
            if i + 1 < nsteps:
                upload(i + 1)
            stream.wait_event(uploaded[i % 2])
            plan.forward(dev_in[i % 2], out=out_lp)
            plan.backward(dev_in[i % 2], out=grads, want=GR)
            consumed[i % 2].record(stream)
            host_lp.copy_(out_lp, non_blocking=True)
            for k in GR:
                host_out[k].copy_(grads[k], non_blocking=True)

    e2e_run(2)
    torch.cuda.synchronize(dev)
    e2e_steps = max(3, args.steps // 2)
    barrier()
    ev0.record(stream)
    e2e_run(e2e_steps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    e2e_ms = max_over_ranks(ev0.elapsed_time(ev1), dev) / e2e_steps
    # an upload's events are re-recorded two uploads later: time each before it is reused
    up_ms = [a.elapsed_time(b) for a, b in copy_ms[-2:]]
    h2d_gbs = h2d / (float(np.mean(up_ms)) * 1e-3) / 1e9 if up_ms else None
    plan.sync_status()

    if rank != 0:
        return
    # ---- roofline of the dominant kernel class ---------------------------------------
    peaks, src = load_peaks()
    flops = algorithmic_flops(p, args.precision)
    dom = max(("edge_fwd", "edge_bwd"), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    launches_per_step = dom_n / args.steps
    per_launch_ms = dom_ms / dom_n
    per_launch_flop = flops[dom] / launches_per_step
    achieved = per_launch_flop / (per_launch_ms * 1e-3)
    if args.precision == "fp32":
        peak = NUM_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6
        roof = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "kernel": dom,
                "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"}
    else:
        peak = peaks["bf16_tflops"] * 1e12
        traffic = traffic_per_launch(p, dom) if args.precision == "fp16" else None
        roof = {"bound": "tensor", "achieved": achieved / 1e12, "peak": peak / 1e12,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                "peak_source": "bf16_tflops (%s)" % src}
    lib_launches = int(sum(v[1] for v in prof.values()))
    try:
        per_step, kernel_names = count_kernel_launches(step, dev)
        if per_step == 0:  # another profiler holds the CUDA activity API (e.g. under ncu)
            raise RuntimeError("no kernel activity recorded")
        total_launches = per_step * args.steps
        launch_src = "CUDA profiler, one step x steps (%d kernels per step, %d distinct)" % (
            per_step, len(kernel_names))
    except Exception as exc:  # profiler unavailable: the library's own count of timed calls
        total_launches, kernel_names = lib_launches, []
        launch_src = "library timing wrappers (profiler unavailable: %s)" % type(exc).__name__

    # ---- the same step on the FP32 CUDA-core path, and the log P agreement ------------
    fp32 = None
    if args.precision != "fp32" and not args.no_fp32_compare:
        lp_ours = out_lp.cpu().numpy()
        ms32, lp32 = time_plan_steps(p, "fp32", dev, steps=3, warmup=1)
        fp32 = {"value": entries / (ms32 * 1e-3), "ms_per_step": ms32,
                "speedup": ms32 / ms_step,
                "max_abs_dlogp_vs_fp32": float(np.max(np.abs(lp_ours - lp32)))}

    # ---- the same step with the per-sample gradients dz / deps as well -----------------
    sample_grads = None
    if args.precision == "fp16" and not args.no_sample_grads:
        want = GR + ("dz", "deps")
        gz = dict(grads)
        gz["dz"] = torch.empty_like(t["eps"])
        gz["deps"] = torch.empty_like(t["eps"])
        for _ in range(2):
            plan.forward(t, out=out_lp)
            plan.backward(t, out=gz, want=want)
        torch.cuda.synchronize(dev)
        nz = max(3, args.steps // 5)
        ev0.record(stream)
        for _ in range(nz):
            plan.forward(t, out=out_lp)
            plan.backward(t, out=gz, want=want)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        ms_z = ev0.elapsed_time(ev1) / nz
        plan.profile_enable(True)
        for _ in range(nz):
            plan.forward(t, out=out_lp)
            plan.backward(t, out=gz, want=want)
        pz = plan.profile_read()
        plan.profile_enable(False)
        plan.sync_status()
        sample_grads = {"ms_per_step": ms_z, "extra_ms_per_step": ms_z - ms_step,
                        "value": entries / (ms_z * 1e-3), "grads": list(want), "steps": nz,
                        "graph": False,
                        "kernel_ms_per_step": {k: v[0] / nz for k, v in pz.items()}}
        del gz

    # ---- materialised-factor baseline (forward only, FP32) ----------------------------
    unfused = None
    if args.compare_unfused:
        ms_f, lp_f = time_forward(p, "fp32", dev, steps=max(3, args.steps), warmup=3)
        ms_u, lp_u = time_forward(p, "fp32_unfused", dev, steps=max(3, args.steps), warmup=3)
        ms_t, lp_t = time_forward(p, args.precision, dev, steps=max(3, args.steps), warmup=3)
        unfused = {"fused_fp32_fwd_ms": ms_f, "unfused_fp32_fwd_ms": ms_u,
                   "fused_speedup": ms_u / ms_f, "%s_fwd_ms" % args.precision: ms_t,
                   "factor_bytes_written": 4 * p.edge_entries(),
                   "max_abs_dlogp_unfused_vs_fused": float(np.max(np.abs(lp_u - lp_f)))}

    # ---- the loopy graph of Fig. 1 (matrix messages) ----------------------------------
    loopy = None
    if not args.no_loopy and ws == 1:
        loopy = loopy_leg(args, dev)
    widening = None
    if not args.no_widening and args.workload == DEFAULT_WORKLOAD and ws == 1 and args.precision == "fp16":
        widening = widening_leg(args, dev)

    # ---- CPU baseline (oracle on a bounded sample) ------------------------------------
    cpu = None
    vs_oracle = None
    if not args.no_cpu_baseline and ws == 1:
        v, ninst, secs, ref_lp = time_oracle_sample(p, target_s=args.cpu_seconds)
        cpu = {"value": v, "unit": "entries/s", "cores": oracle_cores(), "kind": "oracle",
               "sample": "%d of %d instances, fwd+bwd FP64, %.1f s" % (ninst, p.B, secs)}
        # the oracle's log P of those instances against this run's (same inputs)
        d_lp = np.abs(out_lp.cpu().numpy()[:ninst] - ref_lp)
        vs_oracle = {"max_abs_dlogp": float(d_lp.max()), "median_abs_dlogp": float(np.median(d_lp)),
                     "instances": int(ninst), "tolerance": 2e-2 if args.precision == "fp16" else 1e-4}

    line = {
        "metric": "tmc_fwd_bwd_factor_entries_per_s", "value": value, "unit": "entries/s",
        "n_gpus": ws, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp16": "f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": args.workload, "B": int(p.B), "n": int(p.n[0]), "K": int(p.K[0]),
                   "d": int(p.d[0]), "obs": int(p.obs[0]), "precision": args.precision,
                   "cuda_graph": bool(args.graph),
                   "schedule": plan.get_schedule() if args.precision == "fp16" else None,
                   "autotune": tuned,
                   "entries_per_step": entries, "grads": list(GR),
                   "l2": "inputs larger than L2 (eps %.0f MB per step)" % (p.eps.nbytes / 1e6),
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "vs_oracle": vs_oracle,
        "e2e": {"value": entries * ws / (e2e_ms * 1e-3), "unit": "entries/s",
                "h2d_gbs": h2d_gbs, "host_cpus": (sorted(numa)[0], sorted(numa)[-1]) if numa else None,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "fp32_path": fp32,
        "unfused_baseline": unfused,
        "sample_grads": sample_grads,
        "instance_latency": latency,
        "gpu_launches": total_launches,
        "gpu_launches_source": launch_src,
        "kernels": kernel_names,
        "kernel_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
        "clocks": clk.summary(),
        "loopy": loopy,
        "widening": widening,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", default=os.environ.get("TMC_BENCH_PRECISION", "fp16"),
                    choices=["fp32", "fp16"])
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--autotune", action=argparse.BooleanOptionalAction, default=True,
                    help="time every combination of the persistent-launch knobs (work order, prologue "
                         "lead, grid) on the workload first and keep the fastest (default; the loopy leg "
                         "tunes the N tile of its message products)")
    ap.add_argument("--graph", action=argparse.BooleanOptionalAction, default=True,
                    help="capture one step in a CUDA graph and time graph replays (default; "
                         "--no-graph times plain launches)")
    ap.add_argument("--compare-unfused", action="store_true",
                    help="also time the FP32 forward with every K x K factor materialised")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sample-grads", action="store_true",
                    help="skip the extra timing of the step with the per-sample gradients dz, deps")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-loopy", action="store_true",
                    help="skip the loopy-graph (Fig. 1, matrix messages) leg")
    ap.add_argument("--no-widening", action="store_true",
                    help="skip the short timings of the other workloads (trees, layered, coupled, star)")
    ap.add_argument("--loopy-only", action="store_true",
                    help="run only the loopy-graph leg and print its JSON object")
    ap.add_argument("--loopy-workload", default=None,
                    help="diamond:K=..,d=..,obs=..,B=.. (default K=4096,d=128,obs=128,B=4)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.loopy_only:
        import torch
        from paper_1806_08593_gb300.build import build
        build()
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        print(json.dumps(loopy_leg(args, dev)))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
