"""Coupled (non-factorised) proposals on the GPU against the FP64 oracle, through the C-ABI.

Section 2.3 ("Non-factorised proposals"): sample k of latent i is drawn given its parent's
sample k, Q_i = N(m_i + A_i (z_p^k - m_p), diag(exp(2 logs_i))).  Every output is compared:
log P (1e-4 nats on the FP32 path, 2e-2 and a 1e-3 design margin on the tensor-core path) and
each gradient (dz, deps, the proposal's m, logs and A, and W, bias, C) within 1e-3 relative.
"""
import numpy as np
import pytest

from paper_1806_08593_gb300 import workload as wl
from tests.parity import compare, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-4, "fp16": 1e-3}
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _problem(which):
    if which == "prior_chain":   # the paper's comparison: the prior as the proposal
        return wl.couple_proposal(wl.make_chain(5, 96, 12, 20, 3, seed=901), "prior")
    if which == "scaled_chain":
        return wl.couple_proposal(wl.make_chain(4, 200, 70, 40, 2, seed=902), "scaled", alpha=0.6)
    if which == "trees":
        return wl.couple_proposal(wl.tree_batch(B=6, seed=903), "scaled", alpha=0.5)
    # ragged dimensions (one K per instance).  (With the prior as the proposal this chain's
    # log P is about -1300, where FP32 rounding alone exceeds 1e-4 nats.)
    return wl.couple_proposal(wl.layered_chain([4, 8, 16, 32, 64], 40, obs=64, B=3, seed=904), "scaled",
                              alpha=0.5)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("which", ["prior_chain", "scaled_chain", "trees", "layered"])
def test_coupled_matches_oracle(precision, which):
    p = _problem(which)
    go = np.linspace(0.5, 1.5, p.B)
    got = gpu_run(p, precision, grad_out=go)
    ref = oracle_run(p, grad_out=go)
    rep = compare(p, got, ref, TOL[precision], TOL_GRAD)
    print(which, precision, {k: "%.1e" % v for k, v in rep.items()})


def test_coupled_autograd_fp16():
    import torch
    from paper_1806_08593_gb300.tmc import Plan, tmc_log_marginal
    p = _problem("prior_chain")
    ref = oracle_run(p)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    for k in ("eps", "q_mean", "q_logstd", "q_A", "W"):
        t[k].requires_grad_(True)
    lp = tmc_log_marginal(plan, t["eps"], t["q_mean"], t["q_logstd"], t["W"], t["bias"], t["C"], t["x"], t["q_A"])
    lp.sum().backward()
    torch.cuda.synchronize()
    plan.sync_status()
    for name, key in (("eps", "deps"), ("q_mean", "dq_mean"), ("q_logstd", "dq_logstd"), ("q_A", "dq_A"),
                      ("W", "dW")):
        g = t[name].grad.double().cpu().numpy()
        e = np.linalg.norm(g - ref[key]) / np.linalg.norm(ref[key])
        assert e <= TOL_GRAD, (name, e)
    plan.close()
