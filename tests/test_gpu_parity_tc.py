"""Tensor-core (tcgen05, split-fp16) path vs the FP64 oracle through the C-ABI.

Tolerances: |delta log P| <= 2e-2 nats per instance (reduced-precision path) and gradients
within 1e-3 relative per tensor -- the parameter and proposal gradients and the per-sample
gradients dz and deps.  The split hi/lo fp16 operands give ~22-bit products, so the measured
errors are far smaller; TOL_LOGP_DESIGN (1e-3) pins that design margin.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.parity import compare, gpu_run, mixed_roots_problem, oracle_run

pytestmark = pytest.mark.gpu
TOL_LOGP = 2e-2
TOL_LOGP_DESIGN = 1e-3
TOL_GRAD = 1e-3
PARAM_GRADS = ("dq_mean", "dq_logstd", "dW", "dbias", "dC")
ALL_GRADS = PARAM_GRADS + ("dz", "deps")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def _check(p, grad_out=None, want=ALL_GRADS):
    got = gpu_run(p, "fp16", grad_out=grad_out, want=want)
    ref = oracle_run(p, grad_out=grad_out)
    rep = compare(p, got, ref, TOL_LOGP_DESIGN, TOL_GRAD, keys=list(want))
    print(p.name or "problem", {k: "%.1e" % v for k, v in rep.items()})
    assert rep["log_phat_max_abs"] <= TOL_LOGP
    return rep


def test_config1_tc():
    _check(wl.chain_config("chain_n3_K4_d2_B8"))


@pytest.mark.parametrize("n,K,d,obs,B", [
    (5, 100, 24, 40, 3),      # ragged K, d in the 64-wide class
    (4, 300, 64, 50, 2),      # three chunks, d exactly 64
    (3, 260, 100, 129, 2),    # d in the 128-wide class, obs > 128
    (4, 128, 128, 256, 2),    # exact tiles, d = 128
    (1, 77, 9, 5, 3),         # single latent
    (6, 1, 3, 4, 2),          # K = 1
    (3, 1100, 24, 40, 2),     # K > 1024: node moments over two items (atomics), ragged unit
    (2, 1300, 100, 64, 1),    # the same in the 128-wide class
])
def test_chains_tc(n, K, d, obs, B):
    _check(wl.make_chain(n, K, d, obs, B, seed=2000 + n * 7 + K + d), grad_out=np.linspace(0.5, 1.5, B))


@pytest.mark.parametrize("B,layered", [(150, False), (70, True)])
def test_shared_many_instances_tc(B, layered):
    """One model shared by many instances: the gradients of the shared W, bias and C are sums
    over instances (groups of 8 instances, then a tree of 64-row chunks; 150 instances take
    two levels), weighted by a different grad_out per instance."""
    if layered:
        p = wl.layered_chain([4, 8, 16, 32, 64], 20, obs=40, B=B, seed=717)
    else:
        p = wl.make_chain(4, 16, 24, 30, B, seed=716)
    _check(p, grad_out=np.linspace(0.25, 1.75, B))


def test_many_nodes_tc():
    """More than 8192 latents, non-root latents and leaves: the per-node set-up kernels take
    four nodes per CTA (9000 observed children of one root)."""
    _check(wl.star(9000, 16, 2, B=1, seed=1236))


def test_uneven_trees_tc():
    _check(wl.tree_batch(B=10, seed=777))


def test_star_fig2_tc():
    parent = np.array([-1] + [0] * 9, dtype=np.int32)
    _check(wl.make_problem([parent] * 3, [200] * 3, [20] * 3, [7] * 3, shared=True, seed=98))


def test_large_star_tc():
    # the Section 3.1 toy at scale: one latent with 2000 observed children, d = 1
    _check(wl.star(2000, 128, 1, B=2, seed=1234))


@pytest.mark.parametrize("which", ["layered", "trees", "shared_K", "wide"])
def test_ragged_tc(which):
    """A different K_i and d_i per latent (Eq. (is)); W_i of shape d_i x d_parent."""
    if which == "layered":  # the paper's five-layer widths, K = 20, synthetic observations
        p = wl.layered_chain([4, 8, 16, 32, 64], 20, obs=96, B=6, seed=711)
    elif which == "trees":
        p = wl.ragged_trees(8, seed=712, n_choices=(1, 3, 6, 9), Ks=(1, 17, 64, 100, 130),
                            ds=(1, 8, 24, 65), max_depth=4)
    elif which == "shared_K":  # shared model, K_i differing between instances too
        p = wl.make_problem([wl.chain_parents(4)] * 3, [[70, 20, 130, 64], [5, 90, 64, 64], [128] * 4],
                            [[6, 33, 70, 12]] * 3, [24] * 3, shared=True, seed=713)
    else:  # both dimension classes in one instance, several chunks per edge
        p = wl.make_problem([np.array([-1, 0, 1, 1, 0], dtype=np.int32)] * 2,
                            [[300, 129, 260, 90, 200], [64, 256, 128, 300, 40]],
                            [[128, 40, 100, 100, 100], [30, 128, 100, 100, 100]], [64, 70],
                            shared=False, seed=714)
    assert p.ragged
    _check(p, grad_out=np.linspace(0.5, 1.5, p.B))


def test_mixed_roots_tc():
    _check(mixed_roots_problem())


def test_config3_tc_sampled():
    p = wl.chain_config("chain_n8_K256_d64_B128")
    idx = [0, 64, 127]
    go = np.zeros(p.B)
    go[idx] = 1.0
    got = gpu_run(p, "fp16", grad_out=go, want=PARAM_GRADS)
    sub = oracle.subset(p, idx)
    ref = oracle_run(sub)
    err = np.abs(got["log_phat"][idx] - ref["log_phat"]).max()
    assert err <= TOL_LOGP_DESIGN, err
    for k in ("dW", "dbias", "dC"):
        e = np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
        assert e <= TOL_GRAD, (k, e)


def test_sample_gradients_alone():
    """dz / deps requested without any parameter gradient (and the converse, earlier)."""
    p = wl.make_chain(3, 200, 16, 32, 2, seed=5)
    _check(p, want=("dz",))
    _check(p, want=("deps",))


def test_autograd_fp16_plan():
    """torch.autograd through an fp16 plan: every input's gradient, the noise included."""
    import torch
    from paper_1806_08593_gb300.tmc import Plan, tmc_log_marginal
    p = wl.make_chain(4, 150, 12, 20, 3, seed=17)
    ref = oracle_run(p)
    plan = Plan.from_problem(p, "fp16")
    t = plan.to_device(p)
    for k in ("eps", "q_mean", "q_logstd", "W", "bias", "C"):
        t[k].requires_grad_(True)
    lp = tmc_log_marginal(plan, **t)
    lp.sum().backward()
    torch.cuda.synchronize()
    plan.sync_status()
    assert np.abs(lp.detach().cpu().numpy() - ref["log_phat"]).max() <= TOL_LOGP_DESIGN
    for name, key in (("eps", "deps"), ("q_mean", "dq_mean"), ("q_logstd", "dq_logstd"), ("W", "dW"),
                      ("bias", "dbias"), ("C", "dC")):
        g = t[name].grad.double().cpu().numpy()
        e = np.linalg.norm(g - ref[key]) / np.linalg.norm(ref[key])
        assert e <= TOL_GRAD, (name, e)
    plan.close()
