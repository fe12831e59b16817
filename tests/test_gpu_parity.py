"""CUDA path vs the FP64 oracle, through the C-ABI (needs a GB300).

Tolerances: |delta log P| <= 1e-4 nats per instance (FP32 path); gradients within 1e-3
relative (per tensor, ||g - g_ref|| / ||g_ref||).
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.parity import compare, gpu_run, mixed_roots_problem, oracle_run

pytestmark = pytest.mark.gpu
TOL_LOGP_F32 = 1e-4
TOL_GRAD = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1806_08593_gb300.build import build
    build()


def test_config1_fp32_vs_oracle_and_brute_force():
    p = wl.chain_config("chain_n3_K4_d2_B8")
    got = gpu_run(p, "fp32")
    ref = oracle_run(p)
    np.testing.assert_allclose(ref["log_phat"], oracle.brute_force(p), atol=1e-12)
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD)


@pytest.mark.parametrize("n,K,d,obs,B", [
    (5, 100, 24, 40, 3),     # ragged K tile (64 + 36)
    (4, 130, 70, 33, 2),     # three row tiles, d spans two 64-wide tiles, odd obs
    (3, 65, 130, 129, 2),    # d > 128 (second 128-column sweep), obs > 128
    (1, 77, 9, 5, 3),        # single latent (root is the leaf)
    (6, 1, 3, 4, 2),         # K = 1: the single-sample weight
    (2, 3, 1, 1, 4),         # d = obs = 1
])
def test_chains_fp32(n, K, d, obs, B):
    p = wl.make_chain(n, K, d, obs, B, seed=1000 + n * 7 + K + d)
    got = gpu_run(p, "fp32", grad_out=np.linspace(0.5, 1.5, B))
    ref = oracle_run(p, grad_out=np.linspace(0.5, 1.5, B))
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD)


def test_shared_many_instances_fp32():
    """One model shared by 150 instances: the shared gradients are per-instance partials summed
    by a tree of 64-row chunks (two levels here), weighted by a different grad_out each."""
    B = 150
    p = wl.make_chain(4, 16, 24, 30, B, seed=716)
    go = np.linspace(0.25, 1.75, B)
    compare(p, gpu_run(p, "fp32", grad_out=go), oracle_run(p, grad_out=go), TOL_LOGP_F32, TOL_GRAD)


def test_uneven_trees_fp32():
    p = wl.tree_batch(B=12, seed=4242)
    got = gpu_run(p, "fp32")
    ref = oracle_run(p)
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD)


def test_large_star_fp32():
    p = wl.star(2000, 128, 1, B=2, seed=1234)
    compare(p, gpu_run(p, "fp32"), oracle_run(p), TOL_LOGP_F32, TOL_GRAD)


def test_mixed_roots_fp32():
    p = mixed_roots_problem()
    compare(p, gpu_run(p, "fp32"), oracle_run(p), TOL_LOGP_F32, TOL_GRAD)


@pytest.mark.parametrize("which", ["layered", "trees", "shared_K", "wide"])
def test_ragged_fp32(which):
    """A different K_i and d_i per latent (Eq. (is)); W_i of shape d_i x d_parent."""
    if which == "layered":  # the paper's five-layer widths, K = 20, synthetic observations
        p = wl.layered_chain([4, 8, 16, 32, 64], 20, obs=96, B=6, seed=711)
    elif which == "trees":
        p = wl.ragged_trees(8, seed=712, n_choices=(1, 3, 6, 9), Ks=(1, 17, 64, 100, 130),
                            ds=(1, 8, 24, 65), max_depth=4)
    elif which == "shared_K":  # shared model, the same d_i everywhere, K_i differing between instances too
        p = wl.make_problem([wl.chain_parents(4)] * 3, [[70, 20, 130, 64], [5, 90, 64, 64], [128] * 4],
                            [[6, 33, 70, 12]] * 3, [24] * 3, shared=True, seed=713)
    else:  # wide latents of both sizes, several 64-row tiles per edge
        p = wl.make_problem([np.array([-1, 0, 1, 1, 0], dtype=np.int32)] * 2,
                            [[300, 129, 260, 90, 200], [64, 256, 128, 300, 40]],
                            [[128, 40, 100, 100, 100], [30, 128, 100, 100, 100]], [64, 70],
                            shared=False, seed=714)
    assert p.ragged
    got = gpu_run(p, "fp32", grad_out=np.linspace(0.5, 1.5, p.B))
    ref = oracle_run(p, grad_out=np.linspace(0.5, 1.5, p.B))
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD)


def test_star_fig2_fp32():
    parent = np.array([-1] + [0] * 9, dtype=np.int32)
    p = wl.make_problem([parent] * 3, [70] * 3, [5] * 3, [7] * 3, shared=True, seed=99)
    got = gpu_run(p, "fp32")
    ref = oracle_run(p)
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD)


def test_config2_fp32_full():
    p = wl.chain_config("chain_n8_K128_d32_B256")
    got = gpu_run(p, "fp32", grads=False)
    ref = {"log_phat": oracle.log_marginal(p)}
    compare(p, got, ref, TOL_LOGP_F32, TOL_GRAD, keys=[])


def test_config3_fp32_sampled_instances():
    """Full-size launch (B=128); oracle on a sample of instances.  Gradients of shared
    parameters are compared with grad_out selecting only the sampled instances."""
    p = wl.chain_config("chain_n8_K256_d64_B128")
    idx = [0, 37, 127]
    go = np.zeros(p.B)
    go[idx] = 1.0
    got = gpu_run(p, "fp32", grad_out=go, want=("dW", "dbias", "dC", "dq_mean", "dq_logstd"))
    sub = oracle.subset(p, idx)
    ref = oracle_run(sub)
    assert np.abs(got["log_phat"][idx] - ref["log_phat"]).max() <= TOL_LOGP_F32
    for k in ("dW", "dbias", "dC"):
        e = np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])
        assert e <= TOL_GRAD, (k, e)
    # per-instance proposal gradients of the sampled instances
    d, n = 64, 8
    for j, b in enumerate(idx):
        for k in ("dq_mean", "dq_logstd"):
            gg = got[k][b * n * d:(b + 1) * n * d]
            rr = ref[k][j * n * d:(j + 1) * n * d]
            assert np.linalg.norm(gg - rr) / np.linalg.norm(rr) <= TOL_GRAD, (k, b)
