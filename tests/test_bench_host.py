"""Host-side bookkeeping of bench.py (no GPU): workload names, the algorithmic FLOP count the
roofline divides by, the gradients a training step asks for, and the bounded oracle sample."""
import numpy as np

import bench
from paper_1806_08593_gb300 import workload as wl


def test_algorithmic_flops_uniform_chain():
    """Per edge p -> i: forward 2 K_p K_i d_i, adjoint 2 K_p K_i (d_i + d_p); for one K and d per
    instance that is 2 (n - 1) K^2 d and twice that, summed over instances."""
    p = bench.make_workload("chain_n3_K4_d2_B8")
    f = bench.algorithmic_flops(p, "fp16")
    e = float(np.sum((p.n.astype(np.int64) - 1) * p.K.astype(np.int64) ** 2 * p.d.astype(np.int64)))
    assert f["edge_fwd"] == 2.0 * e
    assert f["edge_bwd"] == 4.0 * e


def test_algorithmic_flops_per_latent_sizes():
    p = wl.layered_chain([3, 5, 7], [2, 4, 6], obs=4, B=2, seed=5)
    f = bench.algorithmic_flops(p, "fp16")
    # chain 0 -> 1 -> 2 with (K, d) = (2, 3), (4, 5), (6, 7), twice
    fwd = 2 * (2 * 4 * 5 + 4 * 6 * 7) * 2
    bwd = 2 * (2 * 4 * (5 + 3) + 4 * 6 * (7 + 5)) * 2
    assert f["edge_fwd"] == fwd and f["edge_bwd"] == bwd


def test_workload_names():
    layered = bench.make_workload("layered:B=3,K=5")
    assert layered.B == 3 and list(layered.d_nodes()[:5]) == [4, 8, 16, 32, 64]
    assert bench.step_grads(layered) == bench.GRADS
    coupled = bench.make_workload("coupled:chain_n3_K4_d2_B8")
    assert coupled.q_A is not None and "dq_A" in bench.step_grads(coupled)
    star = bench.make_workload("star:N=5,K=3,d=1")
    assert int(star.n[0]) == 6


def test_oracle_sample_is_bounded():
    p = bench.make_workload("chain_n3_K4_d2_B8")
    value, done, secs, logp = bench.time_oracle_sample(p, target_s=0.05)
    assert 1 <= done <= p.B and len(logp) == done and value > 0
