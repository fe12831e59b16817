"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test names the property of the estimator (Eq. (is), Section 2.1) or of the Gaussian
model that it checks.  Together they make a dropped term, a wrong sign, a swapped index or
a transposed parameter in the oracle fail at least one test.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.gaussian_closed_form import log_px, log_weight_single


# ---------------------------------------------------------------------------------------
# Eq. (is) by brute-force enumeration == summing out one index at a time (Section 2.2).
# ---------------------------------------------------------------------------------------
def test_brute_force_chain_config1():
    p = wl.chain_config("chain_n3_K4_d2_B8")
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-12)


@pytest.mark.parametrize("K,n", [(2, 10), (3, 6), (5, 4), (1, 24)])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_brute_force_chains(K, n, d):
    p = wl.make_chain(n, K, d, obs=2 * d, B=2, seed=100 + K * 7 + n * 3 + d)
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_random_trees(seed):
    rng = np.random.default_rng(seed)
    parents = [wl.random_tree(rng, 5, max_depth=3) for _ in range(3)]
    Ks = [int(rng.integers(1, 5)) for _ in range(3)]
    ds = [int(rng.integers(1, 4)) for _ in range(3)]
    p = wl.make_problem(parents, Ks, ds, [2, 3, 4], shared=False, seed=500 + seed)
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


def test_brute_force_star_of_fig2():
    """The latent-variable model of Fig. 2: one global root with N children."""
    parent = np.array([-1] + [0] * 6, dtype=np.int32)
    p = wl.make_problem([parent] * 2, [3, 3], [2, 2], [3, 3], shared=True, seed=7)
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


def test_brute_force_star_workload():
    # the large-star workload's generator (per-instance models, belief-propagation proposal)
    # at a size brute force can enumerate: 3^5 combinations
    p = wl.star(4, 3, 2, B=2, seed=31)
    assert list(p.n) == [5, 5]
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


# ---------------------------------------------------------------------------------------
# K = 1 reduces to the single-sample (VAE) importance weight P(x, z) / Q(z) (Section 1).
# ---------------------------------------------------------------------------------------
def test_k1_is_single_sample_weight():
    rng = np.random.default_rng(3)
    parents = [wl.random_tree(rng, n, 8) for n in (1, 2, 7, 12)]
    p = wl.make_problem(parents, [1] * 4, [3, 2, 4, 1], [5, 2, 3, 6], shared=False, seed=11)
    got = oracle.log_marginal(p)
    want = [log_weight_single(p, b, [0] * int(p.n[b])) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def test_single_combination_weight_matches_enumeration():
    """Brute force with K=2 on a tiny chain == log-mean-exp of the 2^n hand-built weights."""
    p = wl.make_chain(3, 2, 2, obs=3, B=1, seed=19)
    w = []
    for c in range(8):
        ks = [(c >> i) & 1 for i in range(3)]
        w.append(log_weight_single(p, 0, ks))
    w = np.array(w)
    want = np.log(np.mean(np.exp(w - w.max()))) + w.max()
    np.testing.assert_allclose(oracle.log_marginal(p)[0], want, rtol=0, atol=1e-12)


# ---------------------------------------------------------------------------------------
# Exactness: when the posterior factorises over latents and Q equals it, every importance
# ratio equals p(x), so log P_TMC = log p(x) for any K and any eps.  W = 0 makes the latents
# independent a priori; C with orthogonal columns makes each leaf's posterior covariance
# diagonal, so the factorised diagonal proposal can equal the posterior exactly.
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("K", [1, 3, 16])
def test_exact_when_posterior_factorises_chain(K):
    p = wl.make_chain(5, K, 3, obs=6, B=3, seed=31 + K, zero_W=True, exact_proposal=True,
                     orth_C=True)
    got = oracle.log_marginal(p)
    want = [log_px(p, b) for b in range(p.B)]
    # float32 storage of the proposal limits agreement to ~1e-7 nats
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)
    # with the proposal in float32 the weights are not exactly constant; their spread is tiny
    assert np.ptp(got - np.array(want)) < 5e-6


def test_exact_when_posterior_factorises_trees():
    rng = np.random.default_rng(5)
    parents = [wl.random_tree(rng, n, 4) for n in (1, 3, 6, 9)]
    p = wl.make_problem(parents, [4, 2, 5, 3], [2, 3, 1, 2], [4, 6, 2, 4], shared=False,
                        seed=41, zero_W=True, exact_proposal=True, orth_C=True)
    got = oracle.log_marginal(p)
    want = [log_px(p, b) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


def test_exact_single_latent():
    p = wl.make_chain(1, 9, 4, obs=5, B=4, seed=43, exact_proposal=True, orth_C=True)
    got = oracle.log_marginal(p)
    want = [log_px(p, b) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


def test_exactness_is_sensitive_to_the_proposal():
    """Control for the tests above: a perturbed proposal breaks exactness."""
    p = wl.make_chain(5, 4, 3, obs=6, B=2, seed=33, zero_W=True, exact_proposal=False,
                     orth_C=True)
    got = oracle.log_marginal(p)
    want = [log_px(p, b) for b in range(p.B)]
    assert np.max(np.abs(got - np.array(want))) > 1e-2


# ---------------------------------------------------------------------------------------
# Unbiasedness (Section 2.1): E_Q[P_TMC] = p(x); Jensen: E_Q[log P_TMC] <= log p(x).
# ---------------------------------------------------------------------------------------
def _resampled(p, S, seed_base):
    """S copies of instance 0 of p with independent eps (same model, x and proposal)."""
    base = oracle.subset(p, [0])
    reps = oracle.subset(base, [0] * S)
    reps.eps = np.concatenate([wl.redraw_eps(base, seed_base + s) for s in range(S)])
    return reps


@pytest.mark.parametrize("shape", ["config1", "toy1_star"])
def test_unbiased_and_jensen(shape):
    if shape == "config1":
        p = wl.chain_config("chain_n3_K4_d2_B8")
    else:
        # Toy model of Section 3.1: theta ~ N(0,1), z_i | theta ~ N(theta, 1),
        # x_i | z_i ~ N(z_i, 1); proposals are the generative marginals N(0,1), N(0,2).
        N = 6
        parent = np.array([-1] + [0] * N, dtype=np.int32)
        model = ([np.zeros((1, 1))] + [np.ones((1, 1))] * N, [np.zeros(1)] * (N + 1), np.ones((1, 1)))
        p = wl.make_problem([parent], [8], [1], [1], shared=True, seed=77, obs_var=1.0,
                            model_override=model)
        p.q_mean[:] = 0.0
        p.q_logstd[:] = np.log(np.array([1.0] + [np.sqrt(2.0)] * N, dtype=np.float32))
    S = 100_000
    reps = _resampled(p, S, 1000)
    lp = oracle.log_marginal(reps)
    ref = log_px(p, 0)
    r = np.exp(lp - ref)
    se = r.std(ddof=1) / np.sqrt(S)
    assert abs(r.mean() - 1.0) <= 4 * se, (r.mean(), se)
    assert se < 0.05
    assert lp.mean() <= ref + 4 * lp.std(ddof=1) / np.sqrt(S)


# ---------------------------------------------------------------------------------------
# Invariances of Eq. (is): relabelling samples within a latent, or renumbering the latents
# (keeping parents before children), leaves P_TMC unchanged.
# ---------------------------------------------------------------------------------------
def test_sample_permutation_invariance():
    p = wl.chain_config("chain_n3_K4_d2_B8")
    base = oracle.log_marginal(p)
    e = p.eps.reshape(p.B, 3, 4, 2).copy()
    rng = np.random.default_rng(0)
    for b in range(p.B):
        for i in range(3):
            e[b, i] = e[b, i, rng.permutation(4)]
    np.testing.assert_allclose(oracle.log_marginal(p, eps=e.ravel()), base, rtol=0, atol=1e-12)


def test_node_renumbering_invariance():
    # tree 0 -> {1, 2}, 1 -> {3}; renumber children 1 <-> 2 (3's parent follows)
    parent = np.array([-1, 0, 0, 1], dtype=np.int32)
    p = wl.make_problem([parent], [3], [2], [3], shared=False, seed=9)
    n, K, d = 4, 3, 2
    perm = [0, 2, 1, 3]  # new node j is old node perm[j]
    newpar = np.array([-1, 0, 0, 2], dtype=np.int32)
    q = oracle.subset(p, [0])
    q.parent = newpar
    q.eps = p.eps.reshape(n, K, d)[perm].ravel()
    q.q_mean = p.q_mean.reshape(n, d)[perm].ravel()
    q.q_logstd = p.q_logstd.reshape(n, d)[perm].ravel()
    q.W = p.W.reshape(n, d, d)[perm].ravel()
    q.bias = p.bias.reshape(n, d)[perm].ravel()
    # leaves in node order: old leaves {2, 3} -> new numbers {1, 3}; x order old (2, 3) -> new (1, 3)
    np.testing.assert_allclose(oracle.log_marginal(q), oracle.log_marginal(p), rtol=0, atol=1e-12)
