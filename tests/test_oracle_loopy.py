"""Pins of the FP64 oracle for the loopy graph of Fig. 1 (CPU only).

z1 -> z2, z1 -> z3, {z2, z3} -> z4 -> x: z4 has two parents, so summing out k4 and then k1
leaves factors over two indices (matrix messages, Section 2.2 and Fig. 1 C/D).  Checks:
enumeration of all K^4 combinations of Eq. (is), the K = 1 single-sample weight from the
joint Gaussian density of the graph, exactness when the posterior factorises and the proposal
equals it (closed-form log p(x) from the marginal of x), unbiasedness / Jensen, and
invariance under relabelling the samples.
"""
import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle
from paper_1806_08593_gb300 import workload as wl


@pytest.mark.parametrize("K,d", [(1, 2), (2, 1), (3, 2), (4, 3), (5, 1)])
@pytest.mark.parametrize("shared", [True, False])
def test_diamond_brute_force(K, d, shared):
    p = wl.make_diamond(K, d, 2 * d + 1, 3, seed=1000 + 10 * K + d, shared=shared)
    np.testing.assert_allclose(oracle.diamond_log_marginal(p), oracle.diamond_brute_force(p),
                               rtol=0, atol=1e-11)


def _log_px(p, b):
    W, bias, C, x = p.instance(b)
    mu, S, _ = wl.diamond_joint(W, bias, p.prior_var)
    d = p.d
    cov = C @ S[3 * d:, 3 * d:] @ C.T + p.obs_var * np.eye(p.obs)
    return multivariate_normal(C @ mu[3 * d:], cov).logpdf(x)


def test_diamond_k1_is_single_sample_weight():
    p = wl.make_diamond(1, 3, 5, 4, seed=1101, shared=False)
    got = oracle.diamond_log_marginal(p)
    d = p.d
    for b in range(p.B):
        W, bias, C, x = p.instance(b)
        mu, S, _ = wl.diamond_joint(W, bias, p.prior_var)
        eps = p.eps.reshape(p.B, 4, 1, d)[b, :, 0].astype(np.float64)
        m = p.q_mean.reshape(p.B, 4, d)[b].astype(np.float64)
        ls = p.q_logstd.reshape(p.B, 4, d)[b].astype(np.float64)
        z = (m + np.exp(ls) * eps).ravel()
        lj = multivariate_normal(mu, S).logpdf(z)  # the joint of the DAG, not factor by factor
        lx = multivariate_normal(C @ z[3 * d:], p.obs_var * np.eye(p.obs)).logpdf(x)
        lq = np.sum(-0.5 * eps ** 2 - ls - 0.5 * np.log(2 * np.pi))
        np.testing.assert_allclose(got[b], lj + lx - lq, rtol=0, atol=1e-9)


@pytest.mark.parametrize("K", [1, 3, 8])
def test_diamond_exact_when_posterior_factorises(K):
    p = wl.make_diamond(K, 3, 6, 3, seed=1200 + K, shared=True, zero_W=True, exact_proposal=True,
                        orth_C=True)
    got = oracle.diamond_log_marginal(p)
    want = [_log_px(p, b) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


def test_diamond_unbiased_and_jensen():
    p = wl.make_diamond(2, 1, 2, 1, seed=1301)
    S = 20_000
    rng = np.random.default_rng(77)
    reps = wl.Diamond(**{**p.__dict__, "B": S})
    reps.eps = rng.standard_normal(S * p.eps.size).astype(np.float32)
    reps.q_mean = np.tile(p.q_mean, S)
    reps.q_logstd = np.tile(p.q_logstd, S)
    reps.x = np.tile(p.x, S)
    lp = oracle.diamond_log_marginal(reps)
    ref = _log_px(p, 0)
    r = np.exp(lp - ref)
    se = r.std(ddof=1) / np.sqrt(S)
    assert abs(r.mean() - 1.0) <= 4 * se, (r.mean(), se)
    assert lp.mean() <= ref + 4 * lp.std(ddof=1) / np.sqrt(S)


def test_diamond_sample_permutation_invariance():
    p = wl.make_diamond(6, 2, 3, 2, seed=1401)
    base = oracle.diamond_log_marginal(p)
    e = p.eps.reshape(p.B, 4, p.K, p.d).copy()
    rng = np.random.default_rng(3)
    for b in range(p.B):
        for i in range(4):
            e[b, i] = e[b, i, rng.permutation(p.K)]
    np.testing.assert_allclose(oracle.diamond_log_marginal(p, eps=e.ravel()), base, rtol=0, atol=1e-11)
