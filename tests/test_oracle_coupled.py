"""Pins of the FP64 oracle with a coupled (non-factorised) proposal (CPU only).

Section 2.3 ("Non-factorised proposals") and its appendix: sample k of latent i may be drawn
given samples of other latents, Q_i(z_i^k | x, all samples of qa(i)), and Eq. (is) keeps its
form because the proposal factor is indexed by k_i alone.  Here qa(i) is the model parent and
sample k of latent i is drawn given the parent's sample k:
Q_i = N(m_i + A_i (z_p^k - m_p), diag(exp(2 logs_i))).  Checks: brute-force enumeration, the
K = 1 weight when the proposal is the prior (every transition cancels, leaving the root and
the observations), unbiasedness, A = 0 reducing to the factorised oracle, and central
differences of the elimination and the brute force, couplings included.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.gaussian_closed_form import instance_params, log_px


@pytest.mark.parametrize("mode", ["prior", "scaled"])
@pytest.mark.parametrize("which", ["chain", "trees"])
def test_brute_force_coupled(mode, which):
    if which == "chain":
        p = wl.make_chain(5, 3, 2, obs=3, B=2, seed=801)
    else:
        rng = np.random.default_rng(802)
        parents = [wl.random_tree(rng, n, 3) for n in (4, 6)]
        p = wl.make_problem(parents, [3, 2], [2, 1], [3, 2], shared=False, seed=803)
    q = wl.couple_proposal(p, mode)
    np.testing.assert_allclose(oracle.log_marginal(q), oracle.brute_force(q), rtol=0, atol=1e-11)


def test_k1_prior_proposal_cancels_the_transitions():
    """K = 1, proposal = prior for every non-root latent: the single weight is
    log P(z_0) - log Q_0(z_0) + sum_leaves log N(x_l; C z_l, obs_var), with the z drawn
    ancestrally from eps (z_i = W_i z_p + b_i + prior_std eps_i)."""
    rng = np.random.default_rng(811)
    parents = [wl.chain_parents(6), wl.random_tree(rng, 7, 3)]
    p = wl.couple_proposal(wl.make_problem(parents, [1, 1], [3, 2], [4, 3], shared=False, seed=812), "prior")
    got = oracle.log_marginal(p)
    for b in range(p.B):
        n, Kn, dn, o, par, W, bias, C, x = instance_params(p, b)
        s = p.slices(b)
        eps = p.eps[s["eps"][0]:s["eps"][1]].astype(np.float64)
        m = p.q_mean[s["q"][0]:s["q"][1]].astype(np.float64)
        ls = p.q_logstd[s["q"][0]:s["q"][1]].astype(np.float64)
        oq = np.concatenate([[0], np.cumsum(dn)]).astype(int)
        ow = np.concatenate([[0], np.cumsum(dn * np.array([dn[par[i]] if i else dn[0] for i in range(n)]))]).astype(int)
        Af = p.q_A[s["A"][0]:s["A"][1]].astype(np.float64)
        lg = lambda y, mu, var: -0.5 * np.sum((y - mu) ** 2) / var - 0.5 * len(y) * np.log(2 * np.pi * var)
        # the samples as the proposal draws them (its stored float32 parameters)
        z, lq = [None] * n, 0.0
        for i in range(n):
            mq = m[oq[i]:oq[i + 1]].copy()
            if i:
                A = Af[ow[i]:ow[i + 1]].reshape(dn[i], dn[par[i]])
                mq += A @ (z[par[i]] - m[oq[par[i]]:oq[par[i] + 1]])
            e, sd = eps[oq[i]:oq[i + 1]], np.exp(ls[oq[i]:oq[i + 1]])
            z[i] = mq + sd * e
            lq += np.sum(-0.5 * e ** 2 - np.log(sd) - 0.5 * np.log(2 * np.pi))
        root_and_obs = lg(z[0], bias[0], p.prior_var)
        for a, l in enumerate(p.leaves_of(b)):
            root_and_obs += lg(x[a * o:(a + 1) * o], C @ z[l], p.obs_var)
        trans = sum(lg(z[i], W[i] @ z[par[i]] + bias[i], p.prior_var) for i in range(1, n))
        # the full single-sample weight, from the joint density directly
        np.testing.assert_allclose(got[b], root_and_obs + trans - lq, rtol=0, atol=1e-10)
        # and the cancellation: every transition against its proposal factor (to the float32
        # rounding of the stored proposal)
        lq_trans = lq - np.sum(-0.5 * eps[:dn[0]] ** 2 - ls[:dn[0]] - 0.5 * np.log(2 * np.pi))
        assert abs(trans - lq_trans) < 1e-5
        np.testing.assert_allclose(got[b], root_and_obs - (lq - lq_trans), rtol=0, atol=1e-5)


def test_zero_coupling_is_the_factorised_proposal():
    p = wl.make_chain(4, 3, 2, obs=3, B=2, seed=821)
    q = wl.couple_proposal(p, "scaled", alpha=0.0)
    g0, g1 = oracle.grad(p), oracle.grad(q)
    for k in ("log_phat", "dz", "dq_mean", "dq_logstd", "dW", "dbias", "dC"):
        np.testing.assert_allclose(g1[k], g0[k], rtol=1e-12, atol=1e-12)


def test_coupled_unbiased_and_jensen():
    p = wl.couple_proposal(wl.make_chain(3, 3, 1, obs=2, B=1, seed=831), "prior")
    base = oracle.subset(p, [0])
    S = 50_000
    reps = oracle.subset(base, [0] * S)
    reps.eps = np.concatenate([wl.redraw_eps(base, 9000 + s) for s in range(S)])
    lp = oracle.log_marginal(reps)
    ref = log_px(p, 0)
    r = np.exp(lp - ref)
    se = r.std(ddof=1) / np.sqrt(S)
    assert abs(r.mean() - 1.0) <= 4 * se, (r.mean(), se)
    assert lp.mean() <= ref + 4 * lp.std(ddof=1) / np.sqrt(S)


H = 1e-4


@pytest.mark.parametrize("fn_name", ["log_marginal", "brute_force"])
@pytest.mark.parametrize("shared", [True, False])
def test_coupled_grad_vs_central_differences(fn_name, shared):
    if shared:
        p = wl.couple_proposal(wl.make_chain(3, 3, 2, obs=2, B=2, seed=841), "scaled", alpha=0.7)
    else:
        rng = np.random.default_rng(842)
        parents = [wl.random_tree(rng, 4, 2), wl.chain_parents(3)]
        p = wl.couple_proposal(wl.make_problem(parents, [2, 3], [2, 1], [2, 3], shared=False, seed=843), "prior")
    fn = getattr(oracle, fn_name)
    go = np.array([0.7, -1.3])
    g = oracle.grad(p, grad_out=go)
    s = np.exp(p.q_logstd.astype(np.float64))
    deps = g["dz"].copy()  # dz = (d/d eps) / exp(logs), latent by latent
    oe = oq = 0
    for K, d in zip(p.K_nodes().astype(int), p.d_nodes().astype(int)):
        deps[oe:oe + K * d] *= np.tile(s[oq:oq + d], K)
        oe += K * d
        oq += d
    an = dict(eps=deps, q_mean=g["dq_mean"], q_logstd=g["dq_logstd"], q_A=g["dq_A"], W=g["dW"],
              bias=g["dbias"], C=g["dC"])
    rng = np.random.default_rng(29)
    for name, ga in an.items():
        base = getattr(p, name).astype(np.float64)
        idx = rng.choice(base.size, size=min(base.size, max(4, base.size // 3)), replace=False)
        for i in idx:
            a = base.copy(); a[i] += H
            b = base.copy(); b[i] -= H
            fd = (np.dot(go, fn(p, **{name: a})) - np.dot(go, fn(p, **{name: b}))) / (2 * H)
            assert abs(fd - ga[i]) <= 2e-5 * max(1.0, abs(ga[i])), (name, int(i), fd, ga[i])
