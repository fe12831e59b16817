"""Pins of the FP64 oracle with a different K_i and d_i for every latent (CPU only).

Eq. (is) draws K_i samples for latent i, and the normaliser is 1 / prod_i K_i; a latent's
dimension may differ from its parent's (W_i is d_i x d_parent), as in the paper's five-layer
model with widths 4/8/16/32/64.  The same independent checks as for uniform sizes: brute-force
enumeration, the single-sample weight at K_i = 1, exactness under a factorising exact
posterior against the closed-form marginal, unbiasedness, and finite differences of both the
elimination and the brute force.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl
from tests.gaussian_closed_form import log_px, log_weight_single


@pytest.mark.parametrize("shared", [True, False])
def test_brute_force_ragged_chain(shared):
    parents = [wl.chain_parents(4)] * 2
    Ks = [[2, 3, 1, 4], [3, 1, 2, 2]]
    ds = [[1, 3, 2, 2], [1, 3, 2, 2]]
    p = wl.make_problem(parents, Ks, ds, [3, 3], shared=shared, seed=611)
    assert p.ragged
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


@pytest.mark.parametrize("seed", range(4))
def test_brute_force_ragged_trees(seed):
    p = wl.ragged_trees(5, seed=620 + seed)
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


def test_layered_chain_brute_force():
    # the 4/8/16/32/64 widths (scaled down to brute-force size: 1/2/3/2/4 with K_i <= 3)
    p = wl.layered_chain([1, 2, 3, 2, 4], [3, 2, 3, 2, 3], obs=5, B=2, seed=631)
    np.testing.assert_allclose(oracle.log_marginal(p), oracle.brute_force(p), rtol=0, atol=1e-11)


def test_k1_ragged_is_single_sample_weight():
    rng = np.random.default_rng(41)
    parents = [wl.random_tree(rng, n, 4) for n in (2, 5, 8)]
    ds = []
    for par in parents:
        leaves = set(wl._leaves(par))
        ds.append([3 if i in leaves else int(rng.integers(1, 5)) for i in range(len(par))])
    p = wl.make_problem(parents, [1, 1, 1], ds, [4, 2, 5], shared=False, seed=642)
    got = oracle.log_marginal(p)
    want = [log_weight_single(p, b, [0] * int(p.n[b])) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-10)


def test_ragged_combination_weights_match_enumeration():
    """Brute force == log-mean-exp of the prod K_i hand-built weights (K = 2, 1, 3)."""
    p = wl.make_problem([wl.chain_parents(3)], [[2, 1, 3]], [[2, 1, 3]], [2], shared=False, seed=651)
    w = np.array([log_weight_single(p, 0, [a, 0, c]) for a in range(2) for c in range(3)])
    want = np.log(np.mean(np.exp(w - w.max()))) + w.max()
    np.testing.assert_allclose(oracle.log_marginal(p)[0], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.brute_force(p)[0], want, rtol=0, atol=1e-12)


@pytest.mark.parametrize("K", [[1, 2, 3, 4, 5], [7, 3, 1, 2, 9]])
def test_exact_ragged_when_posterior_factorises(K):
    rng = np.random.default_rng(7)
    parents = [wl.chain_parents(5), wl.random_tree(rng, 5, 2)]
    ds = [[2, 4, 1, 3, 2], None]
    leaves = set(wl._leaves(parents[1]))
    ds[1] = [3 if i in leaves else i + 1 for i in range(5)]
    p = wl.make_problem(parents, [K, K[::-1]], ds, [5, 6], shared=False, seed=661, zero_W=True,
                        exact_proposal=True, orth_C=True)
    got = oracle.log_marginal(p)
    want = [log_px(p, b) for b in range(p.B)]
    np.testing.assert_allclose(got, want, rtol=0, atol=5e-6)


def test_ragged_unbiased_and_jensen():
    p = wl.make_problem([wl.chain_parents(3)], [[3, 1, 2]], [[2, 1, 2]], [2], shared=True, seed=671)
    base = oracle.subset(p, [0])
    S = 50_000
    reps = oracle.subset(base, [0] * S)
    reps.eps = np.concatenate([wl.redraw_eps(base, 5000 + s) for s in range(S)])
    lp = oracle.log_marginal(reps)
    ref = log_px(p, 0)
    r = np.exp(lp - ref)
    se = r.std(ddof=1) / np.sqrt(S)
    assert abs(r.mean() - 1.0) <= 4 * se, (r.mean(), se)
    assert lp.mean() <= ref + 4 * lp.std(ddof=1) / np.sqrt(S)


H = 1e-4  # central differences: truncation error ~h^2 (1e-3 leaves ~6e-4 on dC here)


def _deps(p, dz):
    s = np.exp(p.q_logstd.astype(np.float64))
    Kn, dn = p.K_nodes(), p.d_nodes()
    out = dz.copy()
    oe = oq = 0
    for i in range(len(Kn)):
        K, d = int(Kn[i]), int(dn[i])
        out[oe:oe + K * d] *= np.tile(s[oq:oq + d], K)
        oe += K * d
        oq += d
    return out


@pytest.mark.parametrize("fn_name", ["log_marginal", "brute_force"])
@pytest.mark.parametrize("shared", [True, False])
def test_ragged_grad_vs_central_differences(fn_name, shared):
    if shared:
        p = wl.make_problem([wl.chain_parents(3)] * 2, [[2, 3, 2], [3, 1, 2]], [[2, 3, 1]] * 2, [2, 2],
                            shared=True, seed=681)
    else:
        p = wl.ragged_trees(3, seed=682)
    fn = getattr(oracle, fn_name)
    go = np.array([0.7, -1.3, 0.4])[:p.B]
    g = oracle.grad(p, grad_out=go)
    an = dict(eps=_deps(p, g["dz"]), q_mean=g["dq_mean"], q_logstd=g["dq_logstd"], W=g["dW"],
              bias=g["dbias"], C=g["dC"])
    rng = np.random.default_rng(19)
    for name, ga in an.items():
        base = getattr(p, name).astype(np.float64)
        idx = rng.choice(base.size, size=min(base.size, max(4, base.size // 3)), replace=False)
        for i in idx:
            a = base.copy(); a[i] += H
            b = base.copy(); b[i] -= H
            fd = (np.dot(go, fn(p, **{name: a})) - np.dot(go, fn(p, **{name: b}))) / (2 * H)
            assert abs(fd - ga[i]) <= 2e-5 * max(1.0, abs(ga[i])), (name, int(i), fd, ga[i])


def test_instance_slices_partition_the_flat_arrays():
    """Problem.slices_all (one pass) gives every instance the same slices as slices(b), and the
    per-instance slices of the per-instance arrays tile them without gaps or overlap; subset()
    of every instance reproduces the batch's oracle result."""
    import oracle
    p = wl.ragged_trees(9, seed=641)
    every = p.slices_all()
    assert len(every) == p.B
    for key, arr in (("eps", p.eps), ("q", p.q_mean), ("x", p.x), ("W", p.W), ("C", p.C)):
        end = 0
        for b in range(p.B):
            assert every[b] == p.slices(b)
            lo, hi = every[b][key]
            assert lo == end and hi >= lo
            end = hi
        assert end == arr.size, key
    whole = oracle.log_marginal(p)
    parts = oracle.log_marginal(oracle.subset(p, list(range(p.B))))
    np.testing.assert_array_equal(whole, parts)
