"""Pins of the oracle's analytic gradients (CPU only).

The oracle differentiates log P_TMC by running the message recursion backwards.  These
tests compare it with central finite differences (step 1e-3, FP64) of
  (a) the oracle's own forward value, and
  (b) the brute-force enumeration of Eq. (is), which shares no recursion with it,
on seeded subsets of the entries of every input tensor.
"""
import numpy as np
import pytest

import oracle
from paper_1806_08593_gb300 import workload as wl

H = 1e-3


def _objective(p, fn, go, **over):
    return float(np.dot(go, fn(p, **over)))


def _fd(p, fn, go, name, idx):
    base = getattr(p, name).astype(np.float64)
    out = []
    for i in idx:
        a = base.copy(); a[i] += H
        b = base.copy(); b[i] -= H
        out.append((_objective(p, fn, go, **{name: a}) - _objective(p, fn, go, **{name: b})) / (2 * H))
    return np.array(out)


def _analytic(p, go):
    g = oracle.grad(p, grad_out=go)
    # d/d eps = exp(logs) * dz  (the proposal's own term depends on eps only through z)
    s = np.exp(p.q_logstd.astype(np.float64))
    deps = g["dz"].copy()
    off_e = off_q = 0
    for b in range(p.B):
        n, K, d = int(p.n[b]), int(p.K[b]), int(p.d[b])
        deps[off_e:off_e + n * K * d] *= np.repeat(s[off_q:off_q + n * d].reshape(n, 1, d), K, 1).ravel()
        off_e += n * K * d
        off_q += n * d
    return dict(eps=deps, q_mean=g["dq_mean"], q_logstd=g["dq_logstd"], W=g["dW"],
                bias=g["dbias"], C=g["dC"])


def _problems():
    chain = wl.make_chain(4, 3, 2, obs=3, B=2, seed=201)
    rng = np.random.default_rng(8)
    parents = [wl.random_tree(rng, n, 3) for n in (3, 5)]
    trees = wl.make_problem(parents, [3, 2], [2, 3], [4, 2], shared=False, seed=202)
    return {"chain_shared": chain, "trees_unshared": trees}


@pytest.mark.parametrize("which", ["chain_shared", "trees_unshared"])
@pytest.mark.parametrize("fn_name", ["log_marginal", "brute_force"])
def test_grad_vs_central_differences(which, fn_name):
    p = _problems()[which]
    fn = getattr(oracle, fn_name)
    go = np.array([0.7, -1.3])[:p.B]
    an = _analytic(p, go)
    rng = np.random.default_rng(17)
    for name, g in an.items():
        size = getattr(p, name).size
        k = min(size, max(4, size // 3))
        idx = rng.choice(size, size=k, replace=False)
        fd = _fd(p, fn, go, name, idx)
        err = np.abs(fd - g[idx])
        tol = 2e-5 * np.maximum(1.0, np.abs(g[idx]))
        assert np.all(err <= tol), (name, float(err.max()), list(zip(fd, g[idx]))[:4])


def test_unused_root_weight_has_zero_gradient():
    p = _problems()["chain_shared"]
    g = oracle.grad(p)
    d = int(p.d[0])
    assert np.all(g["dW"][:d * d] == 0.0)


def test_grad_linear_in_grad_out():
    p = _problems()["chain_shared"]
    g1 = oracle.grad(p, grad_out=np.array([1.0, 0.0]))
    g2 = oracle.grad(p, grad_out=np.array([0.0, 1.0]))
    g12 = oracle.grad(p, grad_out=np.array([2.0, -3.0]))
    for k in ("dz", "dq_mean", "dq_logstd", "dW", "dbias", "dC"):
        np.testing.assert_allclose(g12[k], 2 * g1[k] - 3 * g2[k], rtol=1e-12, atol=1e-12)


def test_logstd_gradient_contains_unit_weight_mass():
    """With every other factor independent of a latent's samples (eps = 0 makes all its
    samples equal), d logP/d logs_ij = sum_k q_i[k] = 1 from the proposal's own term plus
    the path term, which vanishes because z - m = 0."""
    p = wl.make_chain(3, 4, 2, obs=2, B=1, seed=5)
    e = p.eps.reshape(3, 4, 2).copy()
    e[1] = 0.0
    g = oracle.grad(p, eps=e.ravel())
    np.testing.assert_allclose(g["dq_logstd"].reshape(3, 2)[1], [1.0, 1.0], rtol=0, atol=1e-12)
