"""Closed-form Gaussian quantities used to pin the oracle (test helper, numpy FP64).

log p(x) for the linear-Gaussian tree is computed from the marginal distribution of the
stacked leaf observations: the latent means/covariances are propagated down the tree
(z_i = W_i z_p + b_i + noise, so Cov(z_i, z_j) = W_i Cov(z_p, z_j) for j < i and
Cov(z_i, z_i) = W_i Cov(z_p, z_p) W_i^T + prior_var I), then x_l = C z_l + noise.  This
route shares nothing with the oracle's message passing or with the generator's
information-form posterior, so agreement between them is evidence for both.  Latents may
have different dimensions d_i (W_i is d_i x d_parent) and sample counts K_i.
"""
import numpy as np


def instance_params(p, b):
    """Per-latent W_i, bias_i lists, C, x, sizes of instance b."""
    s = p.slices(b)
    n, o = int(p.n[b]), int(p.obs[b])
    Kn, dn, dp = p.node_sizes(b)
    Wf = p.W[s["W"][0]:s["W"][1]].astype(np.float64)
    bf = p.bias[s["bias"][0]:s["bias"][1]].astype(np.float64)
    W, bias, ow, ob = [], [], 0, 0
    for i in range(n):
        W.append(Wf[ow:ow + dn[i] * dp[i]].reshape(dn[i], dp[i]))
        bias.append(bf[ob:ob + dn[i]])
        ow += dn[i] * dp[i]
        ob += dn[i]
    dl = int(dn[p.leaves_of(b)[0]])
    C = p.C[s["C"][0]:s["C"][1]].astype(np.float64).reshape(o, dl)
    x = p.x[s["x"][0]:s["x"][1]].astype(np.float64)
    return n, Kn, dn, o, p.parents_of(b), W, bias, C, x


def log_px(p, b):
    n, Kn, dn, o, par, W, bias, C, x = instance_params(p, b)
    off = np.concatenate([[0], np.cumsum(dn)]).astype(int)
    N = int(off[-1])
    blk = lambda i: slice(off[i], off[i + 1])
    mean = [None] * n
    cov = np.zeros((N, N))
    mean[0] = bias[0]
    cov[blk(0), blk(0)] = p.prior_var * np.eye(dn[0])
    for i in range(1, n):
        q = par[i]
        mean[i] = W[i] @ mean[q] + bias[i]
        for j in range(i):
            cov[blk(i), blk(j)] = W[i] @ cov[blk(q), blk(j)]
            cov[blk(j), blk(i)] = cov[blk(i), blk(j)].T
        cov[blk(i), blk(i)] = W[i] @ cov[blk(q), blk(q)] @ W[i].T + p.prior_var * np.eye(dn[i])
    leaves = p.leaves_of(b)
    L = len(leaves)
    mx = np.concatenate([C @ mean[l] for l in leaves])
    cx = np.zeros((L * o, L * o))
    for a, la in enumerate(leaves):
        for c, lc in enumerate(leaves):
            cx[a * o:(a + 1) * o, c * o:(c + 1) * o] = C @ cov[blk(la), blk(lc)] @ C.T
    cx += p.obs_var * np.eye(L * o)
    ch = np.linalg.cholesky(cx)
    r = np.linalg.solve(ch, x - mx)
    return float(-0.5 * r @ r - np.sum(np.log(np.diag(ch))) - 0.5 * L * o * np.log(2 * np.pi))


def log_weight_single(p, b, k_per_node):
    """log P(x, z) - sum_i log Q_i(z_i) for one sample combination (the single-sample
    importance weight of the VAE estimator), from the joint density directly."""
    n, Kn, dn, o, par, W, bias, C, x = instance_params(p, b)
    s = p.slices(b)
    ef = p.eps[s["eps"][0]:s["eps"][1]].astype(np.float64)
    mf = p.q_mean[s["q"][0]:s["q"][1]].astype(np.float64)
    lf = p.q_logstd[s["q"][0]:s["q"][1]].astype(np.float64)
    z, m, ls, oe, oq = [], [], [], 0, 0
    for i in range(n):
        eps_i = ef[oe:oe + Kn[i] * dn[i]].reshape(Kn[i], dn[i])
        m.append(mf[oq:oq + dn[i]])
        ls.append(lf[oq:oq + dn[i]])
        z.append(m[i] + np.exp(ls[i]) * eps_i[k_per_node[i]])
        oe += Kn[i] * dn[i]
        oq += dn[i]
    lg = lambda y, mu, var: -0.5 * np.sum((y - mu) ** 2) / var - 0.5 * len(y) * np.log(2 * np.pi * var)
    v = lg(z[0], bias[0], p.prior_var)
    for i in range(1, n):
        v += lg(z[i], W[i] @ z[par[i]] + bias[i], p.prior_var)
    for a, l in enumerate(p.leaves_of(b)):
        v += lg(x[a * o:(a + 1) * o], C @ z[l], p.obs_var)
    for i in range(n):
        v -= np.sum(-0.5 * ((z[i] - m[i]) / np.exp(ls[i])) ** 2 - ls[i] - 0.5 * np.log(2 * np.pi))
    return float(v)
