"""Seeded synthetic workloads for the TMC hot path (linear-Gaussian chains and trees).

This module only draws inputs; it holds none of the estimator's arithmetic.  Both the
CUDA path and the FP64 oracle consume what it produces.

Generative model (Section 2.2 "Efficient averaging", directed factorisation; Appendix
"Typical choice of factors"):

    z_0        ~ N(b_0, prior_var I)                       (root; b_0 = 0 here)
    z_i | z_p  ~ N(W_i z_p + b_i, prior_var I)             (i >= 1, p = parent[i] < i)
    x_l | z_l  ~ N(C z_l, obs_var I)                       (one observation per leaf l)

Proposal (Section 2.1, factorised): Q_i = N(m_i, diag(exp(logs_i)^2)), samples
z_i^k = m_i + exp(logs_i) * eps_i^k with eps ~ N(0, I).  m_i / logs_i come from the exact
Gaussian posterior marginals of the instance (mean + N(0, 0.5^2) offset, 1.2 x the
posterior std), so the proposal is reasonable but not exact.

Flat layouts (identical to the C-ABI's tmc_inputs; instance b follows instance b-1):
    eps       [b][i][k][j]   n_b*K_b*d_b floats
    q_mean    [b][i][j]      n_b*d_b
    q_logstd  [b][i][j]      n_b*d_b
    W         [i][r][c]      n*d*d   (shared) or per instance n_b*d_b*d_b; mu_r = sum_c W[r][c] z_p[c] + b[r]
    bias      [i][r]         n*d     (shared) or per instance; bias[0] is the root prior mean
    C         [o][c]         obs*d   (shared) or per instance
    x         [b][leaf][o]   leaves in increasing node order, obs_b floats each

Seeds: model parameters come from PCG64(seed); instance b draws from PCG64(seed).jumped(b+1).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

# The five workloads of the hot path, by shape.
CHAIN_CONFIGS = {
    "chain_n3_K4_d2_B8": dict(n=3, K=4, d=2, obs=4, B=8),
    "chain_n8_K128_d32_B256": dict(n=8, K=128, d=32, obs=64, B=256),
    "chain_n8_K256_d64_B128": dict(n=8, K=256, d=64, obs=128, B=128),
    "chain_n16_K1024_d128_B64": dict(n=16, K=1024, d=128, obs=256, B=64),
}
TREE_BATCH = dict(B=512, n_lo=2, n_hi=24, Ks=(32, 64, 128, 256, 512), ds=(16, 32, 64), max_depth=8)
SEED_BASE = 20181806


@dataclass
class Problem:
    """A batch of TMC instances in the C-ABI's flat layout (all float32 / int32)."""

    n: np.ndarray            # [B] int32
    parent: np.ndarray       # [sum n] int32, local indices, parent[0] = -1, parent[i] < i
    K: np.ndarray            # [B] int32
    d: np.ndarray            # [B] int32
    obs: np.ndarray          # [B] int32
    shared: bool
    prior_var: float
    obs_var: float
    eps: np.ndarray
    q_mean: np.ndarray
    q_logstd: np.ndarray
    W: np.ndarray
    bias: np.ndarray
    C: np.ndarray
    x: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.n.shape[0])

    # ---- offsets (pure bookkeeping) -------------------------------------------------
    def parents_of(self, b: int) -> np.ndarray:
        s = int(np.sum(self.n[:b]))
        return self.parent[s:s + int(self.n[b])]

    def leaves_of(self, b: int) -> list[int]:
        par = self.parents_of(b)
        has_child = np.zeros(len(par), dtype=bool)
        for i in range(1, len(par)):
            has_child[par[i]] = True
        return [i for i in range(len(par)) if not has_child[i]]

    def entries(self) -> int:
        """Factor entries per call, B*n*K^2 summed over instances (the metric's unit)."""
        return int(np.sum(self.n.astype(np.int64) * self.K.astype(np.int64) ** 2))

    def edge_entries(self) -> int:
        """Pairwise-factor entries actually formed: sum over edges of K_p*K_i."""
        return int(np.sum((self.n.astype(np.int64) - 1) * self.K.astype(np.int64) ** 2))

    def slices(self, b: int) -> dict:
        """Slices of every flat array belonging to instance b."""
        n, K, d, o = (self.n.astype(np.int64), self.K.astype(np.int64),
                      self.d.astype(np.int64), self.obs.astype(np.int64))
        nl = np.array([len(self.leaves_of(i)) for i in range(self.B)], dtype=np.int64)
        def off(v):
            return int(np.sum(v[:b])), int(np.sum(v[:b + 1]))
        out = dict(eps=off(n * K * d), q=off(n * d), x=off(nl * o), parent=off(n))
        if self.shared:
            out.update(W=(0, self.W.size), bias=(0, self.bias.size), C=(0, self.C.size))
        else:
            out.update(W=off(n * d * d), bias=off(n * d), C=off(o * d))
        return out


# ---------------------------------------------------------------------------------------
# Exact Gaussian posterior, used only to place the proposal (information form, dense).
# ---------------------------------------------------------------------------------------
def _posterior_factor(parent, Ws, C, prior_var, obs_var):
    """Cholesky factor of the posterior precision and the marginal stds (x-independent)."""
    n = len(parent)
    d = Ws[0].shape[0]
    N = n * d
    A = np.eye(N)
    for i in range(1, n):
        p = parent[i]
        A[i * d:(i + 1) * d, p * d:(p + 1) * d] -= Ws[i]
    Lam = A.T @ A / prior_var
    CtC = C.T @ C / obs_var
    for leaf in _leaves(parent):
        sl = slice(leaf * d, (leaf + 1) * d)
        Lam[sl, sl] += CtC
    cf = sla.cho_factor(Lam, lower=True)
    Linv = sla.solve_triangular(cf[0], np.eye(N), lower=True)
    std = np.sqrt(np.sum(Linv * Linv, axis=0)).reshape(n, d)
    return dict(cf=cf, A=A, std=std, n=n, d=d)


def _posterior_mean(fac, bs, C, xs_by_leaf, prior_var, obs_var):
    n, d = fac["n"], fac["d"]
    h = fac["A"].T @ np.concatenate(bs) / prior_var
    for leaf, xl in xs_by_leaf.items():
        h[leaf * d:(leaf + 1) * d] += C.T @ xl / obs_var
    return sla.cho_solve(fac["cf"], h).reshape(n, d)


def _posterior_tree_bp(parent, Ws, bs, C, xs_by_leaf, prior_var, obs_var):
    """Exact posterior marginals of the tree by Gaussian belief propagation in information
    form: eliminate latents from the leaves up, then pass means / covariances down.
    O(n d^3) instead of the dense O((n d)^3)."""
    n = len(parent)
    d = Ws[0].shape[0]
    I = np.eye(d)
    J = [I / prior_var for _ in range(n)]          # diagonal precision blocks
    h = [np.zeros(d) for _ in range(n)]
    h[0] = bs[0] / prior_var
    CtC = C.T @ C / obs_var
    for i in range(1, n):
        p = parent[i]
        J[p] = J[p] + Ws[i].T @ Ws[i] / prior_var
        h[i] = h[i] + bs[i] / prior_var
        h[p] = h[p] - Ws[i].T @ bs[i] / prior_var
    for leaf, xl in xs_by_leaf.items():
        J[leaf] = J[leaf] + CtC
        h[leaf] = h[leaf] + C.T @ xl / obs_var
    # off-diagonal block between child i and parent p: L_ip = -W_i / prior_var
    Jm = [None] * n   # precision of z_i after absorbing its subtree (conditioned on parent)
    hm = [None] * n
    Jacc = [j.copy() for j in J]
    hacc = [v.copy() for v in h]
    for i in range(n - 1, 0, -1):
        p = parent[i]
        Jm[i], hm[i] = Jacc[i], hacc[i]
        L = -Ws[i] / prior_var                       # d x d block (row i, col p)
        Jinv_L = np.linalg.solve(Jm[i], L)
        Jacc[p] = Jacc[p] - L.T @ Jinv_L
        hacc[p] = hacc[p] - L.T @ np.linalg.solve(Jm[i], hm[i])
    mean = np.zeros((n, d))
    cov = [None] * n
    cov[0] = np.linalg.inv(Jacc[0])
    mean[0] = cov[0] @ hacc[0]
    for i in range(1, n):
        p = parent[i]
        L = -Ws[i] / prior_var
        Jinv = np.linalg.inv(Jm[i])
        A = -Jinv @ L                                # z_i | z_p has mean Jinv (h_i - L z_p)
        mean[i] = Jinv @ hm[i] + A @ mean[p]
        cov[i] = Jinv + A @ cov[p] @ A.T
    std = np.sqrt(np.stack([np.diag(c) for c in cov]))
    return mean, std


def _leaves(parent):
    n = len(parent)
    has_child = np.zeros(n, dtype=bool)
    for i in range(1, n):
        has_child[parent[i]] = True
    return [i for i in range(n) if not has_child[i]]


def _draw_model(rng, n, d, obs, orth_C=False):
    Ws = [np.zeros((d, d))] + [rng.standard_normal((d, d)) / np.sqrt(d) for _ in range(1, n)]
    bs = [np.zeros(d)] + [rng.standard_normal(d) for _ in range(1, n)]
    C = rng.standard_normal((obs, d)) / np.sqrt(d)
    if orth_C:
        # orthogonal columns (C^T C diagonal), so a leaf's posterior covariance is diagonal
        q, _ = np.linalg.qr(C)
        C = q * rng.uniform(0.5, 1.5, size=d)
    return Ws, bs, C


def _ancestral_x(rng, parent, Ws, bs, C, prior_var, obs_var):
    n = len(parent)
    d = bs[0].shape[0]
    z = np.zeros((n, d))
    z[0] = bs[0] + np.sqrt(prior_var) * rng.standard_normal(d)
    for i in range(1, n):
        z[i] = Ws[i] @ z[parent[i]] + bs[i] + np.sqrt(prior_var) * rng.standard_normal(d)
    xs = {}
    for leaf in _leaves(parent):
        xs[leaf] = C @ z[leaf] + np.sqrt(obs_var) * rng.standard_normal(C.shape[0])
    return xs


def _instance(rng, parent, K, Ws, bs, C, prior_var, obs_var, exact_proposal, mean_noise, std_scale,
              fac=None):
    """Draw x, the proposal and eps for one instance (model fixed)."""
    n = len(parent)
    d = bs[0].shape[0]
    xs = _ancestral_x(rng, parent, Ws, bs, C, prior_var, obs_var)
    if fac is None:  # per-instance model: exact marginals by tree belief propagation
        pm, ps = _posterior_tree_bp(parent, Ws, bs, C, xs, prior_var, obs_var)
    else:            # shared model: one dense factorisation serves every instance
        pm, ps = _posterior_mean(fac, bs, C, xs, prior_var, obs_var), fac["std"]
    if exact_proposal:
        m, s = pm, ps
    else:
        m = pm + mean_noise * rng.standard_normal((n, d))
        s = std_scale * ps
    eps = rng.standard_normal((n, K, d), dtype=np.float32)
    x = np.concatenate([xs[l] for l in sorted(xs)])
    return x, m, np.log(s), eps


def make_problem(parents, Ks, ds, obss, *, shared, seed, prior_var=1.0, obs_var=0.1,
                 exact_proposal=False, zero_W=False, mean_noise=0.5, std_scale=1.2,
                 name="", model_override=None, orth_C=False) -> Problem:
    """General batch builder.  parents: list of per-instance parent arrays."""
    B = len(parents)
    base = np.random.PCG64(seed)
    model_rng = np.random.Generator(base)
    n_arr = np.array([len(p) for p in parents], dtype=np.int32)
    eps_l, m_l, ls_l, x_l, W_l, b_l, C_l = [], [], [], [], [], [], []
    shared_model = None
    if shared:
        assert len(set(map(tuple, map(list, parents)))) == 1 and len(set(ds)) == 1 and len(set(obss)) == 1
        shared_model = model_override or _draw_model(model_rng, len(parents[0]), ds[0], obss[0], orth_C)
        if zero_W:
            shared_model = ([np.zeros_like(w) for w in shared_model[0]],) + tuple(shared_model[1:])
        shared_fac = _posterior_factor(np.asarray(parents[0], dtype=np.int64), shared_model[0],
                                       shared_model[2], prior_var, obs_var)
    for b in range(B):
        rng = np.random.Generator(base.jumped(b + 1))
        parent = np.asarray(parents[b], dtype=np.int64)
        if shared:
            Ws, bs, C = shared_model
        else:
            Ws, bs, C = _draw_model(rng, len(parent), ds[b], obss[b], orth_C)
            if zero_W:
                Ws = [np.zeros_like(w) for w in Ws]
            W_l.append(np.stack(Ws).ravel()); b_l.append(np.stack(bs).ravel()); C_l.append(C.ravel())
        x, m, ls, eps = _instance(rng, parent, Ks[b], Ws, bs, C, prior_var, obs_var,
                                  exact_proposal, mean_noise, std_scale,
                                  fac=shared_fac if shared else None)
        eps_l.append(eps.ravel()); m_l.append(m.ravel()); ls_l.append(ls.ravel()); x_l.append(x)
    if shared:
        Ws, bs, C = shared_model
        W_l, b_l, C_l = [np.stack(Ws).ravel()], [np.stack(bs).ravel()], [C.ravel()]
    f32 = lambda lst: np.ascontiguousarray(np.concatenate(lst).astype(np.float32))
    return Problem(
        n=n_arr, parent=np.concatenate([np.asarray(p, dtype=np.int32) for p in parents]),
        K=np.asarray(Ks, dtype=np.int32), d=np.asarray(ds, dtype=np.int32),
        obs=np.asarray(obss, dtype=np.int32), shared=bool(shared),
        prior_var=float(prior_var), obs_var=float(obs_var),
        eps=f32(eps_l), q_mean=f32(m_l), q_logstd=f32(ls_l), W=f32(W_l), bias=f32(b_l),
        C=f32(C_l), x=f32(x_l), name=name)


def chain_parents(n: int) -> np.ndarray:
    return np.arange(-1, n - 1, dtype=np.int32)


def make_chain(n, K, d, obs, B, seed, **kw) -> Problem:
    """Chain z_0 -> z_1 -> ... -> z_{n-1} -> x with one model shared by the B instances."""
    return make_problem([chain_parents(n)] * B, [K] * B, [d] * B, [obs] * B,
                        shared=True, seed=seed, **kw)


def chain_config(name: str, B: int | None = None, **kw) -> Problem:
    c = dict(CHAIN_CONFIGS[name])
    idx = list(CHAIN_CONFIGS).index(name)
    if B is not None:
        c["B"] = B
    p = make_chain(c["n"], c["K"], c["d"], c["obs"], c["B"], SEED_BASE + idx, **kw)
    p.name = name
    return p


def random_tree(rng, n, max_depth) -> np.ndarray:
    """Node 0 is the root; each later node picks a parent uniformly among earlier nodes
    whose depth is below max_depth, so the tree depth is at most max_depth."""
    parent = np.full(n, -1, dtype=np.int32)
    depth = np.zeros(n, dtype=np.int32)
    for i in range(1, n):
        cand = np.nonzero(depth[:i] < max_depth)[0]
        p = int(cand[rng.integers(len(cand))])
        parent[i] = p
        depth[i] = depth[p] + 1
    return parent


def tree_batch(B: int | None = None, seed: int | None = None, **kw) -> Problem:
    """Batch of uneven random trees, each instance with its own model, K and d."""
    cfg = dict(TREE_BATCH)
    if B is not None:
        cfg["B"] = B
    seed = SEED_BASE + 4 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed + 1_000_003))
    parents, Ks, ds = [], [], []
    for _ in range(cfg["B"]):
        n = int(rng.integers(cfg["n_lo"], cfg["n_hi"] + 1))
        parents.append(random_tree(rng, n, cfg["max_depth"]))
        Ks.append(int(rng.choice(cfg["Ks"])))
        ds.append(int(rng.choice(cfg["ds"])))
    obss = [2 * d for d in ds]
    p = make_problem(parents, Ks, ds, obss, shared=False, seed=seed, **kw)
    p.name = "trees_B%d" % cfg["B"]
    return p


def star(N: int, K: int, d: int = 1, obs: int | None = None, B: int = 1, seed: int | None = None,
         **kw) -> Problem:
    """The toy of Section 3.1 at scale: one global latent (the root) with N children, each
    child observed (one observation per leaf), K samples per latent.  Per-instance models,
    so the exact posterior comes from belief propagation (no dense factorisation)."""
    seed = SEED_BASE + 6 if seed is None else seed
    parent = np.array([-1] + [0] * N, dtype=np.int32)
    obs = 2 * d if obs is None else obs
    p = make_problem([parent] * B, [K] * B, [d] * B, [obs] * B, shared=False, seed=seed, **kw)
    p.name = "star_N%d_K%d_d%d_B%d" % (N, K, d, B)
    return p


def redraw_eps(p: Problem, seed: int) -> np.ndarray:
    """Fresh proposal noise for the same model/x/proposal (used for unbiasedness checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(p.eps.shape, dtype=np.float32)
