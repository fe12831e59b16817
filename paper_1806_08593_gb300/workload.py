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
    """A batch of TMC instances in the C-ABI's flat layout (all float32 / int32).

    Sizes: K[b] / d[b] apply to every latent of instance b unless the per-latent arrays Kn /
    dn ([sum n], node order) are given (Eq. (is) allows a different K_i for every latent; a
    latent's dimension d_i may differ too, W_i is then d_i x d_parent).  The leaves of an
    instance share one dimension (one observation matrix C per instance)."""

    n: np.ndarray            # [B] int32
    parent: np.ndarray       # [sum n] int32, local indices, parent[0] = -1, parent[i] < i
    K: np.ndarray            # [B] int32
    d: np.ndarray            # [B] int32 (the leaves' dimension when dn is given)
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
    Kn: np.ndarray | None = None   # [sum n] int32 per-latent K, or None
    dn: np.ndarray | None = None   # [sum n] int32 per-latent d, or None
    # coupled (non-factorised) proposal: A_i per latent, laid out like per-instance W blocks
    # (even when the model is shared); Q_i(z_i^k | parent samples) = N(m_i + A_i (z_p^k - m_p),
    # diag(exp(2 logs_i))).  None: the factorised proposal.
    q_A: np.ndarray | None = None

    @property
    def B(self) -> int:
        return int(self.n.shape[0])

    @property
    def ragged(self) -> bool:
        return self.Kn is not None or self.dn is not None

    def K_nodes(self) -> np.ndarray:
        return self.Kn if self.Kn is not None else np.repeat(self.K, self.n).astype(np.int32)

    def d_nodes(self) -> np.ndarray:
        return self.dn if self.dn is not None else np.repeat(self.d, self.n).astype(np.int32)

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
        """Factor entries per call, B*n*K^2 summed over instances (the metric's unit);
        sum over latents of K_i^2 with per-latent K."""
        return int(np.sum(self.K_nodes().astype(np.int64) ** 2))

    def edge_entries(self) -> int:
        """Pairwise-factor entries actually formed: sum over edges of K_p*K_i."""
        Kn = self.K_nodes().astype(np.int64)
        tot, off = 0, 0
        for b in range(self.B):
            par = self.parents_of(b)
            for i in range(1, len(par)):
                tot += Kn[off + par[i]] * Kn[off + i]
            off += len(par)
        return int(tot)

    def node_sizes(self, b: int):
        """(K_i, d_i, d_parent(i)) of instance b's latents (the root's parent dimension is its
        own: its W block is d_0 x d_0 and ignored)."""
        s = int(np.sum(self.n[:b]))
        n = int(self.n[b])
        Kn = self.K_nodes()[s:s + n].astype(np.int64)
        dn = self.d_nodes()[s:s + n].astype(np.int64)
        par = self.parents_of(b)
        dp = np.array([dn[par[i]] if i else dn[0] for i in range(n)], dtype=np.int64)
        return Kn, dn, dp

    def slices(self, b: int) -> dict:
        """Slices of every flat array belonging to instance b."""
        return self.slices_all(b + 1)[b]

    def slices_all(self, upto: int | None = None) -> list[dict]:
        """slices(b) of the instances b < upto (all by default), in one pass."""
        upto = self.B if upto is None else upto
        eps = q = w = x = c = a = 0
        outs = []
        for i in range(upto):
            Kn, dn, dp = self.node_sizes(i)
            leaves = self.leaves_of(i)
            dl = int(dn[leaves[0]])
            se, sq, sw = int(np.sum(Kn * dn)), int(np.sum(dn)), int(np.sum(dn * dp))
            sx, sc = len(leaves) * int(self.obs[i]), int(self.obs[i]) * dl
            n0 = int(np.sum(self.n[:i]))
            out = dict(eps=(eps, eps + se), q=(q, q + sq), x=(x, x + sx), A=(a, a + sw),
                       parent=(n0, n0 + int(self.n[i])))
            if self.shared:
                out.update(W=(0, self.W.size), bias=(0, self.bias.size), C=(0, self.C.size))
            else:
                out.update(W=(w, w + sw), bias=(q, q + sq), C=(c, c + sc))
            outs.append(out)
            eps += se; q += sq; w += sw; x += sx; c += sc; a += sw
        return outs


# ---------------------------------------------------------------------------------------
# Exact Gaussian posterior, used only to place the proposal (information form, dense).
# Latent i has dimension dn[i]; W_i is dn[i] x dn[parent[i]].
# ---------------------------------------------------------------------------------------
def _offsets(dn):
    return np.concatenate([[0], np.cumsum(dn)]).astype(np.int64)


def _posterior_factor(parent, Ws, C, prior_var, obs_var, dn):
    """Cholesky factor of the posterior precision and the marginal stds (x-independent)."""
    n = len(parent)
    o = _offsets(dn)
    N = int(o[-1])
    A = np.eye(N)
    for i in range(1, n):
        p = parent[i]
        A[o[i]:o[i + 1], o[p]:o[p + 1]] -= Ws[i]
    Lam = A.T @ A / prior_var
    CtC = C.T @ C / obs_var
    for leaf in _leaves(parent):
        sl = slice(o[leaf], o[leaf + 1])
        Lam[sl, sl] += CtC
    cf = sla.cho_factor(Lam, lower=True)
    Linv = sla.solve_triangular(cf[0], np.eye(N), lower=True)
    stdv = np.sqrt(np.sum(Linv * Linv, axis=0))
    return dict(cf=cf, A=A, std=[stdv[o[i]:o[i + 1]] for i in range(n)], n=n, o=o)


def _posterior_mean(fac, bs, C, xs_by_leaf, prior_var, obs_var):
    o = fac["o"]
    h = fac["A"].T @ np.concatenate(bs) / prior_var
    for leaf, xl in xs_by_leaf.items():
        h[o[leaf]:o[leaf + 1]] += C.T @ xl / obs_var
    v = sla.cho_solve(fac["cf"], h)
    return [v[o[i]:o[i + 1]] for i in range(fac["n"])]


def _posterior_tree_bp(parent, Ws, bs, C, xs_by_leaf, prior_var, obs_var, dn):
    """Exact posterior marginals of the tree by Gaussian belief propagation in information
    form: eliminate latents from the leaves up, then pass means / covariances down.
    O(n d^3) instead of the dense O((n d)^3)."""
    n = len(parent)
    J = [np.eye(int(dn[i])) / prior_var for i in range(n)]  # diagonal precision blocks
    h = [np.zeros(int(dn[i])) for i in range(n)]
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
        L = -Ws[i] / prior_var                       # d_i x d_p block (row i, col p)
        Jinv_L = np.linalg.solve(Jm[i], L)
        Jacc[p] = Jacc[p] - L.T @ Jinv_L
        hacc[p] = hacc[p] - L.T @ np.linalg.solve(Jm[i], hm[i])
    mean = [None] * n
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
    std = [np.sqrt(np.diag(c)) for c in cov]
    return mean, std


def _leaves(parent):
    n = len(parent)
    has_child = np.zeros(n, dtype=bool)
    for i in range(1, n):
        has_child[parent[i]] = True
    return [i for i in range(n) if not has_child[i]]


def _draw_model(rng, parent, dn, obs, orth_C=False):
    """W_i (d_i x d_p) entries N(0, 1/d_p), b_i ~ N(0, I), C (obs x d_leaf) entries
    N(0, 1/d_leaf); W_0 = 0 and b_0 = 0 (the root's prior mean)."""
    n = len(parent)
    dl = int(dn[_leaves(parent)[0]])
    Ws = [np.zeros((int(dn[0]), int(dn[0])))] + [
        rng.standard_normal((int(dn[i]), int(dn[parent[i]]))) / np.sqrt(dn[parent[i]]) for i in range(1, n)]
    bs = [np.zeros(int(dn[0]))] + [rng.standard_normal(int(dn[i])) for i in range(1, n)]
    C = rng.standard_normal((obs, dl)) / np.sqrt(dl)
    if orth_C:
        # orthogonal columns (C^T C diagonal), so a leaf's posterior covariance is diagonal
        q, _ = np.linalg.qr(C)
        C = q * rng.uniform(0.5, 1.5, size=dl)
    return Ws, bs, C


def _ancestral_x(rng, parent, Ws, bs, C, prior_var, obs_var):
    n = len(parent)
    z = [None] * n
    z[0] = bs[0] + np.sqrt(prior_var) * rng.standard_normal(bs[0].shape[0])
    for i in range(1, n):
        z[i] = Ws[i] @ z[parent[i]] + bs[i] + np.sqrt(prior_var) * rng.standard_normal(bs[i].shape[0])
    xs = {}
    for leaf in _leaves(parent):
        xs[leaf] = C @ z[leaf] + np.sqrt(obs_var) * rng.standard_normal(C.shape[0])
    return xs


def _instance(rng, parent, Kn, dn, Ws, bs, C, prior_var, obs_var, exact_proposal, mean_noise,
              std_scale, fac=None):
    """Draw x, the proposal and eps for one instance (model fixed).  Returns flat arrays."""
    n = len(parent)
    uniform = len(set(Kn)) == 1 and len(set(dn)) == 1
    xs = _ancestral_x(rng, parent, Ws, bs, C, prior_var, obs_var)
    if fac is None:  # per-instance model: exact marginals by tree belief propagation
        pm, ps = _posterior_tree_bp(parent, Ws, bs, C, xs, prior_var, obs_var, dn)
    else:            # shared model: one dense factorisation serves every instance
        pm, ps = _posterior_mean(fac, bs, C, xs, prior_var, obs_var), fac["std"]
    pm, ps = np.concatenate(pm), np.concatenate(ps)
    if exact_proposal:
        m, s = pm, ps
    else:
        m = pm + mean_noise * rng.standard_normal(pm.shape[0])
        s = std_scale * ps
    if uniform:
        eps = rng.standard_normal((n, int(Kn[0]), int(dn[0])), dtype=np.float32).ravel()
    else:
        eps = np.concatenate([rng.standard_normal((int(Kn[i]), int(dn[i])), dtype=np.float32).ravel()
                              for i in range(n)])
    x = np.concatenate([xs[l] for l in sorted(xs)])
    return x, m, np.log(s), eps


def make_problem(parents, Ks, ds, obss, *, shared, seed, prior_var=1.0, obs_var=0.1,
                 exact_proposal=False, zero_W=False, mean_noise=0.5, std_scale=1.2,
                 name="", model_override=None, orth_C=False) -> Problem:
    """General batch builder.  parents: list of per-instance parent arrays; Ks[b] / ds[b]: an
    int (every latent of b) or a list of per-latent values (Eq. (is)'s K_i; d_i with W_i of
    shape d_i x d_parent; the leaves of an instance must share d)."""
    B = len(parents)
    base = np.random.PCG64(seed)
    model_rng = np.random.Generator(base)
    n_arr = np.array([len(p) for p in parents], dtype=np.int32)
    per = lambda v, n: [int(v)] * n if np.isscalar(v) else [int(a) for a in v]
    Kns = [per(Ks[b], len(parents[b])) for b in range(B)]
    dns = [per(ds[b], len(parents[b])) for b in range(B)]
    ragged = any(len(set(k)) > 1 for k in Kns) or any(len(set(v)) > 1 for v in dns)
    for b in range(B):
        dl = {dns[b][l] for l in _leaves(np.asarray(parents[b]))}
        assert len(dl) == 1, "the leaves of an instance share one dimension"
    eps_l, m_l, ls_l, x_l, W_l, b_l, C_l = [], [], [], [], [], [], []
    shared_model = None
    if shared:
        assert len(set(map(tuple, map(list, parents)))) == 1 and len(set(map(tuple, dns))) == 1 \
            and len(set(obss)) == 1
        par0 = np.asarray(parents[0], dtype=np.int64)
        shared_model = model_override or _draw_model(model_rng, par0, dns[0], obss[0], orth_C)
        if zero_W:
            shared_model = ([np.zeros_like(w) for w in shared_model[0]],) + tuple(shared_model[1:])
        shared_fac = _posterior_factor(par0, shared_model[0], shared_model[2], prior_var, obs_var, dns[0])
    for b in range(B):
        rng = np.random.Generator(base.jumped(b + 1))
        parent = np.asarray(parents[b], dtype=np.int64)
        if shared:
            Ws, bs, C = shared_model
        else:
            Ws, bs, C = _draw_model(rng, parent, dns[b], obss[b], orth_C)
            if zero_W:
                Ws = [np.zeros_like(w) for w in Ws]
            W_l.append(np.concatenate([w.ravel() for w in Ws])); b_l.append(np.concatenate(bs))
            C_l.append(C.ravel())
        x, m, ls, eps = _instance(rng, parent, Kns[b], dns[b], Ws, bs, C, prior_var, obs_var,
                                  exact_proposal, mean_noise, std_scale,
                                  fac=shared_fac if shared else None)
        eps_l.append(eps); m_l.append(m); ls_l.append(ls); x_l.append(x)
    if shared:
        Ws, bs, C = shared_model
        W_l, b_l, C_l = [np.concatenate([w.ravel() for w in Ws])], [np.concatenate(bs)], [C.ravel()]
    f32 = lambda lst: np.ascontiguousarray(np.concatenate(lst).astype(np.float32))
    leaf_d = [dns[b][_leaves(np.asarray(parents[b]))[0]] for b in range(B)]
    return Problem(
        n=n_arr, parent=np.concatenate([np.asarray(p, dtype=np.int32) for p in parents]),
        K=np.asarray([k[0] for k in Kns], dtype=np.int32), d=np.asarray(leaf_d, dtype=np.int32),
        obs=np.asarray(obss, dtype=np.int32), shared=bool(shared),
        prior_var=float(prior_var), obs_var=float(obs_var),
        eps=f32(eps_l), q_mean=f32(m_l), q_logstd=f32(ls_l), W=f32(W_l), bias=f32(b_l),
        C=f32(C_l), x=f32(x_l), name=name,
        Kn=np.concatenate([np.asarray(k, dtype=np.int32) for k in Kns]) if ragged else None,
        dn=np.concatenate([np.asarray(v, dtype=np.int32) for v in dns]) if ragged else None)


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


def layered_chain(widths, K, obs, B, seed=None, **kw) -> Problem:
    """A chain whose latents have the given dimensions, root first, each with K samples (or
    a per-latent list), one model shared by the B instances.  The shape of the paper's
    five-layer MNIST model (widths 4/8/16/32/64 from the top, K = 20; Section 4), with a
    synthetic Gaussian observation of dimension obs in place of the images."""
    n = len(widths)
    seed = SEED_BASE + 7 if seed is None else seed
    p = make_problem([chain_parents(n)] * B, [K] * B, [list(widths)] * B, [obs] * B,
                     shared=True, seed=seed, **kw)
    p.name = "layered_chain_%s_K%s_B%d" % ("-".join(map(str, widths)), K, B)
    return p


def ragged_trees(B, seed, n_choices=(1, 2, 3, 5, 7), Ks=(1, 2, 3, 4), ds=(1, 2, 3), max_depth=3,
                 **kw) -> Problem:
    """Random trees whose latents draw their own K_i and d_i (the leaves of an instance share
    one d), each instance with its own model."""
    rng = np.random.Generator(np.random.PCG64(seed + 2_000_003))
    parents, Kns, dns = [], [], []
    for _ in range(B):
        par = random_tree(rng, int(rng.choice(n_choices)), max_depth)
        leaves = set(_leaves(par))
        dl = int(rng.choice(ds))
        parents.append(par)
        Kns.append([int(rng.choice(Ks)) for _ in range(len(par))])
        dns.append([dl if i in leaves else int(rng.choice(ds)) for i in range(len(par))])
    obss = [int(rng.integers(1, 5)) for _ in range(B)]
    return make_problem(parents, Kns, dns, obss, shared=False, seed=seed, **kw)


def couple_proposal(p: Problem, mode: str = "prior", alpha: float = 0.5) -> Problem:
    """The same instances with a coupled (non-factorised) proposal: sample k of latent i is
    drawn given its parent's sample k (Section 2.3, "Non-factorised proposals").
      mode "prior":  Q_i(z_i | z_p) = P(z_i | z_p) for every non-root latent (A_i = W_i,
                     m_i = W_i m_p + b_i, std = prior std), as in the paper's comparison of
                     factorised and non-factorised proposals; the root keeps its proposal.
      mode "scaled": A_i = alpha W_i with the factorised proposal's m_i and std.
    Requires one K per instance (sample k of a latent needs a parent sample k)."""
    import copy
    q = copy.deepcopy(p)
    A_l, m_l, ls_l = [], [], []
    every = p.slices_all()
    for b in range(p.B):
        Kn, dn, dp = p.node_sizes(b)
        assert np.all(Kn == Kn[0]), "a coupled proposal here needs one K per instance"
        s = every[b]
        par = p.parents_of(b)
        Wf = p.W[s["W"][0]:s["W"][1]].astype(np.float64)
        bf = p.bias[s["bias"][0]:s["bias"][1]].astype(np.float64)
        m = p.q_mean[s["q"][0]:s["q"][1]].astype(np.float64).copy()
        ls = p.q_logstd[s["q"][0]:s["q"][1]].astype(np.float64).copy()
        oq = np.concatenate([[0], np.cumsum(dn)]).astype(int)
        ow = np.concatenate([[0], np.cumsum(dn * dp)]).astype(int)
        A = np.zeros(int(ow[-1]))
        for i in range(1, len(par)):
            Wi = Wf[ow[i]:ow[i + 1]].reshape(dn[i], dp[i])
            if mode == "prior":
                A[ow[i]:ow[i + 1]] = Wi.ravel()
                m[oq[i]:oq[i + 1]] = Wi @ m[oq[par[i]]:oq[par[i] + 1]] + bf[oq[i]:oq[i + 1]]
                ls[oq[i]:oq[i + 1]] = 0.5 * np.log(p.prior_var)
            else:
                A[ow[i]:ow[i + 1]] = alpha * Wi.ravel()
        A_l.append(A); m_l.append(m); ls_l.append(ls)
    q.q_A = np.concatenate(A_l).astype(np.float32)
    q.q_mean = np.concatenate(m_l).astype(np.float32)
    q.q_logstd = np.concatenate(ls_l).astype(np.float32)
    q.name = (p.name or "problem") + "_coupled_" + mode
    return q


def redraw_eps(p: Problem, seed: int) -> np.ndarray:
    """Fresh proposal noise for the same model/x/proposal (used for unbiasedness checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(p.eps.shape, dtype=np.float32)


# ---------------------------------------------------------------------------------------
# The loopy graph of Fig. 1: z1 -> z2, z1 -> z3, {z2, z3} -> z4 -> x.
# ---------------------------------------------------------------------------------------
@dataclass
class Diamond:
    """B instances of the Fig. 1 model, K samples of each of its four latents (dimension d).
    Layouts: eps [B][4][K][d], q_mean / q_logstd [B][4][d], W [5][d][d] (W_1: z2|z1,
    W_2: z3|z1, W_3 and W_4: z4|z2 and z4|z3; W_0 unused), bias [4][d], C [obs][d], x [B][obs];
    W, bias, C once when shared, else per instance."""

    B: int
    K: int
    d: int
    obs: int
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

    def entries(self) -> int:
        """Factor entries formed per call: the two matrix messages (K^3 each) and the K^2
        final sum, per instance."""
        return int(self.B * (2 * self.K ** 3 + self.K ** 2))

    def instance(self, b):
        d, obs = self.d, self.obs
        W = self.W.reshape(-1, 5, d, d)[0 if self.shared else b].astype(np.float64)
        bias = self.bias.reshape(-1, 4, d)[0 if self.shared else b].astype(np.float64)
        C = self.C.reshape(-1, obs, d)[0 if self.shared else b].astype(np.float64)
        return W, bias, C, self.x.reshape(self.B, obs)[b].astype(np.float64)


def _diamond_model(rng, d, obs, orth_C=False):
    W = np.zeros((5, d, d))
    W[1] = rng.standard_normal((d, d)) / np.sqrt(d)
    W[2] = rng.standard_normal((d, d)) / np.sqrt(d)
    W[3] = rng.standard_normal((d, d)) / np.sqrt(2 * d)  # two parents: input variance 2d
    W[4] = rng.standard_normal((d, d)) / np.sqrt(2 * d)
    bias = np.zeros((4, d))
    bias[1:] = rng.standard_normal((3, d))
    C = rng.standard_normal((obs, d)) / np.sqrt(d)
    if orth_C:
        q, _ = np.linalg.qr(C)
        C = q * rng.uniform(0.5, 1.5, size=d)
    return W, bias, C


def diamond_joint(W, bias, prior_var):
    """Mean and covariance of (z1, z2, z3, z4) under the Fig. 1 model: z = A z + bias + noise."""
    d = W.shape[1]
    A = np.zeros((4 * d, 4 * d))
    blk = lambda i: slice(i * d, (i + 1) * d)
    A[blk(1), blk(0)] = W[1]
    A[blk(2), blk(0)] = W[2]
    A[blk(3), blk(1)] = W[3]
    A[blk(3), blk(2)] = W[4]
    Minv = np.linalg.inv(np.eye(4 * d) - A)
    return Minv @ bias.ravel(), prior_var * Minv @ Minv.T, A


def make_diamond(K, d, obs, B, seed, shared=True, prior_var=1.0, obs_var=0.1, exact_proposal=False,
                 zero_W=False, orth_C=False, mean_noise=0.5, std_scale=1.2) -> Diamond:
    """Seeded instances of the Fig. 1 model; the proposal is placed from the exact posterior
    marginals (+ N(0, mean_noise^2) mean offset, std_scale x the std), as for the trees."""
    base = np.random.PCG64(seed)
    mrng = np.random.Generator(base)
    models = []
    for b in range(1 if shared else B):
        W, bias, C = _diamond_model(mrng if shared else np.random.Generator(base.jumped(1000 + b)), d, obs, orth_C)
        if zero_W:
            W[:] = 0.0
        models.append((W, bias, C))
    eps_l, m_l, ls_l, x_l = [], [], [], []
    for b in range(B):
        rng = np.random.Generator(base.jumped(b + 1))
        W, bias, C = models[0 if shared else b]
        mu0, S0, A = diamond_joint(W, bias, prior_var)
        z = rng.multivariate_normal(mu0, S0)
        x = C @ z[3 * d:] + np.sqrt(obs_var) * rng.standard_normal(obs)
        # exact posterior of (z1..z4) given x (information form)
        P0 = (np.eye(4 * d) - A).T @ (np.eye(4 * d) - A) / prior_var
        Lam = P0.copy()
        Lam[3 * d:, 3 * d:] += C.T @ C / obs_var
        h = P0 @ mu0
        h[3 * d:] += C.T @ x / obs_var
        cf = sla.cho_factor(Lam, lower=True)
        pm = sla.cho_solve(cf, h)
        ps = np.sqrt(np.diag(sla.cho_solve(cf, np.eye(4 * d))))
        if exact_proposal:
            m, s = pm, ps
        else:
            m = pm + mean_noise * rng.standard_normal(4 * d)
            s = std_scale * ps
        eps_l.append(rng.standard_normal((4, K, d), dtype=np.float32).ravel())
        m_l.append(m); ls_l.append(np.log(s)); x_l.append(x)
    f32 = lambda lst: np.ascontiguousarray(np.concatenate([np.ravel(a) for a in lst]).astype(np.float32))
    return Diamond(B=B, K=K, d=d, obs=obs, shared=bool(shared), prior_var=float(prior_var),
                   obs_var=float(obs_var), eps=f32(eps_l), q_mean=f32(m_l), q_logstd=f32(ls_l),
                   W=f32([m[0] for m in models]), bias=f32([m[1] for m in models]),
                   C=f32([m[2] for m in models]), x=f32(x_l),
                   name="diamond_K%d_d%d_B%d" % (K, d, B))
