/*
 * tmc_oracle.c -- plain, slow, FP64 CPU oracle for the Tensor Monte Carlo estimator
 * (Aitchison, "Tensor Monte Carlo: Particle Methods for the GPU Era", ICML 2019).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no source with the CUDA path.
 *
 * What it computes (all in double precision, plain loops, no blocking or fusion):
 *
 *   Eq. (is):  P_TMC = 1/prod_i K_i * sum_{k_1..k_n} P(x, z_1^{k_1},..,z_n^{k_n}) / prod_i Q(z_i^{k_i})
 *
 *   with K_i samples of latent i (the number may differ from latent to latent, as Eq. (is)
 *   allows) and latent i of dimension d_i.
 *
 *   tmc_oracle_brute_force    -- that sum enumerated literally over all prod_i K_i sample
 *                                combinations (log-sum-exp over combinations).
 *   tmc_oracle_log_marginal   -- the same quantity by summing out one index at a time
 *                                (Section 2.2 "Efficient averaging": the importance ratio is a
 *                                product of factors, Eq. (fac); sums over the indices of leaves
 *                                are pushed inside, as in the latent-variable example of
 *                                Fig. 2), using the factor choice of the Appendix ("Typical
 *                                choice of factors for a directed graphical model").
 *   tmc_oracle_grad           -- the adjoint of that recursion: gradient of log P_TMC with
 *                                respect to the samples, the model parameters and the proposal
 *                                parameters under the reparameterisation z = m + exp(logs)*eps.
 *
 * Model: z_0 ~ N(bias_0, prior_var I); z_i | z_p ~ N(W_i z_p + bias_i, prior_var I) for i >= 1
 * with p = parent[i] < i (W_i is d_i x d_p); every leaf l carries x_l ~ N(C z_l, obs_var I).
 * Proposal: Q_i(z) = N(z; m_i, diag(exp(2 logs_i))), samples z_i^k = m_i + exp(logs_i) eps_i^k,
 * or, with coupling matrices A_i (the non-factorised proposals of Section 2.3 "Non-factorised
 * proposals" and the appendix), Q_i(z_i^k | all samples of the parent) =
 * N(z_i^k; m_i + A_i (z_p^k - m_p), diag(exp(2 logs_i))): sample k of latent i is drawn given
 * the parent's sample with the same index k, so the proposal factor is still indexed by k_i
 * alone and the elimination is unchanged; only the samples and -log Q_i move.
 *
 * Factors (Appendix):  f_i^{(k_i, k_p)} = P(z_i^{k_i} | z_p^{k_p}) / Q_i(z_i^{k_i})   (i >= 1)
 *                      f_0^{k_0}        = P(z_0^{k_0}) / Q_0(z_0^{k_0})
 *                      g_l^{k_l}        = P(x_l | z_l^{k_l})                          (leaves)
 *
 * Log-sum-exp subtracts the maximum of the whole exponent being summed (one combined
 * maximum), which is exact in real arithmetic and cannot underflow every term.
 *
 * Flat layouts: see tmc_oracle.h.
 */
#include "tmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOG_2PI 1.8378770664093454835606594728112

/* ---------------------------------------------------------------------------------------
 * Instance view: pointers into the flat arrays for one instance b, and per-latent offsets.
 *   oz[i]  start of latent i's [K_i][d_i] block (eps, z, dz)
 *   oq[i]  start of latent i's [d_i] vectors (m, logs, bias)
 *   ow[i]  start of W_i, [d_i][d_p] (the root's block is [d_0][d_0] and unused)
 *   ok[i]  start of latent i's [K_i] per-sample scalars
 *   oe[i]  start of edge p -> i's blocks indexed by the PARENT's samples: messages [K_p] and
 *          conditional means [K_p][d_i] (i >= 1)
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int n, obs, dl; /* latents, observation dimension, the leaves' latent dimension */
  const int *parent, *K, *d;
  long long *oz, *oq, *ow, *ok, *oe, *oed;
  const double *eps, *m, *logs, *W, *bias, *C, *x;
  const double* A; /* proposal coupling matrices (layout of W), or NULL: factorised proposal */
  double prior_var, obs_var;
  int* leaf_slot; /* leaf_slot[i] = index of leaf i among the instance's leaves, or -1 */
  long long nz, nq, nw, nk, ne, ned;
} inst_t;

typedef struct {
  long long eps, q, x, W, C, parent, A;
} offs_t;

static int count_leaves(int n, const int* parent, int* leaf_slot) {
  int i, nl = 0;
  for (i = 0; i < n; ++i) leaf_slot[i] = 0;
  for (i = 1; i < n; ++i) leaf_slot[parent[i]] = -1; /* has a child */
  for (i = 0; i < n; ++i) {
    if (leaf_slot[i] == 0) leaf_slot[i] = nl++;
    else leaf_slot[i] = -1;
  }
  return nl;
}

static int validate(int B, const int* n, const int* parent, const int* K, const int* d,
                    const int* obs, int coupled) {
  long long off = 0;
  int b, i, dl;
  for (b = 0; b < B; ++b) {
    if (n[b] < 1 || obs[b] < 1) return TMC_ORACLE_BAD_ARG;
    if (parent[off] != -1) return TMC_ORACLE_BAD_ARG;
    for (i = 0; i < n[b]; ++i)
      if (K[off + i] < 1 || d[off + i] < 1) return TMC_ORACLE_BAD_ARG;
    for (i = 1; i < n[b]; ++i)
      if (parent[off + i] < 0 || parent[off + i] >= i) return TMC_ORACLE_BAD_ARG;
    /* a coupled proposal draws sample k of latent i given the parent's sample k */
    if (coupled)
      for (i = 1; i < n[b]; ++i)
        if (K[off + i] > K[off + parent[off + i]]) return TMC_ORACLE_BAD_ARG;
    /* the leaves of an instance share one dimension (one observation matrix C) */
    dl = -1;
    for (i = 0; i < n[b]; ++i) {
      int j, leaf = 1;
      for (j = i + 1; j < n[b]; ++j)
        if (parent[off + j] == i) leaf = 0;
      if (leaf) {
        if (dl < 0) dl = d[off + i];
        else if (dl != d[off + i]) return TMC_ORACLE_BAD_ARG;
      }
    }
    off += n[b];
  }
  return TMC_ORACLE_OK;
}

#define KI(I, i) ((I)->K[i])
#define DI(I, i) ((I)->d[i])
#define DP(I, i) ((i) ? (I)->d[(I)->parent[i]] : (I)->d[0])

/* Proposal mean of z_i^k: m_i, plus A_i (z_p^k - m_p) with a coupled proposal (zp = the
   parent's sample with the same index k; NULL at the root). */
static void q_mean_of(const inst_t* I, int i, const double* zp, double* mq) {
  int r, c, d = DI(I, i), dp = DP(I, i);
  for (r = 0; r < d; ++r) {
    double s = I->m[I->oq[i] + r];
    if (I->A && i > 0 && zp)
      for (c = 0; c < dp; ++c)
        s += I->A[I->ow[i] + (long long)r * dp + c] * (zp[c] - I->m[I->oq[I->parent[i]] + c]);
    mq[r] = s;
  }
}

/* z_i^k = (proposal mean) + exp(logs_i) * eps_i^k (reparameterised sample). */
static void sample(const inst_t* I, int i, int k, const double* zp, double* z) {
  int j, d = DI(I, i);
  const double* e = I->eps + I->oz[i] + (long long)k * d;
  q_mean_of(I, i, zp, z);
  for (j = 0; j < d; ++j) z[j] += exp(I->logs[I->oq[i] + j]) * e[j];
}

/* log N(y; mean, var I) in dimension dim. */
static double log_normal_iso(const double* y, const double* mean, int dim, double var) {
  double s = 0.0;
  int j;
  for (j = 0; j < dim; ++j) {
    double r = y[j] - mean[j];
    s += r * r;
  }
  return -0.5 * s / var - 0.5 * dim * (LOG_2PI + log(var));
}

/* log Q_i(z | zp) for the diagonal Gaussian proposal, evaluated as a density of z (zp: the
   parent's sample the proposal of this sample was conditioned on). */
static double log_q(const inst_t* I, int i, const double* z, const double* zp) {
  double s = 0.0, mq[1024];
  int j;
  q_mean_of(I, i, zp, mq);
  for (j = 0; j < DI(I, i); ++j) {
    double ls = I->logs[I->oq[i] + j];
    double r = (z[j] - mq[j]) * exp(-ls);
    s += -0.5 * r * r - ls - 0.5 * LOG_2PI;
  }
  return s;
}

/* mean of z_i given its parent sample: W_i zp + bias_i (i >= 1), or bias_0 for the root. */
static void cond_mean(const inst_t* I, int i, const double* zp, double* mu) {
  int r, c, d = DI(I, i), dp = DP(I, i);
  for (r = 0; r < d; ++r) {
    double s = I->bias[I->oq[i] + r];
    if (i > 0)
      for (c = 0; c < dp; ++c) s += I->W[I->ow[i] + (long long)r * dp + c] * zp[c];
    mu[r] = s;
  }
}

/* log P(x_l | z) at leaf l. */
static double log_obs(const inst_t* I, int leaf_slot, const double* z, double* pred) {
  int o, c;
  const double* xl = I->x + (long long)leaf_slot * I->obs;
  for (o = 0; o < I->obs; ++o) {
    double s = 0.0;
    for (c = 0; c < I->dl; ++c) s += I->C[(long long)o * I->dl + c] * z[c];
    pred[o] = s;
  }
  return log_normal_iso(xl, pred, I->obs, I->obs_var);
}

static double logsumexp(const double* v, int len) {
  double mx = -INFINITY, s = 0.0;
  int k;
  for (k = 0; k < len; ++k)
    if (v[k] > mx) mx = v[k];
  if (mx == -INFINITY) return -INFINITY;
  for (k = 0; k < len; ++k) s += exp(v[k] - mx);
  return mx + log(s);
}

/* ---------------------------------------------------------------------------------------
 * Per-instance workspace.
 *   z[i][k][:]      samples
 *   mu[i][kp][:]    conditional mean of z_i given parent sample kp (i >= 1)
 *   node[i][k]      log of everything indexed by k_i alone: -log Q_i, plus log P(z_0) at the
 *                   root, plus log P(x_i | z_i) at a leaf
 *   logg[i][k]      node[i][k] + sum over children c of logmsg[c][k]
 *   logmsg[i][kp]   message of node i to its parent: log(1/K_i sum_k f_i^{(k,kp)} * children)
 * ------------------------------------------------------------------------------------- */
typedef struct {
  double *z, *mu, *node, *logg, *logmsg;
  double* pred;
} ws_t;

static int ws_alloc(ws_t* w, const inst_t* I) {
  w->z = (double*)calloc(I->nz, sizeof(double));
  w->mu = (double*)calloc(I->ned > 0 ? I->ned : 1, sizeof(double));
  w->node = (double*)calloc(I->nk, sizeof(double));
  w->logg = (double*)calloc(I->nk, sizeof(double));
  w->logmsg = (double*)calloc(I->ne > 0 ? I->ne : 1, sizeof(double));
  w->pred = (double*)calloc(I->obs, sizeof(double));
  return (w->z && w->mu && w->node && w->logg && w->logmsg && w->pred) ? 0 : -1;
}

static void ws_free(ws_t* w) {
  free(w->z); free(w->mu); free(w->node); free(w->logg); free(w->logmsg); free(w->pred);
}

#define Z(w, I, i, k) ((w)->z + (I)->oz[i] + (long long)(k) * DI(I, i))
#define MU(w, I, i, kp) ((w)->mu + (I)->oed[i] + (long long)(kp) * DI(I, i))
#define LOGG(w, I, i, k) ((w)->logg[(I)->ok[i] + (k)])
#define MSG(w, I, i, kp) ((w)->logmsg[(I)->oe[i] + (kp)])

/* log f_i^{(k, kp)} for i >= 1: log P(z_i^k | z_p^kp) (the -log Q_i part lives in node[]). */
static double log_pair(const ws_t* w, const inst_t* I, int i, int k, int kp) {
  return log_normal_iso(Z(w, I, i, k), MU(w, I, i, kp), DI(I, i), I->prior_var);
}

/* Forward recursion; returns log P_TMC of the instance. */
static double instance_forward(const inst_t* I, ws_t* w) {
  int n = I->n, i, k, kp;
  for (i = 0; i < n; ++i)  /* parents first: a coupled proposal reads the parent's sample k */
    for (k = 0; k < KI(I, i); ++k) sample(I, i, k, i ? Z(w, I, I->parent[i], k) : NULL, Z(w, I, i, k));
  for (i = 1; i < n; ++i) {
    int p = I->parent[i];
    for (kp = 0; kp < KI(I, p); ++kp) cond_mean(I, i, Z(w, I, p, kp), MU(w, I, i, kp));
  }
  for (i = 0; i < n; ++i)
    for (k = 0; k < KI(I, i); ++k) {
      const double* z = Z(w, I, i, k);
      double v = -log_q(I, i, z, i ? Z(w, I, I->parent[i], k) : NULL);
      if (i == 0) v += log_normal_iso(z, I->bias + I->oq[0], DI(I, 0), I->prior_var);
      if (I->leaf_slot[i] >= 0) v += log_obs(I, I->leaf_slot[i], z, w->pred);
      w->node[I->ok[i] + k] = v;
    }
  /* logg starts as node; children (larger index) add their messages before the parent's
     own message is formed because we sweep i from n-1 down to 0. */
  memcpy(w->logg, w->node, sizeof(double) * (size_t)I->nk);
  for (i = n - 1; i >= 1; --i) {
    int p = I->parent[i], Ki = KI(I, i), Kp = KI(I, p);
#pragma omp parallel for if (Kp >= 64) schedule(static)
    for (kp = 0; kp < Kp; ++kp) {
      double* t = (double*)malloc(sizeof(double) * Ki);
      int kk;
      for (kk = 0; kk < Ki; ++kk) t[kk] = log_pair(w, I, i, kk, kp) + LOGG(w, I, i, kk);
      MSG(w, I, i, kp) = logsumexp(t, Ki) - log((double)Ki);
      free(t);
    }
    for (kp = 0; kp < Kp; ++kp) LOGG(w, I, p, kp) += MSG(w, I, i, kp);
  }
  return logsumexp(w->logg + I->ok[0], KI(I, 0)) - log((double)KI(I, 0));
}

/* Fills the instance view of instance b and its per-latent offset tables (allocated here,
   released by inst_free). */
static int make_instance(inst_t* I, int b, const offs_t* o, int shared, const int* n, const int* parent,
                         const int* K, const int* d, const int* obs, double prior_var,
                         double obs_var, const double* eps, const double* q_mean,
                         const double* q_logstd, const double* q_A, const double* W,
                         const double* bias, const double* C, const double* x, int* leaf_slot) {
  int i, nn = n[b];
  long long z = 0, q = 0, wo = 0, kk = 0, e = 0, ed = 0;
  I->n = nn;
  I->obs = obs[b];
  I->parent = parent + o->parent;
  I->K = K + o->parent;
  I->d = d + o->parent;
  I->oz = (long long*)malloc(sizeof(long long) * 6 * (size_t)nn);
  if (!I->oz) return -1;
  I->oq = I->oz + nn; I->ow = I->oq + nn; I->ok = I->ow + nn; I->oe = I->ok + nn; I->oed = I->oe + nn;
  for (i = 0; i < nn; ++i) {
    int Ki = I->K[i], di = I->d[i], dp = i ? I->d[I->parent[i]] : di, Kp = i ? I->K[I->parent[i]] : 0;
    I->oz[i] = z; I->oq[i] = q; I->ow[i] = wo; I->ok[i] = kk; I->oe[i] = e; I->oed[i] = ed;
    z += (long long)Ki * di; q += di; wo += (long long)di * dp; kk += Ki;
    e += Kp; ed += (long long)Kp * di;
  }
  I->nz = z; I->nq = q; I->nw = wo; I->nk = kk; I->ne = e; I->ned = ed;
  I->dl = 1;
  for (i = 0; i < nn; ++i)
    if (leaf_slot[i] >= 0) I->dl = I->d[i];
  I->eps = eps + o->eps;
  I->m = q_mean + o->q;
  I->logs = q_logstd + o->q;
  I->W = W + o->W;
  I->A = q_A ? q_A + o->A : NULL;
  I->bias = shared ? bias : bias + o->q; /* bias shares q_mean's offsets unless shared */
  I->C = C + o->C;
  I->x = x + o->x;
  I->prior_var = prior_var;
  I->obs_var = obs_var;
  I->leaf_slot = leaf_slot;
  return 0;
}

static void inst_free(inst_t* I) { free(I->oz); }

/* Per-instance offsets into the flat arrays: eps [sum K_i d_i], q_mean / q_logstd / bias
   [sum d_i], W [sum d_i d_p], C [obs d_leaf], x [leaves obs]; W / bias / C are not advanced
   when the parameters are shared. */
static void advance(offs_t* o, const inst_t* I, int shared, int nleaves) {
  o->eps += I->nz;
  o->q += I->nq;
  o->x += (long long)nleaves * I->obs;
  o->parent += I->n;
  o->A += I->nw; /* the proposal is per instance even when the model is shared */
  if (!shared) {
    o->W += I->nw;
    o->C += (long long)I->obs * I->dl;
  }
}

int tmc_oracle_log_marginal(int B, const int* n, const int* parent, const int* K, const int* d,
                            const int* obs, int shared, double prior_var, double obs_var,
                            const double* eps, const double* q_mean, const double* q_logstd,
                            const double* q_A, const double* W, const double* bias,
                            const double* C, const double* x, double* log_phat) {
  offs_t o;
  int b, rc = validate(B, n, parent, K, d, obs, q_A != NULL);
  if (rc) return rc;
  memset(&o, 0, sizeof(o));
  for (b = 0; b < B; ++b) {
    inst_t I;
    ws_t w;
    int* slot = (int*)malloc(sizeof(int) * n[b]);
    int nl = count_leaves(n[b], parent + o.parent, slot);
    if (make_instance(&I, b, &o, shared, n, parent, K, d, obs, prior_var, obs_var, eps, q_mean,
                      q_logstd, q_A, W, bias, C, x, slot)) { free(slot); return TMC_ORACLE_NOMEM; }
    if (ws_alloc(&w, &I)) { inst_free(&I); free(slot); return TMC_ORACLE_NOMEM; }
    log_phat[b] = instance_forward(&I, &w);
    ws_free(&w);
    advance(&o, &I, shared, nl);
    inst_free(&I);
    free(slot);
  }
  return TMC_ORACLE_OK;
}

/* ---------------------------------------------------------------------------------------
 * Adjoint.  With L = log P_TMC:
 *   weight of a root sample   w_0[k]   = exp(logg_0[k] - log K_0 - L)
 *   weight of an edge entry   pi_i[kp][k] = w_p[kp] * exp(log f_i^{(k,kp)} + logg_i[k]
 *                                              - log K_i - logmsg_i[kp])
 *   weight of a sample        w_i[k]   = sum_kp pi_i[kp][k]
 * dL/d(log f_i^{(k,kp)}) = pi_i[kp][k]; dL/d(node_i[k]) = w_i[k].
 * G_i^k = sum over the factors of log P(x, z) touching z_i^k of weight * d(log factor)/dz
 * (every other sample held fixed).  Reparameterisation: z_i^k = mq_i^k + s_i eps_i^k with
 * mq_i^k = m_i (+ A_i (z_p^k - m_p) for a coupled proposal) and s_i = exp(logs_i); in terms
 * of eps, -log Q_i = sum_j (eps_j^2/2 + logs_j + log(2 pi)/2).  With eps held fixed, moving
 * z_i^k moves every descendant's sample k through the couplings, so the total derivative is
 *   T_i^k = G_i^k + sum_{children c} A_c^T T_c^k     (T = G for a factorised proposal),
 * and
 *   d/d eps_i^k = s_i T_i^k + w_i[k] eps_i^k,   reported as dz = that / s_i
 *                 (= G + w (z - m)/s^2 for a factorised proposal: the gradient w.r.t. z with
 *                 Q evaluated as a density of z),
 *   dm_i    = sum_k G_i^k          (m_i moves z_i, and the children's samples not at all),
 *   dlogs_i = sum_k w_i[k] + sum_k T_i^k s_i eps_i^k,
 *   dA_i    = sum_k T_i^k (z_p^k - m_p)^T.
 * ------------------------------------------------------------------------------------- */
static void instance_backward(const inst_t* I, ws_t* w, double L, double go, double* dz,
                              double* dm, double* dlogs, double* dA, double* dW, double* dbias,
                              double* dC) {
  int n = I->n, i, k, kp, j, c;
  const int dl = I->dl;
  double var = I->prior_var;
  double* wt = (double*)calloc((size_t)I->nk, sizeof(double));
  double* dzl = (double*)calloc((size_t)I->nz, sizeof(double));
  double* pred = (double*)calloc(I->obs, sizeof(double));
  const int K0 = KI(I, 0);
  for (k = 0; k < K0; ++k) wt[I->ok[0] + k] = exp(LOGG(w, I, 0, k) - log((double)K0) - L);
  for (i = 1; i < n; ++i) {
    int p = I->parent[i], Ki = KI(I, i), Kp = KI(I, p), d = DI(I, i), dp = DI(I, p);
    double* dmu = (double*)calloc((size_t)Kp * d, sizeof(double));
    /* rows kp: parent sample; columns k: child sample */
#pragma omp parallel for if (Kp >= 64) schedule(static) private(k, j)
    for (kp = 0; kp < Kp; ++kp) {
      const double* mu = MU(w, I, i, kp);
      for (k = 0; k < Ki; ++k) {
        const double* z = Z(w, I, i, k);
        double pi = wt[I->ok[p] + kp] *
                    exp(log_pair(w, I, i, k, kp) + LOGG(w, I, i, k) - log((double)Ki) - MSG(w, I, i, kp));
        for (j = 0; j < d; ++j) dmu[(long long)kp * d + j] += pi * (z[j] - mu[j]) / var;
      }
    }
    /* column direction: weights and sample gradients of the child */
#pragma omp parallel for if (Ki >= 64) schedule(static) private(kp, j)
    for (k = 0; k < Ki; ++k) {
      const double* z = Z(w, I, i, k);
      double acc_w = 0.0;
      for (kp = 0; kp < Kp; ++kp) {
        const double* mu = MU(w, I, i, kp);
        double pi = wt[I->ok[p] + kp] *
                    exp(log_pair(w, I, i, k, kp) + LOGG(w, I, i, k) - log((double)Ki) - MSG(w, I, i, kp));
        acc_w += pi;
        for (j = 0; j < d; ++j) dzl[I->oz[i] + (long long)k * d + j] += pi * (mu[j] - z[j]) / var;
      }
      wt[I->ok[i] + k] = acc_w;
    }
    /* mu_i^kp = W_i z_p^kp + bias_i */
    for (kp = 0; kp < Kp; ++kp) {
      const double* zp = Z(w, I, p, kp);
      for (j = 0; j < d; ++j) {
        double g = dmu[(long long)kp * d + j];
        dbias[I->oq[i] + j] += go * g;
        for (c = 0; c < dp; ++c) {
          dW[I->ow[i] + (long long)j * dp + c] += go * g * zp[c];
          dzl[I->oz[p] + (long long)kp * dp + c] += I->W[I->ow[i] + (long long)j * dp + c] * g;
        }
      }
    }
    free(dmu);
  }
  /* node terms */
  for (i = 0; i < n; ++i) {
    int d = DI(I, i);
    for (k = 0; k < KI(I, i); ++k) {
      const double* z = Z(w, I, i, k);
      double wk = wt[I->ok[i] + k];
      double* g = dzl + I->oz[i] + (long long)k * d;
      if (i == 0)
        for (j = 0; j < d; ++j) {
          double r = (z[j] - I->bias[I->oq[0] + j]) / var;
          g[j] -= wk * r;
          dbias[I->oq[0] + j] += go * wk * r;
        }
      if (I->leaf_slot[i] >= 0) {
        const double* xl = I->x + (long long)I->leaf_slot[i] * I->obs;
        int o;
        for (o = 0; o < I->obs; ++o) {
          double s = 0.0;
          for (c = 0; c < dl; ++c) s += I->C[(long long)o * dl + c] * z[c];
          pred[o] = (xl[o] - s) / I->obs_var; /* residual / obs_var */
        }
        for (o = 0; o < I->obs; ++o)
          for (c = 0; c < dl; ++c) {
            g[c] += wk * I->C[(long long)o * dl + c] * pred[o];
            dC[(long long)o * dl + c] += go * wk * pred[o] * z[c];
          }
      }
    }
  }
  /* T = G, then the couplings, children before parents (a child's index is the larger) */
  {
    double* T = (double*)malloc(sizeof(double) * (size_t)I->nz);
    memcpy(T, dzl, sizeof(double) * (size_t)I->nz);
    if (I->A)
      for (i = n - 1; i >= 1; --i) {
        int p = I->parent[i], d = DI(I, i), dp = DI(I, p);
        for (k = 0; k < KI(I, i); ++k)
          for (c = 0; c < dp; ++c) {
            double s = 0.0;
            for (j = 0; j < d; ++j)
              s += I->A[I->ow[i] + (long long)j * dp + c] * T[I->oz[i] + (long long)k * d + j];
            T[I->oz[p] + (long long)k * dp + c] += s;
          }
      }
    /* outputs */
    for (i = 0; i < n; ++i) {
      int d = DI(I, i);
      double wsum = 0.0;
      for (k = 0; k < KI(I, i); ++k) wsum += wt[I->ok[i] + k];
      for (j = 0; j < d; ++j) {
        double s = exp(I->logs[I->oq[i] + j]), am = 0.0, al = 0.0;
        for (k = 0; k < KI(I, i); ++k) {
          const long long e = I->oz[i] + (long long)k * d + j;
          const double ep = I->eps[e];
          am += dzl[e];
          al += T[e] * s * ep;
          if (dz) dz[e] += go * (T[e] + wt[I->ok[i] + k] * ep / s);
        }
        dm[I->oq[i] + j] += go * am;
        dlogs[I->oq[i] + j] += go * (wsum + al);
      }
      if (I->A && dA && i > 0) {
        int p = I->parent[i], dp = DI(I, p);
        for (j = 0; j < d; ++j)
          for (c = 0; c < dp; ++c) {
            double s = 0.0;
            for (k = 0; k < KI(I, i); ++k)
              s += T[I->oz[i] + (long long)k * d + j] *
                   (Z(w, I, p, k)[c] - I->m[I->oq[p] + c]);
            dA[I->ow[i] + (long long)j * dp + c] += go * s;
          }
      }
    }
    free(T);
  }
  free(wt); free(dzl); free(pred);
}

int tmc_oracle_grad(int B, const int* n, const int* parent, const int* K, const int* d,
                    const int* obs, int shared, double prior_var, double obs_var,
                    const double* eps, const double* q_mean, const double* q_logstd,
                    const double* q_A, const double* W, const double* bias, const double* C,
                    const double* x, const double* grad_out, double* log_phat, double* dz,
                    double* dq_mean, double* dq_logstd, double* dq_A, double* dW, double* dbias,
                    double* dC) {
  offs_t o;
  int b, rc = validate(B, n, parent, K, d, obs, q_A != NULL);
  if (rc) return rc;
  memset(&o, 0, sizeof(o));
  for (b = 0; b < B; ++b) {
    inst_t I;
    ws_t w;
    double L;
    int* slot = (int*)malloc(sizeof(int) * n[b]);
    int nl = count_leaves(n[b], parent + o.parent, slot);
    if (make_instance(&I, b, &o, shared, n, parent, K, d, obs, prior_var, obs_var, eps, q_mean,
                      q_logstd, q_A, W, bias, C, x, slot)) { free(slot); return TMC_ORACLE_NOMEM; }
    if (ws_alloc(&w, &I)) { inst_free(&I); free(slot); return TMC_ORACLE_NOMEM; }
    L = instance_forward(&I, &w);
    if (log_phat) log_phat[b] = L;
    /* the bias gradient lives where bias does: dbias + 0 (shared) or dbias + o.q */
    instance_backward(&I, &w, L, grad_out ? grad_out[b] : 1.0, dz ? dz + o.eps : NULL,
                      dq_mean + o.q, dq_logstd + o.q, dq_A ? dq_A + o.A : NULL, dW + o.W,
                      shared ? dbias : dbias + o.q, dC + o.C);
    ws_free(&w);
    advance(&o, &I, shared, nl);
    inst_free(&I);
    free(slot);
  }
  return TMC_ORACLE_OK;
}

/* ---------------------------------------------------------------------------------------
 * Brute force: enumerate every combination (k_0..k_{n-1}) and evaluate the importance
 * ratio of Eq. (is) from the joint density directly.
 * ------------------------------------------------------------------------------------- */
int tmc_oracle_brute_force(int B, const int* n, const int* parent, const int* K, const int* d,
                           const int* obs, int shared, double prior_var, double obs_var,
                           const double* eps, const double* q_mean, const double* q_logstd,
                           const double* q_A, const double* W, const double* bias,
                           const double* C, const double* x, long long max_combos,
                           double* log_phat) {
  offs_t o;
  int b, rc = validate(B, n, parent, K, d, obs, q_A != NULL);
  if (rc) return rc;
  memset(&o, 0, sizeof(o));
  for (b = 0; b < B; ++b) {
    inst_t I;
    int* slot = (int*)malloc(sizeof(int) * n[b]);
    int nl = count_leaves(n[b], parent + o.parent, slot);
    long long combos = 1, t;
    int i;
    double lognorm = 0.0;
    if (make_instance(&I, b, &o, shared, n, parent, K, d, obs, prior_var, obs_var, eps, q_mean,
                      q_logstd, q_A, W, bias, C, x, slot)) { free(slot); return TMC_ORACLE_NOMEM; }
    for (i = 0; i < I.n; ++i) {
      combos *= KI(&I, i);
      lognorm += log((double)KI(&I, i));
      if (combos > max_combos) { inst_free(&I); free(slot); return TMC_ORACLE_TOO_BIG; }
    }
    {
      double* lw = (double*)malloc(sizeof(double) * combos);
      double* all = (double*)malloc(sizeof(double) * (size_t)I.nz); /* every sample, [i][k][:] */
      double* mu = (double*)malloc(sizeof(double) * (size_t)I.nq);
      double* pred = (double*)malloc(sizeof(double) * I.obs);
      int* kk = (int*)malloc(sizeof(int) * I.n);
      int k;
      /* the samples, parents first (a coupled proposal reads the parent's sample k) */
      for (i = 0; i < I.n; ++i)
        for (k = 0; k < KI(&I, i); ++k)
          sample(&I, i, k, i ? all + I.oz[I.parent[i]] + (long long)k * DI(&I, I.parent[i]) : NULL,
                 all + I.oz[i] + (long long)k * DI(&I, i));
#define ZB(i, k) (all + I.oz[i] + (long long)(k) * DI(&I, i))
      for (t = 0; t < combos; ++t) {
        long long r = t;
        double v = 0.0;
        for (i = 0; i < I.n; ++i) { kk[i] = (int)(r % KI(&I, i)); r /= KI(&I, i); }
        /* log P(x, z) of the combination: root prior, conditionals, observations; then the
           proposal densities, sample k_i of latent i given its parent's sample k_i */
        for (i = 0; i < I.n; ++i) {
          int j;
          const double* zi = ZB(i, kk[i]);
          if (i == 0) {
            for (j = 0; j < DI(&I, 0); ++j) mu[j] = I.bias[I.oq[0] + j];
          } else {
            cond_mean(&I, i, ZB(I.parent[i], kk[I.parent[i]]), mu);
          }
          v += log_normal_iso(zi, mu, DI(&I, i), I.prior_var);
          if (slot[i] >= 0) v += log_obs(&I, slot[i], zi, pred);
          v -= log_q(&I, i, zi, i ? ZB(I.parent[i], kk[i]) : NULL);
        }
        lw[t] = v;
      }
#undef ZB
      log_phat[b] = logsumexp(lw, (int)combos) - lognorm;
      free(lw); free(all); free(mu); free(pred); free(kk);
    }
    advance(&o, &I, shared, nl);
    inst_free(&I);
    free(slot);
  }
  return TMC_ORACLE_OK;
}
