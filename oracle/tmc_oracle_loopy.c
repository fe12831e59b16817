/*
 * tmc_oracle_loopy.c -- FP64 CPU oracle for TMC on the loopy graph of Fig. 1
 * (Section 2.2 "Efficient averaging": a latent with two parents closes a loop, and summing out
 * one index produces a factor over two remaining indices -- a matrix message).
 *
 * TEST INFRASTRUCTURE (only the tests and the benchmark's CPU leg may load it); no code is
 * shared with the CUDA path.
 *
 * Model (one instance; node 0 = z1, 1 = z2, 2 = z3, 3 = z4, all of dimension d):
 *   z1 ~ N(bias_0, prior_var I)
 *   z2 | z1 ~ N(W_1 z1 + bias_1, prior_var I),   z3 | z1 ~ N(W_2 z1 + bias_2, prior_var I)
 *   z4 | z2, z3 ~ N(W_3 z2 + W_4 z3 + bias_3, prior_var I)
 *   x | z4 ~ N(C z4, obs_var I)
 * Proposal: Q_i = N(m_i, diag(exp(2 logs_i))), K samples of every latent.
 *
 * Eq. (is) with the factors of the Appendix: f1 = P(z1)/Q1, f2 = P(z2|z1)/Q2, f3 = P(z3|z1)/Q3,
 * f4 = P(z4|z2,z3) P(x|z4)/Q4.  Summing out k4 and then k1 (Fig. 1 C, D) leaves two factors
 * over (k2, k3):
 *   M4[k2][k3] = log (1/K) sum_k4 f4(k2, k3, k4)
 *   M1[k2][k3] = log (1/K) sum_k1 f1(k1) f2(k1, k2) f3(k1, k3)
 *   log P_TMC  = log (1/K^2) sum_{k2,k3} exp(M4 + M1)
 * Every log-sum-exp subtracts the maximum of the whole exponent it sums (the combined maximum),
 * and every factor is evaluated from its Gaussian density directly (no expansion).
 *
 * Flat layouts (instance b after instance b-1; shared parameters: one instance's):
 *   eps [B][4][K][d], q_mean / q_logstd [B][4][d], W [5][d][d] (W_0 unused), bias [4][d],
 *   C [obs][d], x [B][obs].
 */
#include "tmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LOG_2PI 1.8378770664093454835606594728112

static double lnorm(const double* y, const double* mean, int dim, double var) {
  double s = 0.0;
  int j;
  for (j = 0; j < dim; ++j) {
    double r = y[j] - mean[j];
    s += r * r;
  }
  return -0.5 * s / var - 0.5 * dim * (LOG_2PI + log(var));
}

static double lse(const double* v, long long n) {
  double mx = -INFINITY, s = 0.0;
  long long i;
  for (i = 0; i < n; ++i)
    if (v[i] > mx) mx = v[i];
  if (mx == -INFINITY) return -INFINITY;
  for (i = 0; i < n; ++i) s += exp(v[i] - mx);
  return mx + log(s);
}

typedef struct {
  int K, d, obs;
  double pv, ov;
  const double *eps, *m, *ls, *W, *bias, *C, *x;
  double* z;    /* [4][K][d] samples */
  double* u;    /* [4][K] -log Q_i (+ log P(z1) at node 0, + log P(x | z4) at node 3) */
} dia_t;

#define DZ(I, i, k) ((I)->z + ((long long)(i) * (I)->K + (k)) * (I)->d)
#define DW(I, w) ((I)->W + (long long)(w) * (I)->d * (I)->d)

/* W_w a (+ W_v c if v > 0) + bias_i */
static void affine(const dia_t* I, int w, const double* a, int v, const double* c, int i, double* out) {
  int r, j, d = I->d;
  for (r = 0; r < d; ++r) {
    double s = I->bias[i * d + r];
    for (j = 0; j < d; ++j) s += DW(I, w)[r * d + j] * a[j];
    if (v > 0)
      for (j = 0; j < d; ++j) s += DW(I, v)[r * d + j] * c[j];
    out[r] = s;
  }
}

static void dia_prepare(dia_t* I) {
  int i, k, j, o, K = I->K, d = I->d;
  double* pred = (double*)malloc(sizeof(double) * I->obs);
  for (i = 0; i < 4; ++i)
    for (k = 0; k < K; ++k) {
      double* z = DZ(I, i, k);
      const double* e = I->eps + ((long long)i * K + k) * d;
      double lq = 0.0;
      for (j = 0; j < d; ++j) {
        double s = exp(I->ls[i * d + j]);
        z[j] = I->m[i * d + j] + s * e[j];
        lq += -0.5 * e[j] * e[j] - I->ls[i * d + j] - 0.5 * LOG_2PI;
      }
      I->u[i * K + k] = -lq;
      if (i == 0) I->u[k] += lnorm(z, I->bias, d, I->pv);
      if (i == 3) {
        for (o = 0; o < I->obs; ++o) {
          double s = 0.0;
          for (j = 0; j < d; ++j) s += I->C[(long long)o * d + j] * z[j];
          pred[o] = s;
        }
        I->u[3 * K + k] += lnorm(I->x, pred, I->obs, I->ov);
      }
    }
  free(pred);
}

static double dia_eliminate(const dia_t* I) {
  const int K = I->K, d = I->d;
  double* M = (double*)malloc(sizeof(double) * (size_t)K * K);
  /* the conditional means of z2 and z3 given z1^k1 depend on k1 alone: computed once */
  double* mu2 = (double*)malloc(sizeof(double) * (size_t)K * d);
  double* mu3 = (double*)malloc(sizeof(double) * (size_t)K * d);
  int k2, k;
  for (k = 0; k < K; ++k) {
    affine(I, 1, DZ(I, 0, k), 0, NULL, 1, mu2 + (long long)k * d);
    affine(I, 2, DZ(I, 0, k), 0, NULL, 2, mu3 + (long long)k * d);
  }
#pragma omp parallel for schedule(static)
  for (k2 = 0; k2 < K; ++k2) {
    double* t = (double*)malloc(sizeof(double) * K);
    double* mu = (double*)malloc(sizeof(double) * d);
    int k3, k1, k4;
    for (k3 = 0; k3 < K; ++k3) {
      double m4, m1;
      affine(I, 3, DZ(I, 1, k2), 4, DZ(I, 2, k3), 3, mu); /* mean of z4 | z2^k2, z3^k3 */
      for (k4 = 0; k4 < K; ++k4) t[k4] = I->u[3 * K + k4] + lnorm(DZ(I, 3, k4), mu, d, I->pv);
      m4 = lse(t, K) - log((double)K);
      for (k1 = 0; k1 < K; ++k1) {
        double v = I->u[k1];
        v += lnorm(DZ(I, 1, k2), mu2 + (long long)k1 * d, d, I->pv);
        v += lnorm(DZ(I, 2, k3), mu3 + (long long)k1 * d, d, I->pv);
        t[k1] = v;
      }
      m1 = lse(t, K) - log((double)K);
      M[(long long)k2 * K + k3] = I->u[K + k2] + I->u[2 * K + k3] + m4 + m1;
    }
    free(t);
    free(mu);
  }
  {
    double r = lse(M, (long long)K * K) - 2.0 * log((double)K);
    free(M);
    free(mu2);
    free(mu3);
    return r;
  }
}

static double dia_brute(const dia_t* I) {
  const int K = I->K, d = I->d;
  const long long n = (long long)K * K * K * K;
  double* lw = (double*)malloc(sizeof(double) * n);
  double* mu = (double*)malloc(sizeof(double) * d);
  long long t;
  for (t = 0; t < n; ++t) {
    int k1 = (int)(t % K), k2 = (int)((t / K) % K), k3 = (int)((t / K / K) % K), k4 = (int)(t / K / K / K);
    double v = I->u[k1] + I->u[K + k2] + I->u[2 * K + k3] + I->u[3 * K + k4];
    affine(I, 1, DZ(I, 0, k1), 0, NULL, 1, mu);
    v += lnorm(DZ(I, 1, k2), mu, d, I->pv);
    affine(I, 2, DZ(I, 0, k1), 0, NULL, 2, mu);
    v += lnorm(DZ(I, 2, k3), mu, d, I->pv);
    affine(I, 3, DZ(I, 1, k2), 4, DZ(I, 2, k3), 3, mu);
    v += lnorm(DZ(I, 3, k4), mu, d, I->pv);
    lw[t] = v;
  }
  {
    double r = lse(lw, n) - 4.0 * log((double)K);
    free(lw);
    free(mu);
    return r;
  }
}

static int dia_run(int brute, int B, int K, int d, int obs, int shared, double prior_var,
                   double obs_var, const double* eps, const double* q_mean, const double* q_logstd,
                   const double* W, const double* bias, const double* C, const double* x,
                   long long max_combos, double* log_phat) {
  int b;
  if (B < 1 || K < 1 || d < 1 || obs < 1 || !(prior_var > 0.0) || !(obs_var > 0.0)) return TMC_ORACLE_BAD_ARG;
  if (brute && (double)K * K * K * K > (double)max_combos) return TMC_ORACLE_TOO_BIG;
  for (b = 0; b < B; ++b) {
    dia_t I;
    I.K = K; I.d = d; I.obs = obs; I.pv = prior_var; I.ov = obs_var;
    I.eps = eps + (long long)b * 4 * K * d;
    I.m = q_mean + (long long)b * 4 * d;
    I.ls = q_logstd + (long long)b * 4 * d;
    I.W = W + (shared ? 0 : (long long)b * 5 * d * d);
    I.bias = bias + (shared ? 0 : (long long)b * 4 * d);
    I.C = C + (shared ? 0 : (long long)b * obs * d);
    I.x = x + (long long)b * obs;
    I.z = (double*)malloc(sizeof(double) * 4 * (size_t)K * d);
    I.u = (double*)malloc(sizeof(double) * 4 * (size_t)K);
    if (!I.z || !I.u) { free(I.z); free(I.u); return TMC_ORACLE_NOMEM; }
    dia_prepare(&I);
    log_phat[b] = brute ? dia_brute(&I) : dia_eliminate(&I);
    free(I.z);
    free(I.u);
  }
  return TMC_ORACLE_OK;
}

int tmc_oracle_diamond_log_marginal(int B, int K, int d, int obs, int shared, double prior_var,
                                    double obs_var, const double* eps, const double* q_mean,
                                    const double* q_logstd, const double* W, const double* bias,
                                    const double* C, const double* x, double* log_phat) {
  return dia_run(0, B, K, d, obs, shared, prior_var, obs_var, eps, q_mean, q_logstd, W, bias, C, x,
                 0, log_phat);
}

int tmc_oracle_diamond_brute_force(int B, int K, int d, int obs, int shared, double prior_var,
                                   double obs_var, const double* eps, const double* q_mean,
                                   const double* q_logstd, const double* W, const double* bias,
                                   const double* C, const double* x, long long max_combos,
                                   double* log_phat) {
  return dia_run(1, B, K, d, obs, shared, prior_var, obs_var, eps, q_mean, q_logstd, W, bias, C, x,
                 max_combos, log_phat);
}
