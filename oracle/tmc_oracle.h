/*
 * tmc_oracle.h -- FP64 CPU oracle for the Tensor Monte Carlo estimator.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU baseline may
 * call these functions.  Nothing here is shared with the CUDA path.
 *
 * Batch layout (instance b follows instance b-1 in every flat array, latent i after latent
 * i-1 within it; all arrays are host memory owned by the caller):
 *   n[B], obs[B]                      latents and observation dimension of each instance
 *   K[sum n], d[sum n]                samples K_i and dimension d_i of every latent
 *   parent[sum n]                     local indices; parent[0] = -1, 0 <= parent[i] < i
 *   eps[sum K_i*d_i]     [i][k][j]    proposal noise
 *   q_mean, q_logstd [sum d_i]        proposal mean / log std, [i][j]
 *   W     [sum d_i*d_p]  [i][r][c]    W_i is d_i x d_p (p = parent[i]); the root's block is
 *                                     d_0 x d_0 and unused
 *   bias  [sum d_i]                   bias_0 is the root prior mean
 *   C     [obs*d_leaf] per instance   [o][c]; the leaves of an instance share one dimension
 *   x     [sum leaves*obs]            one observation per leaf, leaves in node order
 * (W, bias and C of one instance only when shared.)  With shared != 0 every instance uses the
 * same W/bias/C (and must have the same n, parent, d_i, obs); their gradients are summed over
 * instances.
 *
 *   q_A   [sum d_i*d_p] per instance, or NULL   proposal couplings (layout of W, root block
 *                                     unused): Q_i(z_i^k | parent samples) =
 *                                     N(m_i + A_i (z_p^k - m_p), diag(exp(2 logs_i))); needs
 *                                     K_i <= K_parent.  NULL: the factorised Q_i = N(m_i, .)
 *
 * Gradient outputs have the layout of the matching input and are ACCUMULATED (+=), each
 * instance's contribution multiplied by grad_out[b] (grad_out may be NULL: all ones).
 * dz (= the gradient w.r.t. eps divided by exp(logs)) and dq_A may be NULL.  Return value:
 * TMC_ORACLE_* status.
 */
#ifndef TMC_ORACLE_H
#define TMC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { TMC_ORACLE_OK = 0, TMC_ORACLE_BAD_ARG = 1, TMC_ORACLE_NOMEM = 2, TMC_ORACLE_TOO_BIG = 3 };

/* log P_TMC per instance by summing out one index at a time (Section 2.2, Appendix). */
int tmc_oracle_log_marginal(int B, const int* n, const int* parent, const int* K, const int* d,
                            const int* obs, int shared, double prior_var, double obs_var,
                            const double* eps, const double* q_mean, const double* q_logstd,
                            const double* q_A, const double* W, const double* bias,
                            const double* C, const double* x, double* log_phat);

/* Analytic gradient of sum_b grad_out[b] * log P_TMC_b (reparameterisation gradients). */
int tmc_oracle_grad(int B, const int* n, const int* parent, const int* K, const int* d,
                    const int* obs, int shared, double prior_var, double obs_var,
                    const double* eps, const double* q_mean, const double* q_logstd,
                    const double* q_A, const double* W, const double* bias, const double* C,
                    const double* x, const double* grad_out, double* log_phat, double* dz,
                    double* dq_mean, double* dq_logstd, double* dq_A, double* dW, double* dbias,
                    double* dC);

/* Eq. (is) enumerated over all prod K_i combinations; TMC_ORACLE_TOO_BIG above max_combos. */
int tmc_oracle_brute_force(int B, const int* n, const int* parent, const int* K, const int* d,
                           const int* obs, int shared, double prior_var, double obs_var,
                           const double* eps, const double* q_mean, const double* q_logstd,
                           const double* q_A, const double* W, const double* bias,
                           const double* C, const double* x, long long max_combos,
                           double* log_phat);

/* The loopy graph of Fig. 1 (z1 -> z2, z1 -> z3, {z2, z3} -> z4 -> x), K samples of every
 * latent, all of dimension d; see tmc_oracle_loopy.c for the model and layouts.  log P_TMC by
 * summing out k4 and k1 (two matrix messages over (k2, k3)), or by enumerating all K^4
 * combinations (TMC_ORACLE_TOO_BIG above max_combos). */
int tmc_oracle_diamond_log_marginal(int B, int K, int d, int obs, int shared, double prior_var,
                                    double obs_var, const double* eps, const double* q_mean,
                                    const double* q_logstd, const double* W, const double* bias,
                                    const double* C, const double* x, double* log_phat);
int tmc_oracle_diamond_brute_force(int B, int K, int d, int obs, int shared, double prior_var,
                                   double obs_var, const double* eps, const double* q_mean,
                                   const double* q_logstd, const double* W, const double* bias,
                                   const double* C, const double* x, long long max_combos,
                                   double* log_phat);

#ifdef __cplusplus
}
#endif
#endif
