/*
 * qem_oracle.c -- plain FP64 CPU oracle for the QEM E-step and M-step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * What it computes (arXiv 2503.08264):
 *  - K samples per latent from a factorised proposal Q (Sec. 3.2, App. A.2);
 *  - the massively parallel importance weights r_k, the marginal-likelihood
 *    estimate P_MP and the moment estimate m_MP of Eq. (mp_iw), i.e.
 *      P_MP = K^-n sum_k r_k,   r_k = P(x, z^k) / prod_i Q(z_i^{k_i}),
 *      w_i[k] = K^-n sum_{k : k_i = k} r_k / P_MP   (marginal weight of sample k of latent i),
 *      m_i = sum_k w_i[k] T(z_i^k)                   (Eq. mp_iw, m(z) = T(z_i));
 *    evaluated by the distributive law over the plate tree (Sec. 6: sum the
 *    child indices out one latent at a time, leaves first), every step in
 *    FP64 with no blocking, fusion or reordering of the sums;
 *  - the moment-matching M-step (Sec. 4, App. B) for Gaussian, Gamma and
 *    Beta proposals and the EMA of the mean parameters (Eq. ema, Alg. 1).
 *
 * The tree recursion is pinned in the tests against a literal enumeration of
 * all K^n index vectors (a separate Python program) and against closed forms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { PRIOR_STD_NORMAL = 0, PRIOR_NORMAL_FIXED_VAR = 1, PRIOR_NORMAL_MEAN_LOGVAR = 2,
       PRIOR_GAMMA = 3, PRIOR_BETA = 4 };
enum { LIK_NONE = 0, LIK_GAUSS = 1, LIK_BERNOULLI_LOGIT = 2, LIK_POISSON_LOG = 3,
       LIK_POISSON_RATE = 4, LIK_BERNOULLI_PROB = 5 };
enum { Q_GAUSS = 0, Q_GAMMA = 1, Q_BETA = 2 };
#define GAMMA_TRIES 8

static const double LOG_2PI = 1.8378770664093454835606594728112;
static const double TWO_PI = 6.283185307179586476925286766559;

typedef struct {
  int64_t n;            /* plate elements at this level */
  int dim;              /* latent dimension D */
  int prior;            /* PRIOR_* */
  double prior_a, prior_b;
  int lik;              /* LIK_* */
  double lik_var;
  int n_obs;
  int qfam;             /* Q_* */
  const int64_t* parent;/* [n] parent element index at level-1 (NULL at level 0) */
  const double* x;      /* [n][n_obs][dim] covariates */
  const double* y;      /* [n][n_obs] observations */
  const double* q;      /* [n][2][dim] proposal parameters */
  const double* eps;    /* [n][K][nps] supplied noise, or NULL: counter-based draws */
  double* z;            /* out [n][K][dim] samples */
  double* w;            /* out [n][K] marginal weights */
  double* mom;          /* out [n][2][dim] E_w[T(z)] */
  double* logL;         /* out [n][K] (levels>0): log mean_k exp S_e[kp][k] per parent sample kp */
  const double* H_extra;/* [n][K] (level 0, or NULL): plate sums of root children that this call does
                           not hold (another shard's), added to the root's children sum */
} orc_level;

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the paper's
 * definition: 10 rounds of two 32x32->64 multiplies with the round constants
 * M0 = 0xD2511F53, M1 = 0xCD9E8D57 and Weyl key increments 0x9E3779B9,
 * 0xBB67AE85.                                                               */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of the noise stream (shared definition with the CUDA side,
 * implemented independently there): key = (seed lo, seed hi); counter =
 * (sample lo, sample hi, level<<24 | block, iteration), sample = e*K + k,
 * block = noise index / 4.  Uniform u = (x + 0.5) 2^-32.  Normal slots use
 * Box-Muller on (u0,u1) and (u2,u3); uniform slots take u directly. */
static int noise_slot_is_uniform(int qfam, int idx) {
  if (qfam == Q_GAUSS) return 0;
  int blk = 2 * GAMMA_TRIES + 1;
  int r = idx % blk;
  return (r == blk - 1) || (r & 1);
}

static double draw_noise(uint64_t seed, uint64_t iter, int level, uint64_t sample, int idx, int qfam) {
  uint32_t ctr[4] = {(uint32_t)sample, (uint32_t)(sample >> 32),
                     ((uint32_t)level << 24) | (uint32_t)(idx / 4), (uint32_t)iter};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t x[4];
  orc_philox4x32_10(ctr, key, x);
  double u[4];
  for (int i = 0; i < 4; ++i) u[i] = ((double)x[i] + 0.5) * (1.0 / 4294967296.0);
  int j = idx % 4;
  if (noise_slot_is_uniform(qfam, idx)) return u[j];
  double ua = u[j & 2], ub = u[(j & 2) + 1];
  double r = sqrt(-2.0 * log(ua));
  return (j & 1) ? r * sin(TWO_PI * ub) : r * cos(TWO_PI * ub);
}

void orc_draw_noise(uint64_t seed, uint64_t iter, int level, int64_t n, int K, int nps, int qfam,
                    double* out) {
  for (int64_t e = 0; e < n; ++e)
    for (int k = 0; k < K; ++k)
      for (int d = 0; d < nps; ++d)
        out[(e * K + k) * nps + d] = draw_noise(seed, iter, level, (uint64_t)e * K + k, d, qfam);
}

/* The same stream for selected elements only: idx[i] is the element's index
 * within its level (the counter uses it, so a sub-model drawn this way gets
 * the noise its elements have in the full model). */
void orc_draw_noise_at(uint64_t seed, uint64_t iter, int level, const int64_t* idx, int64_t n, int K, int nps,
                       int qfam, double* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int k = 0; k < K; ++k)
      for (int d = 0; d < nps; ++d)
        out[(i * K + k) * nps + d] = draw_noise(seed, iter, level, (uint64_t)idx[i] * K + k, d, qfam);
}

/* ------------------------------------------------------------------------- */
/* Special functions, from their series (no vendor code).                    */
/* digamma: psi(x+1) = psi(x) + 1/x to shift x >= 10, then the asymptotic
 * series  ln x - 1/(2x) - sum_n B_2n / (2n x^2n)  (Bernoulli numbers).      */
double orc_digamma(double x) {
  if (!(x > 0.0) || !isfinite(x)) return NAN;  /* defined here for finite x > 0 only */
  double acc = 0.0;
  while (x < 10.0) { acc -= 1.0 / x; x += 1.0; }
  double f = 1.0 / (x * x);
  double t = f * (-1.0 / 12 + f * (1.0 / 120 + f * (-1.0 / 252 + f * (1.0 / 240 + f * (-1.0 / 132 + f * (691.0 / 32760 + f * (-1.0 / 12)))))));
  return acc + log(x) - 0.5 / x + t;
}

/* trigamma: psi'(x) = psi'(x+1) + 1/x^2, then
 *  1/x + 1/(2x^2) + sum_n B_2n / x^(2n+1).                                   */
double orc_trigamma(double x) {
  if (!(x > 0.0) || !isfinite(x)) return NAN;
  double acc = 0.0;
  while (x < 10.0) { acc += 1.0 / (x * x); x += 1.0; }
  double f = 1.0 / (x * x);
  double t = 1.0 / x + f / 2.0 + (f / x) * (1.0 / 6 + f * (-1.0 / 30 + f * (1.0 / 42 + f * (-1.0 / 30 + f * (5.0 / 66 + f * (-691.0 / 2730 + f * (7.0 / 6)))))));
  return acc + t;
}

/* ------------------------------------------------------------------------- */
/* Sampling from the proposal (Alg. 1 "z ~ Q_t").                            */

/* Gamma(shape a, rate 1) by Marsaglia & Tsang (2000) from supplied noise
 * (GAMMA_TRIES normal/uniform pairs, then one uniform for a < 1).           */
static double gamma_from_noise(double a, const double* nz) {
  double ab = a < 1.0 ? a + 1.0 : a;
  double d = ab - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double g = d;  /* deterministic fallback if every attempt is rejected */
  for (int t = 0; t < GAMMA_TRIES; ++t) {
    double xn = nz[2 * t], u = nz[2 * t + 1];
    double v = 1.0 + c * xn;
    if (v <= 0.0) continue;
    v = v * v * v;
    if (log(u) < 0.5 * xn * xn + d - d * v + d * log(v)) { g = d * v; break; }
  }
  if (a < 1.0) g *= pow(nz[2 * GAMMA_TRIES], 1.0 / a);
  return g;
}

static void sample_one(const orc_level* L, int64_t e, const double* nz, double* z) {
  const double* q = L->q + e * 2 * L->dim;
  const int blk = 2 * GAMMA_TRIES + 1;
  for (int d = 0; d < L->dim; ++d) {
    if (L->qfam == Q_GAUSS) {
      z[d] = q[d] + q[L->dim + d] * nz[d];
    } else if (L->qfam == Q_GAMMA) {
      z[d] = gamma_from_noise(q[d], nz + d * blk) / q[L->dim + d];
    } else {
      double g1 = gamma_from_noise(q[d], nz + (2 * d) * blk);
      double g2 = gamma_from_noise(q[L->dim + d], nz + (2 * d + 1) * blk);
      z[d] = g1 / (g1 + g2);
    }
  }
}

static double log_q(const orc_level* L, int64_t e, const double* z) {
  const double* q = L->q + e * 2 * L->dim;
  double s = 0.0;
  for (int d = 0; d < L->dim; ++d) {
    double a = q[d], b = q[L->dim + d];
    if (L->qfam == Q_GAUSS) {
      double t = (z[d] - a) / b;
      s += -0.5 * LOG_2PI - log(b) - 0.5 * t * t;
    } else if (L->qfam == Q_GAMMA) {
      s += a * log(b) - lgamma(a) + (a - 1.0) * log(z[d]) - b * z[d];
    } else {
      s += (a - 1.0) * log(z[d]) + (b - 1.0) * log1p(-z[d]) - (lgamma(a) + lgamma(b) - lgamma(a + b));
    }
  }
  return s;
}

/* log p(z | parent sample zp) of one plate element (the model's prior). */
static double log_prior(const orc_level* L, const double* z, const double* zp) {
  const int D = L->dim;
  double s = 0.0;
  switch (L->prior) {
    case PRIOR_STD_NORMAL:
      for (int d = 0; d < D; ++d) s += -0.5 * log(TWO_PI * L->prior_a) - z[d] * z[d] / (2.0 * L->prior_a);
      break;
    case PRIOR_NORMAL_FIXED_VAR:
      for (int d = 0; d < D; ++d) {
        double t = z[d] - zp[d];
        s += -0.5 * log(TWO_PI * L->prior_a) - t * t / (2.0 * L->prior_a);
      }
      break;
    case PRIOR_NORMAL_MEAN_LOGVAR:
      /* parent sample = (mean (D), log-variance (D)) */
      for (int d = 0; d < D; ++d) {
        double t = z[d] - zp[d], lv = zp[D + d];
        s += -0.5 * LOG_2PI - 0.5 * lv - 0.5 * t * t * exp(-lv);
      }
      break;
    case PRIOR_GAMMA:
      for (int d = 0; d < D; ++d)
        s += L->prior_a * log(L->prior_b) - lgamma(L->prior_a) + (L->prior_a - 1.0) * log(z[d]) - L->prior_b * z[d];
      break;
    case PRIOR_BETA:
      for (int d = 0; d < D; ++d)
        s += (L->prior_a - 1.0) * log(z[d]) + (L->prior_b - 1.0) * log1p(-z[d])
             - (lgamma(L->prior_a) + lgamma(L->prior_b) - lgamma(L->prior_a + L->prior_b));
      break;
  }
  return s;
}

/* sum_n log p(y_n | z, x_n) of one plate element. */
static double log_lik(const orc_level* L, int64_t e, const double* z) {
  const int D = L->dim;
  double s = 0.0;
  for (int n = 0; n < L->n_obs; ++n) {
    const double* xn = L->x + (e * L->n_obs + n) * D;
    double y = L->y[e * L->n_obs + n];
    double lin = 0.0;
    for (int d = 0; d < D; ++d) lin += z[d] * xn[d];
    switch (L->lik) {
      case LIK_GAUSS: s += -0.5 * log(TWO_PI * L->lik_var) - (y - lin) * (y - lin) / (2.0 * L->lik_var); break;
      case LIK_BERNOULLI_LOGIT: {
        /* y s - log(1 + e^s), evaluated without overflow */
        double sp = lin > 0 ? lin + log1p(exp(-lin)) : log1p(exp(lin));
        s += y * lin - sp;
        break;
      }
      case LIK_POISSON_LOG: s += y * lin - exp(lin) - lgamma(y + 1.0); break;
      case LIK_POISSON_RATE: s += y * log(z[0]) - z[0] - lgamma(y + 1.0); break;
      case LIK_BERNOULLI_PROB: s += y * log(z[0]) + (1.0 - y) * log1p(-z[0]); break;
      default: break;
    }
  }
  return s;
}

/* log( (1/K) sum_k exp(v_k) ) with the max shift (any shift is exact). */
static double log_mean_exp(const double* v, int K) {
  double m = -INFINITY;
  for (int k = 0; k < K; ++k) if (v[k] > m) m = v[k];
  if (m == -INFINITY) return -INFINITY;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s += exp(v[k] - m);
  return m + log(s) - log((double)K);
}

/* ------------------------------------------------------------------------- */
/* E-step: MPIW over the plate tree (Eq. mp_iw; Sec. 6 for the recursion).   */
int orc_estep(int n_levels, orc_level* lv, int K, uint64_t seed, uint64_t iter, double* log_pmp) {
  if (n_levels < 1 || K < 1) return 1;
  double** local = calloc((size_t)n_levels, sizeof(double*));  /* log lik - log q  [n][K] */
  double** H = calloc((size_t)n_levels, sizeof(double*));      /* children's sum    [n][K] */
  for (int l = 0; l < n_levels; ++l) {
    orc_level* L = &lv[l];
    local[l] = malloc(sizeof(double) * (size_t)(L->n * K));
    H[l] = calloc((size_t)(L->n * K), sizeof(double));
    int nps = L->qfam == Q_GAUSS ? L->dim : L->dim * (L->qfam == Q_GAMMA ? 1 : 2) * (2 * GAMMA_TRIES + 1);
    /* 1. draw z ~ Q and evaluate the local factor of every sample */
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < L->n; ++e) {
      double* nz = malloc(sizeof(double) * (size_t)nps);
      for (int k = 0; k < K; ++k) {
        if (L->eps) memcpy(nz, L->eps + (e * K + k) * nps, sizeof(double) * (size_t)nps);
        else for (int d = 0; d < nps; ++d) nz[d] = draw_noise(seed, iter, l, (uint64_t)e * K + k, d, L->qfam);
        double* z = L->z + (e * K + k) * L->dim;
        sample_one(L, e, nz, z);
        local[l][e * K + k] = log_lik(L, e, z) - log_q(L, e, z);
      }
      free(nz);
    }
  }
  /* 2. leaves to root: L_e[kp] = log mean_k exp( log p(z_e^k | z_p^kp) + local_e[k] + H_e[k] ),
   *    H_parent[kp] += L_e[kp]   (sum over the plate)                       */
  for (int l = n_levels - 1; l >= 1; --l) {
    orc_level* L = &lv[l];
    const orc_level* P = &lv[l - 1];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < L->n; ++e) {
      double* S = malloc(sizeof(double) * (size_t)K);
      int64_t p = L->parent[e];
      for (int kp = 0; kp < K; ++kp) {
        const double* zp = P->z + (p * K + kp) * P->dim;
        for (int k = 0; k < K; ++k)
          S[k] = log_prior(L, L->z + (e * K + k) * L->dim, zp) + local[l][e * K + k] + H[l][e * K + k];
        L->logL[e * K + kp] = log_mean_exp(S, K);
      }
      free(S);
    }
    for (int64_t e = 0; e < L->n; ++e)      /* plate sum, in element order */
      for (int kp = 0; kp < K; ++kp) H[l - 1][L->parent[e] * K + kp] += L->logL[e * K + kp];
  }
  /* 3. root: a[k] = log p(z_0^k) + local + H;  log P_MP = log mean exp a;  w_0 = softmax a */
  {
    orc_level* R = &lv[0];
    double* a = malloc(sizeof(double) * (size_t)K);
    for (int64_t i = 0; i < R->n; ++i) {
      for (int k = 0; k < K; ++k)
        a[k] = log_prior(R, R->z + (i * K + k) * R->dim, NULL) + local[0][i * K + k] + H[0][i * K + k] +
               (R->H_extra ? R->H_extra[i * K + k] : 0.0);
      double lme = log_mean_exp(a, K);
      log_pmp[i] = lme;
      double lse = lme + log((double)K);
      for (int k = 0; k < K; ++k) R->w[i * K + k] = exp(a[k] - lse);
    }
    free(a);
  }
  /* 4. root to leaves: w_e[k] = sum_kp w_p[kp] exp(S_e[kp][k]) / sum_k' exp(S_e[kp][k']) */
  for (int l = 1; l < n_levels; ++l) {
    orc_level* L = &lv[l];
    const orc_level* P = &lv[l - 1];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < L->n; ++e) {
      int64_t p = L->parent[e];
      double* we = L->w + e * K;
      for (int k = 0; k < K; ++k) we[k] = 0.0;
      for (int kp = 0; kp < K; ++kp) {
        double wp = P->w[p * K + kp];
        if (wp == 0.0) continue;
        const double* zp = P->z + (p * K + kp) * P->dim;
        double lse = L->logL[e * K + kp] + log((double)K);
        for (int k = 0; k < K; ++k) {
          double s = log_prior(L, L->z + (e * K + k) * L->dim, zp) + local[l][e * K + k] + H[l][e * K + k];
          we[k] += wp * exp(s - lse);
        }
      }
    }
  }
  /* 5. moments E_w[T(z)] per element (Eq. momone(z)) */
  for (int l = 0; l < n_levels; ++l) {
    orc_level* L = &lv[l];
    const int D = L->dim;
    for (int64_t e = 0; e < L->n; ++e)
      for (int d = 0; d < D; ++d) {
        double t0 = 0.0, t1 = 0.0;
        for (int k = 0; k < K; ++k) {
          double wk = L->w[e * K + k], zv = L->z[(e * K + k) * D + d];
          if (L->qfam == Q_GAUSS) { t0 += wk * zv; t1 += wk * zv * zv; }
          else if (L->qfam == Q_GAMMA) { t0 += wk * zv; t1 += wk * log(zv); }
          else { t0 += wk * log(zv); t1 += wk * log1p(-zv); }
        }
        L->mom[(e * 2 + 0) * D + d] = t0;
        L->mom[(e * 2 + 1) * D + d] = t1;
      }
  }
  for (int l = 0; l < n_levels; ++l) { free(local[l]); free(H[l]); }
  free(local); free(H);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* M-step (App. B): set the proposal's parameters from its mean parameters.   */

/* Gaussian: mean = E z, var = E z^2 - (E z)^2, floored (the pathology of
 * Sec. 4 when one sample carries all the weight).                            */
void orc_mstep_gauss(const double* m, int64_t n, int D, double var_floor, double* q_out) {
  for (int64_t e = 0; e < n; ++e)
    for (int d = 0; d < D; ++d) {
      double m1 = m[(e * 2) * D + d], m2 = m[(e * 2 + 1) * D + d];
      double v = m2 - m1 * m1;
      double fl = var_floor * (m1 * m1 > 1.0 ? m1 * m1 : 1.0);
      if (!(v > fl)) v = fl;
      q_out[(e * 2) * D + d] = m1;
      q_out[(e * 2 + 1) * D + d] = sqrt(v);
    }
}

/* Gamma(shape a, rate b) from (E z, E log z): log a - psi(a) = log E z - E log z,
 * b = a / E z.  Newton from Minka's (2002) closed-form start.                */
static double gamma_shape(double s) {
  /* Jensen: E log z < log E z for every non-degenerate Gamma, so s > 0 */
  if (!(s > 0.0) || !isfinite(s)) return NAN;
  double a = (3.0 - s + sqrt((s - 3.0) * (s - 3.0) + 24.0 * s)) / (12.0 * s);
  for (int it = 0; it < 100; ++it) {
    double f = log(a) - orc_digamma(a) - s;
    double fp = 1.0 / a - orc_trigamma(a);
    double an = a - f / fp;
    if (an <= 0.0) an = 0.5 * a;
    if (fabs(an - a) <= 1e-15 * a) { a = an; break; }
    a = an;
  }
  return a;
}

void orc_mstep_gamma(const double* m, int64_t n, int D, double* q_out) {
  for (int64_t e = 0; e < n; ++e)
    for (int d = 0; d < D; ++d) {
      double mz = m[(e * 2) * D + d], mlz = m[(e * 2 + 1) * D + d];
      double a = gamma_shape(log(mz) - mlz);
      q_out[(e * 2) * D + d] = a;
      q_out[(e * 2 + 1) * D + d] = a / mz;
    }
}

/* Beta(a, b) from (E log z, E log(1-z)):
 *   psi(a) - psi(a+b) = E log z,  psi(b) - psi(a+b) = E log(1-z).
 * Start from psi(x) ~ log(x - 1/2), then 2-D Newton (Minka 2000).
 * Jensen gives e^{E log z} + e^{E log(1-z)} < E z + E(1-z) = 1 for every
 * Beta; statistics outside that domain (or non-finite) have no solution and
 * give NaN parameters, as does a Newton run that cannot stay positive.      */
void orc_mstep_beta(const double* m, int64_t n, int D, double* q_out) {
  for (int64_t e = 0; e < n; ++e)
    for (int d = 0; d < D; ++d) {
      double la = m[(e * 2) * D + d], lb = m[(e * 2 + 1) * D + d];
      double A = exp(la), B = exp(lb);
      if (!isfinite(la) || !isfinite(lb) || !(A + B < 1.0)) {
        q_out[(e * 2) * D + d] = NAN;
        q_out[(e * 2 + 1) * D + d] = NAN;
        continue;
      }
      double t = 0.5 / (1.0 - A - B);
      double a = 0.5 + A * t, b = 0.5 + B * t;
      for (int it = 0; it < 200; ++it) {
        double pab = orc_digamma(a + b), tab = orc_trigamma(a + b);
        double g1 = orc_digamma(a) - pab - la, g2 = orc_digamma(b) - pab - lb;
        double j11 = orc_trigamma(a) - tab, j22 = orc_trigamma(b) - tab, j12 = -tab;
        double det = j11 * j22 - j12 * j12;
        double da = (j22 * g1 - j12 * g2) / det, db = (j11 * g2 - j12 * g1) / det;
        double an = a - da, bn = b - db;
        int halvings = 0;
        while ((an <= 0.0 || bn <= 0.0) && halvings < 64) { da *= 0.5; db *= 0.5; an = a - da; bn = b - db; ++halvings; }
        if (!(an > 0.0 && bn > 0.0) || !isfinite(an) || !isfinite(bn)) { a = b = NAN; break; }
        double ch = fabs(an - a) / a + fabs(bn - b) / b;
        a = an; b = bn;
        if (ch < 1e-15) break;
      }
      q_out[(e * 2) * D + d] = a;
      q_out[(e * 2 + 1) * D + d] = b;
    }
}

/* EMA of the mean parameters (Eq. ema): m_t = (1 - lambda) m_{t-1} + lambda m_hat. */
void orc_ema(double* m, const double* m_hat, int64_t count, double lambda) {
  for (int64_t i = 0; i < count; ++i) m[i] = (1.0 - lambda) * m[i] + lambda * m_hat[i];
}
