/*
 * Plain FP64 CPU oracle: Lasso by cyclic coordinate descent with GAP SAFE
 * sphere screening, dynamic (every f passes) and sequential (warm starts along
 * a geometric lambda grid) -- Fercoq, Gramfort, Salmon, "Mind the duality gap:
 * safer rules for the Lasso", ICML 2015 (arXiv:1505.03410).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Conventions
 *   - every floating-point value is IEEE double; loops sum left to right;
 *     compiled with -ffp-contract=off so no multiply-add is fused.
 *   - X is column-major: element (i, j) is X[i + j*ldx], ldx >= n.
 *   - the mask of kept (safe-active) features is one bit per feature:
 *     bit (j % 32) of word j / 32.
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   R1  gap tolerance eps = gap_tol_rel * ||y||^2.
 *   R2  dual point theta = alpha * rho, with alpha = 1 / max(lambda,
 *       ||X^T rho||_inf) by default, or the clipped optimal scaling of Eq. (8)
 *       when dual_point == 1 (alpha = y^T rho / (lambda ||rho||^2) when
 *       ||X^T rho||_inf == 0; alpha = 0 when rho == 0).
 *   R3  checks run before the first pass at each lambda and then after every
 *       f passes (Algorithm 1, "k mod f = 1"); one more check follows the
 *       K-th pass so the reported gap belongs to the returned beta.
 *   R4  the safe-active set is reset to all p features at each new lambda
 *       and only shrinks within one lambda.
 *   R5  scope of X^T rho: all p features (default) or the kept features
 *       only (xtr_scope == 1, the O(nq) evaluation of Sec. 4.1).
 *   R6  coordinates are visited in ascending index order; a feature is
 *       screened iff mu_j < 1 (Eq. (6)); zero-norm columns are screened.
 *   R7  the radius uses the gap inflated by a bound on its own FP64 rounding,
 *       tau = 2 (n + p + 8) u (||rho||^2 + lambda ||beta||_1 + ||y||^2 +
 *       ||lambda theta - y||^2), u = 2^-53; the stopping test uses the plain
 *       gap.
 *   R8  when a check does not stop, coefficients of newly screened features
 *       are set to zero and the residual is updated (Remark 3: this can only
 *       move beta closer to the solution); when it stops, beta is returned
 *       unchanged, so the certified gap belongs to the returned beta.
 *   R9  lambda_t = lambda_max * 10^(-delta t / (T-1)), t = 0..T-1 (Sec. 3.3),
 *       passed in as the ratios lambda_t / lambda_max.
 *   (R10-R13 concern the batched problems on row subsets, outside starting
 *   points at lambda_max and the learned start; orc_lasso_batch and
 *   oracle/lista.py state what they need of them.)
 *   R14 GAP SAFE dome (screen_rule == 1, Eq. (11) with the parameters of the
 *       appendix): ball center (y/lambda + theta)/2, ball radius R/2 with
 *       R = ||y/lambda - theta||, unit normal (y/lambda - theta)/R and ratio
 *       alpha_D = 2 r^2/R^2 - 1, where r^2 = (||y||^2 - ||X beta - y||^2 -
 *       2 lambda ||beta||_1)/lambda^2 is the radius of Thm. 2 taken from the
 *       primal point beta (clipped at 0).  The main text prints the normal
 *       with the opposite sign; the appendix's sign is the one for which the
 *       dome contains theta_hat (theta_hat is in the ball with diameter
 *       [theta, y/lambda] because it is the projection of y/lambda on the
 *       dual feasible set, and at distance >= r from y/lambda because
 *       D(theta_hat) <= P(beta)).  As for the sphere, the rounding bound tau of
 *       R7 enlarges the dome: lambda^2 R^2 is taken as ||lambda theta - y||^2
 *       + tau and lambda^2 r^2 as ||y||^2 - 2P - tau.  A feature is screened
 *       when the sphere test or the dome test screens it (both regions are
 *       safe; in exact arithmetic the dome lies inside the sphere, so this is
 *       the dome test).  When theta = y/lambda the dome is a point and only
 *       the sphere test runs.
 *   R15 refined radius (refined_radius == 1, Thm. 2): the sphere's radius is
 *       min(sqrt(2 (G + tau))/lambda, R), with lambda^2 R^2 = ||lambda theta -
 *       y||^2 + tau.  Thm. 2's radius sqrt(R^2 - r(beta)^2) equals sqrt(2 G) /
 *       lambda when ||y||^2 - 2P >= 0 (expand G = P - D) and equals R when the
 *       clipped r(beta) is 0, i.e. for iterates whose primal value exceeds
 *       P(0) = ||y||^2/2; the minimum is that radius with the rounding bound
 *       of R7 on both arguments.
 *   R16 Elastic-Net (enet_alpha < 1, the paper's appendix on the Elastic-Net):
 *       minimise 1/2 ||X beta - y||^2 + lambda a ||beta||_1 + lambda (1 - a)/2
 *       ||beta||^2 (a = enet_alpha) as the Lasso with penalty a lambda on the
 *       augmented design [X; sqrt((1 - a) lambda) I] and response [y; 0].  The
 *       augmented design changes with lambda, so it is built at every lambda
 *       and the whole of Algorithm 1 (checks, screening, passes) runs on it.
 *       lambda_max = ||X^T y||_inf / a (beta = 0 is optimal from there on).  The
 *       residual's first n entries are carried between lambdas as in the
 *       Lasso; its last p entries are -sqrt((1 - a) lambda) beta at the new
 *       lambda.  The stats report lambda (not a lambda) and the objectives of
 *       the augmented Lasso, which are the Elastic-Net's.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_NOT_CONVERGED 5

/* Per-lambda record written by orc_lasso_path (doubles, in this order). */
enum { ST_LAMBDA = 0, ST_PRIMAL, ST_DUAL, ST_GAP, ST_RADIUS, ST_ALPHA, ST_EPOCHS,
       ST_CHECKS, ST_NACTIVE, ST_NNZ, ST_CONVERGED, ST_NFIELDS };

typedef struct {
  int32_t screen_period; /* f */
  int32_t dual_point;    /* 0: rho / max(lambda, ||X^T rho||_inf); 1: Eq. (8) */
  int32_t xtr_scope;     /* 0: all p; 1: kept features only */
  int32_t warm_start;    /* 1: beta carried from the previous lambda */
  int64_t max_epochs;    /* K, passes per lambda */
  double gap_tol_rel;    /* eps / ||y||^2 */
  int32_t screen_rule;   /* 0: GAP SAFE sphere; 1: sphere and GAP SAFE dome (R14) */
  int32_t refined_radius; /* 1: the sphere radius of Thm. 2 (R15) */
  double enet_alpha;     /* a in (0, 1]: 1 is the Lasso, below 1 the Elastic-Net (R16) */
} orc_opts;

typedef struct {
  double alpha;    /* theta = alpha * rho */
  double xtr_inf;  /* max |x_j^T rho| over the scope */
  double primal;   /* P_lambda(beta), Eq. (1) */
  double dual;     /* D_lambda(theta), Eq. (2) */
  double gap;      /* P - D */
  double radius;   /* sqrt(2 (max(gap,0) + tau)) / lambda, Prop. 1 / Eq. (10); Thm. 2's with R15 */
  double tau;      /* rounding inflation of the gap used in the radius (R7) */
  int64_t n_kept;  /* features kept by the test */
  double dome_rad;   /* dome ball radius (R14; 0 when the dome is not used) */
  double dome_alpha; /* dome ratio alpha_D (R14) */
} orc_check_result;

static int mask_get(const uint32_t* m, int64_t j) { return (m[j >> 5] >> (j & 31)) & 1u; }
static void mask_clear(uint32_t* m, int64_t j) { m[j >> 5] &= ~(1u << (j & 31)); }

static double dot_col(const double* X, int64_t ldx, int64_t n, int64_t j, const double* v) {
  const double* x = X + j * ldx;
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += x[i] * v[i];
  return s;
}

/* Column squared norms, c0 = X^T y, lambda_max = ||X^T y||_inf (Sec. 1.2),
 * ||y||^2.  scal[0] = lambda_max, scal[1] = ||y||^2, scal[2] = argmax. */
void orc_precompute(const double* X, int64_t n, int64_t p, int64_t ldx, const double* y,
                    double* norms2, double* c0, double* scal) {
  double lmax = 0.0, yy = 0.0;
  int64_t arg = 0;
  for (int64_t j = 0; j < p; ++j) {
    norms2[j] = dot_col(X, ldx, n, j, X + j * ldx);
    c0[j] = dot_col(X, ldx, n, j, y);
    if (fabs(c0[j]) > lmax) { lmax = fabs(c0[j]); arg = j; }
  }
  for (int64_t i = 0; i < n; ++i) yy += y[i] * y[i];
  scal[0] = lmax;
  scal[1] = yy;
  scal[2] = (double)arg;
}

/* Geometric grid of Sec. 3.3 as ratios lambda_t / lambda_0 (R9). */
void orc_lambda_ratios(int32_t T, double delta, double* ratios) {
  for (int32_t t = 0; t < T; ++t)
    ratios[t] = (T == 1) ? 1.0 : pow(10.0, -delta * (double)t / (double)(T - 1));
}

/* Support function of the dome D(c, rad, alpha, nrm) (appendix, dome test)
 * at a vector x, from the scalars c^T x, nrm^T x and ||x||: the dome is the
 * part of the ball B(c, rad) on the side nrm^T (z - c) <= -alpha rad of its
 * hyperplane.  If x points far enough against nrm, the ball's own extreme
 * point c + rad x/||x|| lies in the dome; otherwise the maximum is on the
 * circle where the hyperplane cuts the sphere. */
double orc_dome_support(double cx, double rad, double alpha, double nx, double xnorm) {
  if (nx < -alpha * xnorm) return cx + rad * xnorm;
  double w = xnorm * xnorm - nx * nx;
  if (w < 0.0) w = 0.0;
  return cx - rad * alpha * nx + rad * sqrt(w * (1.0 - alpha * alpha));
}

/* One GAP SAFE check (Algorithm 1, the "every f passes" block):
 * c = X_scope^T rho, dual point theta (Eq. (8) / R2), P, D, gap, radius
 * r = sqrt(2 G)/lambda (Prop. 1), sphere test |x_j^T theta| + r ||x_j|| >= 1
 * (Eq. (7), Eq. (10)) applied to the kept features of mask_in; with
 * screen_rule == 1 also the dome test max(sigma(x_j), sigma(-x_j)) >= 1
 * (Eq. (11), R14), which needs c0 = X^T y.
 * Reads beta and rho, changes neither.  c (length p, may be NULL) receives
 * x_j^T rho for the scope (0 outside it); mu (length p, may be NULL) receives
 * the test value of each feature of mask_in (the sphere's, or the dome's when
 * the dome runs) and 0 elsewhere. */
void orc_check(const double* X, int64_t n, int64_t p, int64_t ldx, const double* y, double yy,
               const double* norms2, const double* c0, const double* beta, const double* rho,
               const uint32_t* mask_in, double lambda, const orc_opts* o,
               uint32_t* mask_out, double* c, double* mu_out, orc_check_result* res) {
  int64_t words = (p + 31) / 32;
  double* cbuf = c ? c : (double*)malloc(sizeof(double) * (size_t)p);
  double m = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    int in_scope = (o->xtr_scope == 0) || mask_get(mask_in, j);
    double cj = in_scope ? dot_col(X, ldx, n, j, rho) : 0.0;
    cbuf[j] = cj;
    if (in_scope && fabs(cj) > m) m = fabs(cj);
  }
  double rr = 0.0, yr = 0.0, l1 = 0.0;
  for (int64_t i = 0; i < n; ++i) { rr += rho[i] * rho[i]; yr += y[i] * rho[i]; }
  for (int64_t j = 0; j < p; ++j) l1 += fabs(beta[j]);

  double alpha;
  if (o->dual_point == 0) {
    alpha = 1.0 / (lambda > m ? lambda : m);
  } else {
    if (rr == 0.0) alpha = 0.0;
    else {
      double a = yr / (lambda * rr);
      if (m > 0.0) {
        double lim = 1.0 / m;
        if (a < -lim) a = -lim;
        if (a > lim) a = lim;
      }
      alpha = a;
    }
  }
  double d2 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double d = lambda * (alpha * rho[i]) - y[i];
    d2 += d * d;
  }
  double P = 0.5 * rr + lambda * l1;
  double D = 0.5 * yy - 0.5 * d2;
  double G = P - D;
  double u = ldexp(1.0, -53);
  double tau = 2.0 * (double)(n + p + 8) * u * (rr + lambda * l1 + yy + d2);
  double Gs = (G > 0.0 ? G : 0.0) + tau;
  double r = sqrt(2.0 * Gs) / lambda;
  if (o->refined_radius == 1) {
    double Rt = sqrt(d2 + tau) / lambda;   /* ||theta - y/lambda||, enlarged (R15) */
    if (Rt < r) r = Rt;
  }
  double aa = fabs(alpha);

  /* dome parameters (R14) */
  int dome = o->screen_rule == 1 && d2 > 0.0;
  double drad = 0.0, dal = 0.0, dR = 0.0;
  if (dome) {
    double big = d2 + tau;                 /* lambda^2 R^2, enlarged */
    double small = yy - 2.0 * P - tau;     /* lambda^2 r^2, reduced */
    if (small < 0.0) small = 0.0;
    double q = small / big;
    if (q > 1.0) q = 1.0;
    dal = 2.0 * q - 1.0;
    drad = 0.5 * sqrt(big) / lambda;
    dR = sqrt(d2) / lambda;                /* ||y/lambda - theta||, scales the normal */
  }

  memcpy(mask_out, mask_in, (size_t)words * sizeof(uint32_t));
  int64_t kept = 0;
  for (int64_t j = 0; j < p; ++j) {
    if (mu_out) mu_out[j] = 0.0;
    if (!mask_get(mask_in, j)) continue;
    double xn = sqrt(norms2[j]);
    double mu = fabs(cbuf[j]) * aa + r * xn;
    int screen = mu < 1.0;
    if (dome) {
      double xt = alpha * cbuf[j];         /* x_j^T theta */
      double xy = c0[j] / lambda;          /* x_j^T y / lambda */
      double cx = 0.5 * (xy + xt);         /* x_j^T (dome center) */
      double nx = (xy - xt) / dR;          /* x_j^T (unit normal) */
      double sp = orc_dome_support(cx, drad, dal, nx, xn);
      double sm = orc_dome_support(-cx, drad, dal, -nx, xn);
      mu = sp > sm ? sp : sm;
      if (mu < 1.0) screen = 1;
    }
    if (mu_out) mu_out[j] = mu;
    if (screen) mask_clear(mask_out, j);
    else ++kept;
  }
  if (!c) free(cbuf);
  res->alpha = alpha;
  res->xtr_inf = m;
  res->primal = P;
  res->dual = D;
  res->gap = G;
  res->radius = r;
  res->tau = tau;
  res->n_kept = kept;
  res->dome_rad = drad;
  res->dome_alpha = dal;
}

/* One cyclic pass of Algorithm 1 over the ascending list of kept features:
 * beta_j <- ST(lambda/||x_j||^2, beta_j + x_j^T rho / ||x_j||^2), with
 * ST(u, x) = sign(x) (|x| - u)_+, and rho -= (new - old) x_j. */
void orc_cd_pass(const double* X, int64_t n, int64_t ldx, const int64_t* list, int64_t q,
                 const double* norms2, double lambda, double* beta, double* rho) {
  for (int64_t k = 0; k < q; ++k) {
    int64_t j = list[k];
    double n2 = norms2[j];
    if (n2 == 0.0) continue;
    double g = dot_col(X, ldx, n, j, rho);
    double b = beta[j] + g / n2;
    double thr = lambda / n2;
    double ab = fabs(b);
    double nb = (ab > thr) ? (b > 0.0 ? ab - thr : -(ab - thr)) : 0.0;
    if (nb != beta[j]) {
      double d = nb - beta[j];
      const double* x = X + j * ldx;
      for (int64_t i = 0; i < n; ++i) rho[i] -= d * x[i];
      beta[j] = nb;
    }
  }
}

/* Check log for the safety tests (may be NULL): per check, the lambda index,
 * gap, radius, alpha, the residual rho of that check (n values) and the
 * dome's radius and ratio (R14). */
typedef struct {
  int64_t cap;      /* capacity in checks */
  int64_t count;    /* checks written */
  int32_t* t;       /* cap */
  double* gap;      /* cap */
  double* radius;   /* cap */
  double* alpha;    /* cap */
  double* rho;      /* cap * n */
  double* dome_rad;   /* cap */
  double* dome_alpha; /* cap */
} orc_log;

/* Algorithm 1 (CD with GAP SAFE rules) over the grid lambda_t = lambda_max *
 * ratios[t].  beta0 (p, may be NULL = zeros) is the starting point.
 * Outputs: beta_out p*T (column t = solution at lambda_t), mask_out
 * words*T (kept set of the last check at lambda_t, may be NULL),
 * stats ST_NFIELDS*T.  Returns ORC_NOT_CONVERGED if any lambda hit the
 * pass cap, else ORC_OK. */
int orc_lasso_path(const double* X, int64_t n, int64_t p, int64_t ldx, const double* y,
                   const double* ratios, int32_t T, const double* beta0, const orc_opts* o,
                   double* beta_out, uint32_t* mask_out, double* stats, orc_log* log) {
  if (n <= 0 || p <= 0 || ldx < n || T <= 0 || o->screen_period <= 0 || o->max_epochs < 0 ||
      !(o->enet_alpha > 0.0 && o->enet_alpha <= 1.0))
    return ORC_ERR_INVALID;
  int64_t words = (p + 31) / 32;
  /* Elastic-Net (R16): the augmented design, response, residual and tables */
  int enet = o->enet_alpha < 1.0;
  int64_t na = n + p;
  double* Xa = enet ? (double*)malloc(sizeof(double) * (size_t)(na * p)) : NULL;
  double* ya = enet ? (double*)malloc(sizeof(double) * (size_t)na) : NULL;
  double* rhoa = enet ? (double*)malloc(sizeof(double) * (size_t)na) : NULL;
  double* norms2a = enet ? (double*)malloc(sizeof(double) * (size_t)p) : NULL;
  double* c0a = enet ? (double*)malloc(sizeof(double) * (size_t)p) : NULL;
  double* norms2 = (double*)malloc(sizeof(double) * (size_t)p);
  double* c0 = (double*)malloc(sizeof(double) * (size_t)p);
  double* beta = (double*)malloc(sizeof(double) * (size_t)p);
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)p);
  uint32_t* mask = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)words);
  uint32_t* mask2 = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)words);
  double scal[3];
  orc_precompute(X, n, p, ldx, y, norms2, c0, scal);
  double lmax = scal[0] / o->enet_alpha, yy = scal[1];
  double eps = o->gap_tol_rel * yy;
  int status = ORC_OK;

  for (int64_t j = 0; j < p; ++j) beta[j] = beta0 ? beta0[j] : 0.0;
  for (int64_t i = 0; i < n; ++i) rho[i] = y[i];
  for (int64_t j = 0; j < p; ++j)
    if (beta[j] != 0.0)
      for (int64_t i = 0; i < n; ++i) rho[i] -= beta[j] * X[i + j * ldx];

  for (int32_t t = 0; t < T; ++t) {
    double lambda = lmax * ratios[t];
    if (t > 0 && !o->warm_start) {
      for (int64_t j = 0; j < p; ++j) beta[j] = beta0 ? beta0[j] : 0.0;
      for (int64_t i = 0; i < n; ++i) rho[i] = y[i];
      for (int64_t j = 0; j < p; ++j)
        if (beta[j] != 0.0)
          for (int64_t i = 0; i < n; ++i) rho[i] -= beta[j] * X[i + j * ldx];
    }
    for (int64_t w = 0; w < words; ++w) mask[w] = 0xffffffffu;
    if (p % 32) mask[words - 1] = (1u << (p % 32)) - 1u;

    /* the design this lambda's Lasso runs on, and its L1 penalty */
    const double* Xs = X;
    int64_t ns = n, lds = ldx;
    const double* ys = y;
    double* rs = rho;
    const double* n2s = norms2;
    const double* c0s = c0;
    double lam1 = lambda;
    if (enet) {
      double mu = (1.0 - o->enet_alpha) * lambda;
      double sm = sqrt(mu);
      lam1 = o->enet_alpha * lambda;
      for (int64_t j = 0; j < p; ++j) {
        double* col = Xa + j * na;
        for (int64_t i = 0; i < n; ++i) col[i] = X[i + j * ldx];
        for (int64_t i = 0; i < p; ++i) col[n + i] = (i == j) ? sm : 0.0;
      }
      for (int64_t i = 0; i < n; ++i) ya[i] = y[i];
      for (int64_t i = 0; i < p; ++i) ya[n + i] = 0.0;
      for (int64_t i = 0; i < n; ++i) rhoa[i] = rho[i];
      for (int64_t j = 0; j < p; ++j) rhoa[n + j] = -(sm * beta[j]);
      double scal_a[3];
      orc_precompute(Xa, na, p, na, ya, norms2a, c0a, scal_a);
      Xs = Xa;
      ns = na;
      lds = na;
      ys = ya;
      rs = rhoa;
      n2s = norms2a;
      c0s = c0a;
    }

    int64_t epochs = 0, checks = 0;
    int converged = 0;
    orc_check_result cr;
    for (;;) {
      orc_check(Xs, ns, p, lds, ys, yy, n2s, c0s, beta, rs, mask, lam1, o, mask2, NULL, NULL, &cr);
      ++checks;
      if (log && log->count < log->cap) {
        int64_t k = log->count++;
        log->t[k] = t;
        log->gap[k] = cr.gap;
        log->radius[k] = cr.radius;
        log->alpha[k] = cr.alpha;
        memcpy(log->rho + k * n, rs, sizeof(double) * (size_t)n);
        log->dome_rad[k] = cr.dome_rad;
        log->dome_alpha[k] = cr.dome_alpha;
      }
      /* newly screened features whose coefficient is nonzero (R8) */
      if (cr.gap <= eps) {
        memcpy(mask, mask2, sizeof(uint32_t) * (size_t)words);
        converged = 1;
        break;
      }
      if (epochs >= o->max_epochs) {
        memcpy(mask, mask2, sizeof(uint32_t) * (size_t)words);
        break;
      }
      for (int64_t j = 0; j < p; ++j) {
        if (mask_get(mask, j) && !mask_get(mask2, j) && beta[j] != 0.0) {
          double b = beta[j];
          for (int64_t i = 0; i < ns; ++i) rs[i] += b * Xs[i + j * lds];
          beta[j] = 0.0;
        }
      }
      memcpy(mask, mask2, sizeof(uint32_t) * (size_t)words);
      int64_t q = 0;
      for (int64_t j = 0; j < p; ++j)
        if (mask_get(mask, j)) list[q++] = j;
      for (int32_t e = 0; e < o->screen_period && epochs < o->max_epochs; ++e) {
        orc_cd_pass(Xs, ns, lds, list, q, n2s, lam1, beta, rs);
        ++epochs;
      }
    }
    if (enet)
      for (int64_t i = 0; i < n; ++i) rho[i] = rhoa[i];
    if (!converged) status = ORC_ERR_NOT_CONVERGED;
    int64_t nnz = 0;
    for (int64_t j = 0; j < p; ++j) {
      beta_out[j + (int64_t)t * p] = beta[j];
      nnz += (beta[j] != 0.0);
    }
    if (mask_out) memcpy(mask_out + (int64_t)t * words, mask, sizeof(uint32_t) * (size_t)words);
    double* s = stats + (int64_t)t * ST_NFIELDS;
    s[ST_LAMBDA] = lambda;
    s[ST_PRIMAL] = cr.primal;
    s[ST_DUAL] = cr.dual;
    s[ST_GAP] = cr.gap;
    s[ST_RADIUS] = cr.radius;
    s[ST_ALPHA] = cr.alpha;
    s[ST_EPOCHS] = (double)epochs;
    s[ST_CHECKS] = (double)checks;
    s[ST_NACTIVE] = (double)cr.n_kept;
    s[ST_NNZ] = (double)nnz;
    s[ST_CONVERGED] = (double)converged;
  }
  free(norms2); free(c0); free(beta); free(rho); free(list); free(mask); free(mask2);
  free(Xa); free(ya); free(rhoa); free(norms2a); free(c0a);
  return status;
}

/* Many independent paths over one design X (the batched workload): problem b
 * uses the rows i with row_mask[i + b*n] != 0 (all rows when row_mask is
 * NULL) and the response Y[:, b] (n x B, column-major, ld n; entries outside
 * the row subset are ignored) and starts from beta0[b*p .. b*p + p) (zeros
 * when beta0 is NULL).  Each problem is the plain path above on its own row
 * subset, with its own lambda_max; outputs are stacked by problem:
 * beta_out p*T*B, mask_out words*T*B, stats ST_NFIELDS*T*B. */
int orc_lasso_batch(const double* X, int64_t n, int64_t p, int64_t ldx, const double* Y,
                    const uint8_t* row_mask, int64_t B, const double* ratios, int32_t T,
                    const double* beta0, const orc_opts* o, double* beta_out, uint32_t* mask_out,
                    double* stats) {
  int64_t words = (p + 31) / 32;
  int status = ORC_OK;
  double* Xs = (double*)malloc(sizeof(double) * (size_t)(n * p));
  double* ys = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t b = 0; b < B; ++b) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (row_mask && !row_mask[i + b * n]) continue;
      ys[m] = Y[i + b * n];
      ++m;
    }
    if (m == 0) { status = ORC_ERR_INVALID; continue; }
    for (int64_t j = 0; j < p; ++j) {
      int64_t r = 0;
      for (int64_t i = 0; i < n; ++i) {
        if (row_mask && !row_mask[i + b * n]) continue;
        Xs[r + j * m] = X[i + j * ldx];
        ++r;
      }
    }
    int rc = orc_lasso_path(Xs, m, p, m, ys, ratios, T, beta0 ? beta0 + b * p : NULL, o, beta_out + b * p * T,
                            mask_out ? mask_out + b * words * T : NULL,
                            stats + b * ST_NFIELDS * T, NULL);
    if (rc != ORC_OK && status == ORC_OK) status = rc;
  }
  free(Xs); free(ys);
  return status;
}
