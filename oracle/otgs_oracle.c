/*
 * otgs_oracle.c -- plain FP64 CPU oracle for discrete optimal transport with
 * the squared-L2 + group-lasso regulariser (Ida et al., "Fast Regularized
 * Discrete Optimal Transport with Group-Sparse Regularizers", AAAI 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and it never calls it.
 *
 * Everything is FP64, single-threaded, in the order the paper states it.
 * Conventions:
 *   C       float32, m x n row-major (c_ij = C[i*n + j]), widened exactly to
 *           double before use
 *   labels  int32 per source row, values in [0, L)
 *   a, b    FP64 marginals (Sec. 2.1)
 *   group l = the rows with label l, visited in ascending row index
 *   theta   = mu * gamma, the soft-threshold level (Eq. 5, Lemma 2)
 *
 * Parity pins are not in this file: see tests/test_oracle_pins.py.
 */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

typedef struct {
    int64_t m, n;
    int32_t L;
    float *C;
    int32_t *labels;
    double *a, *b;
    double gamma, mu, theta;
    int64_t *goff;   /* L+1 offsets into grows */
    int64_t *grows;  /* rows of group l: grows[goff[l] .. goff[l+1]-1], ascending */
    double *sqrtg;   /* sqrt(g_l) */
} orc_t;

/* ------------------------------------------------------------------ setup */

EXPORT void orc_destroy(orc_t *h)
{
    if (!h) return;
    free(h->C); free(h->labels); free(h->a); free(h->b);
    free(h->goff); free(h->grows); free(h->sqrtg);
    free(h);
}

/* Copies the inputs.  Returns NULL on invalid sizes or labels. */
EXPORT orc_t *orc_create(int64_t m, int64_t n, int32_t L, const float *C,
                         const int32_t *labels, const double *a, const double *b,
                         double gamma, double mu)
{
    if (m <= 0 || n <= 0 || L <= 0 || !(gamma > 0.0) || !(mu >= 0.0)) return NULL;
    for (int64_t i = 0; i < m; i++)
        if (labels[i] < 0 || labels[i] >= L) return NULL;
    orc_t *h = (orc_t *)calloc(1, sizeof(orc_t));
    h->m = m; h->n = n; h->L = L;
    h->gamma = gamma; h->mu = mu; h->theta = mu * gamma;
    h->C = (float *)malloc(sizeof(float) * (size_t)(m * n));
    memcpy(h->C, C, sizeof(float) * (size_t)(m * n));
    h->labels = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    memcpy(h->labels, labels, sizeof(int32_t) * (size_t)m);
    h->a = (double *)malloc(sizeof(double) * (size_t)m);
    h->b = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(h->a, a, sizeof(double) * (size_t)m);
    memcpy(h->b, b, sizeof(double) * (size_t)n);
    /* group lists by counting sort, rows ascending inside each group */
    h->goff = (int64_t *)calloc((size_t)L + 1, sizeof(int64_t));
    h->grows = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    h->sqrtg = (double *)malloc(sizeof(double) * (size_t)L);
    for (int64_t i = 0; i < m; i++) h->goff[labels[i] + 1]++;
    for (int32_t l = 0; l < L; l++) h->goff[l + 1] += h->goff[l];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    for (int32_t l = 0; l < L; l++) fill[l] = h->goff[l];
    for (int64_t i = 0; i < m; i++) h->grows[fill[labels[i]]++] = i;
    free(fill);
    for (int32_t l = 0; l < L; l++) h->sqrtg[l] = sqrt((double)(h->goff[l + 1] - h->goff[l]));
    return h;
}

EXPORT double orc_theta(const orc_t *h) { return h->theta; }

/* ------------------------------------------------------ one block (l, j) */

/* f_i = alpha_i + beta_j - c_ij over the rows of group l (Sec. 2.3). */
static inline double f_of(const orc_t *h, const double *alpha, const double *beta,
                          int64_t i, int64_t j)
{
    return (alpha[i] + beta[j]) - (double)h->C[i * h->n + j];
}

/* z_{l,j} = ||[f_[l]]_+||  (Def. 1) and o_{l,j} = ||[f_[l]]_-||  (Def. 2). */
static void block_norms(const orc_t *h, const double *alpha, const double *beta,
                        int32_t l, int64_t j, double *z, double *o)
{
    double zp = 0.0, zn = 0.0;
    for (int64_t k = h->goff[l]; k < h->goff[l + 1]; k++) {
        double f = f_of(h, alpha, beta, h->grows[k], j);
        if (f > 0.0) zp += f * f; else zn += f * f;
    }
    *z = sqrt(zp);
    *o = sqrt(zn);
}

/*
 * Exact block of the plan and of psi (Eq. 5):
 *   grad psi(f)_[l] = [1 - mu / ||f+_[l]||]_+ f+_[l],  f+ = [f]_+ / gamma,
 * i.e. with z = ||[f_[l]]_+||:  t_{[l],j} = ([z - theta]_+ / (gamma z)) [f_[l]]_+.
 * The conjugate value of the block is psi_{l,j} = [z - theta]_+^2 / (2 gamma)
 * (sup over g >= 0 of f.g - Psi(g), attained at g = t).
 * Adds t into rowacc[i] and returns sum_i t_ij in *colsum; returns psi.
 */
static double block_exact(const orc_t *h, const double *alpha, const double *beta,
                          int32_t l, int64_t j, double *rowacc, double *colsum)
{
    double z, o;
    block_norms(h, alpha, beta, l, j, &z, &o);
    *colsum = 0.0;
    if (!(z > h->theta)) return 0.0;
    double s = (z - h->theta) / (h->gamma * z);
    double cs = 0.0;
    for (int64_t k = h->goff[l]; k < h->goff[l + 1]; k++) {
        int64_t i = h->grows[k];
        double f = f_of(h, alpha, beta, i, j);
        if (f > 0.0) {
            double t = s * f;
            if (rowacc) rowacc[i] += t;
            cs += t;
        }
    }
    *colsum = cs;
    double e = z - h->theta;
    return e * e / (2.0 * h->gamma);
}

static double dot(const double *x, const double *y, int64_t k)
{
    double s = 0.0;
    for (int64_t i = 0; i < k; i++) s += x[i] * y[i];
    return s;
}

/*
 * Dense (unscreened) dual objective and gradient, Eq. 4:
 *   D = alpha.a + beta.b - sum_{j,l} psi_{l,j}
 *   dD/dalpha = a - T 1_n,  dD/dbeta = b - T^T 1_m   (Danskin, Sec. 2.3)
 * Optional zout/oout (L x n, row l = group) receive z_{l,j} and o_{l,j}.
 */
EXPORT void orc_dual(const orc_t *h, const double *alpha, const double *beta,
                     double *D, double *galpha, double *gbeta, double *zout, double *oout)
{
    int64_t m = h->m, n = h->n;
    double *rowacc = (double *)calloc((size_t)m, sizeof(double));
    double psi = 0.0;
    for (int64_t j = 0; j < n; j++) {
        double col = 0.0;
        for (int32_t l = 0; l < h->L; l++) {
            double cs;
            psi += block_exact(h, alpha, beta, l, j, rowacc, &cs);
            col += cs;
            if (zout || oout) {
                double z, o;
                block_norms(h, alpha, beta, l, j, &z, &o);
                if (zout) zout[(int64_t)l * n + j] = z;
                if (oout) oout[(int64_t)l * n + j] = o;
            }
        }
        if (gbeta) gbeta[j] = h->b[j] - col;
    }
    if (galpha)
        for (int64_t i = 0; i < m; i++) galpha[i] = h->a[i] - rowacc[i];
    if (D) *D = dot(alpha, h->a, m) + dot(beta, h->b, n) - psi;
    free(rowacc);
}

/* Plan recovery t_j = grad psi(alpha + beta_j 1 - c_j)  (Sec. 2.3); T m x n. */
EXPORT void orc_plan(const orc_t *h, const double *alpha, const double *beta, double *T)
{
    int64_t n = h->n;
    memset(T, 0, sizeof(double) * (size_t)(h->m * n));
    for (int64_t j = 0; j < n; j++)
        for (int32_t l = 0; l < h->L; l++) {
            double z, o;
            block_norms(h, alpha, beta, l, j, &z, &o);
            if (!(z > h->theta)) continue;
            double s = (z - h->theta) / (h->gamma * z);
            for (int64_t k = h->goff[l]; k < h->goff[l + 1]; k++) {
                int64_t i = h->grows[k];
                double f = f_of(h, alpha, beta, i, j);
                if (f > 0.0) T[i * n + j] = s * f;
            }
        }
}

/* Primal objective of Eq. 2 with the regulariser of Eq. 3:
 *   <T, C> + sum_j gamma (1/2 ||t_j||^2 + mu sum_l ||t_j[l]||). */
EXPORT double orc_primal(const orc_t *h, const double *T)
{
    int64_t n = h->n;
    double lin = 0.0, quad = 0.0, grp = 0.0;
    for (int64_t i = 0; i < h->m; i++)
        for (int64_t j = 0; j < n; j++) {
            double t = T[i * n + j];
            lin += t * (double)h->C[i * n + j];
            quad += t * t;
        }
    for (int64_t j = 0; j < n; j++)
        for (int32_t l = 0; l < h->L; l++) {
            double s2 = 0.0;
            for (int64_t k = h->goff[l]; k < h->goff[l + 1]; k++) {
                double t = T[h->grows[k] * n + j];
                s2 += t * t;
            }
            grp += sqrt(s2);
        }
    return lin + h->gamma * (0.5 * quad + h->mu * grp);
}

/* ------------------------------------------------------ bounds (Sec. 3) */

/* Group statistics of dalpha = alpha - alpha_s:
 *   npos_l = ||[dalpha_[l]]_+||, nabs_l = ||dalpha_[l]||, nneg_l = ||[dalpha_[l]]_-||. */
static void dalpha_stats(const orc_t *h, const double *alpha, const double *alpha_s,
                         double *npos, double *nabs, double *nneg)
{
    for (int32_t l = 0; l < h->L; l++) {
        double p = 0.0, q = 0.0;
        for (int64_t k = h->goff[l]; k < h->goff[l + 1]; k++) {
            int64_t i = h->grows[k];
            double d = alpha[i] - alpha_s[i];
            if (d > 0.0) p += d * d; else q += d * d;
        }
        if (npos) npos[l] = sqrt(p);
        if (nneg) nneg[l] = sqrt(q);
        if (nabs) nabs[l] = sqrt(p + q);
    }
}

/*
 * Upper bound (Def. 1, Eq. 6):  zbar = z~ + ||[dalpha_[l]]_+|| + sqrt(g_l) [dbeta_j]_+
 * Lower bound (Def. 2, Eq. 7):  zlow = k~ - ||dalpha_[l]|| - sqrt(g_l)|dbeta_j|
 *                                      - o~ - ||[dalpha_[l]]_-|| - sqrt(g_l)|[dbeta_j]_-|
 * with k~ = ||f~_[l]|| = sqrt(z~^2 + o~^2) (the positive and negative parts of
 * f~ have disjoint supports).  zt, ot, zup, zlow are L x n (row l = group).
 */
EXPORT void orc_bounds(const orc_t *h, const double *alpha, const double *beta,
                       const double *alpha_s, const double *beta_s,
                       const double *zt, const double *ot, double *zup, double *zlow)
{
    int32_t L = h->L;
    int64_t n = h->n;
    double *npos = (double *)malloc(sizeof(double) * (size_t)L);
    double *nabs = (double *)malloc(sizeof(double) * (size_t)L);
    double *nneg = (double *)malloc(sizeof(double) * (size_t)L);
    dalpha_stats(h, alpha, alpha_s, npos, nabs, nneg);
    for (int32_t l = 0; l < L; l++)
        for (int64_t j = 0; j < n; j++) {
            double db = beta[j] - beta_s[j];
            double dbp = db > 0.0 ? db : 0.0;
            double dbn = db < 0.0 ? -db : 0.0;
            int64_t q = (int64_t)l * n + j;
            if (zup) zup[q] = zt[q] + npos[l] + h->sqrtg[l] * dbp;
            if (zlow) {
                double kt = sqrt(zt[q] * zt[q] + ot[q] * ot[q]);
                zlow[q] = kt - nabs[l] - h->sqrtg[l] * fabs(db) - ot[q] - nneg[l] - h->sqrtg[l] * dbn;
            }
        }
    free(npos); free(nabs); free(nneg);
}

/* ------------------------------------------ screened gradient (Alg. 1, 2) */

typedef struct {
    double *alpha_s, *beta_s;  /* snapshot alpha~, beta~ */
    double *zt, *ot;           /* snapshot z~, o~ (L x n) */
    unsigned char *inN;        /* set N (Def. 3), L x n */
    /* cumulative counters */
    int64_t n_in_N;        /* blocks computed because (l,j) in N  (Alg. 2, first loop) */
    int64_t n_checked;     /* upper bounds evaluated             (Alg. 2, second loop) */
    int64_t n_skipped;     /* checked and skipped (zbar <= theta) */
    int64_t n_unskipped;   /* checked and computed exactly */
    int64_t n_snapshot;    /* blocks touched by snapshot refreshes */
} screen_t;

/*
 * GradPsi (Alg. 2): blocks in N are computed exactly; every other block is
 * checked with the upper bound of Eq. 6 and set to zero when zbar <= theta
 * (Lemma 2), else computed exactly.  Returns D and the gradient like orc_dual.
 * skipped (optional, L x n) receives 1 for each skipped block.
 */
static void gradpsi(const orc_t *h, screen_t *sc, const double *alpha, const double *beta,
                    double *D, double *galpha, double *gbeta, unsigned char *skipped)
{
    int64_t m = h->m, n = h->n;
    int32_t L = h->L;
    double *rowacc = (double *)calloc((size_t)m, sizeof(double));
    double *colacc = (double *)calloc((size_t)n, sizeof(double));
    double *npos = (double *)malloc(sizeof(double) * (size_t)L);
    double psi = 0.0;
    /* first loop: (l, j) in N */
    for (int64_t j = 0; j < n; j++)
        for (int32_t l = 0; l < L; l++) {
            int64_t q = (int64_t)l * n + j;
            if (skipped) skipped[q] = 0;
            if (!sc->inN[q]) continue;
            double cs;
            psi += block_exact(h, alpha, beta, l, j, rowacc, &cs);
            colacc[j] += cs;
            sc->n_in_N++;
        }
    /* ||[dalpha_[l]]_+|| for all l, [dbeta]_+ on the fly */
    dalpha_stats(h, alpha, sc->alpha_s, npos, NULL, NULL);
    /* second loop: (l, j) not in N */
    for (int64_t j = 0; j < n; j++) {
        double db = beta[j] - sc->beta_s[j];
        double dbp = db > 0.0 ? db : 0.0;
        for (int32_t l = 0; l < L; l++) {
            int64_t q = (int64_t)l * n + j;
            if (sc->inN[q]) continue;
            sc->n_checked++;
            double zbar = sc->zt[q] + npos[l] + h->sqrtg[l] * dbp;
            if (zbar <= h->theta) {
                sc->n_skipped++;
                if (skipped) skipped[q] = 1;
                continue;
            }
            double cs;
            psi += block_exact(h, alpha, beta, l, j, rowacc, &cs);
            colacc[j] += cs;
            sc->n_unskipped++;
        }
    }
    if (galpha) for (int64_t i = 0; i < m; i++) galpha[i] = h->a[i] - rowacc[i];
    if (gbeta) for (int64_t j = 0; j < n; j++) gbeta[j] = h->b[j] - colacc[j];
    if (D) *D = dot(alpha, h->a, m) + dot(beta, h->b, n) - psi;
    free(rowacc); free(colacc); free(npos);
}

/* Alg. 1, every r iterations: rebuild N from the lower bound (Eq. 7, Def. 3)
 * against the current snapshot, then refresh the snapshot at (alpha, beta). */
static void rebuild_N_and_snapshot(const orc_t *h, screen_t *sc, const double *alpha,
                                   const double *beta, int use_lower)
{
    int64_t m = h->m, n = h->n;
    int64_t LN = (int64_t)h->L * n;
    if (use_lower) {
        double *zlow = (double *)malloc(sizeof(double) * (size_t)LN);
        orc_bounds(h, alpha, beta, sc->alpha_s, sc->beta_s, sc->zt, sc->ot, NULL, zlow);
        for (int64_t q = 0; q < LN; q++) sc->inN[q] = zlow[q] > h->theta;
        free(zlow);
    } else {
        memset(sc->inN, 0, (size_t)LN);
    }
    orc_dual(h, alpha, beta, NULL, NULL, NULL, sc->zt, sc->ot);
    memcpy(sc->alpha_s, alpha, sizeof(double) * (size_t)m);
    memcpy(sc->beta_s, beta, sizeof(double) * (size_t)n);
    sc->n_snapshot += LN;
}

/*
 * One screened evaluation for tests: GradPsi (Alg. 2) against explicit
 * snapshot arrays (FP64) and set N.  counts[4] += {in_N, checked, skipped,
 * unskipped}.  skipped (L x n) receives the skip decisions.
 */
EXPORT void orc_gradpsi(const orc_t *h, const double *alpha, const double *beta,
                        const double *alpha_s, const double *beta_s, const double *zt,
                        const unsigned char *inN, double *D, double *galpha, double *gbeta,
                        unsigned char *skipped, int64_t *counts)
{
    screen_t sc;
    memset(&sc, 0, sizeof(sc));
    sc.alpha_s = (double *)alpha_s; sc.beta_s = (double *)beta_s;
    sc.zt = (double *)zt; sc.inN = (unsigned char *)inN;
    gradpsi(h, &sc, alpha, beta, D, galpha, gbeta, skipped);
    if (counts) {
        counts[0] += sc.n_in_N; counts[1] += sc.n_checked;
        counts[2] += sc.n_skipped; counts[3] += sc.n_unskipped;
    }
}

/* ------------------------------------------------------------- L-BFGS */

/*
 * The dual (Eq. 4) is concave; the solver minimises F = -D over
 * x = (alpha, beta) in R^{m+n} with L-BFGS (Liu & Nocedal), memory M,
 * the two-loop recursion with H0 = (s.y / y.y) I (Nocedal & Wright, Alg. 7.4)
 * and the strong-Wolfe line search below.
 */
typedef struct {
    const orc_t *h;
    screen_t *sc;      /* NULL = dense evaluation (the paper's "origin") */
    int64_t N;         /* m + n */
    int64_t evals;
    double *ga, *gb;   /* scratch for dD/dalpha, dD/dbeta */
} solver_t;

/* F(x) = -D(x), G = -grad D. */
static double evalF(solver_t *s, const double *x, double *G)
{
    const orc_t *h = s->h;
    double D;
    if (s->sc) gradpsi(h, s->sc, x, x + h->m, &D, s->ga, s->gb, NULL);
    else orc_dual(h, x, x + h->m, &D, s->ga, s->gb, NULL, NULL);
    for (int64_t i = 0; i < h->m; i++) G[i] = -s->ga[i];
    for (int64_t j = 0; j < h->n; j++) G[h->m + j] = -s->gb[j];
    s->evals++;
    return -D;
}

static double inf_norm(const double *x, int64_t k)
{
    double r = 0.0;
    for (int64_t i = 0; i < k; i++) { double v = fabs(x[i]); if (v > r) r = v; }
    return r;
}

/* Step inside the bracket (lo, hi).  When phi' changes sign across it the
 * zero of the secant of phi' (the minimiser of the quadratic model) is used;
 * otherwise the minimiser of the quadratic through phi(lo), phi'(lo), phi(hi).
 * The step is kept inside [lo + 0.1 w, hi - 0.1 w]; bisection otherwise. */
static double bracket_step(double lo, double Flo, double dlo, double hi, double Fhi, double dhi)
{
    double w = hi - lo, t = lo + 0.5 * w;
    if (dlo < 0.0 && dhi > 0.0) {
        t = lo - dlo * w / (dhi - dlo);
    } else {
        double den = 2.0 * (Fhi - Flo - dlo * w);
        if (den > 0.0) t = lo - dlo * w * w / den;
    }
    if (!(t >= lo + 0.1 * w && t <= hi - 0.1 * w)) t = lo + 0.5 * w;
    return t;
}

#define LS_C1 1e-4
#define LS_C2 0.9
#define LS_EPS_F 1e-12
#define LS_MAX_EVALS 40

/*
 * Line search along the descent direction d from x (F0, slope dphi0 < 0),
 * returning a step that meets the strong Wolfe conditions (Nocedal & Wright,
 * Ch. 3): sufficient decrease F <= F0 + c1 t dphi0 and |dphi| <= c2 |dphi0|.
 * F is convex, so the bracket is driven by the sign of dphi: a point that
 * fails sufficient decrease or has dphi >= 0 becomes the upper end, any other
 * the lower end; the step doubles until an upper end exists.  Near the
 * optimum F differences reach FP64 resolution; there sufficient decrease is
 * taken in Hager & Zhang's approximate form (F - F0 <= eps |F0| and
 * dphi <= (2 c1 - 1) dphi0), which uses the exact derivative instead.
 * On success xt/Ft/Gt hold the accepted point and 0 is returned, else -1.
 */
static int line_search(solver_t *s, const double *x, double F0, double dphi0,
                       const double *d, double t_init, double *xt, double *Ft,
                       double *Gt, double *tacc)
{
    int64_t N = s->N;
    double *xl = (double *)malloc(sizeof(double) * (size_t)N);
    double *Gl = (double *)malloc(sizeof(double) * (size_t)N);
    int rc = -1, have_hi = 0;
    double lo = 0.0, Flo = F0, dlo = dphi0, hi = 0.0, Fhi = 0.0, dhi = 0.0;
    double t = t_init;
    for (int evals = 1; ; evals++) {
        for (int64_t k = 0; k < N; k++) xt[k] = x[k] + t * d[k];
        double F = evalF(s, xt, Gt);
        double dphi = dot(Gt, d, N);
        int suff = (F <= F0 + LS_C1 * t * dphi0) ||
                   (F - F0 <= LS_EPS_F * fabs(F0) && dphi <= (2.0 * LS_C1 - 1.0) * dphi0);
        if (suff && fabs(dphi) <= -LS_C2 * dphi0) { *Ft = F; *tacc = t; rc = 0; break; }
        if (!suff || dphi >= 0.0) {
            hi = t; Fhi = F; dhi = dphi; have_hi = 1;
        } else {
            lo = t; Flo = F; dlo = dphi;
            memcpy(xl, xt, sizeof(double) * (size_t)N);
            memcpy(Gl, Gt, sizeof(double) * (size_t)N);
        }
        if (evals >= LS_MAX_EVALS || (have_hi && hi - lo <= 1e-15 * hi)) {
            /* out of budget: keep the last sufficient-decrease point, if any */
            if (lo > 0.0) {
                memcpy(xt, xl, sizeof(double) * (size_t)N);
                memcpy(Gt, Gl, sizeof(double) * (size_t)N);
                *Ft = Flo; *tacc = lo; rc = 0;
            }
            break;
        }
        t = have_hi ? bracket_step(lo, Flo, dlo, hi, Fhi, dhi) : 2.0 * t;
    }
    free(xl); free(Gl);
    return rc;
}

/*
 * Solve max D with L-BFGS from the given (alpha, beta) (zero start = the
 * start of Alg. 1).  screening = 1 runs Alg. 1: GradPsi for every evaluation, and
 * every r accepted iterations the set N is rebuilt from Eq. 7 (use_lower = 1)
 * and the snapshot refreshed.  Stops when ||grad D||_inf <= tol.
 *
 *   out_D            final D
 *   counts[10]       iters, evals, status (0 ok, -4 maxit, -6 line search),
 *                    in_N, checked, skipped, unskipped, snapshot blocks,
 *                    ls failures (0/1), reserved
 *   trace[trace_cap] D after each accepted iteration (trace[0] = start)
 *   ginf             final ||grad D||_inf
 */
EXPORT int orc_solve(const orc_t *h, double *alpha, double *beta, double tol, int maxit,
                     int M, int screening, int use_lower, int r, double *out_D,
                     int64_t *counts, double *trace, int trace_cap, double *ginf)
{
    int64_t m = h->m, n = h->n, N = m + n, LN = (int64_t)h->L * n;
    solver_t s;
    memset(&s, 0, sizeof(s));
    s.h = h; s.N = N;
    s.ga = (double *)malloc(sizeof(double) * (size_t)m);
    s.gb = (double *)malloc(sizeof(double) * (size_t)n);
    screen_t sc;
    memset(&sc, 0, sizeof(sc));
    double *x = (double *)malloc(sizeof(double) * (size_t)N);
    memcpy(x, alpha, sizeof(double) * (size_t)m);
    memcpy(x + m, beta, sizeof(double) * (size_t)n);
    if (screening) {
        sc.alpha_s = (double *)malloc(sizeof(double) * (size_t)m);
        sc.beta_s = (double *)malloc(sizeof(double) * (size_t)n);
        sc.zt = (double *)malloc(sizeof(double) * (size_t)LN);
        sc.ot = (double *)malloc(sizeof(double) * (size_t)LN);
        sc.inN = (unsigned char *)calloc((size_t)LN, 1);
        /* as Alg. 1 starts: snapshot at the start point, N empty */
        orc_dual(h, x, x + m, NULL, NULL, NULL, sc.zt, sc.ot);
        memcpy(sc.alpha_s, x, sizeof(double) * (size_t)m);
        memcpy(sc.beta_s, x + m, sizeof(double) * (size_t)n);
        sc.n_snapshot += LN;
        s.sc = &sc;
    }
    double *G = (double *)malloc(sizeof(double) * (size_t)N);
    double *d = (double *)malloc(sizeof(double) * (size_t)N);
    double *xt = (double *)malloc(sizeof(double) * (size_t)N);
    double *Gt = (double *)malloc(sizeof(double) * (size_t)N);
    double *S = (double *)malloc(sizeof(double) * (size_t)(N * M));
    double *Y = (double *)malloc(sizeof(double) * (size_t)(N * M));
    double *rho = (double *)malloc(sizeof(double) * (size_t)M);
    double *al = (double *)malloc(sizeof(double) * (size_t)M);
    int npairs = 0, head = 0;  /* ring buffer: newest pair at (head-1) mod M */
    double F = evalF(&s, x, G);
    if (trace && trace_cap > 0) trace[0] = -F;
    int iter = 0, status = -4, lsfail = 0;
    for (;;) {
        if (inf_norm(G, N) <= tol) { status = 0; break; }
        if (iter >= maxit) { status = -4; break; }
        /* two-loop recursion: d = -H G */
        memcpy(d, G, sizeof(double) * (size_t)N);
        for (int k = 0; k < npairs; k++) {
            int idx = ((head - 1 - k) % M + M) % M;
            al[idx] = rho[idx] * dot(S + (int64_t)idx * N, d, N);
            double *yv = Y + (int64_t)idx * N;
            for (int64_t q = 0; q < N; q++) d[q] -= al[idx] * yv[q];
        }
        if (npairs > 0) {
            int nw = ((head - 1) % M + M) % M;
            double *yv = Y + (int64_t)nw * N;
            double h0 = dot(S + (int64_t)nw * N, yv, N) / dot(yv, yv, N);
            for (int64_t q = 0; q < N; q++) d[q] *= h0;
        }
        for (int k = npairs - 1; k >= 0; k--) {
            int idx = ((head - 1 - k) % M + M) % M;
            double be = rho[idx] * dot(Y + (int64_t)idx * N, d, N);
            double *sv = S + (int64_t)idx * N;
            for (int64_t q = 0; q < N; q++) d[q] += (al[idx] - be) * sv[q];
        }
        for (int64_t q = 0; q < N; q++) d[q] = -d[q];
        double dphi0 = dot(G, d, N);
        if (!(dphi0 < 0.0)) {  /* not a descent direction: restart from -G */
            for (int64_t q = 0; q < N; q++) d[q] = -G[q];
            dphi0 = dot(G, d, N);
            npairs = 0;
        }
        double t0 = (iter == 0 && npairs == 0) ? 1.0 / inf_norm(G, N) : 1.0;
        double Ft, tacc;
        if (line_search(&s, x, F, dphi0, d, t0, xt, &Ft, Gt, &tacc) != 0) {
            status = -6; lsfail = 1; break;
        }
        /* curvature pair */
        double *sv = S + (int64_t)head * N, *yv = Y + (int64_t)head * N;
        for (int64_t q = 0; q < N; q++) { sv[q] = xt[q] - x[q]; yv[q] = Gt[q] - G[q]; }
        double sy = dot(sv, yv, N);
        double ss = dot(sv, sv, N), yy = dot(yv, yv, N);
        if (sy > 1e-12 * sqrt(ss * yy)) {
            rho[head] = 1.0 / sy;
            head = (head + 1) % M;
            if (npairs < M) npairs++;
        }
        memcpy(x, xt, sizeof(double) * (size_t)N);
        memcpy(G, Gt, sizeof(double) * (size_t)N);
        F = Ft;
        iter++;
        if (trace && iter < trace_cap) trace[iter] = -F;
        if (screening && iter % r == 0) rebuild_N_and_snapshot(h, &sc, x, x + m, use_lower);
    }
    memcpy(alpha, x, sizeof(double) * (size_t)m);
    memcpy(beta, x + m, sizeof(double) * (size_t)n);
    if (out_D) *out_D = -F;
    if (ginf) *ginf = inf_norm(G, N);
    if (counts) {
        counts[0] = iter; counts[1] = s.evals; counts[2] = status;
        counts[3] = sc.n_in_N; counts[4] = sc.n_checked; counts[5] = sc.n_skipped;
        counts[6] = sc.n_unskipped; counts[7] = sc.n_snapshot; counts[8] = lsfail; counts[9] = 0;
    }
    free(G); free(d); free(xt); free(Gt); free(S); free(Y); free(rho); free(al); free(x);
    free(s.ga); free(s.gb);
    if (screening) { free(sc.alpha_s); free(sc.beta_s); free(sc.zt); free(sc.ot); free(sc.inN); }
    return status;
}

/* ------------------------------------- FP32 screening rule of the GPU path */

/*
 * Bit-for-bit replica of the screening decisions the CUDA path takes, written
 * from the rule it implements (Eq. 6-8 in FP32 with directed rounding), to
 * check the GPU's skip set and set N exactly.  Reading of the paper: Eq. 6 is
 * evaluated with every operation rounded toward +inf (so Lemma 1 holds for the
 * computed bound) and a block is skipped when zbar <= RD(theta - tau_l),
 * tau_l = 2^-36 (sqrt(g_l) M + g_l theta), a margin that covers the rounding of
 * the evaluation kernel; Eq. 7 is evaluated round-to-nearest.
 *
 * Group sums follow the GPU order: lane k (0..31) adds rows k, k+32, ... of
 * the group (ascending row index), then the 32 lane values meet in a xor tree
 * with offsets 16, 8, 4, 2, 1.
 *
 *   alpha, beta, alpha_s, beta_s   current iterate and snapshot (caller order)
 *   zt, ot                          FP32 snapshot values, row l at zt + l*ldz
 *   Nmask_in                        set N as L x ntiles words (bit = column % 32)
 *   skip_out (optional)             L x ntiles words: blocks skipped by Eq. 6
 *   N_out (optional)                L x ntiles words: N rebuilt from Eq. 7
 *   counts[3] (optional)            += in N, checked, skipped
 *
 * Pinned against the paper's rule in FP64 (orc_bounds) by
 * tests/test_oracle_screen_rule.py: every block this rule skips has an FP64
 * upper bound below theta by at least half the margin, every block whose FP64
 * bound is below theta by more than the FP32 error bound is skipped, the set
 * N differs from the FP64 one only within the rounding band of theta, and on
 * dyadic inputs (every FP32 operation exact) the decisions equal the FP64
 * rule's except on ties zbar == theta.
 */
static void xor_tree_f(float *v)
{
    float w[32];
    for (int off = 16; off >= 1; off >>= 1) {
        for (int x = 0; x < 32; x++) w[x] = v[x] + v[x ^ off];
        for (int x = 0; x < 32; x++) v[x] = w[x];
    }
}

EXPORT void orc_gpu_screen(const orc_t *h, const double *alpha, const double *beta,
                           const double *alpha_s, const double *beta_s, const float *zt,
                           const float *ot, int64_t ldz, const uint32_t *Nmask_in,
                           int64_t ntiles, uint32_t *skip_out, uint32_t *N_out, int64_t *counts)
{
    const int32_t L = h->L;
    const int64_t n = h->n;
    const int old_mode = fegetround();
    float *npos = (float *)malloc(sizeof(float) * (size_t)L);
    float *nabs = (float *)malloc(sizeof(float) * (size_t)L);
    float *nneg = (float *)malloc(sizeof(float) * (size_t)L);
    float *sgru = (float *)malloc(sizeof(float) * (size_t)L);
    float *sgrn = (float *)malloc(sizeof(float) * (size_t)L);
    float *dbp = (float *)malloc(sizeof(float) * (size_t)n);
    float *dba = (float *)malloc(sizeof(float) * (size_t)n);
    float *dbn = (float *)malloc(sizeof(float) * (size_t)n);
    float amax = 0.f, asmax = 0.f, bmax = 0.f, bsmax = 0.f, cmax = 0.f;
    for (int64_t q = 0; q < h->m * n; q++) if (h->C[q] > cmax) cmax = h->C[q];
    for (int32_t l = 0; l < L; l++) {
        float pu[32], a2[32], n2[32];
        for (int x = 0; x < 32; x++) { pu[x] = 0.f; a2[x] = 0.f; n2[x] = 0.f; }
        int64_t g = h->goff[l + 1] - h->goff[l];
        for (int64_t k = 0; k < g; k++) {
            int64_t i = h->grows[h->goff[l] + k];
            int x = (int)(k % 32);
            fesetround(FE_UPWARD);
            volatile double du = alpha[i] - alpha_s[i];
            float dp = (float)du;
            if (!(dp > 0.f)) dp = 0.f;
            pu[x] = pu[x] + dp * dp;
            float ar = (float)fabs(alpha[i]), asr = (float)fabs(alpha_s[i]);
            if (ar > amax) amax = ar;
            if (asr > asmax) asmax = asr;
            fesetround(FE_TONEAREST);
            volatile double dd = alpha[i] - alpha_s[i];
            float d = (float)dd;
            a2[x] = a2[x] + d * d;
            float dn = d < 0.f ? d : 0.f;
            n2[x] = n2[x] + dn * dn;
        }
        fesetround(FE_TONEAREST);
        double sg = sqrt((double)g);
        fesetround(FE_UPWARD);
        xor_tree_f(pu);
        npos[l] = sqrtf(pu[0]);
        sgru[l] = (float)sg;
        fesetround(FE_TONEAREST);
        xor_tree_f(a2);
        xor_tree_f(n2);
        nabs[l] = sqrtf(a2[0]);
        nneg[l] = sqrtf(n2[0]);
        sgrn[l] = (float)sqrt((double)g);
    }
    for (int64_t j = 0; j < n; j++) {
        fesetround(FE_UPWARD);
        volatile double du = beta[j] - beta_s[j];
        float p = (float)du;
        dbp[j] = p > 0.f ? p : 0.f;
        float br = (float)fabs(beta[j]), bsr = (float)fabs(beta_s[j]);
        if (br > bmax) bmax = br;
        if (bsr > bsmax) bsmax = bsr;
        fesetround(FE_TONEAREST);
        volatile double dd = beta[j] - beta_s[j];
        float d = (float)dd;
        dba[j] = fabsf(d);
        dbn[j] = d < 0.f ? -d : 0.f;
    }
    fesetround(FE_TONEAREST);
    double M = (((double)amax + (double)bmax) + (double)asmax) + (double)bsmax + (double)cmax;
    const double theta = h->theta;
    const float theta_f = (float)theta;
    int64_t c_in = 0, c_chk = 0, c_skip = 0;
    for (int32_t l = 0; l < L; l++) {
        int64_t g = h->goff[l + 1] - h->goff[l];
        fesetround(FE_TONEAREST);
        double tau = ldexp(sqrt((double)g) * M + (double)g * theta, -36);
        double tdiff = theta - tau;
        fesetround(FE_DOWNWARD);
        float th_skip = (float)tdiff;
        for (int64_t jt = 0; jt < ntiles; jt++) {
            uint32_t sw = 0, nw = 0, Nw = Nmask_in ? Nmask_in[l * ntiles + jt] : 0u;
            for (int lane = 0; lane < 32; lane++) {
                int64_t j = jt * 32 + lane;
                if (j >= n || g == 0) continue;
                const float z = zt[l * ldz + j], o = ot[l * ldz + j];
                int inN = (Nw >> lane) & 1u;
                if (inN) c_in++;
                else {
                    c_chk++;
                    fesetround(FE_UPWARD);
                    float zbar = (z + npos[l]) + sgru[l] * dbp[j];
                    if (zbar <= th_skip) { sw |= 1u << lane; c_skip++; }
                }
                fesetround(FE_TONEAREST);
                float kt = sqrtf(z * z + o * o);
                float zl = kt - nabs[l];
                zl = zl - sgrn[l] * dba[j];
                zl = zl - o;
                zl = zl - nneg[l];
                zl = zl - sgrn[l] * dbn[j];
                if (zl > theta_f) nw |= 1u << lane;
            }
            if (skip_out) skip_out[l * ntiles + jt] = sw;
            if (N_out) N_out[l * ntiles + jt] = nw;
        }
    }
    fesetround(old_mode);
    if (counts) { counts[0] += c_in; counts[1] += c_chk; counts[2] += c_skip; }
    free(npos); free(nabs); free(nneg); free(sgru); free(sgrn); free(dbp); free(dba); free(dbn);
}
