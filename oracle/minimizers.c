/*
 * FP64 oracle: line searches and minimizers of arXiv 1810.03358
 * (TEST INFRASTRUCTURE ONLY, see ffmin_oracle.h).
 *
 *   LS_H    Algorithm 5 (Section 5.2)
 *   LS_PAR  Algorithm 6 (Section 5.2)
 *   GD      adaptive steepest descent, Eq. 4, step from LS_PAR (Section 3)
 *   FGM     Algorithm 1 (Section 5.1)
 *   CG      Algorithm 2, beta variants of Section 4 / Section 5.1
 *   L-BFGS  Algorithms 3 and 4 (Section 5.1)
 *   parab   gradient-free random-atom moves (Section 3)
 *   HB      the heavy-ball method of Section 4 (Eq. 8) with constant alpha, beta
 *   OGM     the optimized gradient method of Section 4 (Eq. 11) with its
 *           step 1/L replaced by a line search over h (the variant the
 *           paper gives right after Eq. 13)
 *
 * Readings where the paper is silent:
 *  - every search direction is normalised to unit 2-norm before the line
 *    search (Section 5.1), so h is the 2-norm of the step;
 *  - the step accepted in one search is the next search's h0 (Section 5.2);
 *  - a failed search restarts the method once from the antigradient with
 *    momentum / history cleared and h0 reset; a second consecutive failure
 *    stops with ORC_LINESEARCH (Section 5.1: stop or change direction);
 *  - convergence: max_k |dE/dx_k| < gtol_inf after a gradient evaluation;
 *  - LS_PAR with K = 2 runs the refinement loop once (3 evaluations);
 *    degenerate parabolas (curvature <= 0, non-finite vertex) step to
 *    k_plus times the best non-zero step (half the smallest step when the
 *    best point is h = 0); a refined vertex is clamped to 8 x max|h|;
 *  - a non-finite trial energy counts as +inf inside a line search;
 *  - L-BFGS scales H0 by <s,y>/<y,y> of the newest stored pair and skips
 *    pairs with <s,y> <= 0;
 *  - CG: beta uses the previous unnormalised direction; restart every
 *    cg_restart_every iterations and whenever <g+, r+> >= 0;
 *  - FGM: Algorithm 1 as printed (non-monotone, no momentum restart; the
 *    best point x_* is what is returned); stop when |grad f(w)|_inf < tol
 *    and return the better of the best iterate and w.  Option fgm_restart
 *    adds the function-value adaptive restart of O'Donoghue and Candes
 *    (theta <- 1, x^{k-1} <- x^{k+1} whenever f(x^{k+1}) > f(x^k)), which
 *    the paper does not use in Algorithm 1.
 *  - OGM: t_0 = 1; the gradient is evaluated at y (the base of the line
 *    search, which takes LS_PAR with G0 by default, steps of either sign);
 *    stop when |grad f(x^k)|_inf < tol; no momentum restart (the method is
 *    kept literal: restarts measured on convex quadratics break its Eq. 12
 *    rate), except the common one after a failed search (x^0 <- x^k,
 *    t <- 1, the gradient sum restarted at x^k).
 * A trial point x + h r is formed as fma(h, r_k, x_k) per component.
 */
#include "ffmin_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------- trace of the last run ---------------- */
#define TRACE_CAP 200000
static double tr_f[TRACE_CAP], tr_h[TRACE_CAP], tr_th[TRACE_CAP], tr_b[TRACE_CAP];
static int32_t tr_n;
static void trace_reset(void) { tr_n = 0; }
static void trace_add(double f, double h, double th, double b) {
    if (tr_n < TRACE_CAP) {
        tr_f[tr_n] = f; tr_h[tr_n] = h; tr_th[tr_n] = th; tr_b[tr_n] = b; tr_n++;
    }
}
int32_t orc_trace(double *f, double *h, double *theta, double *beta, int32_t cap) {
    int32_t n = tr_n < cap ? tr_n : cap;
    for (int32_t k = 0; k < n; k++) {
        if (f) f[k] = tr_f[k];
        if (h) h[k] = tr_h[k];
        if (theta) theta[k] = tr_th[k];
        if (beta) beta[k] = tr_b[k];
    }
    return n;
}

/* ---------------- SplitMix64 ---------------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
int32_t orc_pick_atom(uint64_t seed, uint64_t k, int32_t n) {
    unsigned __int128 p = (unsigned __int128)orc_splitmix64(seed, k) * (uint64_t)n;
    return (int32_t)(p >> 64);
}

void orc_options_default(orc_options *o) {
    memset(o, 0, sizeof(*o));
    o->method = ORC_LBFGS;
    o->cg_variant = ORC_CG_PRP;
    o->ls = ORC_LS_DEFAULT;
    o->lbfgs_m = 10;
    o->gtol_inf = 0.1;
    o->max_iter = 100000;
    o->max_evals = 1000000;
    o->cg_restart_every = 0; /* 0 -> number of variables */
    o->h0 = 0.1;
    o->k_plus = 2.0;
    o->k_minus = 0.5;
    o->eps_h = 1e-10;
    o->ls_par_K = 2;
    o->ls_par_g0 = 1;
    o->gradfree_delta = 0.05;
    o->seed = 12345;
    o->precond_d = NULL;
    o->pc_window = 200;
    o->pc_rel = 1e-5;
    o->pc_gfar = 100.0;
}

static double finite_or_inf(double f) { return isfinite(f) ? f : HUGE_VAL; }

/* ---------------- LS_H (Algorithm 5) ---------------- */
double orc_ls_h(orc_line_fn phi, void *ctx, double f_star, double h0, double eps_h,
                double k_plus, double k_minus, double *f_out, int32_t *n_evals) {
    int32_t ne = 0;
    double f0 = finite_or_inf(phi(ctx, h0)); ne++;
    if (f0 < f_star) {
        double h1 = k_plus * h0;
        double f1 = finite_or_inf(phi(ctx, h1)); ne++;
        *n_evals = ne;
        if (f1 < f0) { *f_out = f1; return h1; }
        *f_out = f0;
        return h0;
    }
    double h2 = k_minus * h0;
    double f2 = finite_or_inf(phi(ctx, h2)); ne++;
    while (f2 > f_star) {
        h2 = k_minus * h2;
        if (h2 <= eps_h) { *n_evals = ne; *f_out = f_star; return 0.0; }
        f2 = finite_or_inf(phi(ctx, h2)); ne++;
    }
    *n_evals = ne;
    *f_out = f2;
    return h2;
}

/* ---------------- LS_PAR (Algorithm 6) ---------------- */
/* Vertex of the parabola through three points (Newton form
 * p(h) = f0 + d1 (h - h0) + A (h - h0)(h - h1)); returns 0 when the
 * curvature A is not positive or the vertex is not finite. */
static int parabola3(const double *h, const double *f, double *vertex) {
    double d1 = (f[1] - f[0]) / (h[1] - h[0]);
    double d2 = (f[2] - f[1]) / (h[2] - h[1]);
    double A = (d2 - d1) / (h[2] - h[0]);
    if (!(A > 0.0) || !isfinite(A)) return 0;
    double v = 0.5 * (h[0] + h[1]) - d1 / (2.0 * A);
    if (!isfinite(v)) return 0;
    *vertex = v;
    return 1;
}

/* order two points: by f ascending, then by |h| ascending */
static int point_less(double ha, double fa, double hb, double fb) {
    if (fa < fb) return 1;
    if (fa > fb) return 0;
    return fabs(ha) < fabs(hb);
}

static void sort_points(double *h, double *f, int n) {
    for (int a = 1; a < n; a++) { /* insertion sort, stable */
        double hh = h[a], ff = f[a];
        int b = a - 1;
        while (b >= 0 && point_less(hh, ff, h[b], f[b])) {
            h[b + 1] = h[b]; f[b + 1] = f[b]; b--;
        }
        h[b + 1] = hh; f[b + 1] = ff;
    }
}

double orc_ls_par(orc_line_fn phi, void *ctx, double f_star, double slope, double h0,
                  int32_t K, int32_t g0, double k_plus, double *f_out, int32_t *n_evals) {
    int32_t ne = 0;
    double h[4], f[4];
    h[0] = 0.0; f[0] = f_star;
    if (g0) {
        h[1] = h0;
        f[1] = finite_or_inf(phi(ctx, h[1])); ne++;
        /* parabola through f(0) = f*, f'(0) = slope and (h1, f1) */
        double a = (f[1] - f_star - slope * h[1]) / (h[1] * h[1]);
        double v = -slope / (2.0 * a);
        if (a > 0.0 && isfinite(a) && isfinite(v)) h[2] = v;
        else h[2] = k_plus * h[1];
        f[2] = finite_or_inf(phi(ctx, h[2])); ne++;
    } else {
        h[1] = -0.5 * h0;
        f[1] = finite_or_inf(phi(ctx, h[1])); ne++;
        h[2] = 0.5 * h0;
        f[2] = finite_or_inf(phi(ctx, h[2])); ne++;
    }
    for (int32_t k = 2; k <= K; k++) {
        double v;
        double hmax = fmax(fabs(h[0]), fmax(fabs(h[1]), fabs(h[2])));
        if (!parabola3(h, f, &v)) {
            /* degenerate: step beyond the best non-zero point, or back
             * towards 0 when h = 0 is the best point */
            int ib = 0;
            for (int a = 1; a < 3; a++)
                if (point_less(h[a], f[a], h[ib], f[ib])) ib = a;
            if (h[ib] != 0.0) {
                v = k_plus * h[ib];
            } else {
                int ic = -1;
                for (int a = 0; a < 3; a++)
                    if (h[a] != 0.0 && (ic < 0 || fabs(h[a]) < fabs(h[ic]))) ic = a;
                v = ic >= 0 ? 0.5 * h[ic] : h0;
            }
        }
        if (fabs(v) > 8.0 * hmax) v = copysign(8.0 * hmax, v);
        h[3] = v;
        f[3] = finite_or_inf(phi(ctx, h[3])); ne++;
        sort_points(h, f, 4);
    }
    if (K == 2) sort_points(h, f, 3); /* the paper's extra sort; already sorted */
    *n_evals = ne;
    if (f[0] < f_star) { *f_out = f[0]; return h[0]; }
    *f_out = f_star;
    return 0.0;
}

/* ---------------- minimizers ---------------- */
typedef struct {
    int32_t n;
    orc_fg_fn fg;
    void *ctx;
    int32_t ne, neg;
    int32_t status;
} obj_t;

static double obj_e(obj_t *o, const double *x) {
    int32_t st = 0;
    double f = o->fg(o->ctx, x, NULL, &st);
    o->ne++;
    if (st) return INFINITY;
    return f;
}
static double obj_eg(obj_t *o, const double *x, double *g) {
    int32_t st = 0;
    double f = o->fg(o->ctx, x, g, &st);
    o->neg++;
    if (st || !isfinite(f)) o->status = ORC_NONFINITE;
    return f;
}

typedef struct {
    obj_t *o;
    const double *x, *r;
    double *xt;
} line_t;

static double line_phi(void *ctx, double h) {
    line_t *l = (line_t *)ctx;
    for (int32_t k = 0; k < l->o->n; k++) l->xt[k] = fma(h, l->r[k], l->x[k]);
    return obj_e(l->o, l->xt);
}

static double dotn(int32_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int32_t k = 0; k < n; k++) s += a[k] * b[k];
    return s;
}
static double infnorm(int32_t n, const double *a) {
    double m = 0.0;
    for (int32_t k = 0; k < n; k++) m = fmax(m, fabs(a[k]));
    return m;
}

/* direction normalisation (Section 5.1): rhat = r * (1/|r|_2) */
static void normalise(int32_t n, const double *r, double *rhat) {
    double inv = 1.0 / sqrt(dotn(n, r, r));
    for (int32_t k = 0; k < n; k++) rhat[k] = r[k] * inv;
}

static double line_search(const orc_options *op, int method, obj_t *o, const double *x,
                          const double *rhat, double *xt, double f_star, double slope,
                          double h0, double *f_out, int32_t *ne) {
    line_t l = {o, x, rhat, xt};
    int ls = op->ls;
    if (ls == ORC_LS_DEFAULT) ls = (method == ORC_FGM) ? ORC_LS_H : ORC_LS_PAR;
    if (ls == ORC_LS_H)
        return orc_ls_h(line_phi, &l, f_star, h0, op->eps_h, op->k_plus, op->k_minus, f_out, ne);
    return orc_ls_par(line_phi, &l, f_star, slope, h0, op->ls_par_K, op->ls_par_g0,
                      op->k_plus, f_out, ne);
}

/* L-BFGS two-loop recursion, Algorithm 3 (readings: scale by the newest
 * pair; loops over the stored pairs; optional H0 diagonal d). */
void orc_lbfgs_direction(int32_t n, const double *g, int32_t count, const double *s,
                         const double *y, const double *d, double *r) {
    for (int32_t k = 0; k < n; k++) r[k] = -g[k];
    if (count == 0) return;
    double *alpha = (double *)malloc(sizeof(double) * count);
    double *rho = (double *)malloc(sizeof(double) * count);
    for (int32_t i = 0; i < count; i++) rho[i] = 1.0 / dotn(n, s + (size_t)i * n, y + (size_t)i * n);
    for (int32_t i = count - 1; i >= 0; i--) { /* newest -> oldest */
        const double *si = s + (size_t)i * n, *yi = y + (size_t)i * n;
        alpha[i] = rho[i] * dotn(n, si, r);
        for (int32_t k = 0; k < n; k++) r[k] -= alpha[i] * yi[k];
    }
    const double *sn = s + (size_t)(count - 1) * n, *yn = y + (size_t)(count - 1) * n;
    double gamma = dotn(n, sn, yn) / dotn(n, yn, yn);
    for (int32_t k = 0; k < n; k++) r[k] = d ? gamma * d[k] * r[k] : gamma * r[k];
    for (int32_t i = 0; i < count; i++) { /* oldest -> newest */
        const double *si = s + (size_t)i * n, *yi = y + (size_t)i * n;
        double beta = rho[i] * dotn(n, yi, r);
        for (int32_t k = 0; k < n; k++) r[k] += (alpha[i] - beta) * si[k];
    }
    free(alpha);
    free(rho);
}

static double cg_beta(int variant, int32_t n, const double *gp, const double *g,
                      const double *d) {
    /* y = g+ - g ; d = previous unnormalised direction */
    double gpy = 0.0, dy = 0.0, gpgp = dotn(n, gp, gp), gg = dotn(n, g, g), dg = dotn(n, d, g);
    for (int32_t k = 0; k < n; k++) {
        double yk = gp[k] - g[k];
        gpy += gp[k] * yk;
        dy += d[k] * yk;
    }
    switch (variant) {
    case ORC_CG_HS: return gpy / dy;
    case ORC_CG_FR: return gpgp / gg;
    case ORC_CG_PRP_PLUS: return fmax(0.0, gpy / gg);
    case ORC_CG_CD: return gpgp / (-dg);
    case ORC_CG_LS: return gpy / (-dg);
    case ORC_CG_DY: return gpgp / dy;
    case ORC_CG_PRP:
    default: return gpy / gg;
    }
}

#define CAP_HIT(it, o) ((it) >= op->max_iter || (o).ne + (o).neg >= op->max_evals)

/* optional per-iteration H0 diagonal of the force-field L-BFGS (the network) */
typedef struct {
    const orc_ff *ff;
    const double *w;
    int32_t *n8;
} diag_ctx_t;
static diag_ctx_t *g_diag = NULL;

int orc_minimize(int32_t n, orc_fg_fn fg, void *ctx, double *x, const orc_options *op,
                 orc_result *res) {
    obj_t o = {n, fg, ctx, 0, 0, ORC_OK};
    int method = op->method;
    trace_reset();
    memset(res, 0, sizeof(*res));
    if (method == ORC_GRADFREE) { res->status = ORC_BAD_ARG; return ORC_BAD_ARG; }
    size_t nb = sizeof(double) * (size_t)n;
    double *g = malloc(nb), *r = malloc(nb), *rhat = malloc(nb), *xt = malloc(nb),
           *gn = malloc(nb), *xn = malloc(nb), *xp = malloc(nb), *xb = malloc(nb);
    int m = op->lbfgs_m > 0 ? op->lbfgs_m : 1;
    double *S = malloc(nb * m), *Y = malloc(nb * m);
    int32_t hist = 0;
    int32_t restart_every = op->cg_restart_every > 0 ? op->cg_restart_every : n;
    int status = ORC_OK;
    int32_t it = 0, lsf = 0;
    double h0 = op->h0;
    int fresh = 1;
    double f = obj_eg(&o, x, g);
    double ginf = infnorm(n, g);
    double result_f = f, result_ginf = ginf;
    if (o.status) { status = o.status; goto done; }

    if (method == ORC_FGM) {
        /* Algorithm 1: x_* <- x0, x^{-1} <- x0, theta_{-1} <- 1 */
        double th_prev = 1.0, fb = f, fw = f, fx = f;
        memcpy(xp, x, nb);
        memcpy(xb, x, nb);
        double *w = xn, *gw = gn;
        memcpy(w, x, nb);
        memcpy(gw, g, nb);
        int have_w = 1; /* w^0 = x^0: its E and gradient are already known */
        int xb_is_w_grad = 1; /* gradient at xb known (= gw) */
        double xb_ginf = ginf;
        for (;;) {
            double th = 0.5 * th_prev * (sqrt(th_prev * th_prev + 4.0) - th_prev);
            double beta = th_prev * (1.0 - th_prev) / (th_prev * th_prev + th);
            if (!have_w) {
                for (int32_t k = 0; k < n; k++) w[k] = fma(beta, x[k] - xp[k], x[k]);
                fw = obj_eg(&o, w, gw);
                if (o.status) { status = o.status; break; }
            }
            have_w = 0;
            double gwinf = infnorm(n, gw);
            if (gwinf < op->gtol_inf) {
                if (fw < fb) { memcpy(xb, w, nb); fb = fw; xb_ginf = gwinf; xb_is_w_grad = 1; }
                status = ORC_OK;
                break;
            }
            if (CAP_HIT(it, o)) { status = ORC_MAX_ITER; break; }
            for (int32_t k = 0; k < n; k++) r[k] = -gw[k];
            normalise(n, r, rhat);
            int32_t ne = 0;
            double fnew, h;
            if (op->fgm_step > 0.0) {
                /* fixed step 1/L (tests): x^{k+1} = w^k - grad f(w^k) / L, i.e.
                 * h = |grad f(w^k)|_2 / L along r^k; f(x^{k+1}) for the best point */
                line_t l = {&o, w, rhat, xt};
                h = op->fgm_step * sqrt(dotn(n, gw, gw));
                fnew = line_phi(&l, h);
            } else {
                h = line_search(op, method, &o, w, rhat, xt, fw, dotn(n, gw, rhat), h0, &fnew, &ne);
            }
            if (h == 0.0) {
                lsf++;
                if (fresh) { status = ORC_LINESEARCH; break; }
                fresh = 1;
                th_prev = 1.0;
                memcpy(x, w, nb);
                memcpy(xp, w, nb);
                fx = fw;
                h0 = op->h0;
                continue;
            }
            fresh = 0;
            memcpy(xp, x, nb);
            for (int32_t k = 0; k < n; k++) x[k] = fma(h, rhat[k], w[k]);
            trace_add(fnew, h, th, beta);
            if (op->fgm_restart && fnew > fx) {
                /* optional adaptive restart (function scheme of O'Donoghue and
                 * Candes; not part of Algorithm 1): the new iterate is worse
                 * than the previous one, so the momentum is dropped */
                th_prev = 1.0;
                memcpy(xp, x, nb);
            } else {
                th_prev = th;
            }
            fx = fnew;
            h0 = h;
            it++;
            if (fnew < fb) { memcpy(xb, x, nb); fb = fnew; xb_is_w_grad = 0; }
        }
        memcpy(x, xb, nb);
        result_f = fb;
        if (status != ORC_NONFINITE) {
            if (xb_is_w_grad) {
                result_ginf = xb_ginf;
            } else { /* report the gradient of the returned point */
                result_f = obj_eg(&o, x, g);
                result_ginf = infnorm(n, g);
            }
        }
        goto done;
    }

    if (method == ORC_HB) {
        /* Eq. 8: x^{k+1} = x^k - alpha grad f(x^k) + beta (x^k - x^{k-1}),
         * x^{-1} = x^0, formed as fma(beta, x^k - x^{k-1}, fma(-alpha, g, x^k)) */
        if (!(op->hb_alpha > 0.0) || !(op->hb_beta >= 0.0)) { status = ORC_BAD_ARG; goto done; }
        memcpy(xp, x, nb);
        for (;;) {
            if (ginf < op->gtol_inf) { status = ORC_OK; break; }
            if (CAP_HIT(it, o)) { status = ORC_MAX_ITER; break; }
            for (int32_t k = 0; k < n; k++)
                xn[k] = fma(op->hb_beta, x[k] - xp[k], fma(-op->hb_alpha, g[k], x[k]));
            double fn = obj_eg(&o, xn, gn);
            /* a failed evaluation ends the run at the last good iterate */
            if (o.status) { status = o.status; break; }
            memcpy(xp, x, nb);
            memcpy(x, xn, nb);
            memcpy(g, gn, nb);
            f = fn;
            ginf = infnorm(n, g);
            it++;
            trace_add(fn, op->hb_alpha, 0.0, op->hb_beta);
        }
        result_f = f;
        result_ginf = ginf;
        goto done;
    }

    if (method == ORC_OGM) {
        /* Eq. 11: y = (1 - 1/t') x^k + (1/t') x^0,
         *         d = (1 - 1/t') grad f(x^k) + (2/t') sum_j t_j grad f(x^j),
         *         x^{k+1} = y - h d with h from a line search,
         * t' = t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2 */
        double *x0 = malloc(nb), *ds = malloc(nb), *y = malloc(nb), *gy = malloc(nb);
        double t = 1.0;
        memcpy(x0, x, nb);
        memcpy(ds, g, nb); /* t_0 grad f(x^0) */
        for (;;) {
            if (ginf < op->gtol_inf) { status = ORC_OK; break; }
            if (CAP_HIT(it, o)) { status = ORC_MAX_ITER; break; }
            const double tn = 0.5 * (1.0 + sqrt(4.0 * t * t + 1.0));
            const double a = 1.0 - 1.0 / tn, b = 1.0 / tn, c2 = 2.0 / tn;
            for (int32_t k = 0; k < n; k++) {
                y[k] = fma(a, x[k], b * x0[k]);
                r[k] = -fma(a, g[k], c2 * ds[k]);
            }
            normalise(n, r, rhat);
            const double fy = obj_eg(&o, y, gy);
            if (o.status) { status = o.status; break; }
            const double slope = dotn(n, gy, rhat);
            int32_t ne = 0;
            double fnew;
            /* x^{k+1} = y - (1/L) d, i.e. h = |d| / L along rhat (fixed-step
             * form, for tests), else a line search over h */
            double h = op->ogm_step > 0.0 ? op->ogm_step * sqrt(dotn(n, r, r))
                                          : line_search(op, method, &o, y, rhat, xt, fy, slope, h0, &fnew, &ne);
            if (h == 0.0) {
                lsf++;
                if (fresh) { status = ORC_LINESEARCH; break; }
                fresh = 1;
                t = 1.0;
                memcpy(x0, x, nb);
                memcpy(ds, g, nb);
                h0 = op->h0;
                continue;
            }
            fresh = 0;
            for (int32_t k = 0; k < n; k++) xn[k] = fma(h, rhat[k], y[k]);
            double fn = obj_eg(&o, xn, gn);
            if (o.status) { status = o.status; memcpy(x, xn, nb); f = fn; break; }
            it++;
            h0 = fabs(h);
            trace_add(fn, h, tn, 0.0);
            t = tn;
            for (int32_t k = 0; k < n; k++) ds[k] = fma(tn, gn[k], ds[k]);
            memcpy(x, xn, nb);
            memcpy(g, gn, nb);
            f = fn;
            ginf = infnorm(n, g);
        }
        free(x0); free(ds); free(y); free(gy);
        result_f = f;
        result_ginf = ginf;
        goto done;
    }

    /* GD, CG, L-BFGS */
    if (ginf < op->gtol_inf) goto done;
    for (int32_t k = 0; k < n; k++) r[k] = -g[k];
    int pc_on = g_diag != NULL; /* learned diagonal in use, and its safeguard's mark */
    int32_t pc_it = it;
    double pc_f = f;
    for (;;) {
        if (CAP_HIT(it, o)) { status = ORC_MAX_ITER; break; }
        if (method == ORC_LBFGS && g_diag && pc_on && hist > 0) {
            /* learned diagonal; plain L-BFGS when it gives no descent direction */
            orc_precond_diag(g_diag->ff, g_diag->w, g_diag->n8, g, xt);
            orc_lbfgs_direction(n, g, hist, S, Y, xt, r);
            if (!(dotn(n, g, r) < 0.0)) orc_lbfgs_direction(n, g, hist, S, Y, NULL, r);
        } else if (method == ORC_LBFGS)
            orc_lbfgs_direction(n, g, hist, S, Y, op->precond_d, r);
        else if (method == ORC_GD)
            for (int32_t k = 0; k < n; k++) r[k] = -g[k];
        normalise(n, r, rhat);
        double slope = dotn(n, g, rhat);
        int32_t ne = 0;
        double fnew;
        double h = line_search(op, method, &o, x, rhat, xt, f, slope, h0, &fnew, &ne);
        if (h == 0.0) {
            lsf++;
            if (fresh) { status = ORC_LINESEARCH; break; }
            fresh = 1;
            hist = 0;
            for (int32_t k = 0; k < n; k++) r[k] = -g[k];
            h0 = op->h0;
            continue;
        }
        fresh = 0;
        for (int32_t k = 0; k < n; k++) xn[k] = fma(h, rhat[k], x[k]);
        double fn = obj_eg(&o, xn, gn);
        if (o.status) { status = o.status; memcpy(x, xn, nb); f = fn; break; }
        it++;
        h0 = fabs(h);
        trace_add(fn, h, 0.0, 0.0);
        double gninf = infnorm(n, gn);
        if (method == ORC_LBFGS) {
            /* s = x+ - x, y = g+ - g; keep the pair only if <s,y> > 0 */
            double *sn = S + (size_t)(hist < m ? hist : m - 1) * n;
            double *yn = Y + (size_t)(hist < m ? hist : m - 1) * n;
            double sy = 0.0;
            for (int32_t k = 0; k < n; k++) sy += (xn[k] - x[k]) * (gn[k] - g[k]);
            if (sy > 0.0) {
                if (hist == m) { /* drop the oldest pair */
                    memmove(S, S + n, nb * (m - 1));
                    memmove(Y, Y + n, nb * (m - 1));
                } else {
                    hist++;
                }
                for (int32_t k = 0; k < n; k++) { sn[k] = xn[k] - x[k]; yn[k] = gn[k] - g[k]; }
            }
        } else if (method == ORC_CG) {
            if (gninf >= op->gtol_inf) {
                double *rn = xt; /* scratch */
                if (it % restart_every == 0) {
                    for (int32_t k = 0; k < n; k++) rn[k] = -gn[k];
                } else {
                    double beta = cg_beta(op->cg_variant, n, gn, g, r);
                    for (int32_t k = 0; k < n; k++) rn[k] = -gn[k] + beta * r[k];
                    if (dotn(n, gn, rn) >= 0.0)
                        for (int32_t k = 0; k < n; k++) rn[k] = -gn[k];
                }
                memcpy(r, rn, nb);
            }
        }
        memcpy(x, xn, nb);
        memcpy(g, gn, nb);
        f = fn;
        ginf = gninf;
        if (ginf < op->gtol_inf) { status = ORC_OK; break; }
        if (pc_on && op->pc_window > 0 && it - pc_it >= op->pc_window) {
            /* the energy stalled far from a stationary point: plain L-BFGS */
            if (ginf > op->pc_gfar * op->gtol_inf && !(pc_f - f >= op->pc_rel * fabs(pc_f))) pc_on = 0;
            pc_it = it;
            pc_f = f;
        }
    }
    result_f = f;
    result_ginf = ginf;
done:
    res->energy = result_f;
    res->grad_inf = result_ginf;
    res->iterations = it;
    res->energy_evals = o.ne;
    res->grad_evals = o.neg;
    res->ls_failures = lsf;
    res->status = status;
    free(g); free(r); free(rhat); free(xt); free(gn); free(xn); free(xp); free(xb);
    free(S); free(Y);
    return status;
}

/* ---------------- force-field objective ---------------- */
static double ff_fg(void *ctx, const double *x, double *g, int32_t *status) {
    orc_terms t;
    *status = orc_energy_terms((const orc_ff *)ctx, x, g, &t);
    return t.total;
}

/* one gradient-free move of atom i in x: the best of 7 axis points (current,
 * +-delta on x, y, z) and the vertex of the per-axis parabolas (8 row
 * energies, Section 3) */
static double move_row(const orc_ff *ff, const double *x, int32_t i, const double *p, double r_far) {
    return r_far > 0.0 ? orc_row_energy_taylor(ff, x, i, p, r_far) : orc_row_energy(ff, x, i, p);
}

static void parab_move(const orc_ff *ff, double *x, int32_t i, double dl, double r_far) {
    double p[8][3], fv[8];
    for (int c = 0; c < 8; c++)
        for (int a = 0; a < 3; a++) p[c][a] = x[3 * i + a];
    for (int a = 0; a < 3; a++) {
        p[1 + 2 * a][a] += dl; /* +delta */
        p[2 + 2 * a][a] -= dl; /* -delta */
    }
    for (int c = 0; c < 7; c++) fv[c] = move_row(ff, x, i, p[c], r_far);
    for (int a = 0; a < 3; a++) {
        double fp = fv[1 + 2 * a], fm = fv[2 + 2 * a];
        double curv = fm - 2.0 * fv[0] + fp;
        double ts = curv > 0.0 ? dl * (fm - fp) / (2.0 * curv) : 0.0;
        p[7][a] = x[3 * i + a] + ts;
    }
    fv[7] = move_row(ff, x, i, p[7], r_far);
    int best = 0;
    for (int c = 1; c < 8; c++)
        if (fv[c] < fv[best]) best = c;
    for (int a = 0; a < 3; a++) x[3 * i + a] = p[best][a];
}

/* gradient-free "parab" (Section 3): move one random atom per step to the
 * best of 7 axis points (current, +-delta on x, y, z) and the vertex of the
 * per-axis parabolas; check |grad|_inf once per sweep of N moves. */
static int parab(const orc_ff *ff, double *x, const orc_options *op, orc_result *res) {
    const int32_t n = ff->n_atoms;
    const double dl = op->gradfree_delta;
    size_t nb = sizeof(double) * 3 * (size_t)n;
    double *g = malloc(nb);
    orc_terms t;
    int status = orc_energy_terms(ff, x, g, &t);
    int32_t neg = 1, ne = 0, moves = 0;
    double ginf = infnorm(3 * n, g);
    trace_reset();
    if (status == ORC_OK && !(ginf < op->gtol_inf)) {
        for (;;) {
            for (int32_t sweep = 0; sweep < n; sweep++) {
                if (moves >= op->max_iter) { status = ORC_MAX_ITER; break; }
                int32_t i = orc_pick_atom(op->seed, (uint64_t)moves, n);
                parab_move(ff, x, i, dl, op->gradfree_taylor_r);
                ne += 8;
                moves++;
            }
            if (status == ORC_MAX_ITER) break;
            status = orc_energy_terms(ff, x, g, &t);
            neg++;
            ginf = infnorm(3 * n, g);
            trace_add(t.total, 0.0, 0.0, 0.0);
            if (status != ORC_OK) break;
            if (ginf < op->gtol_inf) break;
        }
    }
    if (status == ORC_MAX_ITER) { /* report the returned point */
        orc_energy_terms(ff, x, g, &t);
        neg++;
        ginf = infnorm(3 * n, g);
    }
    res->energy = t.total;
    res->grad_inf = ginf;
    res->iterations = moves;
    res->energy_evals = ne;
    res->grad_evals = neg;
    res->ls_failures = 0;
    res->status = status;
    free(g);
    return status;
}

/* ---- parallel epochs of the gradient-free search (Section 3's proposal) ----
 * Epoch e cuts the molecule into P parts by recursive bisection: a set of
 * atoms meant for p parts is ordered by (coordinate on its axis of largest
 * extent, index) and split at rank round(|A| floor(p/2) / p) (halves up) plus a random
 * shift in [-span/2, span/2], span = max(1, |A| / (2p)) (node k of the
 * bisection tree draws pick(seed, 2^62 + e 2^20 + k, span)), clamped to
 * [1, |A| - 1]; the cut plane lies halfway between the two atoms on either
 * side, and the halves recurse (left first) into floor(p/2) and the rest.
 * Each part is a box bounded by its cut planes.  An atom is movable when it
 * is at least `margin` from every cut plane of its box.  Every part q then
 * runs |L_q| moves (L_q: its movable atoms in index order; move m picks
 * L_q[pick(seed, q 2^40 + e N + m, |L_q|)]) on its own copy of the epoch's
 * starting positions: it sees its own moves and the other parts as they
 * were at the start of the epoch.  The parts' atoms are then merged and the
 * gradient checked.  A cap on the total moves truncates part q to
 * max_iter - (moves so far) - (moves of parts < q).  With P = 1 this is the
 * sequential method (one epoch = one sweep). */
#define EPOCH_CUT_STREAM (1ULL << 62)
typedef struct { double c; int32_t a; } rank_t;
static int cmp_rank(const void *u, const void *v) {
    const rank_t *x = (const rank_t *)u, *y = (const rank_t *)v;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return x->a < y->a ? -1 : (x->a > y->a ? 1 : 0);
}

typedef struct {
    const double *x;
    uint64_t seed, e;
    int32_t *part;   /* [N] part of each atom */
    double *box;     /* [P][6]: lo xyz, hi xyz */
    int32_t next;    /* next part id */
    rank_t *rk;      /* scratch [N] */
} cut_ctx_t;

static void bisect(cut_ctx_t *cc, int32_t *A, int32_t na, int32_t p, const double lo[3],
                   const double hi[3], uint64_t node) {
    if (p == 1) {
        const int32_t q = cc->next++;
        for (int32_t k = 0; k < na; k++) cc->part[A[k]] = q;
        for (int k = 0; k < 3; k++) { cc->box[6 * q + k] = lo[k]; cc->box[6 * q + 3 + k] = hi[k]; }
        return;
    }
    int axis = 0;
    double ext[3];
    for (int k = 0; k < 3; k++) {
        double mn = cc->x[3 * A[0] + k], mx = mn;
        for (int32_t t = 1; t < na; t++) {
            mn = fmin(mn, cc->x[3 * A[t] + k]);
            mx = fmax(mx, cc->x[3 * A[t] + k]);
        }
        ext[k] = mx - mn;
    }
    if (ext[1] > ext[axis]) axis = 1;
    if (ext[2] > ext[axis]) axis = 2;
    for (int32_t t = 0; t < na; t++) { cc->rk[t].c = cc->x[3 * A[t] + axis]; cc->rk[t].a = A[t]; }
    qsort(cc->rk, (size_t)na, sizeof(rank_t), cmp_rank);
    for (int32_t t = 0; t < na; t++) A[t] = cc->rk[t].a;
    const int32_t p1 = p / 2;
    const int32_t span = na / (2 * p) > 1 ? na / (2 * p) : 1;
    /* round(na p1 / p), halves up, in integers */
    int32_t c = (int32_t)((2LL * na * p1 + p) / (2LL * p)) +
                orc_pick_atom(cc->seed, EPOCH_CUT_STREAM + (cc->e << 20) + node, span) - span / 2;
    if (c < 1) c = 1;
    if (c > na - 1) c = na - 1;
    const double plane = 0.5 * (cc->x[3 * A[c - 1] + axis] + cc->x[3 * A[c] + axis]);
    double hl[3] = {hi[0], hi[1], hi[2]}, lr[3] = {lo[0], lo[1], lo[2]};
    hl[axis] = plane;
    lr[axis] = plane;
    bisect(cc, A, c, p1, lo, hl, 2 * node + 1);
    bisect(cc, A + c, na - c, p - p1, lr, hi, 2 * node + 2);
}

static int parab_epochs(const orc_ff *ff, double *x, const orc_options *op, orc_result *res) {
    const int32_t n = ff->n_atoms, P = op->gradfree_parts < n ? op->gradfree_parts : n;
    const double dl = op->gradfree_delta, w = op->gradfree_margin;
    size_t nb = sizeof(double) * 3 * (size_t)n;
    double *g = malloc(nb), *xs = malloc(nb), *xv = malloc(nb);
    double *box = malloc(sizeof(double) * 6 * (size_t)P);
    rank_t *rk = malloc(sizeof(rank_t) * (size_t)n);
    int32_t *part = malloc(sizeof(int32_t) * (size_t)n), *list = malloc(sizeof(int32_t) * (size_t)n);
    int32_t *all = malloc(sizeof(int32_t) * (size_t)n), *mov = malloc(sizeof(int32_t) * (size_t)P);
    orc_terms t;
    int status = orc_energy_terms(ff, x, g, &t);
    int32_t neg = 1, ne = 0, moves = 0;
    double ginf = infnorm(3 * n, g);
    trace_reset();
    if (status == ORC_OK && !(ginf < op->gtol_inf)) {
        for (uint64_t e = 0;; e++) {
            if (moves >= op->max_iter) { status = ORC_MAX_ITER; break; }
            for (int32_t a = 0; a < n; a++) all[a] = a;
            const double inf3[3] = {-HUGE_VAL, -HUGE_VAL, -HUGE_VAL}, sup3[3] = {HUGE_VAL, HUGE_VAL, HUGE_VAL};
            cut_ctx_t cc = {x, op->seed, e, part, box, 0, rk};
            bisect(&cc, all, n, P, inf3, sup3, 0);
            memcpy(xs, x, nb);
            int32_t off = 0, truncated = 0;
            for (int32_t q = 0; q < P; q++) {
                const double *bx = box + 6 * q;
                int32_t m_q = 0;
                for (int32_t a = 0; a < n; a++) {
                    if (part[a] != q) continue;
                    int ok = 1;
                    for (int k = 0; k < 3; k++)
                        if (xs[3 * a + k] - bx[k] < w || bx[3 + k] - xs[3 * a + k] < w) ok = 0;
                    if (ok) list[m_q++] = a;
                }
                int32_t allowed = op->max_iter - moves - off;
                if (allowed > m_q) allowed = m_q;
                if (allowed < 0) allowed = 0;
                if (allowed < m_q) truncated = 1;
                mov[q] = allowed;
                memcpy(xv, xs, nb);
                for (int32_t m = 0; m < allowed; m++) {
                    const uint64_t k = ((uint64_t)q << 40) + e * (uint64_t)n + (uint64_t)m;
                    parab_move(ff, xv, list[orc_pick_atom(op->seed, k, m_q)], dl, op->gradfree_taylor_r);
                    ne += 8;
                }
                for (int32_t a = 0; a < n; a++)
                    if (part[a] == q)
                        for (int k = 0; k < 3; k++) x[3 * a + k] = xv[3 * a + k];
                off += m_q;
            }
            for (int32_t q = 0; q < P; q++) moves += mov[q];
            if (truncated) { status = ORC_MAX_ITER; break; }
            status = orc_energy_terms(ff, x, g, &t);
            neg++;
            ginf = infnorm(3 * n, g);
            trace_add(t.total, (double)off, 0.0, 0.0);
            if (status != ORC_OK) break;
            if (ginf < op->gtol_inf) break;
            if (off == 0) { status = ORC_MAX_ITER; break; } /* nothing movable */
        }
    }
    if (status == ORC_MAX_ITER) { /* report the returned point */
        orc_energy_terms(ff, x, g, &t);
        neg++;
        ginf = infnorm(3 * n, g);
    }
    res->energy = t.total;
    res->grad_inf = ginf;
    res->iterations = moves;
    res->energy_evals = ne;
    res->grad_evals = neg;
    res->ls_failures = 0;
    res->status = status;
    free(g); free(xs); free(xv); free(box); free(rk); free(part); free(list); free(all); free(mov);
    return status;
}

int orc_minimize_ff(const orc_ff *ff, double *x, const orc_options *o, orc_result *res) {
    if (o->method == ORC_GRADFREE && o->gradfree_parts >= 1) return parab_epochs(ff, x, o, res);
    if (o->method == ORC_GRADFREE) return parab(ff, x, o, res);
    orc_options op = *o;
    if (op.cg_restart_every <= 0) op.cg_restart_every = 3 * ff->n_atoms;
    diag_ctx_t dc;
    int32_t *n8 = NULL;
    if (o->mlp_w && o->method == ORC_LBFGS) {
        /* neighbour counts of the starting structure */
        n8 = malloc(sizeof(int32_t) * (size_t)(ff->n_atoms > 0 ? ff->n_atoms : 1));
        for (int i = 0; i < ff->n_atoms; i++) n8[i] = orc_neighbour_count(ff, x, i, 8.0);
        dc.ff = ff;
        dc.w = o->mlp_w;
        dc.n8 = n8;
        g_diag = &dc;
    }
    int st = orc_minimize(3 * ff->n_atoms, ff_fg, (void *)ff, x, &op, res);
    g_diag = NULL;
    free(n8);
    return st;
}

/* ---------------- monotonic basin hopping ---------------- */
/* Perturbation of one coordinate: step * (2u - 1), u = the top 53 bits of
 * the SplitMix64 output of `seed` at counter `k`, scaled to [0, 1). */
static double mbh_offset(uint64_t seed, uint64_t k, double step) {
    const double u = (double)(orc_splitmix64(seed, k) >> 11) * 0x1.0p-53;
    return step * (2.0 * u - 1.0);
}

typedef int (*local_fn)(void *ctx, double *x, const orc_options *o, orc_result *r);

/* Monotonic basin hopping on top of a local minimizer (the construction of
 * Wales and Doye that Section 2 mentions, in its monotonic form): minimize
 * locally from x; then `hops` times perturb the best point coordinate by
 * coordinate (x_k + step * (2u - 1), counter hop * n + k), minimize locally
 * and keep the new point when its energy is lower (any finite result: a
 * converged run, a capped one, or one whose line search found no further
 * step).  res: the kept point's energy,
 * gradient norm and status; iterations and evaluations summed over all
 * local runs. */
static int mbh(int32_t n, local_fn local, void *ctx, double *x, const orc_options *o, int32_t hops,
               double step, uint64_t seed, orc_result *res, int32_t *accepted) {
    size_t nb = sizeof(double) * (size_t)n;
    double *best = malloc(nb), *trial = malloc(nb);
    orc_result r, rb;
    int32_t acc = 0, it = 0, ne = 0, neg = 0, lsf = 0;
    local(ctx, x, o, &rb);
    it += rb.iterations; ne += rb.energy_evals; neg += rb.grad_evals; lsf += rb.ls_failures;
    memcpy(best, x, nb);
    for (int32_t h = 0; h < hops; h++) {
        for (int32_t k = 0; k < n; k++)
            trial[k] = best[k] + mbh_offset(seed, (uint64_t)h * (uint64_t)n + (uint64_t)k, step);
        local(ctx, trial, o, &r);
        it += r.iterations; ne += r.energy_evals; neg += r.grad_evals; lsf += r.ls_failures;
        const int usable = r.status != ORC_NONFINITE && isfinite(r.energy);
        if (usable && (!isfinite(rb.energy) || r.energy < rb.energy)) {
            memcpy(best, trial, nb);
            rb = r;
            acc++;
        }
    }
    memcpy(x, best, nb);
    *res = rb;
    res->iterations = it;
    res->energy_evals = ne;
    res->grad_evals = neg;
    res->ls_failures = lsf;
    if (accepted) *accepted = acc;
    free(best);
    free(trial);
    return res->status;
}

typedef struct {
    int32_t n;
    orc_fg_fn fg;
    void *ctx;
} fn_ctx_t;
static int local_fn_generic(void *ctx, double *x, const orc_options *o, orc_result *r) {
    fn_ctx_t *c = (fn_ctx_t *)ctx;
    return orc_minimize(c->n, c->fg, c->ctx, x, o, r);
}
static int local_fn_ff(void *ctx, double *x, const orc_options *o, orc_result *r) {
    return orc_minimize_ff((const orc_ff *)ctx, x, o, r);
}

int orc_basin_hop(int32_t n, orc_fg_fn fg, void *ctx, double *x, const orc_options *o, int32_t hops,
                  double step, uint64_t seed, orc_result *res, int32_t *accepted) {
    fn_ctx_t c = {n, fg, ctx};
    return mbh(n, local_fn_generic, &c, x, o, hops, step, seed, res, accepted);
}

int orc_basin_hop_ff(const orc_ff *ff, double *x, const orc_options *o, int32_t hops, double step,
                     uint64_t seed, orc_result *res, int32_t *accepted) {
    return mbh(3 * ff->n_atoms, local_fn_ff, (void *)ff, x, o, hops, step, seed, res, accepted);
}
