/*
 * FP64 CPU oracle for the force-field minimization of arXiv 1810.03358.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of what the paper computes: the OPLS-style energy and its
 * analytic gradient (Section 2), the line searches LS_H and LS_PAR
 * (Section 5.2, Algorithms 5 and 6), the minimizers FGM, CG and L-BFGS
 * (Section 5.1, Algorithms 1-4), adaptive gradient descent (Section 3,
 * Eq. 4) and the gradient-free "parab" atom moves (Section 3).  It shares no
 * code with the CUDA library; only tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load it.
 *
 * Everything is FP64, single-threaded, with no blocking or reordering beyond
 * what the definitions state.  Built with -ffp-contract=off so that a*b+c is
 * two roundings unless fma() is written explicitly.
 */
#ifndef FFMIN_ORACLE_H
#define FFMIN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Force-field description (host arrays, borrowed). */
typedef struct {
    int32_t n_atoms;
    const double *charge, *sigma, *epsilon;          /* [N] */
    int32_t n_bonds;
    const int32_t *bond_idx;                         /* [nb*2] */
    const double *bond_k, *bond_r0;                  /* [nb] */
    int32_t n_angles;
    const int32_t *angle_idx;                        /* [na*3], vertex in the middle */
    const double *angle_k, *angle_theta0;            /* [na], theta0 in radians */
    int32_t n_dihedrals;
    const int32_t *dihedral_idx;                     /* [nd*4] */
    const double *dihedral_v;                        /* [nd*4] V1..V4 */
    double coulomb_c;
    /* 0: every pair interacts (Section 2).  1: a force-field variant (not in
     * the paper): pairs joined by a bond or by the ends of an angle are
     * excluded, the end atoms of a dihedral interact scaled by scale14. */
    int32_t exclusions;
    double scale14;
} orc_ff;

/* Energy split by term plus the sum of |term| over every term and pair. */
typedef struct {
    double stretch, bend, torsion, coulomb, vdw, total, sum_abs;
    int32_t degenerate_dihedrals;
} orc_terms;

/* Return codes. */
enum { ORC_OK = 0, ORC_NONFINITE = 1, ORC_LINESEARCH = 2, ORC_MAX_ITER = 3, ORC_BAD_ARG = 4 };

/* Energy (and gradient if grad != NULL, [3N]) at x [3N] (xyz per atom).
 * Returns ORC_OK, or ORC_NONFINITE when two atoms coincide or a value is
 * not finite. */
int orc_energy_terms(const orc_ff *ff, const double *x, double *grad, orc_terms *out);

/* orc_energy_terms restricted to the pairs (i, j), i < j, with i in [i0, i1)
 * (plus the bonded terms when i0 == 0); the gradient of these terms is ADDED
 * into grad [3N] (may be NULL).  The blocks of a partition of [0, N) sum to
 * the whole energy and gradient: independent workers may split the rows. */
int orc_energy_rows(const orc_ff *ff, const double *x, int32_t i0, int32_t i1, double *grad,
                    orc_terms *out);

/* E(xp) - E(x) summed term by term (each term at xp minus itself at x),
 * *sum_abs = sum over terms of |difference|: the definition of a line-search
 * trial's energy change.  Pairs (i, j), i < j, with i in [i0, i1); the
 * bonded terms only when i0 == 0 (callers may split the rows). */
int orc_energy_delta(const orc_ff *ff, const double *x, const double *xp, int32_t i0, int32_t i1,
                     double *delta, double *sum_abs);

/* Energy of every term that contains atom i, with atom i placed at p[3]
 * and every other atom at x: the part of E that changes when only atom i
 * moves (pair terms with i plus bonded terms containing i). */
double orc_row_energy(const orc_ff *ff, const double *x, int32_t i, const double p[3]);

/* The same with the Coulomb terms of every atom at least r_far from x_i
 * replaced by their first-order Taylor expansion about x_i (Section 3's
 * amortised construction for the gradient-free moves); r_far = +inf gives
 * orc_row_energy. */
double orc_row_energy_taylor(const orc_ff *ff, const double *x, int32_t i, const double p[3],
                             double r_far);

/* Gradient of E with respect to atom i alone (g3[3]); pair row plus the
 * bonded terms that contain atom i. */
int orc_atom_gradient(const orc_ff *ff, const double *x, int32_t i, double *g3);

/* Neighbour count of atom i: atoms j != i with |x_i - x_j| < rc. */
int32_t orc_neighbour_count(const orc_ff *ff, const double *x, int32_t i, double rc);

/* ---- generic objective for the minimizers -------------------------------- */
/* f(x); writes the gradient when g != NULL; *status != 0 on failure. */
typedef double (*orc_fg_fn)(void *ctx, const double *x, double *g, int32_t *status);

/* 1-D function phi(h) for the line searches. */
typedef double (*orc_line_fn)(void *ctx, double h);

/* LS_H (Algorithm 5).  f_star = phi(0).  Returns the step (0 on failure);
 * *f_out = phi(step) (f_star on failure); *n_evals = phi calls made. */
double orc_ls_h(orc_line_fn phi, void *ctx, double f_star, double h0, double eps_h,
                double k_plus, double k_minus, double *f_out, int32_t *n_evals);

/* LS_PAR (Algorithm 6).  slope = phi'(0) (used when g0 != 0).  k_plus and
 * the clamp of 8 x max|h| handle degenerate parabolas (the paper is silent). */
double orc_ls_par(orc_line_fn phi, void *ctx, double f_star, double slope, double h0,
                  int32_t K, int32_t g0, double k_plus, double *f_out, int32_t *n_evals);

/* Minimizer options / results. */
enum { ORC_GD = 0, ORC_FGM = 1, ORC_CG = 2, ORC_LBFGS = 3, ORC_GRADFREE = 4, ORC_OGM = 5, ORC_HB = 6 };
enum { ORC_CG_PRP = 0, ORC_CG_HS, ORC_CG_FR, ORC_CG_PRP_PLUS, ORC_CG_CD, ORC_CG_LS, ORC_CG_DY };
enum { ORC_LS_DEFAULT = 0, ORC_LS_H = 1, ORC_LS_PAR = 2 };

typedef struct {
    int32_t method, cg_variant, ls, lbfgs_m;
    double gtol_inf;
    int32_t max_iter, max_evals, cg_restart_every;
    double h0, k_plus, k_minus, eps_h;
    int32_t ls_par_K, ls_par_g0;
    double gradfree_delta;
    uint64_t seed;
    /* gradient-free search: 0 = one atom at a time (Section 3); P >= 1 =
     * parallel epochs over P slabs (Section 3's proposal), atoms closer
     * than gradfree_margin A to a slab boundary stay put in that epoch */
    int32_t gradfree_parts;
    double gradfree_margin;
    double gradfree_taylor_r;  /* > 0: moves use orc_row_energy_taylor with this r_far */
    const double *precond_d;   /* optional fixed per-variable H0 diagonal [n] (L-BFGS) */
    const double *mlp_w;       /* optional network [ORC_MLP_NW]: H0 diagonal per iteration (force field) */
    double ogm_step;           /* OGM: fixed step 1/L instead of the line search when > 0 (tests) */
    double hb_alpha, hb_beta;  /* heavy ball (Eq. 8): constant step alpha > 0 and momentum beta >= 0 */
    int32_t fgm_restart;       /* FGM: 1 adds the function-value momentum restart (not in Algorithm 1) */
    double fgm_step;           /* FGM: fixed step 1/L instead of the line search when > 0 (tests) */
    /* L-BFGS with mlp_w (not in the paper): every pc_window accepted steps
     * (0: never) E is compared with its value at the last check (first: the
     * start); if it fell by less than pc_rel |E| while |grad|_inf >
     * pc_gfar * gtol_inf, the rest of the run is plain L-BFGS */
    int32_t pc_window;
    double pc_rel, pc_gfar;
} orc_options;

typedef struct {
    double energy, grad_inf;
    int32_t iterations, energy_evals, grad_evals, ls_failures, status;
} orc_result;

void orc_options_default(orc_options *o);

/* Minimize a generic objective of n variables in place. */
int orc_minimize(int32_t n, orc_fg_fn fg, void *ctx, double *x, const orc_options *o,
                 orc_result *res);

/* Minimize the force field in place (every method, including GRADFREE). */
int orc_minimize_ff(const orc_ff *ff, double *x, const orc_options *o, orc_result *res);

/* Monotonic basin hopping (the construction of Wales and Doye that Section 2
 * mentions, monotonic form) on top of the local minimizer of `o`: minimize
 * from x; then hops times perturb the best point coordinate by coordinate
 * by step * (2u - 1), u = (SplitMix64(seed, h * n + k) >> 11) * 2^-53,
 * minimize locally and keep the result when its energy is lower (any
 * finite result).  x: the kept point on return; res:
 * its energy, gradient norm and status with iterations and evaluations
 * summed over all local runs; *accepted: hops kept. */
int orc_basin_hop(int32_t n, orc_fg_fn fg, void *ctx, double *x, const orc_options *o, int32_t hops,
                  double step, uint64_t seed, orc_result *res, int32_t *accepted);
int orc_basin_hop_ff(const orc_ff *ff, double *x, const orc_options *o, int32_t hops, double step,
                     uint64_t seed, orc_result *res, int32_t *accepted);

/* Optional per-iteration trace of the last orc_minimize* call (f after each
 * accepted step, step length, FGM theta and beta).  Returns entries copied. */
int32_t orc_trace(double *f, double *h, double *theta, double *beta, int32_t cap);

/* L-BFGS direction (Algorithm 3): r = -H g from `count` stored pairs given
 * oldest first (s[k*n..], y[k*n..]); d is an optional H0 diagonal. */
void orc_lbfgs_direction(int32_t n, const double *g, int32_t count, const double *s,
                         const double *y, const double *d, double *r);

/* ---- preconditioner network (not in the paper) ---- */
#define ORC_MLP_NW 449
double orc_mlp_forward(const double *w, const double *f, double *h);
double orc_mlp_loss_grad(const double *w, const double *feat, const double *target, int64_t n,
                         double *grad);
void orc_mlp_features(double q, double sigma, double eps, int32_t n8, double gnorm, double *f);
void orc_precond_diag(const orc_ff *ff, const double *w, const int32_t *n8, const double *g, double *d);

/* SplitMix64 (Steele, Lea, Flood 2014): the k-th output of the counter-based
 * stream with the given seed, and the atom it picks among n. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k);
int32_t orc_pick_atom(uint64_t seed, uint64_t k, int32_t n);

#ifdef __cplusplus
}
#endif
#endif
