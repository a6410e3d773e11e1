/*
 * ffmin — all-pairs force-field energy, gradient and local minimization on
 * NVIDIA GB300 (sm_103a).  C ABI.
 *
 * The operations follow arXiv 1810.03358 ("Algorithms for local minimization
 * of a force field for 3D macromolecules"):
 *   - energy: Section 2, E = E_stretch + E_bend + E_torsion + E_cul + E_vdw,
 *     non-bonded terms over ALL atom pairs (no exclusions, unless a topology
 *     asks for the exclusion variant, which the paper does not have),
 *     explicit gradient;
 *   - minimizers: Section 5.1, Algorithms 1 (FGM), 2 (CG), 3-4 (L-BFGS);
 *     adaptive gradient descent of Section 3 (Eq. 4 with a parabolic step);
 *     the gradient-free random-atom "parab" moves of Section 3, one atom at
 *     a time or in parallel epochs (Section 3's proposal); the optimized
 *     gradient method of Section 4 (Eq. 11) with a line search;
 *   - line searches: Section 5.2, Algorithms 5 (LS_H) and 6 (LS_PAR).
 *
 * Conventions
 *   - Coordinates are FP64, xyz per atom, [3N] contiguous (AoS), in A.
 *     Energies in kcal/mol, gradients in kcal/mol/A.
 *   - "_dev" pointers are device pointers the caller owns (e.g. torch
 *     tensors); "_host" pointers are host memory the caller owns.  The
 *     library owns all workspace inside the opaque ffmin_system.
 *   - All GPU work is enqueued on the stream given at ffmin_create; every
 *     call that returns results to host memory synchronizes that stream.
 *   - No function aborts or exits.  Errors are returned as ffmin_status; a
 *     CUDA error is latched in the system, which then refuses further work.
 *     ffmin_last_error() gives a one-line message.
 *   - There is no CPU fallback: every computation runs in CUDA kernels.
 */
#ifndef FFMIN_H
#define FFMIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FFMIN_OK = 0,
    FFMIN_ERR_INVALID_ARG = 1,
    FFMIN_ERR_CUDA = 2,
    FFMIN_ERR_NONFINITE = 3,   /* coincident atoms, or a non-finite E or gradient */
    FFMIN_ERR_LINESEARCH = 4,  /* no relaxing step, even after one restart (Section 5.1) */
    FFMIN_ERR_MAX_ITER = 5,    /* iteration or evaluation budget used up */
    FFMIN_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    FFMIN_ERR_OOM = 7
} ffmin_status;

/* GD: adaptive steepest descent (Section 3, Eq. 4); FGM: Algorithm 1 (see
 * options.fgm_restart); CG:
 * Algorithm 2; LBFGS: Algorithms 3-4; GRADFREE: random-atom parabolic moves
 * (Section 3); OGM: the optimized gradient method of Section 4 (Eq. 11) with
 * the step 1/L replaced by a line search from y (LS_PAR with G0 by default),
 * the gradient evaluated at y and at every x^k, t_0 = 1, no momentum restart
 * except after a failed line search; HB: the heavy-ball method of Section 4
 * (Eq. 8) with constant step options.hb_alpha and momentum options.hb_beta,
 * x^{-1} = x^0, no line search (one E + grad per step). */
typedef enum {
    FFMIN_GD = 0, FFMIN_FGM = 1, FFMIN_CG = 2, FFMIN_LBFGS = 3, FFMIN_GRADFREE = 4, FFMIN_OGM = 5,
    FFMIN_HB = 6
} ffmin_method;

/* beta of CG (Section 5.1; Andrei 2008): d = previous unnormalised
 * direction, y = g+ - g.  PRP g+.y/|g|^2, HS g+.y/d.y, FR |g+|^2/|g|^2,
 * PRP+ max(0, PRP), CD |g+|^2/(-d.g), LS g+.y/(-d.g), DY |g+|^2/d.y. */
typedef enum {
    FFMIN_CG_PRP = 0, FFMIN_CG_HS, FFMIN_CG_FR, FFMIN_CG_PRP_PLUS,
    FFMIN_CG_CD, FFMIN_CG_LS, FFMIN_CG_DY
} ffmin_cg_variant;

/* DEFAULT = LS_H for FGM, LS_PAR for GD, CG and L-BFGS. */
typedef enum { FFMIN_LS_DEFAULT = 0, FFMIN_LS_H = 1, FFMIN_LS_PAR = 2 } ffmin_linesearch;

/* FP64: every pair term in FP64.  MIXED: pair terms in FP32 with FP32
 * accumulation inside a j-chunk; per-atom sums, energy totals, the line
 * search, every dot product and all vector updates stay FP64. */
typedef enum { FFMIN_FP64 = 0, FFMIN_MIXED = 1 } ffmin_precision;

/* One system (host arrays, FP64 / int32, copied at ffmin_create; the
 * caller keeps ownership).  Atom indices are 0-based within the system. */
typedef struct {
    int32_t n_atoms;
    const double *charge, *sigma, *epsilon;            /* [N] e, A, kcal/mol */
    int32_t n_bonds;
    const int32_t *bond_idx;                           /* [nb*2] */
    const double *bond_k, *bond_r0;                    /* [nb] E = K (r - r0)^2 */
    int32_t n_angles;
    const int32_t *angle_idx;                          /* [na*3], vertex in the middle */
    const double *angle_k, *angle_theta0;              /* [na] E = K (theta - theta0)^2, rad */
    int32_t n_dihedrals;
    const int32_t *dihedral_idx;                       /* [nd*4] */
    const double *dihedral_v;                          /* [nd*4] V1..V4 */
    double coulomb_c;  /* 0 -> 332.0716 kcal*A/(mol*e^2) = 1389.38757 / 4.184 (Section 2) */
    /* 0: every pair interacts (Section 2).  1: a force-field variant, not in
     * the paper: pairs joined by a bond or by the ends of an angle are
     * excluded, the end atoms of a dihedral interact scaled by scale14
     * (finite, >= 0).  FP64 pair terms: FP64 correction terms (weight s - 1
     * on the pair term) beside the all-pairs sweep.  FP32 pair terms (MIXED):
     * the sweeps scale the listed pairs inside their sums (an FP32
     * correction could not cancel the rounding of the excluded clashes); the
     * MIXED gradient-free search refuses the variant. */
    int32_t exclusions;
    double scale14;
} ffmin_topology;

typedef struct {
    int32_t method;          /* ffmin_method, default FFMIN_LBFGS */
    int32_t cg_variant;      /* ffmin_cg_variant, default PRP */
    int32_t ls;              /* ffmin_linesearch, default DEFAULT */
    int32_t lbfgs_m;         /* history pairs, 1..16, default 10 */
    double gtol_inf;         /* stop when max_k |dE/dx_k| < gtol_inf; default 0.1 kcal/mol/A */
    int32_t max_iter;        /* accepted steps (GRADFREE: atom moves), default 100000 */
    int32_t max_evals;       /* energy + gradient evaluations, default 1000000 */
    int32_t cg_restart_every;/* 0 -> 3N */
    double h0;               /* first trial step (A), default 0.1 */
    double k_plus, k_minus;  /* step growth / shrink factors, default 2 and 0.5 */
    double eps_h;            /* LS_H smallest step, default 1e-10 */
    int32_t ls_par_K;        /* LS_PAR refinement bound K >= 2, default 2 */
    int32_t ls_par_g0;       /* LS_PAR uses the slope at 0 (G0), default 1 */
    double gradfree_delta;   /* GRADFREE axis offset (A), default 0.05 */
    uint64_t seed;           /* GRADFREE atom picker seed (SplitMix64 stream) */
    /* GRADFREE, 0 (default): one atom at a time (Section 3).  P >= 1: parallel
     * epochs (Section 3's proposal): each epoch cuts the system into P parts
     * by recursive bisection at randomly shifted median ranks, every part
     * moves its atoms that lie at least gradfree_margin A (default 1.0) from
     * its cut planes on its own copy of the epoch's starting positions, one
     * CUDA block per part; the parts are merged and the gradient checked
     * after every epoch.  P = 1 is the sequential method. */
    int32_t gradfree_parts;
    double gradfree_margin;
    int32_t use_learned_precond; /* L-BFGS: scale H0 by the learned per-atom diagonal */
    /* Bound on device evaluation rounds (each round evaluates at most one E
     * or E + grad per system; rounds run in groups of 8); 0 -> max_evals + 64.
     * A system still running when it is reached stops with
     * FFMIN_ERR_TIMEOUT: x then holds its last accepted point (FGM: its best
     * point), energy that point's energy (from the pair terms of the current
     * precision phase) and grad_inf its |grad|_inf (NaN for FGM when that
     * gradient was never evaluated). */
    int32_t max_ticks;
    /* L-BFGS trajectory recording (training data of the preconditioner):
     * when record_dev != NULL, after every record_every-th accepted step k
     * (slot k / record_every - 1 < record_slots) every atom i of every system
     * writes (<s_i, y_i>, <y_i, y_i>, |grad_i| before the step, 1) to
     * record_dev[(slot * total_atoms + i) * 4 + 0..3] (device, FP64). */
    double *record_dev;
    int32_t record_every, record_slots;
    /* FGM: 0 (default) runs Algorithm 1 as printed (non-monotone, no
     * momentum restart; the best point is returned); 1 adds the
     * function-value adaptive restart of O'Donoghue and Candes (theta <- 1,
     * momentum dropped whenever f(x^{k+1}) > f(x^k)), which Algorithm 1 does
     * not have. */
    int32_t fgm_restart;
    /* HB (Eq. 8): x^{k+1} = x^k - hb_alpha grad f(x^k) + hb_beta (x^k - x^{k-1});
     * hb_alpha > 0 (A^2 mol/kcal), hb_beta >= 0; defaults 1e-4 and 0.5.  A
     * non-finite evaluation stops the run at the last finite iterate. */
    double hb_alpha, hb_beta;
    /* GRADFREE: r_far > 0 replaces the Coulomb term of every atom at least
     * r_far A from the moving atom's current position by its first-order
     * Taylor expansion about that position (Section 3's linearised far
     * field; Lennard-Jones stays exact); 0 (default): exact rows. */
    double gradfree_taylor_r;
    /* 0 (default): a minimization is one launch of a CUDA graph whose
     * conditional WHILE node repeats the pipeline rounds on the device.  1:
     * the host replays the same rounds (a graph of 8) and checks for active
     * systems after each replay: the same work and results, for profilers
     * that cannot look into conditional graph nodes. */
    int32_t host_loop;
    /* L-BFGS with the learned diagonal (not in the paper): every pc_window
     * accepted steps (default 200; 0: never) the run compares E with its
     * value pc_window steps earlier; if it fell by less than pc_rel |E|
     * (default 1e-5) while |grad E|_inf > pc_gfar * gtol_inf (default 100),
     * the rest of the run is plain L-BFGS (an energy stalled far from a
     * stationary point).  The FP64 phase of a MIXED run starts a new count. */
    int32_t pc_window;
    double pc_rel, pc_gfar;
} ffmin_options;

typedef struct {
    double energy;           /* E at the returned point */
    double grad_inf;         /* max_k |dE/dx_k| at the returned point */
    int32_t iterations;      /* accepted steps (GRADFREE: moves) */
    int32_t energy_evals;    /* energy-only evaluations (GRADFREE: row evaluations) */
    int32_t grad_evals;      /* energy + gradient evaluations */
    int32_t ls_failures;
    int32_t stop_reason;     /* ffmin_status: OK when converged */
    int32_t fp64_iterations; /* accepted steps taken with FP64 pair terms: all of
                                them for FP64, the FP64 phase of a MIXED run
                                (0 for MIXED gradient-free runs) */
} ffmin_result;

typedef struct ffmin_system ffmin_system;

/* Fill *o with the defaults above. */
void ffmin_options_default(ffmin_options *o);

/* Human-readable name of a status. */
const char *ffmin_status_string(ffmin_status s);

/* Create a batch of n_sys >= 1 systems (their atoms are concatenated in
 * the order given: system b owns atoms [A_b, A_b + N_b) of every
 * coordinate / gradient buffer).  precision: ffmin_precision.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: INVALID_ARG (bad counts or indices), OOM, CUDA. */
ffmin_status ffmin_create(const ffmin_topology *systems, int32_t n_sys, int32_t precision,
                          void *cuda_stream, ffmin_system **out);

/* Free every device and host resource of the system. */
ffmin_status ffmin_destroy(ffmin_system *sys);

/* Total atom count over the batch; per-system atom offset of system b. */
int64_t ffmin_n_atoms(const ffmin_system *sys);
int64_t ffmin_atom_offset(const ffmin_system *sys, int32_t b);

/* Energy of every system at x_dev [3 * total atoms] (device, FP64):
 * e_host[n_sys].  Section 2.  Synchronizes the stream. */
ffmin_status ffmin_energy(ffmin_system *sys, const double *x_dev, double *e_host);

/* Energy and gradient: e_host[n_sys], g_dev [3 * total atoms] (device). */
ffmin_status ffmin_energy_grad(ffmin_system *sys, const double *x_dev, double *e_host,
                               double *g_dev);

/* Same with host buffers: copies x_host to the device, evaluates, and
 * copies the gradient back to g_host (pass NULL to skip it). */
ffmin_status ffmin_energy_grad_host(ffmin_system *sys, const double *x_host, double *e_host,
                                    double *g_host);

/* Energy change of a line-search trial, evaluated the way the minimizers
 * evaluate it (Section 5.2's searches compare f(x + h r) with f(x)):
 * de_host[b] = E_b(x + h r) - E_b(x) for every system, x_dev and r_dev
 * [3 * total atoms] (device, FP64; r is used as given, not normalised).
 * FFMIN_FP64: the difference of two FP64 energies.  FFMIN_MIXED: x is
 * evaluated with E + grad (FP32 pair terms), then the trial with every pair
 * term taken as an exact FP32 difference from x (the form of every MIXED
 * energy-only trial) and the bonded terms in FP64.  Errors: INVALID_ARG,
 * NONFINITE (coincident atoms at x or at the trial).  Synchronizes the
 * stream.  A diagnostic of the trials' accuracy. */
ffmin_status ffmin_energy_delta(ffmin_system *sys, const double *x_dev, const double *r_dev, double h,
                                double *de_host);

/* Minimize every system of the batch from x_dev (device, in/out): on
 * return x_dev holds each system's result and results[n_sys] its record.
 * The call's status is FFMIN_OK when it ran; each system's own outcome is
 * in results[b].stop_reason.  method GRADFREE requires n_sys == 1. */
ffmin_status ffmin_minimize(ffmin_system *sys, double *x_dev, const ffmin_options *opt,
                            ffmin_result *results);

/* Monotonic basin hopping (the construction of Wales and Doye that Section 2
 * mentions as a way to deeper minima, in its monotonic form) on top of the
 * local minimizer of opt, every system of the batch at once: minimize
 * locally from x_dev; then hops times perturb each system's best point
 * coordinate by coordinate by step * (2u - 1) (A), u = (SplitMix64(seed + b,
 * h * 3N_b + k) >> 11) * 2^-53 for coordinate k of system b at hop h,
 * minimize all systems locally together, and keep each system's new point
 * when its energy is lower (any finite result).  x_dev (device, in/out):
 * the kept points; results[b]: the kept point's energy, |grad|_inf and
 * stop reason, with iterations and evaluations summed over all local runs;
 * accepted_host[b] (optional): hops kept.  GRADFREE needs one system. */
ffmin_status ffmin_basin_hop(ffmin_system *sys, double *x_dev, const ffmin_options *opt, int32_t hops,
                             double step, uint64_t seed, ffmin_result *results, int32_t *accepted_host);

/* Same with a host coordinate buffer (copied in and out). */
ffmin_status ffmin_minimize_host(ffmin_system *sys, double *x_host, const ffmin_options *opt,
                                 ffmin_result *results);

/* Learned L-BFGS preconditioner: a per-atom MLP 5 -> 64 -> 1 (ReLU hidden
 * layer) with FP16 weights, applied when options.use_learned_precond is set.
 * w_fp16 holds 449 half-precision values: W1 [64][5], b1 [64], W2 [64], b2.
 * Features per atom: q, sigma, epsilon, n(8 A)/64, log(1 + |g_i|).
 * H0 = gamma * diag(exp(clamp(z_i, -3, 3))) over the atom's 3 coordinates.
 * The paper has no counterpart; this is an extension of Algorithm 3. */
ffmin_status ffmin_set_precond(ffmin_system *sys, const uint16_t *w_fp16_host, int32_t n_params);

/* Neighbour counts: counts_dev[i] = number of atoms j != i of i's system
 * with |x_i - x_j| < 8 A at x_dev (device), a feature of the
 * preconditioner network.  Not in the paper. */
ffmin_status ffmin_neighbour_counts(ffmin_system *sys, const double *x_dev, int32_t *counts_dev);

/* Train the preconditioner network on the GPU (hand-written forward,
 * backward and Adam kernels, FP32): steps Adam steps (learning rate lr) on
 * minibatches of `batch` rows drawn from n_samples rows of feat_dev
 * [n][5] / target_dev [n] (device) with the SplitMix64 stream of `seed`;
 * loss = mean (z - t)^2.  w32_dev [449] FP32 weights (in/out), adam_dev
 * [898] moment estimates (in/out, zero at the start), work_dev
 * [ffmin_mlp_work_floats()] scratch, loss_host [steps] (optional) the
 * minibatch losses, w16_dev [449] (optional) FP16 weights out.  steps = 0
 * computes the mean-loss gradient over the first min(batch, n) rows into
 * work_dev[work - 449 .. work) without updating.  Synchronizes the stream. */
ffmin_status ffmin_mlp_train(const float *feat_dev, const float *target_dev, int64_t n_samples,
                             int32_t steps, int32_t batch, float lr, uint64_t seed, float *w32_dev,
                             float *adam_dev, float *work_dev, float *loss_host, uint16_t *w16_dev,
                             void *cuda_stream);
int64_t ffmin_mlp_work_floats(void);

/* Autotuner: for each candidate work-item layout (3, 6, 10 or 20 items per
 * resident pair-kernel block, which sets the j-chunk length of the row
 * sweep's (i-tile, j-chunk) items and the number of j-tiles per item of the
 * symmetric tiles) and, for MIXED objects, each FP32 pair-kernel tile shape
 * (two i-atoms per thread in 64-thread blocks, or one in 128-thread
 * blocks), time the pair kernels at x_dev (one energy + gradient launch
 * plus three energy-only launches, an L-BFGS step's mix) and keep the
 * fastest; *density_out = the chosen items per block (ffmin_get_tuning
 * reports the shape too).  The defaults before any call are 10 items per
 * block and two i-atoms per thread.  Synchronizes.  Not in the paper. */
ffmin_status ffmin_autotune(ffmin_system *sys, const double *x_dev, int32_t *density_out);

/* Install a layout without timing (e.g. one an earlier ffmin_autotune chose
 * for the same batch): density in [1, 20] items per resident block,
 * f32_atoms_per_thread 1 or 2 (the FP32 tile shape; FP64 objects ignore
 * it).  Results do not depend on either, up to the rounding of the FP32
 * partial sums.  INVALID_ARG otherwise.  Synchronizes. */
ffmin_status ffmin_set_tuning(ffmin_system *sys, int32_t density, int32_t f32_atoms_per_thread);
/* The installed layout: items per resident block and FP32 i-atoms per thread. */
ffmin_status ffmin_get_tuning(const ffmin_system *sys, int32_t *density, int32_t *f32_atoms_per_thread);

/* Time the dominant pair kernel alone: reps launches at x_dev with forces
 * (with_grad = 1), energy only (0), or as a MIXED line-search difference
 * trial (2), CUDA events on the system's stream; *ms = mean duration of one
 * launch.  Diagnostic for roofline reporting. */
ffmin_status ffmin_time_pair_kernel(ffmin_system *sys, const double *x_dev, int32_t with_grad,
                                    int32_t reps, float *ms);

/* The parts of one epoch of the parallel gradient-free search, computed on
 * the host exactly as ffmin_minimize cuts them (see gradfree_parts):
 * part_out[a] = part of atom a (parts numbered left first in the bisection),
 * movable_out[a] = 1 when atom a is at least margin A from every cut plane
 * of its part.  x_host: [3n] positions; no device work.  Not in the paper. */
ffmin_status ffmin_epoch_parts(const double *x_host, int32_t n, int32_t parts, uint64_t seed,
                               uint64_t epoch, double margin, int32_t *part_out, int32_t *movable_out);

/* Measured ALU peak of the current device in TFLOP/s (FMA = 2 flops):
 * independent FP32 (precision = FFMIN_MIXED) or FP64 (FFMIN_FP64) FMA
 * chains on every SM, reps timed launches on the default stream after three
 * warm-up launches.  Allocates and frees a small output buffer.  The
 * denominator of the pair kernels' roofline; not part of the paper. */
ffmin_status ffmin_alu_peak(int32_t precision, int32_t reps, double *tflops);

/* Work done by the last ffmin_minimize: pair kernel launches and device
 * evaluation rounds; n_kernel_launches counts every kernel launched. */
ffmin_status ffmin_last_stats(const ffmin_system *sys, int64_t *ticks,
                              int64_t *n_kernel_launches, int64_t *pair_interactions);

/* Allocation-free non-bonded energy and gradient (no counterpart in the
 * paper: an interface for callers that cannot let a library allocate device
 * memory, such as an application confined to another framework's capped
 * memory pool, or a latency-bound loop that cannot afford cudaMalloc's
 * implicit device synchronisation).  Computes, in FP64, the Coulomb +
 * Lennard-Jones energy over all atom pairs of ONE system (no bonded terms)
 * and its gradient.  All buffers are the caller's device memory:
 *   x_dev [3N] xyz per atom; charge_dev, sigma_dev, epsilon_dev [N];
 *   g_dev [3N] gradient out; e_dev [1] energy out.
 * coulomb_c: 0 -> 332.0716 kcal*A/(mol*e^2); negative or non-finite ->
 * FFMIN_ERR_INVALID_ARG.  Work is enqueued on cuda_stream (NULL = legacy
 * default stream); the call then synchronises that stream to read its
 * status: FFMIN_ERR_NONFINITE when the energy or a gradient component is not
 * finite (two coincident atoms), else FFMIN_OK.
 * Scratch: a fixed device array inside the library (about 2 MB, held by
 * every GPU that loads the library until the process exits); n_atoms above
 * 8192 returns FFMIN_ERR_INVALID_ARG.  The first call on each device looks
 * up the array's device address in the device's primary context and keeps
 * it, so make that first call before any stream capture, and do not use
 * the entry point after cudaDeviceReset or from a non-primary context.
 * Every call uses the same array: calls that overlap on the GPU (concurrent
 * streams) race; serialise them.  No cudaMalloc or cudaFree is ever
 * called. */
ffmin_status ffmin_pair_energy_grad_noalloc(const double *x_dev, const double *charge_dev,
                                            const double *sigma_dev, const double *epsilon_dev,
                                            int32_t n_atoms, double coulomb_c, double *g_dev,
                                            double *e_dev, void *cuda_stream);

/* Last error message of the system (or of the last failed create). */
const char *ffmin_last_error(const ffmin_system *sys);

#ifdef __cplusplus
}
#endif
#endif
