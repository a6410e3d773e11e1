// Internal structures shared by the ffmin CUDA translation units.
//
// Layout in HBM (one batch of n_sys systems, atoms concatenated):
//   - vectors: V_NSLOT FP64 arrays of vstride doubles (3 per atom, xyz AoS):
//     current point X, gradient G, direction R, trial point XT and its
//     gradient GT, FGM's w / momentum / best point, the learned H0 diagonal
//     and the L-BFGS ring of (s, y) pairs (m + 1 physical slots each);
//   - pair-kernel inputs rewritten for every evaluation: per atom float4 or
//     double4_32a (x, y, z, q*sqrt(C)) and constant float2 / double2
//     (sigma, sqrt(24 eps));
//   - per-(tile, j-chunk) partial row sums of the pair kernel
//     ([n_items][TI] float4 or double4_32a: gx, gy, gz, row energy);
//   - bonded terms (FP64) with a per-atom incidence list, so that every
//     atom gathers its own bonded gradient without atomics;
//   - per-system control state (SysState) driven by the last block of the
//     per-tile kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ffmin.h"

namespace ffm {

constexpr int TI = 128;        // atoms per tile = threads of every per-tile kernel
constexpr int TJ = 128;        // j atoms staged per shared-memory tile in the pair kernel
constexpr int MAXM = 16;       // largest L-BFGS memory
constexpr int NRING = MAXM + 1;  // ring slots (m committed pairs + one staging slot)
constexpr int NRED = 2 * NRING + 4;  // reduction values per tile

enum Slot : int {
    V_X = 0, V_G, V_R, V_XT, V_GT, V_W, V_P, V_XB, V_D, V_XIN, V_X0, V_DS,
    V_S0, V_Y0 = V_S0 + NRING, V_NSLOT = V_Y0 + NRING
};

enum EvKind : int { EV_NONE = 0, EV_E = 1, EV_EG = 2 };

enum UpdKind : int {
    U_NONE = 0,
    U_ACCEPT,        // X <- XT, G <- GT
    U_PUSH,          // L-BFGS: s = XT - X, y = GT - G into the staging slot, dots, then ACCEPT
    U_FGM_W,         // W <- XT, G <- GT (optionally XB <- XT)
    U_FGM_ACCEPT,    // Xn = fma(h, R * inv, W); P <- Xn - X (0 on restart); X <- Xn (XB <- Xn)
    U_FGM_RESET,     // X <- W, P <- 0
    U_FGM_BEST_W,    // XB <- W
    U_OGM,           // OGM: (accept) X <- XT, G <- GT; (restart) X0 <- X, DS <- G, else
                     // (accept) DS += h G; then W = a X + b X0, R = -(a G + inv DS), <R, R>
    U_HB             // heavy ball: P <- X (start: P <- XT), X <- XT, G <- GT;
                     // then XT = fma(b, X - P, fma(-a, G, X)), the next iterate
};

enum Phase : int {
    PH_IDLE = 0, PH_START, PH_DIR, PH_LS, PH_ACCEPT, PH_FGM_W, PH_FINAL, PH_EVAL_ONLY, PH_DONE,
    PH_OGM_UPD, PH_OGM_Y, PH_HB
};

// a pair item (i-tile, j-chunk); tile < 0 marks a bonded item whose j0, nj
// is a range of bonded terms (of one type and one system, diag = system).
// Row-sweep lists (FP32, and FP64 when the symmetric list would not fit):
// every j of the system's row, slot unused.  Symmetric FP64 list: j-chunks
// of whole tiles at or right of the i-tile; the item writes its i-side
// partial rows to slot and the j-side rows of its q-th j-tile to slot + 1 + q.
struct Item { int32_t tile, j0, nj, diag, slot, pad0, pad1, pad2; };
constexpr int BONDED_ITEM_TERMS = 64;

// item0 / nitem: the tile's items in the row-sweep list; row64: its first
// item in the symmetric list (row of tile pairs (tile, J >= tile)), chunk64:
// j-tiles per symmetric item of its system, tloc: index inside its system;
// slot64: the partial-row slot of its row's first symmetric item (the row's
// items hold consecutive slots, 1 + chunk64 per item, so the q-th item of
// the row starts at slot64 + q * (1 + chunk64));
// xlo / xhi: the smallest and largest scaled partner (exclusion variant) of
// its atoms, xlo > xhi when there is none
struct Tile { int32_t sys, a0, na, item0, nitem, row64, chunk64, tloc, xlo, xhi, slot64, pad1; };

struct DirOp {
    int32_t on, use_d, dots;  // dots: 1 -> |R|^2, <G,R>; 2 -> <Y_j, R> for the Y list
    int32_t nS, nY;
    int32_t sS[NRING], sY[NRING];
    double a, b, outer;
    double cS[NRING], cY[NRING];
};

struct UpdOp {
    int32_t op, best, restart, stage;  // stage: physical ring slot for U_PUSH
    int32_t nS, sS[NRING];             // committed s slots (U_PUSH dots)
    int32_t accept;                    // U_OGM: the step to XT was accepted
    double h, inv, a, b;
};

struct SysState {
    // geometry of the system inside the batch
    int32_t atom0, natoms, tile0, ntile;
    // options
    int32_t method, cg_variant, ls, m, max_iter, max_evals, restart_every, K, g0, use_d;
    double gtol, h0_init, kplus, kminus, eps_h;
    // status and counters
    int32_t active, status, iter, ne, neg, lsf, fresh, phase;
    // current point
    double f, gg, ginf, rg;
    double h0, h_acc;
    // requests for the next kernels
    UpdOp upd;
    DirOp dir[2];
    int32_t ev_kind, ev_base, ev_dir, cg_check;
    double ev_h, ev_scale;
    // FP32 line-search trials are evaluated as energy differences from the
    // search's base point: E = epair_base + sum of pair differences + bonded
    int32_t ev_delta, delta_pad;
    double epair_last, epair_base;
    // line search
    int32_t ls_kind, ls_step, ls_k, ls_pad;
    double lh[4], lf[4], fstar, slope, rnorm, ls_f0, ls_h0v;
    // L-BFGS ring (physical slots 0..m): committed pairs oldest first
    int32_t ring_count, ring_pad;
    int32_t ring[NRING];
    double rho[NRING], yy[NRING];
    double SY[NRING][NRING];  // SY[a][b] = <s_a, y_b>, a older than b
    double sg[NRING];         // <s_a, g> at the current point
    double alpha[NRING];
    // FGM
    double th_prev, fx, fb, fw, xb_ginf;
    double ogm_t;  // OGM: t_k
    int32_t xb_known, result_slot;
    int32_t fgm_restart, fgm_pad;  // 1: function-value momentum restart (not in Algorithm 1)
    double hb_alpha, hb_beta;      // heavy ball (Eq. 8): constant step and momentum
    // result
    double res_f, res_ginf;
    // learned preconditioner in use for this run
    int32_t precond_on;
    // precision: mixed = 1 for a MIXED object; mode 0 = FP32 pair terms,
    // mode 1 = FP64 pair terms (the FP64 phase of a mixed run, or always)
    int32_t mixed, mode;
    int32_t iter_fp64_0;  // S.iter when the FP64 phase began (0: FP64 throughout)
    // learned-diagonal safeguard: every pc_window accepted steps with the
    // diagonal, E must have fallen by pc_rel |E| since the mark (pc_mark_*)
    // while |grad|_inf > pc_gfar * gtol, else the run continues without it
    int32_t pc_window, pc_mark_iter;
    double pc_rel, pc_gfar, pc_mark_f;
    // preconditioner: 1 when the current direction used the learned diagonal
    int32_t dir_used_d, rec_every;
    int32_t rec_slots, rec_pad;
    double *rec_ptr;
};

// FP32 -> FP64 hand-over of a MIXED run: when the FP32 |grad|_inf falls
// below this multiple of the tolerance (the FP64 phase then certifies the
// point); a failed FP32 line search also hands over
constexpr double MIXED_SWITCH_RATIO = 1.0;

// batches of at least this many systems reduce and run their control steps
// in k_sysreduce (one block per system); smaller ones in the last block of
// each per-tile kernel
constexpr int LB_MAX_SYS = 8;

struct Ctx {
    int32_t n_sys, n_tiles, n_items, n_atoms;
    int64_t vstride;
    int32_t prec;           // ffmin_precision
    int32_t sep_reduce;     // 1: per-system reductions + control in separate kernels (large batches)
    int32_t f32_ipt;        // FP32 pair-kernel shape: i-atoms per thread (1 or 2; host-side dispatch)
    const Tile *tiles;
    const Item *items;
    SysState *st;
    double *vec;            // [V_NSLOT][vstride]
    // pair kernel inputs / outputs
    float4 *posf;
    float4 *dispf;          // FP32 displacement of the trial point from the base (difference trials)
    const float2 *parf;
    double4_32a *posd;
    const double2 *pard;
    const double *qs;       // q * sqrt(C) per atom (FP64)
    float4 *gpf;            // [n_items][TI]
    float4 *gpf_sym;        // [slots of items64][TI]: FP32 energy-only rows (i-side) on the symmetric list
    double4_32a *gpd;
    // bonded terms
    const int32_t *inc_off; // [n_atoms + 1]
    const int2 *inc;        // x: (type << 2) | position, y: term index
    const int2 *bidx;
    const double2 *bpar;
    const int4 *aidx;
    const double2 *apar;
    const int4 *didx;
    const double4_32a *dpar;
    int32_t n_bonds, n_angles, n_terms, n_pair_items;  // batch totals
    int32_t n_dihedrals, n_excl;  // n_excl: exclusion corrections (type 3, after the dihedrals)
    const int2 *xidx;             // [n_excl] atom pair of each correction
    const double *xw;             // [n_excl] weight s_ij - 1 of its pair term
    // the same scaled pairs per atom (CSR: partners of atom a in
    // xs_part[xs_off[a] .. xs_off[a + 1]), scale s_ij in xs_val): the FP32
    // sweeps scale those pairs inside their sums (MIXED objects only)
    const int32_t *xs_off, *xs_part;
    const float *xs_val;
    const int32_t *term_sys;  // [n_terms] system of each bonded term
    const int2 *sys_items;  // [n_sys] (first, count) of each system's work items (contiguous)
    // FP64 pair terms: sym64 = 1 evaluates each unordered pair once
    // (symmetric tiles, list items64 / sys_items64, partial rows gpd
    // [slots][TI]); 0 uses the row sweep over items / sys_items
    int32_t sym64, n_items64;
    const Item *items64;
    const int2 *sys_items64;
    int32_t *act;           // per work queue L: [L * (2 n_sys + 2)]: active systems, their items,
                            // item prefix [n_sys], system ids [n_sys] (rebuilt every launch)
    double *te;             // [n_terms] energy of each bonded term
    double *tg;             // [2 nb + 3 na + 4 nd][3] gradient of each term at each position
    // reductions
    double *red;            // [n_tiles][NRED]
    unsigned int *counters; // one per kernel kind, reset by the last block
    int32_t *nactive;       // systems still minimizing
    int32_t *nmode;         // [2] active systems per pair-kernel precision mode
    // learned preconditioner features
    const float *feat;      // [n_atoms][3] (q, sigma, eps)
    int32_t *ncount;        // [n_atoms] neighbours within 8 A (pair kernel EG, optional)
    const uint16_t *mlp_w;  // 449 FP16 weights
};

inline __host__ __device__ double *vslot(const Ctx &c, int slot) { return c.vec + (int64_t)slot * c.vstride; }

// SplitMix64 (Steele, Lea and Flood 2014): the k-th output of the
// counter-based stream of `seed` (the gradient-free atom picker and the
// basin-hopping perturbations)
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// counters[] indices
enum { CNT_PAIR = 0, CNT_PAIR_EXIT = 1, CNT_FIN = 2, CNT_UPD = 3, CNT_DIR1 = 4, CNT_DIR2 = 5,
       CNT_PARAB = 6, CNT_PARAB2 = 7, CNT_PAIR64 = 8, CNT_PAIR64_EXIT = 9, CNT_PAIR32E = 10, CNT_N = 11 };

// work queues of the pair kernels (one active list each): FP32 E + grad,
// FP64 terms, FP32 energy only (plain and difference trials)
enum { LIST_F32_EG = 0, LIST_F64 = 1, LIST_F32_E = 2, N_LISTS = 3 };

// ---- launchers (defined in the .cu files) ----
cudaError_t launch_prepare(const Ctx &c, cudaStream_t s);
cudaError_t launch_ncount(const Ctx &c, const double *x, int32_t *out, cudaStream_t s);
// launches the FP32 kernel (MIXED objects) and the FP64 kernel; each skips
// the systems of the other precision mode and exits at once when none is
// in its mode
cudaError_t launch_pair(const Ctx &c, int grid32, int grid32e, int grid64, cudaStream_t s);
// side streams and events for parallel branches of one round: work forked
// from the main stream (event fork) and joined back (events join[k])
struct Branches {
    cudaStream_t side[2];
    cudaEvent_t fork, join[2];
};
cudaError_t launch_activelist(const Ctx &c, cudaStream_t s);
// the pair kernels alone (launch_pair = active lists, then these in turn);
// with br, the FP32 energy-only and FP64 kernels run on br's side streams
cudaError_t launch_pair_kernels(const Ctx &c, int grid32, int grid32e, int grid64, cudaStream_t s,
                                const Branches *br);
cudaError_t launch_finalize(const Ctx &c, cudaStream_t s);
cudaError_t launch_update(const Ctx &c, cudaStream_t s);
cudaError_t launch_dir(const Ctx &c, int which, cudaStream_t s);
// per-system reduction + control step after a stage (only when sep_reduce):
// stage 0 update, 1 / 2 direction passes, 3 finalize
cudaError_t launch_sysreduce(const Ctx &c, int stage, cudaStream_t s);
// basin hopping: out = best + step (2u - 1) per coordinate, u from the
// SplitMix64 stream of seed + b at counter hop * 3N_b + k (system b); and the
// copy of x into best for the systems whose flag is set
cudaError_t launch_mbh_perturb(const Ctx &c, const double *best, double *out, double step, uint64_t seed,
                               int64_t hop, cudaStream_t s);
cudaError_t launch_mbh_accept(const Ctx &c, const int32_t *flags, const double *x, double *best, cudaStream_t s);
// resident blocks of the pair kernel of a mode: 0 FP32 E + grad row sweep,
// 1 FP64 row sweep, 2 FP64 symmetric tiles, 3 FP32 energy only
int pair_grid_size(int mode, int f32_ipt = 2);

// arguments of one epoch of the parallel gradient-free search (one block
// per part, each on its own copy of the positions)
struct EpochArgs {
    double *view;           // [P][3N] FP64 positions of each part's copy
    float4 *viewf;          // [P][N] FP32 (x, y, z, q') copies (MIXED)
    const int32_t *list;    // movable atoms of every part, concatenated
    const int32_t *loff;    // [P + 1] offsets into list
    const int32_t *allowed; // [P] moves of each part in this epoch
    const int32_t *members; // atoms of every part, concatenated
    const int32_t *moff;    // [P + 1] offsets into members
    int n, mode;
    uint64_t seed, epoch;
    double delta;
    double taylor_r2;       // squared far-field radius of the linearised Coulomb rows, 0 = exact
};

}  // namespace ffm
