// C ABI of the ffmin library (declared in include/ffmin.h): creation of a
// batch of systems, energy / gradient evaluation and the minimization driver.
//
// The driver keeps every decision on the device: a minimization is one
// launch of a CUDA graph whose conditional WHILE node repeats a body of
// TICKS_PER_GRAPH pipeline rounds (update, two direction passes, prepare,
// pair, finalize) until no system is active or the round bound is reached;
// where the runtime cannot build that graph, the host replays the body graph
// and reads back the count of still-active systems after each replay.
#include <algorithm>
#include <array>
#include <limits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ffmin_internal.cuh"

using namespace ffm;

// NVTX range over one entry point (visible to profilers; no cost otherwise)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// work-item densities (items per resident pair-kernel block) the autotuner tries
static const int AUTOTUNE_DENSITIES[] = {3, 6, 10, 20};
static const int AUTOTUNE_N = 4;

namespace ffm {
struct ParabState;
cudaError_t launch_parab_move(const Ctx &c, ParabState *ps, int grid, cudaStream_t s);
size_t parab_state_bytes();
void parab_state_init(void *host_buf, int n, int atom0, int mode, int max_moves, uint64_t seed,
                      double delta, double taylor_r);
size_t parab_offset_move();
size_t parab_offset_stop();
cudaError_t launch_epoch(const Ctx &c, const EpochArgs &a, int parts, cudaStream_t s);
}  // namespace ffm
static ffmin_status parab_minimize(ffmin_system *sys, const ffmin_options *o, ffmin_result *res);
static ffmin_status epoch_minimize(ffmin_system *sys, const ffmin_options *o, ffmin_result *res);

struct ffmin_system {
    int n_sys = 0;
    int64_t n_atoms = 0;
    int prec = 0;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    Branches br{};  // side streams of a round's parallel branches
    bool broken = false;
    std::string err;
    Ctx c{};
    std::vector<void *> allocs;
    std::vector<int64_t> atom_off;
    std::vector<int32_t> sys_natoms;
    std::vector<SysState> hst;
    int grid32 = 0, grid32e = 0, grid64 = 0;
    int graph_ticks = 0;
    cudaGraphExec_t graph = nullptr;
    int32_t *h_nactive = nullptr;  // pinned
    // a minimization as one graph launch: a conditional WHILE node whose body
    // is TICKS_PER_GRAPH rounds and the loop-condition kernel; d_loop / h_loop
    // [2]: rounds run, round bound (device / pinned host)
    cudaGraphExec_t loop_exec = nullptr;
    bool loop_failed = false;
    int64_t *d_loop = nullptr, *h_loop = nullptr;
    // gradient-free path: device state and a graph of PARAB_MOVES moves
    void *parab_state = nullptr;
    cudaGraphExec_t parab_graph = nullptr;
    int parab_grid = 0;
    // parallel-epoch gradient-free path: per-part copies and part lists
    int ep_parts = 0;
    double *ep_view = nullptr;
    float4 *ep_viewf = nullptr;
    int32_t *ep_ints = nullptr;  // list [N], members [N], loff, moff [P + 1], allowed [P]
    // learned preconditioner
    bool have_precond = false;
    // some system uses the exclusion variant
    bool has_excl = false;
    // basin hopping: best points [3N] and per-system accept flags
    double *mbh_best = nullptr;
    int32_t *mbh_flags = nullptr;
    // stats of the last minimize
    int64_t last_ticks = 0, last_launches = 0, last_pairs = 0;
    // host copies of the topology needed by the gradient-free path
    std::vector<int32_t> inc_off_h;
    // work-item layout (rebuilt by the autotuner)
    std::vector<Tile> tiles_h;
    int n_bitems = 0, n_terms = 0, density = 10, grid32_max = 0, grid32e_max = 0, grid64_max = 0;
    int grid32_max_s[2] = {0, 0}, grid32e_max_s[2] = {0, 0};  // per FP32 shape (1 or 2 i-atoms per thread)
    int64_t items_cap = 0;
    Tile *d_tiles = nullptr;
    Item *d_items = nullptr;
    int2 *d_sys_items = nullptr;
    // symmetric list (rebuilt by the autotuner with the same density;
    // capacities are those of the densest layout)
    int64_t n_slots64 = 0;
    int n_items64 = 0, grid_sym = 0;
    Item *d_items64 = nullptr;
    int2 *d_sys_items64 = nullptr;
    std::vector<int32_t> term_off[4];  // per-system offsets of bonds, angles, dihedrals, corrections
    int nb_total = 0, na_total = 0, nd_total = 0;
};

// j-chunk length of a system: a multiple of TJ, chosen so that the whole
// batch exposes `density` work items per resident pair-kernel block (the
// queue's tail then costs about 1/density of a block's share, against more
// partial rows to write and sum); ffmin_autotune picks the density
static int chunk_len(int32_t n, int64_t total_tiles, int grid, int density) {
    int64_t want_items = (int64_t)density * grid;
    int64_t chunks = std::max<int64_t>(1, (want_items + total_tiles - 1) / std::max<int64_t>(total_tiles, 1));
    int64_t len = (n + chunks - 1) / chunks;
    len = ((len + TJ - 1) / TJ) * TJ;
    len = std::max<int64_t>(len, TJ);
    return (int)len;
}

// bonded work items of system b (bonds, angles, dihedrals, exclusion
// corrections; global term indices), appended to items
static void bonded_items(const ffmin_system *sys, int b, std::vector<Item> &items) {
    const int starts[4] = {sys->term_off[0][b], sys->nb_total + sys->term_off[1][b],
                           sys->nb_total + sys->na_total + sys->term_off[2][b],
                           sys->nb_total + sys->na_total + sys->nd_total + sys->term_off[3][b]};
    for (int ty = 0; ty < 4; ty++) {
        const int count = sys->term_off[ty][b + 1] - sys->term_off[ty][b];
        for (int k = 0; k < count; k += BONDED_ITEM_TERMS) {
            Item it{};
            it.tile = -1;
            it.j0 = starts[ty] + k;
            it.nj = std::min(BONDED_ITEM_TERMS, count - k);
            it.diag = b;
            items.push_back(it);
        }
    }
}

// Work items for a given density, system by system: the system's bonded
// items (latency-bound FP64 work that overlaps the FP32 pair items), then its
// (tile, j-chunk) pair items; every system's items are contiguous so that
// the pair kernels can run over the active systems only.
static void build_items(ffmin_system *sys, int density, std::vector<Item> &items, std::vector<Tile> &tiles,
                        std::vector<int2> &sys_items) {
    items.clear();
    tiles = sys->tiles_h;
    sys_items.assign(sys->n_sys, make_int2(0, 0));
    const int chunk_grid = sys->prec == FFMIN_MIXED ? sys->grid32_max : sys->grid64_max;
    const int64_t total_tiles = (int64_t)tiles.size();
    size_t t = 0;
    for (int b = 0; b < sys->n_sys; b++) {
        const int first = (int)items.size();
        bonded_items(sys, b, items);
        const int64_t A = sys->atom_off[b];
        const int n = sys->sys_natoms[b];
        const int L = chunk_len(n, total_tiles, chunk_grid, density);
        for (; t < tiles.size() && tiles[t].sys == b; t++) {
            Tile &tl = tiles[t];
            const int a0 = (int)(tl.a0 - A);
            tl.item0 = (int)items.size();
            int cnt = 0;
            for (int j0 = 0; j0 < n; j0 += L) {
                Item it{};
                it.tile = (int)t;
                it.j0 = (int)(A + j0);
                it.nj = std::min(L, n - j0);
                it.diag = (a0 >= j0 && a0 < j0 + it.nj) ? 1 : 0;
                items.push_back(it);
                cnt++;
            }
            tl.nitem = cnt;
        }
        sys_items[b] = make_int2(first, (int)items.size() - first);
    }
}

// Symmetric FP64 list: per system its bonded items, then for every i-tile I
// the chunks of `chunk` j-tiles covering tiles [I, nT) of the system (the
// first chunk starts with the diagonal tile).  Item slots: the i-side rows,
// then one row block per j-tile of the chunk.  chunk is chosen so that the
// batch exposes about `want` items; tiles get row64 / chunk64 / tloc.
static void build_items64(ffmin_system *sys, int64_t want, std::vector<Item> &items,
                          std::vector<int2> &sys_items, int64_t *n_slots) {
    items.clear();
    sys_items.assign(sys->n_sys, make_int2(0, 0));
    std::vector<Tile> &tiles = sys->tiles_h;
    int64_t pairs = 0;
    for (int b = 0; b < sys->n_sys; b++) {
        const int64_t nT = (sys->sys_natoms[b] + TI - 1) / TI;
        pairs += nT * (nT + 1) / 2;
    }
    const int chunk = (int)std::max<int64_t>(1, pairs / std::max<int64_t>(want, 1));
    int64_t slots = 0;
    size_t t = 0;
    for (int b = 0; b < sys->n_sys; b++) {
        const int first = (int)items.size();
        bonded_items(sys, b, items);
        const size_t t0 = t;
        while (t < tiles.size() && tiles[t].sys == b) t++;
        const int nT = (int)(t - t0);
        for (int I = 0; I < nT; I++) {
            Tile &tl = tiles[t0 + I];
            tl.row64 = (int)items.size();
            tl.chunk64 = chunk;
            tl.tloc = I;
            tl.slot64 = (int)slots;
            for (int J = I; J < nT; J += chunk) {
                const int nJ = std::min(chunk, nT - J);
                const Tile &last = tiles[t0 + J + nJ - 1];
                Item it{};
                it.tile = (int)(t0 + I);
                it.j0 = tiles[t0 + J].a0;
                it.nj = last.a0 + last.na - it.j0;
                it.diag = J == I ? 1 : 0;
                it.slot = (int)slots;
                slots += 1 + nJ;
                items.push_back(it);
            }
        }
        sys_items[b] = make_int2(first, (int)items.size() - first);
    }
    *n_slots = slots;
}

// FP64 partial rows of the symmetric list above this size fall back to the
// row sweep (its partial rows grow as the square of the atom count)
static const int64_t SYM64_MAX_BYTES = 4LL << 30;

static void set_item_counts(ffmin_system *sys, int n_items) {
    sys->c.n_items = n_items;
    sys->c.n_pair_items = n_items;
    // no more resident blocks than work items: idle blocks would only pay
    // for queue atomics
    sys->grid32 = std::max(1, std::min(sys->grid32_max, n_items));
    sys->grid32e = std::max(1, std::min(sys->grid32e_max, sys->c.sym64 ? sys->n_items64 : n_items));
    sys->grid64 = std::max(1, std::min(sys->grid64_max, sys->c.sym64 ? sys->n_items64 : n_items));
}

static thread_local std::string g_create_err;

static ffmin_status fail(ffmin_system *s, ffmin_status st, const std::string &msg) {
    if (s) s->err = msg;
    else g_create_err = msg;
    return st;
}

static ffmin_status cuda_fail(ffmin_system *s, cudaError_t e, const char *where) {
    if (s) {
        s->broken = true;
        s->err = std::string(where) + ": " + cudaGetErrorString(e);
    } else {
        g_create_err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? FFMIN_ERR_OOM : FFMIN_ERR_CUDA;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(sys, e_, #call);     \
    } while (0)

template <typename T>
static cudaError_t dalloc(ffmin_system *sys, T **p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) return e;
    sys->allocs.push_back(*p);
    return cudaMemsetAsync(*p, 0, bytes, sys->stream);
}

template <typename T>
static cudaError_t upload(ffmin_system *sys, T **p, const std::vector<T> &h) {
    cudaError_t e = dalloc(sys, p, h.size());
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, sys->stream);
}

extern "C" {

void ffmin_options_default(ffmin_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->method = FFMIN_LBFGS;
    o->cg_variant = FFMIN_CG_PRP;
    o->ls = FFMIN_LS_DEFAULT;
    o->lbfgs_m = 10;
    o->gtol_inf = 0.1;
    o->max_iter = 100000;
    o->max_evals = 1000000;
    o->cg_restart_every = 0;
    o->h0 = 0.1;
    o->k_plus = 2.0;
    o->k_minus = 0.5;
    o->eps_h = 1e-10;
    o->ls_par_K = 2;
    o->ls_par_g0 = 1;
    o->gradfree_delta = 0.05;
    o->gradfree_margin = 1.0;
    o->seed = 12345;
    o->use_learned_precond = 0;
    o->max_ticks = 0;
    o->record_dev = nullptr;
    o->record_every = 0;
    o->record_slots = 0;
    o->fgm_restart = 0;
    o->hb_alpha = 1e-4;
    o->hb_beta = 0.5;
    o->gradfree_taylor_r = 0.0;
    o->host_loop = 0;
    o->pc_window = 200;
    o->pc_rel = 1e-5;
    o->pc_gfar = 100.0;
}

const char *ffmin_status_string(ffmin_status s) {
    switch (s) {
    case FFMIN_OK: return "ok";
    case FFMIN_ERR_INVALID_ARG: return "invalid argument";
    case FFMIN_ERR_CUDA: return "cuda error";
    case FFMIN_ERR_NONFINITE: return "non-finite energy or gradient";
    case FFMIN_ERR_LINESEARCH: return "line search failed";
    case FFMIN_ERR_MAX_ITER: return "iteration limit";
    case FFMIN_ERR_TIMEOUT: return "device round limit";
    case FFMIN_ERR_OOM: return "out of memory";
    }
    return "unknown";
}

const char *ffmin_last_error(const ffmin_system *sys) {
    return sys ? sys->err.c_str() : g_create_err.c_str();
}

int64_t ffmin_n_atoms(const ffmin_system *sys) { return sys ? sys->n_atoms : 0; }

int64_t ffmin_atom_offset(const ffmin_system *sys, int32_t b) {
    if (!sys || b < 0 || b > sys->n_sys) return -1;
    return sys->atom_off[b];
}

ffmin_status ffmin_destroy(ffmin_system *sys) {
    if (!sys) return FFMIN_ERR_INVALID_ARG;
    if (sys->stream) cudaStreamSynchronize(sys->stream);
    if (sys->graph) cudaGraphExecDestroy(sys->graph);
    if (sys->loop_exec) cudaGraphExecDestroy(sys->loop_exec);
    if (sys->h_loop) cudaFreeHost(sys->h_loop);
    if (sys->parab_graph) cudaGraphExecDestroy(sys->parab_graph);
    for (void *p : sys->allocs) cudaFree(p);
    if (sys->h_nactive) cudaFreeHost(sys->h_nactive);
    if (sys->ev_in) cudaEventDestroy(sys->ev_in);
    if (sys->ev_out) cudaEventDestroy(sys->ev_out);
    for (int k = 0; k < 2; k++) {
        if (sys->br.side[k]) cudaStreamDestroy(sys->br.side[k]);
        if (sys->br.join[k]) cudaEventDestroy(sys->br.join[k]);
    }
    if (sys->br.fork) cudaEventDestroy(sys->br.fork);
    if (sys->stream) cudaStreamDestroy(sys->stream);
    delete sys;
    return FFMIN_OK;
}

static bool idx_ok(const int32_t *idx, int64_t count, int32_t n) {
    for (int64_t k = 0; k < count; k++)
        if (idx[k] < 0 || idx[k] >= n) return false;
    return true;
}

ffmin_status ffmin_create(const ffmin_topology *tops, int32_t n_sys, int32_t precision,
                          void *cuda_stream, ffmin_system **out) {
    if (!out) return fail(nullptr, FFMIN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!tops || n_sys < 1) return fail(nullptr, FFMIN_ERR_INVALID_ARG, "need n_sys >= 1 topologies");
    if (precision != FFMIN_FP64 && precision != FFMIN_MIXED)
        return fail(nullptr, FFMIN_ERR_INVALID_ARG, "precision must be FFMIN_FP64 or FFMIN_MIXED");
    int64_t total = 0;
    for (int b = 0; b < n_sys; b++) {
        const ffmin_topology &t = tops[b];
        if (t.n_atoms < 1 || t.n_bonds < 0 || t.n_angles < 0 || t.n_dihedrals < 0)
            return fail(nullptr, FFMIN_ERR_INVALID_ARG, "negative or zero count in topology " + std::to_string(b));
        if (!t.charge || !t.sigma || !t.epsilon)
            return fail(nullptr, FFMIN_ERR_INVALID_ARG, "missing per-atom arrays in topology " + std::to_string(b));
        if ((t.n_bonds && (!t.bond_idx || !t.bond_k || !t.bond_r0)) ||
            (t.n_angles && (!t.angle_idx || !t.angle_k || !t.angle_theta0)) ||
            (t.n_dihedrals && (!t.dihedral_idx || !t.dihedral_v)))
            return fail(nullptr, FFMIN_ERR_INVALID_ARG, "missing bonded arrays in topology " + std::to_string(b));
        if (!idx_ok(t.bond_idx, 2LL * t.n_bonds, t.n_atoms) || !idx_ok(t.angle_idx, 3LL * t.n_angles, t.n_atoms) ||
            !idx_ok(t.dihedral_idx, 4LL * t.n_dihedrals, t.n_atoms))
            return fail(nullptr, FFMIN_ERR_INVALID_ARG, "atom index out of range in topology " + std::to_string(b));
        for (int a = 0; a < t.n_atoms; a++)
            if (!(t.sigma[a] >= 0.0) || !(t.epsilon[a] >= 0.0) || !std::isfinite(t.charge[a]))
                return fail(nullptr, FFMIN_ERR_INVALID_ARG, "sigma/epsilon must be >= 0 and charges finite");
        if ((t.exclusions != 0 && t.exclusions != 1) ||
            (t.exclusions && !(t.scale14 >= 0.0 && std::isfinite(t.scale14))))
            return fail(nullptr, FFMIN_ERR_INVALID_ARG, "exclusions must be 0 or 1, scale14 finite and >= 0");
        // FP64 terms: FP64 correction terms cancel the excluded terms of the
        // all-pairs sweep; FP32 terms (MIXED): the sweeps scale the listed
        // pairs inside their sums, since an FP32 correction could not cancel
        // the rounding of bonded-neighbour clashes (up to 1e10 kcal/mol at a
        // jittered start)
        total += t.n_atoms;
    }
    if (total > (1LL << 30)) return fail(nullptr, FFMIN_ERR_INVALID_ARG, "too many atoms");

    ffmin_system *sys = new ffmin_system();
    sys->n_sys = n_sys;
    sys->n_atoms = total;
    sys->prec = precision;
    sys->user_stream = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaStreamCreateWithFlags(&sys->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { ffmin_status st = cuda_fail(nullptr, e, "cudaStreamCreate"); delete sys; return st; }
    cudaEventCreateWithFlags(&sys->ev_in, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&sys->ev_out, cudaEventDisableTiming);
    e = cudaEventCreateWithFlags(&sys->br.fork, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaStreamCreateWithFlags(&sys->br.side[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sys->br.join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        ffmin_status st = cuda_fail(nullptr, e, "side streams");
        ffmin_destroy(sys);
        return st;
    }
    if (cudaMallocHost((void **)&sys->h_nactive, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost((void **)&sys->h_loop, 2 * sizeof(int64_t)) != cudaSuccess) {
        ffmin_destroy(sys);
        return fail(nullptr, FFMIN_ERR_OOM, "pinned allocation failed");
    }
    sys->grid32 = pair_grid_size(0);
    sys->grid64 = pair_grid_size(1);

    // ---- tiles, items, per-atom data, bonded terms ----
    std::vector<Tile> tiles;
    std::vector<Item> items;
    std::vector<int32_t> tile0(n_sys), ntile(n_sys);
    sys->atom_off.assign(n_sys + 1, 0);
    for (int b = 0; b < n_sys; b++) sys->atom_off[b + 1] = sys->atom_off[b] + tops[b].n_atoms;
    int64_t total_tiles = 0;
    for (int b = 0; b < n_sys; b++) total_tiles += (tops[b].n_atoms + TI - 1) / TI;
    std::vector<double> qs(total), sig(total), aa(total);
    std::vector<float2> parf(total);
    std::vector<double2> pard(total);
    std::vector<float> feat(3 * total);
    std::vector<int2> bidx, aidx_dummy;
    std::vector<double2> bpar, apar;
    std::vector<int4> aidx, didx;
    std::vector<double4_32a> dpar;
    std::vector<int2> xidx;          // exclusion corrections: atom pairs
    std::vector<double> xw;          // and weights s_ij - 1
    std::vector<int32_t> xcount(n_sys, 0);
    std::vector<std::vector<int2>> inc_lists(total);
    std::vector<std::vector<std::pair<int32_t, float>>> xs_lists(total);  // scaled partners per atom
    for (int b = 0; b < n_sys; b++) {
        const ffmin_topology &t = tops[b];
        const int64_t A = sys->atom_off[b];
        const double C = t.coulomb_c > 0.0 ? t.coulomb_c : 1389.38757 / 4.184;
        const double sc = std::sqrt(C);
        for (int a = 0; a < t.n_atoms; a++) {
            qs[A + a] = t.charge[a] * sc;
            sig[A + a] = t.sigma[a];
            aa[A + a] = std::sqrt(24.0 * t.epsilon[a]);
            const double s3 = sig[A + a] * sig[A + a] * sig[A + a];
            const double c6 = aa[A + a] * s3, c12 = aa[A + a] * s3 * s3;
            parf[A + a] = make_float2((float)c6, (float)c12);
            pard[A + a] = make_double2(c6, c12);
            feat[3 * (A + a)] = (float)t.charge[a];
            feat[3 * (A + a) + 1] = (float)t.sigma[a];
            feat[3 * (A + a) + 2] = (float)t.epsilon[a];
        }
        for (int k = 0; k < t.n_bonds; k++) {
            int term = (int)bidx.size();
            int i = t.bond_idx[2 * k], j = t.bond_idx[2 * k + 1];
            bidx.push_back(make_int2((int)(A + i), (int)(A + j)));
            bpar.push_back(make_double2(t.bond_k[k], t.bond_r0[k]));
            inc_lists[A + i].push_back(make_int2((0 << 2) | 0, term));
            inc_lists[A + j].push_back(make_int2((0 << 2) | 1, term));
        }
        for (int k = 0; k < t.n_angles; k++) {
            int term = (int)aidx.size();
            const int32_t *q = t.angle_idx + 3 * k;
            aidx.push_back(make_int4((int)(A + q[0]), (int)(A + q[1]), (int)(A + q[2]), 0));
            apar.push_back(make_double2(t.angle_k[k], t.angle_theta0[k]));
            for (int p = 0; p < 3; p++) inc_lists[A + q[p]].push_back(make_int2((1 << 2) | p, term));
        }
        for (int k = 0; k < t.n_dihedrals; k++) {
            int term = (int)didx.size();
            const int32_t *q = t.dihedral_idx + 4 * k;
            didx.push_back(make_int4((int)(A + q[0]), (int)(A + q[1]), (int)(A + q[2]), (int)(A + q[3])));
            const double *v = t.dihedral_v + 4 * k;
            dpar.push_back(make_double4_32a(v[0], v[1], v[2], v[3]));
            for (int p = 0; p < 4; p++) inc_lists[A + q[p]].push_back(make_int2((2 << 2) | p, term));
        }
        if (t.exclusions) {
            // s_ij = 0 for bonded and angle-end pairs, scale14 for dihedral
            // ends (the smallest scale wins for a pair listed twice); one
            // correction term of weight s_ij - 1 per pair with s_ij != 1,
            // in ascending pair order
            std::map<int64_t, double> scale;
            auto add = [&](int i, int j, double s) {
                const int64_t key = (int64_t)std::min(i, j) * t.n_atoms + std::max(i, j);
                auto it = scale.find(key);
                if (it == scale.end()) scale[key] = s;
                else it->second = std::min(it->second, s);
            };
            for (int k = 0; k < t.n_bonds; k++) add(t.bond_idx[2 * k], t.bond_idx[2 * k + 1], 0.0);
            for (int k = 0; k < t.n_angles; k++) add(t.angle_idx[3 * k], t.angle_idx[3 * k + 2], 0.0);
            for (int k = 0; k < t.n_dihedrals; k++)
                add(t.dihedral_idx[4 * k], t.dihedral_idx[4 * k + 3], t.scale14);
            for (const auto &kv : scale) {
                const double w = kv.second - 1.0;
                const int i = (int)(kv.first / t.n_atoms), j = (int)(kv.first % t.n_atoms);
                if (w == 0.0 || i == j) continue;
                const int term = (int)xidx.size();
                xidx.push_back(make_int2((int)(A + i), (int)(A + j)));
                xw.push_back(w);
                inc_lists[A + i].push_back(make_int2((3 << 2) | 0, term));
                inc_lists[A + j].push_back(make_int2((3 << 2) | 1, term));
                xs_lists[A + i].push_back(std::make_pair((int32_t)(A + j), (float)kv.second));
                xs_lists[A + j].push_back(std::make_pair((int32_t)(A + i), (float)kv.second));
                xcount[b]++;
            }
        }
        // tiles of 128 atoms (never straddling systems)
        tile0[b] = (int)tiles.size();
        for (int a0 = 0; a0 < t.n_atoms; a0 += TI) {
            Tile tl{};
            tl.sys = b;
            tl.a0 = (int)(A + a0);
            tl.na = std::min(TI, t.n_atoms - a0);
            tl.xlo = std::numeric_limits<int32_t>::max();
            tl.xhi = -1;
            for (int a = tl.a0; a < tl.a0 + tl.na; a++)
                for (const auto &pr : xs_lists[a]) {
                    tl.xlo = std::min(tl.xlo, pr.first);
                    tl.xhi = std::max(tl.xhi, pr.first);
                }
            tiles.push_back(tl);
        }
        ntile[b] = (int)tiles.size() - tile0[b];
    }
    // bonded work items go first in the queue: they are latency-bound FP64
    // work and overlap with the FP32 pair items that follow
    const int n_terms = (int)(bidx.size() + aidx.size() + didx.size() + xidx.size());
    std::vector<int32_t> term_sys(std::max(n_terms, 1), 0);
    {
        int t = 0;
        for (int b = 0; b < n_sys; b++) for (int k = 0; k < tops[b].n_bonds; k++) (void)k, term_sys[t++] = b;
        for (int b = 0; b < n_sys; b++) for (int k = 0; k < tops[b].n_angles; k++) (void)k, term_sys[t++] = b;
        for (int b = 0; b < n_sys; b++) for (int k = 0; k < tops[b].n_dihedrals; k++) (void)k, term_sys[t++] = b;
        for (int b = 0; b < n_sys; b++) for (int k = 0; k < xcount[b]; k++) (void)k, term_sys[t++] = b;
    }
    sys->n_terms = n_terms;
    sys->n_bitems = (n_terms + BONDED_ITEM_TERMS - 1) / BONDED_ITEM_TERMS;
    sys->tiles_h = tiles;
    sys->nb_total = (int)bidx.size();
    sys->na_total = (int)aidx.size();
    sys->nd_total = (int)didx.size();
    for (int ty = 0; ty < 4; ty++) sys->term_off[ty].assign(n_sys + 1, 0);
    for (int b = 0; b < n_sys; b++) {
        sys->term_off[0][b + 1] = sys->term_off[0][b] + tops[b].n_bonds;
        sys->term_off[1][b + 1] = sys->term_off[1][b] + tops[b].n_angles;
        sys->term_off[2][b + 1] = sys->term_off[2][b] + tops[b].n_dihedrals;
        sys->term_off[3][b + 1] = sys->term_off[3][b] + xcount[b];
    }
    std::vector<int2> sys_items;
    sys->sys_natoms.resize(n_sys);
    for (int b = 0; b < n_sys; b++) sys->sys_natoms[b] = tops[b].n_atoms;
    for (int k = 0; k < 2; k++) {
        sys->grid32_max_s[k] = pair_grid_size(0, k + 1);
        sys->grid32e_max_s[k] = pair_grid_size(3, k + 1);
    }
    sys->c.f32_ipt = 2;
    // the row list's capacity below takes the FP32 shape with more
    // resident blocks (more items at a given density)
    sys->grid32_max = std::max(sys->grid32_max_s[0], sys->grid32_max_s[1]);
    sys->grid32e_max = sys->grid32e_max_s[1];
    sys->grid64_max = sys->grid64;
    // symmetric list: `density` items per resident block of the symmetric
    // FP64 kernel (the autotuner rebuilds it with the row list); capacity
    // from the densest layout the autotuner may choose.  It also fills the
    // tiles' row64 / chunk64 / tloc, which build_items copies
    std::vector<Item> items64;
    std::vector<int2> sys_items64;
    const int grid_sym = pair_grid_size(2);
    sys->grid_sym = grid_sym;
    int64_t slots_cap = 0;
    build_items64(sys, (int64_t)AUTOTUNE_DENSITIES[AUTOTUNE_N - 1] * grid_sym, items64, sys_items64, &slots_cap);
    const size_t items64_cap = items64.size();
    build_items64(sys, (int64_t)sys->density * grid_sym, items64, sys_items64, &sys->n_slots64);
    sys->n_items64 = (int)items64.size();
    const bool sym64 = slots_cap * TI * (int64_t)sizeof(double4_32a) <= SYM64_MAX_BYTES;
    if (sym64) sys->grid64_max = grid_sym;
    sys->c.sym64 = sym64 ? 1 : 0;
    sys->c.n_items64 = sym64 ? sys->n_items64 : 0;
    sys->n_slots64 = slots_cap;  // allocation size of the partial rows
    // capacity: the densest layout the autotuner may choose
    build_items(sys, AUTOTUNE_DENSITIES[AUTOTUNE_N - 1], items, tiles, sys_items);
    sys->items_cap = (int64_t)items.size();
    sys->grid32_max = sys->grid32_max_s[1];
    build_items(sys, sys->density, items, tiles, sys_items);
    std::vector<int32_t> inc_off(total + 1, 0);
    std::vector<int2> inc;
    for (int64_t a = 0; a < total; a++) {
        inc_off[a] = (int32_t)inc.size();
        for (const int2 &x : inc_lists[a]) inc.push_back(x);
    }
    inc_off[total] = (int32_t)inc.size();
    sys->inc_off_h = inc_off;

    Ctx &c = sys->c;
    c.n_sys = n_sys;
    c.n_tiles = (int)tiles.size();
    set_item_counts(sys, (int)items.size());
    c.n_bonds = (int)bidx.size();
    c.n_angles = (int)aidx.size();
    c.n_dihedrals = (int)didx.size();
    c.n_excl = (int)xidx.size();
    c.n_terms = n_terms;
    c.n_atoms = (int)total;
    c.vstride = ((3 * total + 31) / 32) * 32;
    c.prec = precision;
    c.sep_reduce = n_sys >= LB_MAX_SYS ? 1 : 0;

#define CKC(call)                                                              \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) {                                               \
            ffmin_status st_ = cuda_fail(nullptr, e_, #call);                  \
            ffmin_destroy(sys);                                                \
            return st_;                                                        \
        }                                                                      \
    } while (0)

    Tile *d_tiles; Item *d_items;
    CKC(upload(sys, &d_tiles, tiles));
    CKC(dalloc(sys, &d_items, (size_t)sys->items_cap));
    CKC(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice, sys->stream));
    c.tiles = d_tiles;
    c.items = d_items;
    sys->d_tiles = d_tiles;
    sys->d_items = d_items;
    int2 *d_sys_items;
    CKC(upload(sys, &d_sys_items, sys_items));
    c.sys_items = d_sys_items;
    sys->d_sys_items = d_sys_items;
    if (sym64) {
        CKC(dalloc(sys, &sys->d_items64, items64_cap));
        CKC(cudaMemcpyAsync(sys->d_items64, items64.data(), items64.size() * sizeof(Item), cudaMemcpyHostToDevice,
                            sys->stream));
        CKC(upload(sys, &sys->d_sys_items64, sys_items64));
        c.items64 = sys->d_items64;
        c.sys_items64 = sys->d_sys_items64;
    }
    CKC(dalloc(sys, &c.act, N_LISTS * (2 * (size_t)n_sys + 2)));
    SysState *d_st;
    CKC(dalloc(sys, &d_st, n_sys));
    c.st = d_st;
    CKC(dalloc(sys, &c.vec, (size_t)V_NSLOT * c.vstride));
    double *d_qs;
    CKC(upload(sys, &d_qs, qs));
    c.qs = d_qs;
    {
        // FP64 pair inputs always; FP32 ones too for MIXED objects, whose
        // runs start with FP32 pair terms and finish with FP64 ones
        double2 *d_pard;
        CKC(dalloc(sys, &c.posd, total));
        CKC(upload(sys, &d_pard, pard));
        c.pard = d_pard;
        CKC(dalloc(sys, &c.gpd, (size_t)(sym64 ? sys->n_slots64 : sys->items_cap) * TI));
        if (precision == FFMIN_MIXED) {
            float2 *d_parf;
            CKC(dalloc(sys, &c.posf, total));
            CKC(dalloc(sys, &c.dispf, total));
            CKC(upload(sys, &d_parf, parf));
            c.parf = d_parf;
            CKC(dalloc(sys, &c.gpf, (size_t)sys->items_cap * TI));
            if (sym64) CKC(dalloc(sys, &c.gpf_sym, (size_t)sys->n_slots64 * TI));
        }
    }
    int32_t *d_inc_off; int2 *d_inc, *d_bidx; double2 *d_bpar, *d_apar; int4 *d_aidx, *d_didx; double4_32a *d_dpar;
    CKC(upload(sys, &d_inc_off, inc_off));
    CKC(upload(sys, &d_inc, inc));
    CKC(upload(sys, &d_bidx, bidx));
    CKC(upload(sys, &d_bpar, bpar));
    CKC(upload(sys, &d_aidx, aidx));
    CKC(upload(sys, &d_apar, apar));
    CKC(upload(sys, &d_didx, didx));
    CKC(upload(sys, &d_dpar, dpar));
    c.inc_off = d_inc_off; c.inc = d_inc; c.bidx = d_bidx; c.bpar = d_bpar;
    c.aidx = d_aidx; c.apar = d_apar; c.didx = d_didx; c.dpar = d_dpar;
    int2 *d_xidx;
    double *d_xw;
    CKC(upload(sys, &d_xidx, xidx));
    CKC(upload(sys, &d_xw, xw));
    c.xidx = d_xidx;
    c.xw = d_xw;
    sys->has_excl = !xidx.empty();
    if (sys->has_excl && precision == FFMIN_MIXED) {  // per-atom scaled partners for the FP32 sweeps
        std::vector<int32_t> xs_off(total + 1, 0), xs_part;
        std::vector<float> xs_val;
        for (int64_t a = 0; a < total; a++) {
            xs_off[a] = (int32_t)xs_part.size();
            for (const auto &pr : xs_lists[a]) {
                xs_part.push_back(pr.first);
                xs_val.push_back(pr.second);
            }
        }
        xs_off[total] = (int32_t)xs_part.size();
        int32_t *d_xs_off, *d_xs_part;
        float *d_xs_val;
        CKC(upload(sys, &d_xs_off, xs_off));
        CKC(upload(sys, &d_xs_part, xs_part));
        CKC(upload(sys, &d_xs_val, xs_val));
        c.xs_off = d_xs_off;
        c.xs_part = d_xs_part;
        c.xs_val = d_xs_val;
    }
    int32_t *d_term_sys;
    CKC(upload(sys, &d_term_sys, term_sys));
    c.term_sys = d_term_sys;
    CKC(dalloc(sys, &c.te, std::max(n_terms, 1)));
    CKC(dalloc(sys, &c.tg, 3 * (2 * bidx.size() + 3 * aidx.size() + 4 * didx.size() + 2 * xidx.size()) + 3));
    CKC(dalloc(sys, &c.red, (size_t)c.n_tiles * NRED));
    CKC(dalloc(sys, &c.counters, CNT_N));
    CKC(dalloc(sys, &c.nactive, 1));
    CKC(dalloc(sys, &c.nmode, 2));
    float *d_feat;
    CKC(upload(sys, &d_feat, feat));
    c.feat = d_feat;
    CKC(dalloc(sys, &c.ncount, total));
    uint16_t *d_w;
    CKC(dalloc(sys, &d_w, 512));
    c.mlp_w = d_w;

    // host mirror of the per-system state (geometry part)
    sys->hst.assign(n_sys, SysState{});
    for (int b = 0; b < n_sys; b++) {
        SysState &S = sys->hst[b];
        std::memset(&S, 0, sizeof(S));
        S.atom0 = (int)sys->atom_off[b];
        S.natoms = tops[b].n_atoms;
        S.tile0 = tile0[b];
        S.ntile = ntile[b];
        S.mixed = precision == FFMIN_MIXED ? 1 : 0;
        S.mode = precision == FFMIN_MIXED ? 0 : 1;
    }
    CKC(cudaMemcpyAsync(d_st, sys->hst.data(), sizeof(SysState) * n_sys, cudaMemcpyHostToDevice, sys->stream));
    CKC(cudaStreamSynchronize(sys->stream));
#undef CKC
    *out = sys;
    return FFMIN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- helpers
static ffmin_status enter(ffmin_system *sys) {
    if (!sys) return FFMIN_ERR_INVALID_ARG;
    if (sys->broken) return FFMIN_ERR_CUDA;
    cudaError_t e = cudaEventRecord(sys->ev_in, sys->user_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sys->stream, sys->ev_in, 0);
    if (e != cudaSuccess) return cuda_fail(sys, e, "stream ordering");
    return FFMIN_OK;
}

static ffmin_status leave(ffmin_system *sys) {
    cudaError_t e = cudaEventRecord(sys->ev_out, sys->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sys->user_stream, sys->ev_out, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sys->stream);
    if (e != cudaSuccess) return cuda_fail(sys, e, "stream sync");
    return FFMIN_OK;
}

static ffmin_status upload_states(ffmin_system *sys) {
    CK(cudaMemcpyAsync(sys->c.st, sys->hst.data(), sizeof(SysState) * sys->n_sys, cudaMemcpyHostToDevice,
                       sys->stream));
    return FFMIN_OK;
}

static ffmin_status download_states(ffmin_system *sys) {
    CK(cudaMemcpyAsync(sys->hst.data(), sys->c.st, sizeof(SysState) * sys->n_sys, cudaMemcpyDeviceToHost,
                       sys->stream));
    CK(cudaStreamSynchronize(sys->stream));
    return FFMIN_OK;
}

// active-system counters read by the kernels: all systems start in the
// object's precision mode (FP32 for MIXED, FP64 otherwise)
static ffmin_status set_counts(ffmin_system *sys) {
    int32_t h[3] = {sys->n_sys, 0, 0};
    h[sys->prec == FFMIN_MIXED ? 1 : 2] = sys->n_sys;
    CK(cudaMemcpyAsync(sys->c.nactive, &h[0], sizeof(int32_t), cudaMemcpyHostToDevice, sys->stream));
    CK(cudaMemcpyAsync(sys->c.nmode, &h[1], 2 * sizeof(int32_t), cudaMemcpyHostToDevice, sys->stream));
    return FFMIN_OK;
}

// One evaluation's kernels: the active lists (built from the control state)
// beside the trial point, then the pair kernels, then the finalize.  The
// active-list kernel and k_prepare read the same state and write disjoint
// buffers, so they run on parallel branches.
static cudaError_t launch_eval(ffmin_system *sys, cudaStream_t s) {
    const Ctx &c = sys->c;
    const Branches &br = sys->br;
    cudaError_t e;
    if ((e = cudaEventRecord(br.fork, s)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(br.side[0], br.fork, 0)) != cudaSuccess) return e;
    if ((e = launch_activelist(c, br.side[0])) != cudaSuccess) return e;
    if ((e = launch_prepare(c, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(br.join[0], br.side[0])) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, br.join[0], 0)) != cudaSuccess) return e;
    if ((e = launch_pair_kernels(c, sys->grid32, sys->grid32e, sys->grid64, s, &br)) != cudaSuccess) return e;
    if ((e = launch_finalize(c, s)) != cudaSuccess) return e;
    if (c.sep_reduce) return launch_sysreduce(c, 3, s);
    return cudaSuccess;
}

static cudaError_t launch_tick(ffmin_system *sys) {
    const Ctx &c = sys->c;
    cudaStream_t s = sys->stream;
    cudaError_t e;
    if ((e = launch_update(c, s)) != cudaSuccess) return e;
    if (c.sep_reduce && (e = launch_sysreduce(c, 0, s)) != cudaSuccess) return e;
    if ((e = launch_dir(c, 0, s)) != cudaSuccess) return e;
    if (c.sep_reduce && (e = launch_sysreduce(c, 1, s)) != cudaSuccess) return e;
    if ((e = launch_dir(c, 1, s)) != cudaSuccess) return e;
    if (c.sep_reduce && (e = launch_sysreduce(c, 2, s)) != cudaSuccess) return e;
    return launch_eval(sys, s);
}

constexpr int TICKS_PER_GRAPH = 8;

// Loop condition of the device-driven minimization: counts the rounds and
// keeps the WHILE node running while a system is active and the round bound
// is not reached (so the loop always ends within loop[1] + 8 rounds).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int32_t *nactive, int64_t *loop) {
    const int64_t t = loop[0] + TICKS_PER_GRAPH;
    loop[0] = t;
    cudaGraphSetConditional(h, (*nactive > 0 && t < loop[1]) ? 1u : 0u);
}
static int kernels_per_tick(const ffmin_system *sys) {
    return (sys->prec == FFMIN_MIXED ? 8 : 6) + (sys->c.sep_reduce ? 4 : 0);
}

static ffmin_status ensure_graph(ffmin_system *sys) {
    if (sys->graph) return FFMIN_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(sys->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < TICKS_PER_GRAPH && e == cudaSuccess; t++) e = launch_tick(sys);
    cudaError_t e2 = cudaStreamEndCapture(sys->stream, &g);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(sys, e, "graph capture"); }
    if (e2 != cudaSuccess) return cuda_fail(sys, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&sys->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(sys, e, "cudaGraphInstantiate");
    sys->graph_ticks = TICKS_PER_GRAPH;
    return FFMIN_OK;
}

// The whole minimization as one graph: a WHILE node over TICKS_PER_GRAPH
// rounds plus k_loop_cond.  When the runtime cannot build it, minimize_dev
// replays the plain graph of rounds from the host instead.
static ffmin_status ensure_loop(ffmin_system *sys) {
    if (sys->loop_exec || sys->loop_failed) return FFMIN_OK;
    if (!sys->d_loop) CK(dalloc(sys, &sys->d_loop, 2));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle h{};
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
    if (e == cudaSuccess) {
        cudaGraph_t body = p.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(sys->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaSuccess;
            for (int t = 0; t < TICKS_PER_GRAPH && e1 == cudaSuccess; t++) e1 = launch_tick(sys);
            if (e1 == cudaSuccess) {
                k_loop_cond<<<1, 1, 0, sys->stream>>>(h, sys->c.nactive, sys->d_loop);
                e1 = cudaGetLastError();
            }
            cudaGraph_t out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(sys->stream, &out);
            e = e1 != cudaSuccess ? e1 : e2;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&sys->loop_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {  // fall back to the host-replayed graph of rounds
        (void)cudaGetLastError();
        sys->loop_exec = nullptr;
        sys->loop_failed = true;
    }
    return FFMIN_OK;
}

// one evaluation (E or EG) of every system at the vector in `slot`, or at
// slot + h * dir when dir >= 0; delta = 1 takes a MIXED energy-only trial
// the way a line search does: pair terms as exact FP32 differences from the
// pair energy of the last E + grad evaluation (at `slot`), bonded terms in FP64
static ffmin_status eval_slot(ffmin_system *sys, int slot, int kind, int dir = -1, double h = 0.0,
                              int delta = 0) {
    const Ctx &c = sys->c;
    for (int b = 0; b < sys->n_sys; b++) {
        SysState &S = sys->hst[b];
        S.active = 1;
        S.phase = PH_EVAL_ONLY;
        S.upd.op = U_NONE;
        S.dir[0].on = S.dir[1].on = 0;
        S.ev_kind = kind;
        S.ev_base = slot;
        S.ev_dir = dir;
        S.ev_h = h;
        S.ev_scale = 1.0;
        S.ne = S.neg = 0;
        S.mode = sys->prec == FFMIN_MIXED ? 0 : 1;
        S.ev_delta = (delta && S.mode == 0 && kind == EV_E && dir >= 0) ? 1 : 0;
        S.epair_base = S.epair_last;
    }
    ffmin_status st = upload_states(sys);
    if (st != FFMIN_OK) return st;
    if ((st = set_counts(sys)) != FFMIN_OK) return st;
    CK(launch_eval(sys, sys->stream));
    return download_states(sys);
}

// one evaluation (E or EG) of every system at x (device)
static ffmin_status eval_all(ffmin_system *sys, const double *x_dev, int kind) {
    CK(cudaMemcpyAsync(vslot(sys->c, V_XIN), x_dev, sizeof(double) * 3 * sys->n_atoms,
                       cudaMemcpyDeviceToDevice, sys->stream));
    return eval_slot(sys, V_XIN, kind);
}

extern "C" {

ffmin_status ffmin_energy(ffmin_system *sys, const double *x_dev, double *e_host) {
    NvtxRange nvtx_range("ffmin_energy");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !e_host) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    st = eval_all(sys, x_dev, EV_E);
    if (st != FFMIN_OK) return st;
    ffmin_status res = FFMIN_OK;
    for (int b = 0; b < sys->n_sys; b++) {
        e_host[b] = sys->hst[b].res_f;
        if (sys->hst[b].status == FFMIN_ERR_NONFINITE) res = FFMIN_ERR_NONFINITE;
    }
    st = leave(sys);
    return st != FFMIN_OK ? st : res;
}

ffmin_status ffmin_energy_grad(ffmin_system *sys, const double *x_dev, double *e_host, double *g_dev) {
    NvtxRange nvtx_range("ffmin_energy_grad");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !e_host || !g_dev) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    st = eval_all(sys, x_dev, EV_EG);
    if (st != FFMIN_OK) return st;
    CK(cudaMemcpyAsync(g_dev, vslot(sys->c, V_GT), sizeof(double) * 3 * sys->n_atoms, cudaMemcpyDeviceToDevice,
                       sys->stream));
    ffmin_status res = FFMIN_OK;
    for (int b = 0; b < sys->n_sys; b++) {
        e_host[b] = sys->hst[b].res_f;
        if (sys->hst[b].status == FFMIN_ERR_NONFINITE) res = FFMIN_ERR_NONFINITE;
    }
    st = leave(sys);
    return st != FFMIN_OK ? st : res;
}

ffmin_status ffmin_energy_grad_host(ffmin_system *sys, const double *x_host, double *e_host, double *g_host) {
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_host || !e_host) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    const size_t bytes = sizeof(double) * 3 * sys->n_atoms;
    double *stage = vslot(sys->c, V_XT);  // scratch: overwritten by the evaluation anyway
    CK(cudaMemcpyAsync(stage, x_host, bytes, cudaMemcpyHostToDevice, sys->stream));
    st = eval_all(sys, stage, g_host ? EV_EG : EV_E);
    if (st != FFMIN_OK) return st;
    if (g_host) {
        CK(cudaMemcpyAsync(g_host, vslot(sys->c, V_GT), bytes, cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
    }
    ffmin_status res = FFMIN_OK;
    for (int b = 0; b < sys->n_sys; b++) {
        e_host[b] = sys->hst[b].res_f;
        if (sys->hst[b].status == FFMIN_ERR_NONFINITE) res = FFMIN_ERR_NONFINITE;
    }
    st = leave(sys);
    return st != FFMIN_OK ? st : res;
}

ffmin_status ffmin_energy_delta(ffmin_system *sys, const double *x_dev, const double *r_dev, double h,
                                double *de_host) {
    NvtxRange nvtx_range("ffmin_energy_delta");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !r_dev || !de_host || !std::isfinite(h)) return fail(sys, FFMIN_ERR_INVALID_ARG, "bad argument");
    const size_t bytes = sizeof(double) * 3 * sys->n_atoms;
    CK(cudaMemcpyAsync(vslot(sys->c, V_XIN), x_dev, bytes, cudaMemcpyDeviceToDevice, sys->stream));
    CK(cudaMemcpyAsync(vslot(sys->c, V_R), r_dev, bytes, cudaMemcpyDeviceToDevice, sys->stream));
    // the base of a line search is an E + grad evaluation
    if ((st = eval_slot(sys, V_XIN, EV_EG)) != FFMIN_OK) return st;
    ffmin_status res = FFMIN_OK;
    std::vector<double> base(sys->n_sys);
    for (int b = 0; b < sys->n_sys; b++) {
        base[b] = sys->hst[b].res_f;
        if (sys->hst[b].status == FFMIN_ERR_NONFINITE) res = FFMIN_ERR_NONFINITE;
    }
    if ((st = eval_slot(sys, V_XIN, EV_E, V_R, h, 1)) != FFMIN_OK) return st;
    for (int b = 0; b < sys->n_sys; b++) {
        de_host[b] = sys->hst[b].res_f - base[b];
        if (sys->hst[b].status == FFMIN_ERR_NONFINITE) res = FFMIN_ERR_NONFINITE;
    }
    st = leave(sys);
    return st != FFMIN_OK ? st : res;
}

static ffmin_status check_options(ffmin_system *sys, const ffmin_options *o) {
    if (!o) return fail(sys, FFMIN_ERR_INVALID_ARG, "options is NULL");
    if (o->method < FFMIN_GD || o->method > FFMIN_HB) return fail(sys, FFMIN_ERR_INVALID_ARG, "bad method");
    if (o->method == FFMIN_HB && !(o->hb_alpha > 0.0 && std::isfinite(o->hb_alpha) && o->hb_beta >= 0.0 &&
                                   std::isfinite(o->hb_beta)))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "HB needs hb_alpha > 0 and hb_beta >= 0, both finite");
    if (o->cg_variant < 0 || o->cg_variant > FFMIN_CG_DY) return fail(sys, FFMIN_ERR_INVALID_ARG, "bad cg_variant");
    if (o->ls < 0 || o->ls > FFMIN_LS_PAR) return fail(sys, FFMIN_ERR_INVALID_ARG, "bad line search");
    if (o->method == FFMIN_LBFGS && (o->lbfgs_m < 1 || o->lbfgs_m > MAXM))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "lbfgs_m must be in [1, 16]");
    if (!(o->h0 > 0.0) || !(o->k_plus > 1.0) || !(o->k_minus > 0.0 && o->k_minus < 1.0) ||
        !(o->eps_h > 0.0 && o->eps_h < 1.0) || o->ls_par_K < 2 || !(o->gtol_inf >= 0.0) || o->max_iter < 0 ||
        o->max_evals < 1)
        return fail(sys, FFMIN_ERR_INVALID_ARG, "line-search / stopping parameter out of range");
    if (o->method == FFMIN_GRADFREE && !(o->gradfree_taylor_r >= 0.0))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "gradfree_taylor_r must be >= 0");
    if (o->method == FFMIN_GRADFREE && (o->gradfree_parts < 0 || !(o->gradfree_margin >= 0.0)))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "GRADFREE needs gradfree_parts >= 0 and gradfree_margin >= 0");
    if (o->method == FFMIN_GRADFREE && sys->has_excl && sys->prec == FFMIN_MIXED)
        return fail(sys, FFMIN_ERR_INVALID_ARG,
                    "GRADFREE with exclusions needs FFMIN_FP64 (its FP32 rows do not mask the excluded pairs)");
    if (o->method == FFMIN_GRADFREE && (sys->n_sys != 1 || !(o->gradfree_delta > 0.0)))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "GRADFREE needs one system and delta > 0");
    if (o->use_learned_precond && !sys->have_precond)
        return fail(sys, FFMIN_ERR_INVALID_ARG, "no preconditioner weights set");
    if (o->host_loop != 0 && o->host_loop != 1) return fail(sys, FFMIN_ERR_INVALID_ARG, "host_loop must be 0 or 1");
    if (o->pc_window < 0 || !(o->pc_rel >= 0.0) || !(o->pc_gfar >= 0.0))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "pc_window >= 0, pc_rel >= 0, pc_gfar >= 0");
    if (o->fgm_restart != 0 && o->fgm_restart != 1)
        return fail(sys, FFMIN_ERR_INVALID_ARG, "fgm_restart must be 0 or 1");
    if (o->record_dev && (o->record_every < 1 || o->record_slots < 1))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "recording needs record_every >= 1 and record_slots >= 1");
    return FFMIN_OK;
}

static ffmin_status minimize_dev(ffmin_system *sys, double *x_dev, const ffmin_options *o, ffmin_result *res) {
    const Ctx &c = sys->c;
    const size_t bytes = sizeof(double) * 3 * sys->n_atoms;
    if (o->method == FFMIN_GRADFREE) {
        CK(cudaMemcpyAsync(vslot(c, V_X), x_dev, bytes, cudaMemcpyDeviceToDevice, sys->stream));
        ffmin_status st = o->gradfree_parts >= 1 ? epoch_minimize(sys, o, res) : parab_minimize(sys, o, res);
        if (st != FFMIN_OK) return st;
        CK(cudaMemcpyAsync(x_dev, vslot(c, V_X), bytes, cudaMemcpyDeviceToDevice, sys->stream));
        return FFMIN_OK;
    }
    CK(cudaMemcpyAsync(vslot(c, V_X), x_dev, bytes, cudaMemcpyDeviceToDevice, sys->stream));
    CK(cudaMemsetAsync(vslot(c, V_P), 0, bytes, sys->stream));
    CK(cudaMemsetAsync(vslot(c, V_R), 0, bytes, sys->stream));
    if (o->use_learned_precond) CK(launch_ncount(c, vslot(c, V_X), c.ncount, sys->stream));
    for (int b = 0; b < sys->n_sys; b++) {
        SysState &S = sys->hst[b];
        const int32_t atom0 = S.atom0, natoms = S.natoms, tile0 = S.tile0, ntile = S.ntile;
        std::memset(&S, 0, sizeof(S));
        S.atom0 = atom0; S.natoms = natoms; S.tile0 = tile0; S.ntile = ntile;
        S.method = o->method;
        S.cg_variant = o->cg_variant;
        S.ls = o->ls;
        S.m = o->lbfgs_m;
        S.max_iter = o->max_iter;
        S.max_evals = o->max_evals;
        S.restart_every = o->cg_restart_every > 0 ? o->cg_restart_every : 3 * natoms;
        S.K = o->ls_par_K;
        S.g0 = o->ls_par_g0;
        S.gtol = o->gtol_inf;
        S.h0_init = o->h0;
        S.kplus = o->k_plus;
        S.kminus = o->k_minus;
        S.eps_h = o->eps_h;
        S.fgm_restart = o->fgm_restart;
        S.hb_alpha = o->hb_alpha;
        S.hb_beta = o->hb_beta;
        S.precond_on = (o->use_learned_precond && o->method == FFMIN_LBFGS) ? 1 : 0;
        S.rec_ptr = o->record_dev;
        S.rec_every = o->record_dev ? o->record_every : 0;
        S.rec_slots = o->record_dev ? o->record_slots : 0;
        S.mixed = sys->prec == FFMIN_MIXED ? 1 : 0;
        S.mode = S.mixed ? 0 : 1;
        S.pc_window = o->pc_window;
        S.pc_rel = o->pc_rel;
        S.pc_gfar = o->pc_gfar;
        S.pc_mark_iter = 0;
        S.pc_mark_f = 0.0;
        S.active = 1;
        S.phase = PH_START;
        S.result_slot = o->method == FFMIN_FGM ? V_XB : V_X;
        S.ev_kind = EV_EG;
        S.ev_base = V_X;
        S.ev_dir = -1;
        S.ev_h = 0.0;
        S.ev_scale = 1.0;
    }
    ffmin_status st = upload_states(sys);
    if (st != FFMIN_OK) return st;
    if ((st = set_counts(sys)) != FFMIN_OK) return st;
    st = ensure_graph(sys);
    if (st != FFMIN_OK) return st;
    if ((st = ensure_loop(sys)) != FFMIN_OK) return st;
    const int64_t max_ticks = o->max_ticks > 0 ? o->max_ticks : (int64_t)o->max_evals + 64;
    int64_t ticks = 0;
    bool timeout = false;
    if (sys->loop_exec && !o->host_loop) {  // one graph launch runs the whole minimization
        sys->h_loop[0] = 0;
        sys->h_loop[1] = max_ticks;
        CK(cudaMemcpyAsync(sys->d_loop, sys->h_loop, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, sys->stream));
        CK(cudaGraphLaunch(sys->loop_exec, sys->stream));
        CK(cudaMemcpyAsync(sys->h_loop, sys->d_loop, sizeof(int64_t), cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaMemcpyAsync(sys->h_nactive, c.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
        ticks = sys->h_loop[0];
        timeout = *sys->h_nactive > 0;
        sys->last_launches = ticks * kernels_per_tick(sys) + ticks / TICKS_PER_GRAPH;
    } else {
        for (;;) {
            CK(cudaGraphLaunch(sys->graph, sys->stream));
            ticks += sys->graph_ticks;
            CK(cudaMemcpyAsync(sys->h_nactive, c.nactive, sizeof(int32_t), cudaMemcpyDeviceToHost, sys->stream));
            CK(cudaStreamSynchronize(sys->stream));
            if (*sys->h_nactive <= 0) break;
            if (ticks >= max_ticks) { timeout = true; break; }
        }
        sys->last_launches = ticks * kernels_per_tick(sys);
    }
    sys->last_ticks = ticks;
    if (timeout) {
        // a step accepted in the last round is written into X (FGM: the best
        // point) by the next round's update kernel: run that update once more
        // so that the returned point is the one the counters describe
        CK(launch_update(c, sys->stream));
        if (c.sep_reduce) CK(launch_sysreduce(c, 0, sys->stream));
        sys->last_launches += 1 + (c.sep_reduce ? 1 : 0);
    }
    st = download_states(sys);
    if (st != FFMIN_OK) return st;
    const int slot = o->method == FFMIN_FGM ? V_XB : V_X;
    CK(cudaMemcpyAsync(x_dev, vslot(c, slot), bytes, cudaMemcpyDeviceToDevice, sys->stream));
    int64_t pairs = 0;
    for (int b = 0; b < sys->n_sys; b++) {
        const SysState &S = sys->hst[b];
        ffmin_result &r = res[b];
        r.energy = S.res_f;
        r.grad_inf = S.res_ginf;
        r.iterations = S.iter;
        r.energy_evals = S.ne;
        r.grad_evals = S.neg;
        r.ls_failures = S.lsf;
        r.stop_reason = (timeout && S.active) ? FFMIN_ERR_TIMEOUT : S.status;
        r.fp64_iterations = S.mode == 1 ? S.iter - S.iter_fp64_0 : 0;
        if (timeout && S.active) {  // still running: the last accepted (FGM: best) point
            const bool fgm = S.method == FFMIN_FGM;
            r.energy = fgm ? S.fb : S.f;
            r.grad_inf = fgm ? (S.xb_known ? S.xb_ginf : std::nan("")) : S.ginf;
        }
        const int64_t nb = S.natoms;
        pairs += (int64_t)(S.ne + S.neg) * nb * (nb - 1) / 2;
    }
    sys->last_pairs = pairs;
    return FFMIN_OK;
}

ffmin_status ffmin_minimize(ffmin_system *sys, double *x_dev, const ffmin_options *o, ffmin_result *res) {
    NvtxRange nvtx_range("ffmin_minimize");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !res) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    if ((st = check_options(sys, o)) != FFMIN_OK) return st;
    st = minimize_dev(sys, x_dev, o, res);
    if (st != FFMIN_OK) return st;
    return leave(sys);
}

ffmin_status ffmin_basin_hop(ffmin_system *sys, double *x_dev, const ffmin_options *o, int32_t hops, double step,
                             uint64_t seed, ffmin_result *results, int32_t *accepted_host) {
    NvtxRange nvtx_range("ffmin_basin_hop");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !results) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    if (hops < 0 || !(step >= 0.0) || !std::isfinite(step))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "need hops >= 0 and a finite step >= 0");
    if ((st = check_options(sys, o)) != FFMIN_OK) return st;
    const Ctx &c = sys->c;
    const size_t bytes = sizeof(double) * 3 * sys->n_atoms;
    if (!sys->mbh_best) {
        CK(dalloc(sys, &sys->mbh_best, 3 * (size_t)sys->n_atoms));
        CK(dalloc(sys, &sys->mbh_flags, (size_t)sys->n_sys));
    }
    const int n = sys->n_sys;
    std::vector<ffmin_result> kept(n), cur(n);
    std::vector<int64_t> tot(5 * (size_t)n, 0);  // iterations, energy / grad evaluations, line-search failures, FP64 steps
    std::vector<int32_t> acc(n, 0), flags(n, 0);
    int64_t ticks = 0, launches = 0, pairs = 0;
    auto add = [&](const std::vector<ffmin_result> &r) {
        for (int b = 0; b < n; b++) {
            tot[5 * b] += r[b].iterations;
            tot[5 * b + 1] += r[b].energy_evals;
            tot[5 * b + 2] += r[b].grad_evals;
            tot[5 * b + 3] += r[b].ls_failures;
            tot[5 * b + 4] += r[b].fp64_iterations;
        }
        ticks += sys->last_ticks;
        launches += sys->last_launches;
        pairs += sys->last_pairs;
    };
    // the local minimum of the start
    if ((st = minimize_dev(sys, x_dev, o, kept.data())) != FFMIN_OK) return st;
    add(kept);
    CK(cudaMemcpyAsync(sys->mbh_best, x_dev, bytes, cudaMemcpyDeviceToDevice, sys->stream));
    for (int32_t h = 0; h < hops; h++) {
        CK(launch_mbh_perturb(c, sys->mbh_best, x_dev, step, seed, h, sys->stream));
        if ((st = minimize_dev(sys, x_dev, o, cur.data())) != FFMIN_OK) return st;
        add(cur);
        for (int b = 0; b < n; b++) {  // keep any finite lower result
            const bool usable = cur[b].stop_reason != FFMIN_ERR_NONFINITE && std::isfinite(cur[b].energy);
            flags[b] = usable && (!std::isfinite(kept[b].energy) || cur[b].energy < kept[b].energy) ? 1 : 0;
            if (flags[b]) {
                kept[b] = cur[b];
                acc[b]++;
            }
        }
        CK(cudaMemcpyAsync(sys->mbh_flags, flags.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice,
                           sys->stream));
        CK(launch_mbh_accept(c, sys->mbh_flags, x_dev, sys->mbh_best, sys->stream));
        CK(cudaStreamSynchronize(sys->stream));  // flags is reused by the next hop
        launches += 2;
    }
    CK(cudaMemcpyAsync(x_dev, sys->mbh_best, bytes, cudaMemcpyDeviceToDevice, sys->stream));
    for (int b = 0; b < n; b++) {
        results[b] = kept[b];
        results[b].iterations = (int32_t)std::min<int64_t>(tot[5 * b], INT32_MAX);
        results[b].energy_evals = (int32_t)std::min<int64_t>(tot[5 * b + 1], INT32_MAX);
        results[b].grad_evals = (int32_t)std::min<int64_t>(tot[5 * b + 2], INT32_MAX);
        results[b].ls_failures = (int32_t)std::min<int64_t>(tot[5 * b + 3], INT32_MAX);
        results[b].fp64_iterations = (int32_t)std::min<int64_t>(tot[5 * b + 4], INT32_MAX);
        if (accepted_host) accepted_host[b] = acc[b];
    }
    sys->last_ticks = ticks;
    sys->last_launches = launches;
    sys->last_pairs = pairs;
    return leave(sys);
}

ffmin_status ffmin_minimize_host(ffmin_system *sys, double *x_host, const ffmin_options *o, ffmin_result *res) {
    NvtxRange nvtx_range("ffmin_minimize_host");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_host || !res) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    if ((st = check_options(sys, o)) != FFMIN_OK) return st;
    const size_t bytes = sizeof(double) * 3 * sys->n_atoms;
    double *stage = vslot(sys->c, V_XIN);
    CK(cudaMemcpyAsync(stage, x_host, bytes, cudaMemcpyHostToDevice, sys->stream));
    st = minimize_dev(sys, stage, o, res);
    if (st != FFMIN_OK) return st;
    CK(cudaMemcpyAsync(x_host, stage, bytes, cudaMemcpyDeviceToHost, sys->stream));
    return leave(sys);
}

ffmin_status ffmin_time_pair_kernel(ffmin_system *sys, const double *x_dev, int32_t with_grad, int32_t reps,
                                    float *ms) {
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !ms || reps < 1 || with_grad < 0 || with_grad > 2 ||
        (with_grad == 2 && sys->prec != FFMIN_MIXED))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "bad argument");
    // one full evaluation leaves the positions of x in the pair-kernel inputs
    st = eval_all(sys, x_dev, with_grad == 1 ? EV_EG : EV_E);
    if (st != FFMIN_OK) return st;
    if (with_grad == 2) CK(cudaMemsetAsync(sys->c.dispf, 0, sizeof(float4) * sys->n_atoms, sys->stream));
    for (int b = 0; b < sys->n_sys; b++) {
        sys->hst[b].ev_kind = with_grad == 1 ? EV_EG : EV_E;
        sys->hst[b].ev_delta = with_grad == 2 ? 1 : 0;
    }
    if ((st = upload_states(sys)) != FFMIN_OK) return st;
    if ((st = set_counts(sys)) != FFMIN_OK) return st;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(launch_pair(sys->c, sys->grid32, sys->grid32e, sys->grid64, sys->stream));  // warm-up
    CK(cudaEventRecord(e0, sys->stream));
    for (int r = 0; r < reps; r++) CK(launch_pair(sys->c, sys->grid32, sys->grid32e, sys->grid64, sys->stream));
    CK(cudaEventRecord(e1, sys->stream));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / (float)reps;
    for (int b = 0; b < sys->n_sys; b++) {
        sys->hst[b].ev_kind = EV_NONE;
        sys->hst[b].ev_delta = 0;
    }
    if ((st = upload_states(sys)) != FFMIN_OK) return st;
    return leave(sys);
}

ffmin_status ffmin_neighbour_counts(ffmin_system *sys, const double *x_dev, int32_t *counts_dev) {
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev || !counts_dev) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    // the kernel reads each system's atom range from the device state
    if ((st = upload_states(sys)) != FFMIN_OK) return st;
    CK(launch_ncount(sys->c, x_dev, counts_dev, sys->stream));
    return leave(sys);
}

// Installs the work-item layout of a density (both lists, the tiles' list
// fields, grid sizes) and the FP32 kernel shape; the captured graphs are
// rebuilt at the next minimization.
static ffmin_status install_layout(ffmin_system *sys, int dens, int ipt) {
    sys->c.f32_ipt = ipt;
    sys->grid32_max = sys->grid32_max_s[ipt - 1];
    sys->grid32e_max = sys->grid32e_max_s[ipt - 1];
    std::vector<Item> items, items64;
    std::vector<Tile> tiles;
    std::vector<int2> sys_items, sys_items64;
    if (sys->c.sym64) {  // the symmetric list first: it sets the tiles' row64 / chunk64 / slot64
        int64_t slots = 0;
        build_items64(sys, (int64_t)dens * sys->grid_sym, items64, sys_items64, &slots);
        CK(cudaMemcpyAsync(sys->d_items64, items64.data(), items64.size() * sizeof(Item), cudaMemcpyHostToDevice,
                           sys->stream));
        CK(cudaMemcpyAsync(sys->d_sys_items64, sys_items64.data(), sys_items64.size() * sizeof(int2),
                           cudaMemcpyHostToDevice, sys->stream));
        sys->n_items64 = (int)items64.size();
        sys->c.n_items64 = sys->n_items64;
    }
    build_items(sys, dens, items, tiles, sys_items);
    CK(cudaMemcpyAsync(sys->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice,
                       sys->stream));
    CK(cudaMemcpyAsync(sys->d_sys_items, sys_items.data(), sys_items.size() * sizeof(int2), cudaMemcpyHostToDevice,
                       sys->stream));
    CK(cudaMemcpyAsync(sys->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                       sys->stream));
    set_item_counts(sys, (int)items.size());
    sys->density = dens;
    if (sys->graph) {  // kernel parameters (item count, grid, shape) changed
        cudaGraphExecDestroy(sys->graph);
        sys->graph = nullptr;
    }
    if (sys->loop_exec) {
        cudaGraphExecDestroy(sys->loop_exec);
        sys->loop_exec = nullptr;
    }
    return FFMIN_OK;
}

ffmin_status ffmin_autotune(ffmin_system *sys, const double *x_dev, int32_t *density_out) {
    NvtxRange nvtx_range("ffmin_autotune");
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (!x_dev) return fail(sys, FFMIN_ERR_INVALID_ARG, "NULL argument");
    float best_ms = 0.f;
    int best = sys->density, best_ipt = sys->c.f32_ipt;
    bool have = false;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // FP32 shapes: both for MIXED objects, whose FP32 kernels do the work
    const int n_shapes = sys->prec == FFMIN_MIXED ? 2 : 1;
    for (int sh = 0; sh < n_shapes; sh++) {
        const int ipt = 2 - sh;
        for (int k = 0; k < AUTOTUNE_N; k++) {
            const int dens = AUTOTUNE_DENSITIES[k];
            if ((st = install_layout(sys, dens, ipt)) != FFMIN_OK) return st;
            if ((st = eval_all(sys, x_dev, EV_EG)) != FFMIN_OK) return st;
            // score: one E + grad launch and three energy-only launches, the
            // mix of an L-BFGS step with LS_PAR (the row list serves the FP32
            // E + grad, the symmetric list the FP64 terms and every
            // energy-only pass)
            float ms = 0.f;
            for (int kind : {EV_EG, EV_E}) {
                for (int b = 0; b < sys->n_sys; b++) sys->hst[b].ev_kind = kind;
                if ((st = upload_states(sys)) != FFMIN_OK) return st;
                if ((st = set_counts(sys)) != FFMIN_OK) return st;
                CK(launch_pair(sys->c, sys->grid32, sys->grid32e, sys->grid64, sys->stream));
                CK(cudaEventRecord(e0, sys->stream));
                for (int r = 0; r < 3; r++) CK(launch_pair(sys->c, sys->grid32, sys->grid32e, sys->grid64, sys->stream));
                CK(cudaEventRecord(e1, sys->stream));
                CK(cudaEventSynchronize(e1));
                float t = 0.f;
                CK(cudaEventElapsedTime(&t, e0, e1));
                ms += kind == EV_EG ? t / 3.f : t;
            }
            if (!have || ms < best_ms) { best_ms = ms; best = dens; best_ipt = ipt; have = true; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((st = install_layout(sys, best, best_ipt)) != FFMIN_OK) return st;
    for (int b = 0; b < sys->n_sys; b++) sys->hst[b].ev_kind = EV_NONE;
    if ((st = upload_states(sys)) != FFMIN_OK) return st;
    if (density_out) *density_out = best;
    return leave(sys);
}

ffmin_status ffmin_set_tuning(ffmin_system *sys, int32_t density, int32_t f32_atoms_per_thread) {
    ffmin_status st = enter(sys);
    if (st != FFMIN_OK) return st;
    if (density < 1 || density > AUTOTUNE_DENSITIES[AUTOTUNE_N - 1] ||
        (f32_atoms_per_thread != 1 && f32_atoms_per_thread != 2))
        return fail(sys, FFMIN_ERR_INVALID_ARG, "density in [1, 20], f32_atoms_per_thread 1 or 2");
    if ((st = install_layout(sys, density, f32_atoms_per_thread)) != FFMIN_OK) return st;
    return leave(sys);
}

ffmin_status ffmin_get_tuning(const ffmin_system *sys, int32_t *density, int32_t *f32_atoms_per_thread) {
    if (!sys) return FFMIN_ERR_INVALID_ARG;
    if (density) *density = sys->density;
    if (f32_atoms_per_thread) *f32_atoms_per_thread = sys->c.f32_ipt;
    return FFMIN_OK;
}

ffmin_status ffmin_last_stats(const ffmin_system *sys, int64_t *ticks, int64_t *launches, int64_t *pairs) {
    if (!sys) return FFMIN_ERR_INVALID_ARG;
    if (ticks) *ticks = sys->last_ticks;
    if (launches) *launches = sys->last_launches;
    if (pairs) *pairs = sys->last_pairs;
    return FFMIN_OK;
}

ffmin_status ffmin_set_precond(ffmin_system *sys, const uint16_t *w, int32_t n_params) {
    if (!sys || !w || n_params != 449) return fail(sys, FFMIN_ERR_INVALID_ARG, "need 449 FP16 weights");
    cudaError_t e = cudaMemcpy((void *)sys->c.mlp_w, w, sizeof(uint16_t) * 449, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(sys, e, "ffmin_set_precond");
    sys->have_precond = true;
    return FFMIN_OK;
}

}  // extern "C"


// ---------------------------------------------------------------- parab
static const int PARAB_MOVES = 64;  // moves per graph replay

static ffmin_status parab_minimize(ffmin_system *sys, const ffmin_options *o, ffmin_result *res) {
    const Ctx &c = sys->c;
    const int n = sys->hst[0].natoms;
    const int mode = sys->prec == FFMIN_MIXED ? 0 : 1;
    if (!sys->parab_state) {
        CK(cudaMalloc(&sys->parab_state, parab_state_bytes()));
        sys->allocs.push_back(sys->parab_state);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        sys->parab_grid = std::max(1, std::min((n + TI - 1) / TI, 2 * sms));
    }
    std::vector<char> hbuf(parab_state_bytes());
    parab_state_init(hbuf.data(), n, (int)sys->atom_off[0], mode, o->max_iter, o->seed, o->gradfree_delta,
                     o->gradfree_taylor_r);
    CK(cudaMemcpyAsync(sys->parab_state, hbuf.data(), hbuf.size(), cudaMemcpyHostToDevice, sys->stream));
    ffm::ParabState *ps = (ffm::ParabState *)sys->parab_state;
    if (!sys->parab_graph) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(sys->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < PARAB_MOVES && e == cudaSuccess; k++) e = launch_parab_move(c, ps, sys->parab_grid, sys->stream);
        cudaError_t e2 = cudaStreamEndCapture(sys->stream, &g);
        if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(sys, e, "parab capture"); }
        if (e2 != cudaSuccess) return cuda_fail(sys, e2, "parab capture end");
        e = cudaGraphInstantiate(&sys->parab_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(sys, e, "parab instantiate");
    }
    // initial evaluation (also writes the pair-kernel positions of X)
    ffmin_status st = eval_slot(sys, V_X, EV_EG);
    if (st != FFMIN_OK) return st;
    int32_t neg = 1, moves = 0, status = FFMIN_OK;
    double f = sys->hst[0].res_f, ginf = sys->hst[0].res_ginf;
    int64_t launches = 3, ticks = 0;
    if (sys->hst[0].status == FFMIN_ERR_NONFINITE) status = FFMIN_ERR_NONFINITE;
    // a sweep is N moves; the stopping test follows each complete sweep; an
    // iteration cap that cuts a sweep (or starts one) ends with one more
    // evaluation that reports the returned point
    while (status == FFMIN_OK && !(ginf < o->gtol_inf)) {
        bool truncated = moves >= o->max_iter;
        if (!truncated) {
            const int32_t stop = (int32_t)std::min<int64_t>((int64_t)moves + n, o->max_iter);
            truncated = stop < moves + n;
            CK(cudaMemcpyAsync((char *)sys->parab_state + parab_offset_stop(), &stop, sizeof(int32_t),
                               cudaMemcpyHostToDevice, sys->stream));
            for (int32_t k = moves; k < stop; k += PARAB_MOVES) {
                CK(cudaGraphLaunch(sys->parab_graph, sys->stream));
                launches += 2 * PARAB_MOVES;
                ticks += PARAB_MOVES;
            }
            CK(cudaMemcpyAsync(sys->h_nactive, (char *)sys->parab_state + parab_offset_move(), sizeof(int32_t),
                               cudaMemcpyDeviceToHost, sys->stream));
            CK(cudaStreamSynchronize(sys->stream));
            moves = *sys->h_nactive;
            if (moves != stop) return fail(sys, FFMIN_ERR_CUDA, "gradient-free moves did not all run");
        }
        st = eval_slot(sys, V_X, EV_EG);
        if (st != FFMIN_OK) return st;
        neg++;
        launches += 3;
        f = sys->hst[0].res_f;
        ginf = sys->hst[0].res_ginf;
        if (sys->hst[0].status == FFMIN_ERR_NONFINITE) { status = FFMIN_ERR_NONFINITE; break; }
        if (truncated) { status = FFMIN_ERR_MAX_ITER; break; }
    }
    res[0].energy = f;
    res[0].grad_inf = ginf;
    res[0].iterations = moves;
    res[0].energy_evals = 8 * moves;
    res[0].grad_evals = neg;
    res[0].ls_failures = 0;
    res[0].stop_reason = status;
    res[0].fp64_iterations = sys->prec == FFMIN_MIXED ? 0 : moves;
    sys->last_ticks = ticks;
    sys->last_launches = launches;
    sys->last_pairs = (int64_t)moves * 8 * (n - 1) + (int64_t)neg * n * (int64_t)(n - 1) / 2;
    return FFMIN_OK;
}

// ---------------------------------------------------------------------------
// Parallel epochs of the gradient-free search (options.gradfree_parts >= 1).
// The host cuts the parts every epoch (recursive bisection of the current
// positions: a set meant for p parts is ordered by (coordinate on its axis of
// largest extent, index) and split at rank round(|A| floor(p/2) / p), halves
// up, plus a shift pick(seed, 2^62 + e 2^20 + node, span) - span / 2,
// span = max(1, |A| / (2p)), clamped to [1, |A| - 1]; the cut plane lies
// halfway between the atoms on either side; left half first), lists every
// part's atoms and its movable atoms (at least `margin` from each cut plane
// of its box, index order) and the moves each part may make under the cap;
// one block per part then runs the epoch (k_epoch) and the gradient is
// checked on the merged positions.
static uint64_t host_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static int32_t host_pick(uint64_t seed, uint64_t k, int32_t n) {
    return (int32_t)(((unsigned __int128)host_splitmix64(seed, k) * (uint64_t)n) >> 64);
}

struct Cutter {
    const double *x;
    uint64_t seed, e;
    std::vector<int32_t> part;
    std::vector<std::array<double, 6>> box;
    void run(std::vector<int32_t> &A, size_t a0, size_t na, int p, std::array<double, 6> b, uint64_t node) {
        if (p == 1) {
            const int32_t q = (int32_t)box.size();
            for (size_t t = a0; t < a0 + na; t++) part[A[t]] = q;
            box.push_back(b);
            return;
        }
        int axis = 0;
        double ext[3];
        for (int k = 0; k < 3; k++) {
            double mn = x[3 * A[a0] + k], mx = mn;
            for (size_t t = a0 + 1; t < a0 + na; t++) {
                mn = std::min(mn, x[3 * A[t] + k]);
                mx = std::max(mx, x[3 * A[t] + k]);
            }
            ext[k] = mx - mn;
        }
        if (ext[1] > ext[axis]) axis = 1;
        if (ext[2] > ext[axis]) axis = 2;
        const int p1 = p / 2;
        const int32_t span = std::max<int32_t>(1, (int32_t)(na / (2 * (size_t)p)));
        int64_t c = (2LL * (int64_t)na * p1 + p) / (2LL * p) +
                    host_pick(seed, (1ULL << 62) + (e << 20) + node, span) - span / 2;
        c = std::max<int64_t>(1, std::min<int64_t>(c, (int64_t)na - 1));
        // the order (coordinate, index) is strict, so the c smallest atoms
        // and the atoms on either side of the cut are unique: a selection
        // (linear time) instead of a sort
        auto less = [&](int32_t u, int32_t v) {
            const double cu = x[3 * u + axis], cv = x[3 * v + axis];
            return cu < cv || (cu == cv && u < v);
        };
        std::nth_element(A.begin() + a0, A.begin() + a0 + c, A.begin() + a0 + na, less);
        const int32_t right = A[a0 + c];
        const int32_t left = *std::max_element(A.begin() + a0, A.begin() + a0 + c, less);
        const double plane = 0.5 * (x[3 * left + axis] + x[3 * right + axis]);
        std::array<double, 6> bl = b, br = b;
        bl[3 + axis] = plane;
        br[axis] = plane;
        run(A, a0, (size_t)c, p1, bl, 2 * node + 1);
        run(A, a0 + (size_t)c, na - (size_t)c, p - p1, br, 2 * node + 2);
    }
};

static ffmin_status epoch_minimize(ffmin_system *sys, const ffmin_options *o, ffmin_result *res) {
    Ctx &c = sys->c;
    const int n = sys->hst[0].natoms;
    const int P = std::min(o->gradfree_parts, n);
    const int mode = sys->prec == FFMIN_MIXED ? 0 : 1;
    if (sys->ep_parts < P) {  // per-part copies (kept for later runs)
        for (void *p : {(void *)sys->ep_view, (void *)sys->ep_viewf, (void *)sys->ep_ints}) {
            if (!p) continue;
            cudaFree(p);
            sys->allocs.erase(std::remove(sys->allocs.begin(), sys->allocs.end(), p), sys->allocs.end());
        }
        sys->ep_view = nullptr;
        sys->ep_viewf = nullptr;
        sys->ep_ints = nullptr;
        CK(cudaMalloc(&sys->ep_view, sizeof(double) * 3 * (size_t)n * P));
        sys->allocs.push_back(sys->ep_view);
        if (sys->prec == FFMIN_MIXED) {
            CK(cudaMalloc(&sys->ep_viewf, sizeof(float4) * (size_t)n * P));
            sys->allocs.push_back(sys->ep_viewf);
        }
        CK(cudaMalloc(&sys->ep_ints, sizeof(int32_t) * (2 * (size_t)n + 3 * (size_t)P + 2)));
        sys->allocs.push_back(sys->ep_ints);
        sys->ep_parts = P;
    }
    int32_t *d_list = sys->ep_ints, *d_members = d_list + n, *d_loff = d_members + n;
    int32_t *d_moff = d_loff + P + 1, *d_allowed = d_moff + P + 1;
    ffmin_status st = eval_slot(sys, V_X, EV_EG);
    if (st != FFMIN_OK) return st;
    int32_t neg = 1, moves = 0, status = FFMIN_OK;
    double f = sys->hst[0].res_f, ginf = sys->hst[0].res_ginf;
    int64_t launches = 3, ticks = 0;
    if (sys->hst[0].status == FFMIN_ERR_NONFINITE) status = FFMIN_ERR_NONFINITE;
    std::vector<double> xh(3 * (size_t)n);
    std::vector<int32_t> A(n), ints(2 * (size_t)n + 3 * (size_t)P + 2);
    const double w = o->gradfree_margin;
    const double inf = std::numeric_limits<double>::infinity();
    bool report = false;  // a cap or an empty epoch: one more evaluation reports the point
    for (uint64_t e = 0; status == FFMIN_OK && !(ginf < o->gtol_inf); e++) {
        if (moves >= o->max_iter) { status = FFMIN_ERR_MAX_ITER; report = true; break; }
        CK(cudaMemcpyAsync(xh.data(), vslot(c, V_X), sizeof(double) * xh.size(), cudaMemcpyDeviceToHost,
                           sys->stream));
        CK(cudaStreamSynchronize(sys->stream));
        Cutter cut{xh.data(), o->seed, e, std::vector<int32_t>(n, 0), {}};
        for (int a = 0; a < n; a++) A[a] = a;
        cut.run(A, 0, (size_t)n, P, {-inf, -inf, -inf, inf, inf, inf}, 0);
        int32_t *list = ints.data(), *members = list + n, *loff = members + n, *moff = loff + P + 1;
        int32_t *allowed = moff + P + 1;
        int32_t nl = 0, off = 0, sum = 0;
        bool truncated = false;
        // members of every part in index order (counting sort by part)
        for (int q = 0; q <= P; q++) moff[q] = 0;
        for (int a = 0; a < n; a++) moff[cut.part[a] + 1]++;
        for (int q = 0; q < P; q++) moff[q + 1] += moff[q];
        {
            std::vector<int32_t> fill(moff, moff + P);
            for (int a = 0; a < n; a++) members[fill[cut.part[a]]++] = a;
        }
        for (int q = 0; q < P; q++) {
            loff[q] = nl;
            const std::array<double, 6> &b = cut.box[q];
            for (int t = moff[q]; t < moff[q + 1]; t++) {
                const int a = members[t];
                bool ok = true;
                for (int k = 0; k < 3; k++)
                    if (xh[3 * a + k] - b[k] < w || b[3 + k] - xh[3 * a + k] < w) ok = false;
                if (ok) list[nl++] = a;
            }
            const int32_t m_q = nl - loff[q];
            int64_t al = (int64_t)o->max_iter - moves - off;
            al = std::max<int64_t>(0, std::min<int64_t>(al, m_q));
            if (al < m_q) truncated = true;
            allowed[q] = (int32_t)al;
            sum += (int32_t)al;
            off += m_q;
        }
        loff[P] = nl;
        CK(cudaMemcpyAsync(sys->ep_ints, ints.data(), sizeof(int32_t) * ints.size(), cudaMemcpyHostToDevice,
                           sys->stream));
        EpochArgs ea{sys->ep_view, sys->ep_viewf, d_list, d_loff, d_allowed, d_members, d_moff,
                     n, mode, o->seed, e, o->gradfree_delta,
                     o->gradfree_taylor_r > 0.0 ? o->gradfree_taylor_r * o->gradfree_taylor_r : 0.0};
        CK(launch_epoch(c, ea, P, sys->stream));
        launches += 1;
        ticks += 1;
        moves += sum;
        if (truncated) { status = FFMIN_ERR_MAX_ITER; report = true; break; }
        st = eval_slot(sys, V_X, EV_EG);
        if (st != FFMIN_OK) return st;
        neg++;
        launches += 3;
        f = sys->hst[0].res_f;
        ginf = sys->hst[0].res_ginf;
        if (sys->hst[0].status == FFMIN_ERR_NONFINITE) { status = FFMIN_ERR_NONFINITE; break; }
        if (ginf < o->gtol_inf) break;
        if (off == 0) { status = FFMIN_ERR_MAX_ITER; report = true; break; }
    }
    if (report) {
        st = eval_slot(sys, V_X, EV_EG);
        if (st != FFMIN_OK) return st;
        neg++;
        launches += 3;
        f = sys->hst[0].res_f;
        ginf = sys->hst[0].res_ginf;
    }
    res[0].energy = f;
    res[0].grad_inf = ginf;
    res[0].iterations = moves;
    res[0].energy_evals = 8 * moves;
    res[0].grad_evals = neg;
    res[0].ls_failures = 0;
    res[0].stop_reason = status;
    res[0].fp64_iterations = sys->prec == FFMIN_MIXED ? 0 : moves;
    sys->last_ticks = ticks;
    sys->last_launches = launches;
    sys->last_pairs = (int64_t)moves * 8 * (n - 1) + (int64_t)neg * n * (int64_t)(n - 1) / 2;
    return FFMIN_OK;
}

extern "C" ffmin_status ffmin_epoch_parts(const double *x_host, int32_t n, int32_t parts, uint64_t seed,
                                          uint64_t epoch, double margin, int32_t *part_out,
                                          int32_t *movable_out) {
    if (!x_host || n < 1 || parts < 1 || !part_out || !movable_out || !(margin >= 0.0))
        return FFMIN_ERR_INVALID_ARG;
    const int P = std::min<int32_t>(parts, n);
    const double inf = std::numeric_limits<double>::infinity();
    Cutter cut{x_host, seed, epoch, std::vector<int32_t>(n, 0), {}};
    std::vector<int32_t> A(n);
    for (int a = 0; a < n; a++) A[a] = a;
    cut.run(A, 0, (size_t)n, P, {-inf, -inf, -inf, inf, inf, inf}, 0);
    for (int a = 0; a < n; a++) {
        part_out[a] = cut.part[a];
        const std::array<double, 6> &b = cut.box[cut.part[a]];
        bool ok = true;
        for (int k = 0; k < 3; k++)
            if (x_host[3 * a + k] - b[k] < margin || b[3 + k] - x_host[3 * a + k] < margin) ok = false;
        movable_out[a] = ok ? 1 : 0;
    }
    return FFMIN_OK;
}
