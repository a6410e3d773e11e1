// Gradient-free "parab" minimization (arXiv 1810.03358, Section 3): each move
// picks a random atom i, evaluates the part of E that depends on atom i at
// its position and at +-delta along each axis (7 points), fits a parabola
// per axis through the three values on that axis, evaluates its vertex (the
// 8th point) and moves the atom to the best of the 8 (ties: the earlier
// point).  |grad E|_inf is checked after every sweep of N moves.
//
// With a far-field radius r_far > 0 (options.gradfree_taylor_r), the Coulomb
// term of every atom j at least r_far from atom i's current position x_i is
// replaced by its first-order Taylor expansion about x_i, e0 (1 + d0.(p -
// x_i) / r0^2) with d0 = x_j - x_i and e0 its value at x_i (Section 3's
// linearised far field for single-atom moves); Lennard-Jones stays exact.
//
// The random atom of move k is the k-th output of the counter-based
// SplitMix64 stream (Steele, Lea and Flood 2014) with the user's seed, scaled
// to [0, N) by a 64x64 -> 128-bit multiply (high word).
//
// A move costs two launches over all j (7 rows, then the vertex row); the
// last block of each launch reduces the block partials in a fixed order and
// takes the move's decision, so the moves of a sweep replay as a CUDA graph
// with no host involvement.
#include <cmath>
#include <cstring>

#include "bonded.cuh"
#include "ffmin_internal.cuh"
#include "reduce.cuh"

struct ffmin_system;

namespace ffm {

struct ParabState {
    int32_t move, stop_at, max_moves, n;
    int32_t atom0, mode, atom, best;
    uint64_t seed;
    double delta;
    double taylor_r2;  // r_far^2 of the linearised far field, 0 = exact rows
    double f[8];
    double p[8][3];
};

__device__ __forceinline__ int pick_atom(uint64_t seed, uint64_t k, int n) {
    return (int)__umul64hi(splitmix64(seed, k), (uint64_t)n);
}

// Pair part of the row energy of atom i placed at each of NP positions,
// this thread's share of the j atoms: j = j0, j0 + stride, ... (FP64
// accumulation of FP64 terms, or FP32 sums of FP32 terms in the mixed form);
// pos / posf give the other atoms, xi atom i's current position, tr2 the
// squared far-field radius (0: exact rows).
template <int NP>
__device__ void row_sums(const Ctx &c, int mode, const double4_32a *pos, const float4 *posf,
                         const double2 *par, const float2 *parf, int n, int i, const double (*p)[3],
                         const double *xi, double tr2, int j0, int stride, double *acc) {
    for (int q = 0; q < NP; q++) acc[q] = 0.0;
    if (mode == 1) {
        const double qi = pos[i].w;
        const double2 ci = par[i];
        for (int j = j0; j < n; j += stride) {
            if (j == i) continue;
            const double4_32a pj = pos[j];
            const double2 cj = par[j];
            const double c6 = ci.x * cj.x, c12 = ci.y * cj.y, qq = qi * pj.w;
            bool far = false;
            double e0 = 0.0, fac = 0.0;
            const double d0x = pj.x - xi[0], d0y = pj.y - xi[1], d0z = pj.z - xi[2];
            if (tr2 > 0.0) {
                const double r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                if (r02 >= tr2) {
                    far = true;
                    e0 = qq * rsqrt(r02);
                    fac = e0 / r02;
                }
            }
            for (int q = 0; q < NP; q++) {
                const double dx = pj.x - p[q][0], dy = pj.y - p[q][1], dz = pj.z - p[q][2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = rsqrt(r2);
                const double ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
                const double lj = ri6 * (c12 * ri6 - c6) * (1.0 / 6.0);
                if (far) {
                    const double dd = d0x * (p[q][0] - xi[0]) + d0y * (p[q][1] - xi[1]) + d0z * (p[q][2] - xi[2]);
                    acc[q] += e0 + fac * dd + lj;
                } else {
                    acc[q] += qq * ri + lj;
                }
            }
        }
    } else {
        const float qi = posf[i].w;
        const float2 ci = parf[i];
        float pf[NP][3], accf[NP];
        for (int q = 0; q < NP; q++) {
            accf[q] = 0.f;
            for (int a = 0; a < 3; a++) pf[q][a] = (float)p[q][a];
        }
        const float xf[3] = {(float)xi[0], (float)xi[1], (float)xi[2]};
        const float tr2f = (float)tr2;
        // FP32 sums of this thread's j (tile-local FP32 accumulation of the
        // mixed form), FP64 from the block reduction on
        for (int j = j0; j < n; j += stride) {
            if (j == i) continue;
            const float4 pj = posf[j];
            const float2 cj = parf[j];
            const float c6 = ci.x * cj.x, c12 = ci.y * cj.y, qq = qi * pj.w;
            bool far = false;
            float e0 = 0.f, fac = 0.f;
            const float d0x = pj.x - xf[0], d0y = pj.y - xf[1], d0z = pj.z - xf[2];
            if (tr2f > 0.f) {
                const float r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                if (r02 >= tr2f) {
                    far = true;
                    e0 = qq * rsqrtf(r02);
                    fac = e0 / r02;
                }
            }
            for (int q = 0; q < NP; q++) {
                const float dx = pj.x - pf[q][0], dy = pj.y - pf[q][1], dz = pj.z - pf[q][2];
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float ri = rsqrtf(r2);
                const float ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
                const float lj = ri6 * (c12 * ri6 - c6) * (1.0f / 6.0f);
                if (far) {
                    const float dd = d0x * (pf[q][0] - xf[0]) + d0y * (pf[q][1] - xf[1]) + d0z * (pf[q][2] - xf[2]);
                    accf[q] += e0 + fac * dd + lj;
                } else {
                    accf[q] += qq * ri + lj;
                }
            }
        }
        for (int q = 0; q < NP; q++) acc[q] = (double)accf[q];
    }
}

// the grid's share of one row evaluation over the system's atoms
template <int NP>
__device__ void row_partial(const Ctx &c, const ParabState *ps, int i, const double (*p)[3], const double *xi,
                            double *acc) {
    const int a0 = ps->atom0;
    row_sums<NP>(c, ps->mode, c.posd + a0, c.posf + a0, c.pard + a0, c.parf + a0, ps->n, i, p, xi, ps->taylor_r2,
                 blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, acc);
}

// bonded terms containing atom i (global index a) with atom i at p
__device__ double row_bonded(const Ctx &c, int a, const double *p) {
    const double *x = vslot(c, V_X);
    double e = 0.0;
    for (int k = c.inc_off[a]; k < c.inc_off[a + 1]; k++) {
        const int2 in = c.inc[k];
        e += bonded_term(c, x, in.x >> 2, in.y, in.x & 3, nullptr, nullptr, a, p);
    }
    return e;
}

// 7 row energies: current position and +-delta along x, y, z
__global__ void __launch_bounds__(TI) k_parab_rows(Ctx c, ParabState *ps) {
    if (ps->move >= ps->stop_at) return;
    const int n = ps->n, atom0 = ps->atom0;
    const int i = pick_atom(ps->seed, (uint64_t)ps->move, n);
    const double *X = vslot(c, V_X);
    double p[7][3];
    for (int q = 0; q < 7; q++)
        for (int a = 0; a < 3; a++) p[q][a] = X[3 * (atom0 + i) + a];
    for (int a = 0; a < 3; a++) {
        p[1 + 2 * a][a] = p[1 + 2 * a][a] + ps->delta;
        p[2 + 2 * a][a] = p[2 + 2 * a][a] - ps->delta;
    }
    double acc[7];
    row_partial<7>(c, ps, i, p, p[0], acc);  // p[0]: the current position
    double v[7];
    for (int q = 0; q < 7; q++) v[q] = acc[q];
    block_reduce_store<7>(v, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    if (!last_block(&c.counters[CNT_PARAB])) return;
    __shared__ double tot[7];
    if (threadIdx.x < 7) {
        const int q = threadIdx.x;
        double t = 0.0;
        for (int b = 0; b < gridDim.x; b++) t += __ldcg(&c.red[(int64_t)b * NRED + q]);
        tot[q] = t + row_bonded(c, atom0 + i, p[q]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ps->atom = i;
        for (int q = 0; q < 7; q++) {
            ps->f[q] = tot[q];
            for (int a = 0; a < 3; a++) ps->p[q][a] = p[q][a];
        }
        for (int a = 0; a < 3; a++) {  // per-axis parabola vertex
            const double fp = tot[1 + 2 * a], fm = tot[2 + 2 * a];
            const double curv = fm - 2.0 * tot[0] + fp;
            const double ts = curv > 0.0 ? ps->delta * (fm - fp) / (2.0 * curv) : 0.0;
            ps->p[7][a] = p[0][a] + ts;
        }
        c.counters[CNT_PARAB] = 0;
    }
}

// the vertex row, the decision and the move
__global__ void __launch_bounds__(TI) k_parab_vertex(Ctx c, ParabState *ps) {
    if (ps->move >= ps->stop_at) return;
    const int atom0 = ps->atom0, i = ps->atom;
    double p[1][3];
    for (int a = 0; a < 3; a++) p[0][a] = ps->p[7][a];
    double acc[1];
    row_partial<1>(c, ps, i, p, ps->p[0], acc);  // ps->p[0]: the current position
    double v[1] = {acc[0]};
    block_reduce_store<1>(v, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    if (!last_block(&c.counters[CNT_PARAB2])) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < gridDim.x; b++) t += __ldcg(&c.red[(int64_t)b * NRED]);
        ps->f[7] = t + row_bonded(c, atom0 + i, p[0]);
        int best = 0;
        for (int q = 1; q < 8; q++)
            if (ps->f[q] < ps->f[best]) best = q;
        ps->best = best;
        const int a = atom0 + i;
        double *X = vslot(c, V_X);
        for (int k = 0; k < 3; k++) X[3 * a + k] = ps->p[best][k];
        const double q = c.qs[a];
        if (ps->mode == 1)
            c.posd[a] = make_double4_32a(X[3 * a], X[3 * a + 1], X[3 * a + 2], q);
        else
            c.posf[a] = make_float4((float)X[3 * a], (float)X[3 * a + 1], (float)X[3 * a + 2], (float)q);
        ps->move = ps->move + 1;
        __threadfence();
        c.counters[CNT_PARAB2] = 0;
    }
}

cudaError_t launch_parab_move(const Ctx &c, ParabState *ps, int grid, cudaStream_t s) {
    k_parab_rows<<<grid, TI, 0, s>>>(c, ps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_parab_vertex<<<grid, TI, 0, s>>>(c, ps);
    return cudaGetLastError();
}

size_t parab_state_bytes() { return sizeof(ParabState); }

void parab_state_init(void *host_buf, int n, int atom0, int mode, int max_moves, uint64_t seed,
                      double delta, double taylor_r) {
    ParabState ps;
    std::memset(&ps, 0, sizeof(ps));
    ps.n = n;
    ps.atom0 = atom0;
    ps.mode = mode;
    ps.max_moves = max_moves;
    ps.stop_at = 0;
    ps.seed = seed;
    ps.delta = delta;
    ps.taylor_r2 = taylor_r > 0.0 ? taylor_r * taylor_r : 0.0;
    std::memcpy(host_buf, &ps, sizeof(ps));
}

size_t parab_offset_move() { return offsetof(ParabState, move); }
size_t parab_offset_stop() { return offsetof(ParabState, stop_at); }

// ---------------------------------------------------------------------------
// Parallel epochs of the gradient-free search (Section 3's proposal: cut the
// molecule into parts, move atoms away from the cuts in every part at once,
// merge, cut again).  One block per part q works on its own copy of the
// epoch's starting positions (FP64 [3N] and, for MIXED, FP32 (x, y, z, q')),
// so it sees its own moves and the other parts as they were at the start of
// the epoch; moves are those of the sequential method (7 rows, per-axis
// parabola vertices, the best of 8) with row sums reduced by the block in a
// fixed order.  Move m of part q picks its movable atom list entry
// pick(seed, q 2^40 + e N + m, |L_q|).  The host cuts the parts.
constexpr int EPOCH_THREADS = 256;

// row sums of NP positions of atom i over the part's copy: this thread's j
// (the part's FP64 copy V is read through a double4-free view: positions
// from V, charges q' from c.qs)
template <int NP>
__device__ void epoch_rows(const Ctx &c, const EpochArgs &a, const double *V, const float4 *Vf, int i,
                           const double (*p)[3], double *acc) {
    for (int q = 0; q < NP; q++) acc[q] = 0.0;
    const double xi[3] = {V[3 * i], V[3 * i + 1], V[3 * i + 2]};  // current position
    if (a.mode == 1) {
        const double qi = c.qs[i];
        const double2 ci = c.pard[i];
        for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
            if (j == i) continue;
            const double xj = V[3 * j], yj = V[3 * j + 1], zj = V[3 * j + 2];
            const double2 cj = c.pard[j];
            const double c6 = ci.x * cj.x, c12 = ci.y * cj.y, qq = qi * c.qs[j];
            bool far = false;
            double e0 = 0.0, fac = 0.0;
            const double d0x = xj - xi[0], d0y = yj - xi[1], d0z = zj - xi[2];
            if (a.taylor_r2 > 0.0) {
                const double r02 = d0x * d0x + d0y * d0y + d0z * d0z;
                if (r02 >= a.taylor_r2) {
                    far = true;
                    e0 = qq * rsqrt(r02);
                    fac = e0 / r02;
                }
            }
            for (int q = 0; q < NP; q++) {
                const double dx = xj - p[q][0], dy = yj - p[q][1], dz = zj - p[q][2];
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = rsqrt(r2);
                const double ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
                const double lj = ri6 * (c12 * ri6 - c6) * (1.0 / 6.0);
                if (far) {
                    const double dd = d0x * (p[q][0] - xi[0]) + d0y * (p[q][1] - xi[1]) + d0z * (p[q][2] - xi[2]);
                    acc[q] += e0 + fac * dd + lj;
                } else {
                    acc[q] += qq * ri + lj;
                }
            }
        }
    } else {  // FP32 sums of this thread's j
        row_sums<NP>(c, 0, nullptr, Vf, nullptr, c.parf, a.n, i, p, xi, a.taylor_r2, threadIdx.x, blockDim.x, acc);
    }
}

// fixed-order block sum of NP values (warp shuffles, then warps in order)
template <int NP>
__device__ void block_sum_bcast(double (&v)[NP], double *out) {
    __shared__ double sh[EPOCH_THREADS / 32][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < NP; q++) {
        double x = v[q];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < NP) {
        double t = 0.0;
        for (int k = 0; k < EPOCH_THREADS / 32; k++) t += sh[k][threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(EPOCH_THREADS) k_epoch(Ctx c, EpochArgs a) {
    const int qp = blockIdx.x;
    double *V = a.view + (int64_t)qp * 3 * a.n;
    float4 *Vf = a.mode == 0 ? a.viewf + (int64_t)qp * a.n : nullptr;
    const double *X = vslot(c, V_X);
    for (int j = threadIdx.x; j < a.n; j += blockDim.x) {
        for (int k = 0; k < 3; k++) V[3 * j + k] = X[3 * j + k];
        if (Vf) Vf[j] = make_float4((float)X[3 * j], (float)X[3 * j + 1], (float)X[3 * j + 2], (float)c.qs[j]);
    }
    __syncthreads();
    const int l0 = a.loff[qp], cnt = a.loff[qp + 1] - l0, moves = a.allowed[qp];
    __shared__ double tot[8];
    __shared__ double pv[3];
    __shared__ int atom;
    for (int m = 0; m < moves; m++) {
        if (threadIdx.x == 0)
            atom = a.list[l0 + pick_atom(a.seed, ((uint64_t)qp << 40) + a.epoch * (uint64_t)a.n + (uint64_t)m, cnt)];
        __syncthreads();
        const int i = atom;
        double p[7][3];
        for (int q = 0; q < 7; q++)
            for (int k = 0; k < 3; k++) p[q][k] = V[3 * i + k];
        for (int k = 0; k < 3; k++) {
            p[1 + 2 * k][k] = p[1 + 2 * k][k] + a.delta;
            p[2 + 2 * k][k] = p[2 + 2 * k][k] - a.delta;
        }
        double acc[7];
        epoch_rows<7>(c, a, V, Vf, i, p, acc);
        block_sum_bcast<7>(acc, tot);
        if (threadIdx.x < 7) {  // bonded terms of atom i on this copy, one position per thread
            const int q = threadIdx.x;
            double e = 0.0;
            for (int k = c.inc_off[i]; k < c.inc_off[i + 1]; k++) {
                const int2 in = c.inc[k];
                e += bonded_term(c, V, in.x >> 2, in.y, in.x & 3, nullptr, nullptr, i, p[q]);
            }
            tot[q] += e;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < 3; k++) {  // per-axis parabola vertex
                const double fp = tot[1 + 2 * k], fm = tot[2 + 2 * k];
                const double curv = fm - 2.0 * tot[0] + fp;
                const double ts = curv > 0.0 ? a.delta * (fm - fp) / (2.0 * curv) : 0.0;
                pv[k] = p[0][k] + ts;
            }
        }
        __syncthreads();
        double p7[1][3] = {{pv[0], pv[1], pv[2]}};
        double acc7[1];
        epoch_rows<1>(c, a, V, Vf, i, p7, acc7);
        __shared__ double t7[1];
        block_sum_bcast<1>(acc7, t7);
        if (threadIdx.x == 0) {
            double e = 0.0;
            for (int k = c.inc_off[i]; k < c.inc_off[i + 1]; k++) {
                const int2 in = c.inc[k];
                e += bonded_term(c, V, in.x >> 2, in.y, in.x & 3, nullptr, nullptr, i, p7[0]);
            }
            const double f7 = t7[0] + e;
            int best = 0;
            double fb = tot[0];
            for (int q = 1; q < 7; q++)
                if (tot[q] < fb) { fb = tot[q]; best = q; }
            const double *pb = best < 7 ? p[best] : p7[0];
            if (f7 < fb) pb = p7[0];
            for (int k = 0; k < 3; k++) V[3 * i + k] = pb[k];
            if (Vf) Vf[i] = make_float4((float)pb[0], (float)pb[1], (float)pb[2], Vf[i].w);
        }
        __syncthreads();
    }
    // the part's atoms go back to X
    double *Xw = vslot(c, V_X);
    for (int t = a.moff[qp] + threadIdx.x; t < a.moff[qp + 1]; t += blockDim.x) {
        const int j = a.members[t];
        for (int k = 0; k < 3; k++) Xw[3 * j + k] = V[3 * j + k];
    }
}

cudaError_t launch_epoch(const Ctx &c, const EpochArgs &a, int parts, cudaStream_t s) {
    k_epoch<<<parts, EPOCH_THREADS, 0, s>>>(c, a);
    return cudaGetLastError();
}

}  // namespace ffm
