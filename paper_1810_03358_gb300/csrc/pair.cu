// Non-bonded pair energy and gradient: the O(N^2) hot loop of the method.
//
// E_cul + E_vdw over all atom pairs (arXiv 1810.03358, Section 2), evaluated
// as a row sweep parallel over the outer sum (Section 3: one inner sum per
// GPU thread).  Every thread owns one i-atom of a 128-atom tile in registers
// and walks a j-chunk staged through shared memory; the pair (i, j) is
// evaluated in row i and again in row j, so no force is ever scattered and
// no atomic touches a force (Newton's third law is not used).
//
// Work items are (i-tile, j-chunk) pairs taken from a device queue (reset by
// a memset before each launch) by a persistent grid; each item writes its
// partial row sums (gx, gy, gz, row energy) to its own slot, and the
// finalize kernel sums the slots of an atom in a fixed order, so results are
// deterministic for a given chunking.  Bonded-term items share the queue.
//
// Per pair (d = x_j - x_i, r^-1 = rsqrt(r^2), q' = q sqrt(C), and the
// per-atom Lennard-Jones factors c6 = a sigma^3, c12 = a sigma^6 with
// a = sqrt(24 eps), so that c6_i c6_j = 24 eps_ij sigma_ij^6 and
// c12_i c12_j = 24 eps_ij sigma_ij^12 under the geometric combining rule):
//   e_cul  = q'_i q'_j r^-1
//   6 e_lj = r^-6 (C12 r^-6 - C6),              C6 = c6_i c6_j, C12 = c12_i c12_j
//   F      = (e_cul + r^-6 (2 C12 r^-6 - C6)) r^-2,   grad_i += F d
// which is C q_i q_j / r + 4 sqrt(eps_i eps_j)((s/r)^12 - (s/r)^6) and its
// derivative.  The row energy sum_j (e_cul + e_lj) counts each pair twice;
// the finalize kernel halves it.  The FP32 kernel flushes denormals (none
// occur for separations above 1e-6 A) and takes r^-1 from the hardware
// reciprocal square root (rsqrt.approx.ftz.f32).
#include <cstdio>

#include "bonded.cuh"
#include "ffmin_internal.cuh"

namespace ffm {

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename T> struct VT;
template <> struct VT<float> {
    using V4 = float4;
    using V2 = float2;
    static __device__ __forceinline__ float rsq(float x) { return rsqrt_approx(x); }
};
template <> struct VT<double> {
    using V4 = double4_32a;
    using V2 = double2;
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
};

// scale of the pair (i, j) in the exclusion variant (1 for every pair not
// listed); i must be a real atom
__device__ __forceinline__ float pair_xscale(const Ctx &c, int i, int j) {
    float s = 1.f;
    for (int m = c.xs_off[i]; m < c.xs_off[i + 1]; m++)
        if (c.xs_part[m] == j) s = c.xs_val[m];
    return s;
}

// IPT i-atoms per thread share every j load from shared memory.  DM: 0 an
// off-diagonal tile; 1 the i-tile itself (j == i skipped); 2 the i-tile
// itself on the symmetric list (only j > i: each pair once).  MASK: the j
// tile holds scaled partners of the i tile (exclusion variant, FP32): every
// pair is multiplied by its scale s_ij inside the sums (ig: the i atoms'
// global indices, -1 for padding; jt: the j tile's first atom).
template <typename T, int IPT, bool GRAD, int DM, bool MASK = false>
__device__ __forceinline__ void sweep(const typename VT<T>::V4 *__restrict__ sp,
                                      const typename VT<T>::V2 *__restrict__ sq,
                                      const typename VT<T>::V4 (&pi)[IPT],
                                      const typename VT<T>::V2 (&ci)[IPT], const int (&dk)[IPT],
                                      T (&gx)[IPT], T (&gy)[IPT], T (&gz)[IPT], T (&ec)[IPT],
                                      T (&lj)[IPT], const Ctx *cx = nullptr, const int *ig = nullptr,
                                      int jt = 0) {
    // the masked form runs on a few tiles only: kept rolled (smaller kernel)
#pragma unroll(MASK ? 1 : 8)
    for (int k = 0; k < TJ; k++) {
        const typename VT<T>::V4 pj = sp[k];
        const typename VT<T>::V2 qj = sq[k];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const T dx = pj.x - pi[u].x, dy = pj.y - pi[u].y, dz = pj.z - pi[u].z;
            const T r2 = dx * dx + dy * dy + dz * dz;
            T ri = VT<T>::rsq(r2);
            if (DM == 1) ri = (k == dk[u]) ? T(0) : ri;
            if (DM == 2) ri = (k <= dk[u]) ? T(0) : ri;
            T sc = T(1);
            if (MASK) {
                if (ig[u] >= 0) sc = (T)pair_xscale(*cx, ig[u], jt + k);
            }
            const T ri2 = ri * ri;
            const T e = MASK ? pi[u].w * pj.w * sc * ri : pi[u].w * pj.w * ri;
            const T ri6 = ri2 * ri2 * ri2;
            const T c6 = MASK ? ci[u].x * qj.x * sc : ci[u].x * qj.x;
            const T c12 = MASK ? ci[u].y * qj.y * sc : ci[u].y * qj.y;
            const T t1 = c12 * ri6 - c6;
            ec[u] += e;
            lj[u] += ri6 * t1;
            if (GRAD) {
                const T t2 = c12 * ri6 + t1;
                const T f = (ri6 * t2 + e) * ri2;
                gx[u] += f * dx;
                gy[u] += f * dy;
                gz[u] += f * dz;
            }
        }
    }
}

// FP32 line-search trial as an energy difference from the base point: with
// d = x_j - x_i at the base and dd = the difference of the two atoms'
// displacements, r'^2 - r^2 = dd.(2 d + dd) is formed without cancellation,
// and so are
//   r'^-2 - r^-2 = -(r'^2 - r^2) r^-2 r'^-2,
//   r'^-1 - r^-1 = (r'^-2 - r^-2) / (r^-1 + r'^-1),
//   r'^-6 - r^-6 = (r'^-2 - r^-2)(r'^-4 + r'^-2 r^-2 + r^-4),
//   r'^-12 - r^-12 = (r'^-6 - r^-6)(r'^-6 + r^-6);
// the row then accumulates the exact-difference form of
// e_cul + 6 e_lj, whose rounding error is relative to the difference, not to
// the energies (FP32 coordinates of the trial point would add noise of order
// u |x| |F| per pair, larger than the line search's energy decrements).
template <int IPT, int DM, bool MASK = false>
__device__ __forceinline__ void sweep_delta(const float4 *__restrict__ sp, const float2 *__restrict__ sq,
                                            const float4 *__restrict__ sd, const float4 (&pi)[IPT],
                                            const float2 (&ci)[IPT], const float4 (&di)[IPT],
                                            const int (&dk)[IPT], float (&ec)[IPT], float (&lj)[IPT],
                                            const Ctx *cx = nullptr, const int *ig = nullptr, int jt = 0) {
#pragma unroll(MASK ? 1 : 4)
    for (int k = 0; k < TJ; k++) {
        const float4 pj = sp[k];
        const float2 qj = sq[k];
        const float4 dj = sd[k];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const float dx = pj.x - pi[u].x, dy = pj.y - pi[u].y, dz = pj.z - pi[u].z;
            const float ex = dj.x - di[u].x, ey = dj.y - di[u].y, ez = dj.z - di[u].z;
            float r2 = dx * dx + dy * dy + dz * dz;
            if (DM != 0) r2 = (k == dk[u]) ? 1.f : r2;  // j == i: dd = 0, every difference vanishes
            float D = ex * (2.f * dx + ex) + ey * (2.f * dy + ey) + ez * (2.f * dz + ez);
            if (DM == 2) D = (k <= dk[u]) ? 0.f : D;  // each pair once: j < i contributes nothing
            const float ri = rsqrt_approx(r2), rp = rsqrt_approx(r2 + D);
            const float ri2 = ri * ri, rp2 = rp * rp;
            const float X = -D * ri2 * rp2;
            float inv;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(ri + rp));
            const float d1 = X * inv;
            const float ri4 = ri2 * ri2, rp4 = rp2 * rp2;
            const float d6 = X * (rp4 + rp2 * ri2 + ri4);
            const float d12 = d6 * (rp4 * rp2 + ri4 * ri2);
            float sc = 1.f;
            if (MASK) {
                if (ig[u] >= 0) sc = pair_xscale(*cx, ig[u], jt + k);
            }
            const float c6 = MASK ? ci[u].x * qj.x * sc : ci[u].x * qj.x;
            const float c12 = MASK ? ci[u].y * qj.y * sc : ci[u].y * qj.y;
            ec[u] += MASK ? pi[u].w * pj.w * sc * d1 : pi[u].w * pj.w * d1;
            lj[u] += c12 * d12 - c6 * d6;
        }
    }
}

// Energy-only forms with the i atom's factors outside the sums: per i the
// sums of q'_j X1, c6_j X6 and c12_j X12 (X = r^-1, r^-6, r^-12 for a plain
// energy; the exact differences r'^-1 - r^-1, ... for a difference trial),
// combined with q'_i, c6_i, c12_i once per item.  fa, f6, f12 accumulate
// across the item's j tiles.
template <int IPT, int DM>
__device__ __forceinline__ void sweep_e_factored(const float4 *__restrict__ sp, const float2 *__restrict__ sq,
                                                 const float4 (&pi)[IPT], const int (&dk)[IPT], float (&fa)[IPT],
                                                 float (&f6)[IPT], float (&f12)[IPT]) {
#pragma unroll 8
    for (int k = 0; k < TJ; k++) {
        const float4 pj = sp[k];
        const float2 qj = sq[k];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const float dx = pj.x - pi[u].x, dy = pj.y - pi[u].y, dz = pj.z - pi[u].z;
            const float r2 = dx * dx + dy * dy + dz * dz;
            float ri = rsqrt_approx(r2);
            if (DM == 1) ri = (k == dk[u]) ? 0.f : ri;
            if (DM == 2) ri = (k <= dk[u]) ? 0.f : ri;
            const float ri2 = ri * ri;
            const float ri6 = ri2 * ri2 * ri2;
            fa[u] = fmaf(pj.w, ri, fa[u]);
            f6[u] = fmaf(qj.x, ri6, f6[u]);
            f12[u] = fmaf(qj.y, ri6 * ri6, f12[u]);
        }
    }
}

template <int IPT, int DM>
__device__ __forceinline__ void sweep_delta_factored(const float4 *__restrict__ sp, const float2 *__restrict__ sq,
                                                     const float4 *__restrict__ sd, const float4 (&pi)[IPT],
                                                     const float4 (&di)[IPT], const int (&dk)[IPT],
                                                     float (&fa)[IPT], float (&f6)[IPT], float (&f12)[IPT]) {
#pragma unroll 4
    for (int k = 0; k < TJ; k++) {
        const float4 pj = sp[k];
        const float2 qj = sq[k];
        const float4 dj = sd[k];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const float dx = pj.x - pi[u].x, dy = pj.y - pi[u].y, dz = pj.z - pi[u].z;
            const float ex = dj.x - di[u].x, ey = dj.y - di[u].y, ez = dj.z - di[u].z;
            float r2 = dx * dx + dy * dy + dz * dz;
            if (DM != 0) r2 = (k == dk[u]) ? 1.f : r2;  // j == i: dd = 0, every difference vanishes
            float D = ex * (2.f * dx + ex) + ey * (2.f * dy + ey) + ez * (2.f * dz + ez);
            if (DM == 2) D = (k <= dk[u]) ? 0.f : D;  // each pair once: j < i contributes nothing
            const float ri = rsqrt_approx(r2), rp = rsqrt_approx(r2 + D);
            const float ri2 = ri * ri, rp2 = rp * rp;
            const float X = -D * ri2 * rp2;
            float inv;
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(ri + rp));
            const float d1 = X * inv;
            const float ri4 = ri2 * ri2, rp4 = rp2 * rp2;
            const float d6 = X * (rp4 + rp2 * ri2 + ri4);
            const float d12 = d6 * (rp4 * rp2 + ri4 * ri2);
            fa[u] = fmaf(pj.w, d1, fa[u]);
            f6[u] = fmaf(qj.x, d6, f6[u]);
            f12[u] = fmaf(qj.y, d12, f12[u]);
        }
    }
}

// NT threads per block, IPT i-atoms per thread, NT * IPT == TI (one tile).
// FP32 shapes: two i-atoms per thread (64-thread blocks: every j load from
// shared memory serves two pairs) or one (128-thread blocks: twice the warps
// per work item, which pays when an object has few items); the autotuner
// picks one per object.  Register caps: FP32 kernels run 768 threads per SM
// (12 blocks of 64 or 6 of 128, 80 registers; measured on GB300 faster than
// 1,024 threads at 64 registers and than 4 i-atoms per thread), the FP64
// kernel 8 blocks of 128 (64 registers); the rarely-run bonded items may
// spill.  FFMIN_F32_THREADS_PER_SM overrides the FP32 cap (registers per
// thread follow: 65536 / threads).
#ifndef FFMIN_F32_THREADS_PER_SM
#define FFMIN_F32_THREADS_PER_SM 768
#endif
// XS: the object carries the exclusion variant (FP32 sweeps scale the listed
// pairs); a separate instantiation keeps the masked code out of the kernel
// every other object runs
// EONLY (FP32): the energy-only kernel (plain energies and difference
// trials, on the symmetric list) with its own work queue; the other FP32
// instantiation runs the E + grad row sweep only.  The FP64 row sweep (the
// fallback of batches too large for the symmetric list) takes both kinds.
template <typename T, int NT, int IPT, bool XS = false, bool EONLY = false>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? FFMIN_F32_THREADS_PER_SM / NT : 8)) k_pair(Ctx c);
template <typename T, int NT, int IPT, bool XS, bool EONLY>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 ? FFMIN_F32_THREADS_PER_SM / NT : 8)) k_pair(Ctx c) {
    static_assert(NT * IPT == TI, "a block covers one i-tile");
    using V4 = typename VT<T>::V4;
    using V2 = typename VT<T>::V2;
    __shared__ V4 sp[TJ];
    __shared__ V2 sq[TJ];
    __shared__ float4 sd[sizeof(T) == 4 ? TJ : 1];  // displacements (FP32 difference trials)
    __shared__ int s_item;
    const V4 *__restrict__ pos;
    const V2 *__restrict__ par;
    V4 *__restrict__ out;
    if constexpr (sizeof(T) == 4) {
        pos = c.posf; par = c.parf; out = c.gpf;
    } else {
        pos = c.posd; par = c.pard; out = c.gpd;
    }
    constexpr int MODE = sizeof(T) == 4 ? 0 : 1;
    constexpr int LIST = MODE == 1 ? LIST_F64 : (EONLY ? LIST_F32_E : LIST_F32_EG);
    constexpr int CNT = MODE == 1 ? CNT_PAIR64 : (EONLY ? CNT_PAIR32E : CNT_PAIR);
    // the queue runs over the items of the systems evaluating in this
    // precision and kind only (active list rebuilt before every launch)
    const int32_t *A = c.act + LIST * (2 * c.n_sys + 2);
    const int n_act = A[0], total = A[1];
    if (total == 0) return;
    const int32_t *aoff = A + 2, *asys = A + 2 + c.n_sys;
    const int tid = threadIdx.x;
    __shared__ int s_sym;
    for (;;) {
        if (tid == 0) {
            const int q = (int)atomicAdd(&c.counters[CNT], 1u);
            if (q < total) {  // last active system whose first item is <= q
                int lo = 0, hi = n_act - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (aoff[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                // FP32 energy-only evaluations (plain or difference trials)
                // run on the symmetric list: each pair once, no forces
                const int b = asys[lo];
                const int sym = MODE == 0 && EONLY && c.sym64;
                s_item = (sym ? c.sys_items64 : c.sys_items)[b].x + (q - aoff[lo]);
                s_sym = sym;
            } else {
                s_item = -1;
            }
        }
        __syncthreads();
        const int it = s_item;
        const bool sym = MODE == 0 && s_sym;
        __syncthreads();
        if (it < 0) break;
        const Item I = sym ? c.items64[it] : c.items[it];
        if (I.tile < 0) {  // bonded terms (FP64), overlapping the pair items of other warps
            bonded_item(c, I.j0, I.nj, MODE);
            continue;
        }
        const Tile tl = c.tiles[I.tile];
        const int kind = c.st[tl.sys].ev_kind;
        if (kind == EV_NONE || c.st[tl.sys].mode != MODE) continue;
        if (MODE == 0 && (kind == EV_E) != EONLY) continue;  // the other FP32 queue's system
        const bool delta = MODE == 0 && c.st[tl.sys].ev_delta;
        V4 pi[IPT];
        V2 ci[IPT];
        int ig[IPT];
        T gx[IPT], gy[IPT], gz[IPT], ec[IPT], lj[IPT];
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            const int li = tid + u * NT;
            ig[u] = tl.a0 + li;
            if (li < tl.na) {
                pi[u] = pos[ig[u]];
                ci[u] = par[ig[u]];
            } else {  // padding atom far away with no charge and no LJ
                pi[u].x = T(-1e6); pi[u].y = T(-1e6); pi[u].z = T(-1e6); pi[u].w = T(0);
                ci[u].x = T(0); ci[u].y = T(0);
            }
            gx[u] = gy[u] = gz[u] = ec[u] = lj[u] = T(0);
        }
        float4 di[IPT];
        if constexpr (MODE == 0) {
#pragma unroll
            for (int u = 0; u < IPT; u++)
                di[u] = (delta && tid + u * NT < tl.na) ? c.dispf[ig[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int jend = I.j0 + I.nj;
        for (int jt = I.j0; jt < jend; jt += TJ) {
#pragma unroll
            for (int q = tid; q < TJ; q += NT) {
                const int jl = jt + q;
                if constexpr (MODE == 0) {
                    if (delta) sd[q] = jl < jend ? c.dispf[jl] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                if (jl < jend) {
                    sp[q] = pos[jl];
                    sq[q] = par[jl];
                } else {
                    V4 d; d.x = T(1e6); d.y = T(1e6); d.z = T(1e6); d.w = T(0);
                    V2 z; z.x = T(0); z.y = T(0);
                    sp[q] = d;
                    sq[q] = z;
                }
            }
            __syncthreads();
            // the i tile lies inside this j tile when jt == a0 (tiles and
            // chunks are aligned to TJ == TI inside a system)
            const bool diag = I.diag && jt == tl.a0;
            int dk[IPT];
#pragma unroll
            for (int u = 0; u < IPT; u++) dk[u] = ig[u] - jt;
            if constexpr (MODE == 0) {
                // exclusion variant: this j tile holds scaled partners of
                // the i tile (near the diagonal of a chain); -1 marks padding
                const bool masked = XS && tl.xlo <= tl.xhi && tl.xhi >= jt && tl.xlo < jt + TJ;
                int igm[IPT];
#pragma unroll
                for (int u = 0; u < IPT; u++) igm[u] = tid + u * NT < tl.na ? ig[u] : -1;
                if constexpr (EONLY) {  // energy only: plain or difference trial
                    if (masked) {
                        if (delta) {
                            if (diag && sym) sweep_delta<IPT, 2, true>(sp, sq, sd, pi, ci, di, dk, ec, lj, &c, igm, jt);
                            else if (diag) sweep_delta<IPT, 1, true>(sp, sq, sd, pi, ci, di, dk, ec, lj, &c, igm, jt);
                            else sweep_delta<IPT, 0, true>(sp, sq, sd, pi, ci, di, dk, ec, lj, &c, igm, jt);
                        } else {
                            if (diag && sym) sweep<T, IPT, false, 2, true>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj, &c, igm, jt);
                            else if (diag) sweep<T, IPT, false, 1, true>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj, &c, igm, jt);
                            else sweep<T, IPT, false, 0, true>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj, &c, igm, jt);
                        }
                    } else if (delta) {  // factored sums in the (idle) gradient registers
                        if (diag && sym) sweep_delta_factored<IPT, 2>(sp, sq, sd, pi, di, dk, gx, gy, gz);
                        else if (diag) sweep_delta_factored<IPT, 1>(sp, sq, sd, pi, di, dk, gx, gy, gz);
                        else sweep_delta_factored<IPT, 0>(sp, sq, sd, pi, di, dk, gx, gy, gz);
                    } else {
                        if (diag && sym) sweep_e_factored<IPT, 2>(sp, sq, pi, dk, gx, gy, gz);
                        else if (diag) sweep_e_factored<IPT, 1>(sp, sq, pi, dk, gx, gy, gz);
                        else sweep_e_factored<IPT, 0>(sp, sq, pi, dk, gx, gy, gz);
                    }
                } else {  // E + grad row sweep
                    if (masked) {
                        if (diag) sweep<T, IPT, true, 1, true>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj, &c, igm, jt);
                        else sweep<T, IPT, true, 0, true>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj, &c, igm, jt);
                    } else {
                        if (diag) sweep<T, IPT, true, 1>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
                        else sweep<T, IPT, true, 0>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
                    }
                }
            } else if (kind == EV_EG) {  // FP64 row sweep (fallback of very large batches)
                if (diag) sweep<T, IPT, true, 1>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
                else sweep<T, IPT, true, 0>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
            } else {
                if (diag) sweep<T, IPT, false, 1>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
                else sweep<T, IPT, false, 0>(sp, sq, pi, ci, dk, gx, gy, gz, ec, lj);
            }
            __syncthreads();
        }
        // symmetric list (FP32 energy only): the i-side rows of the item's slot
        V4 *dst = out + (int64_t)it * TI;
        if constexpr (MODE == 0) {
            if (sym) dst = c.gpf_sym + (int64_t)I.slot * TI;
        }
        // FP32 energy only: masked tiles summed the pair terms into ec / lj,
        // the others the factored sums into gx, gy, gz
        constexpr bool factored = MODE == 0 && EONLY;
#pragma unroll
        for (int u = 0; u < IPT; u++) {
            V4 o;
            if (factored) {
                o.x = T(0); o.y = T(0); o.z = T(0);
                o.w = ec[u] + lj[u] * T(1.0 / 6.0) + pi[u].w * gx[u] +
                      (ci[u].y * gz[u] - ci[u].x * gy[u]) * T(1.0 / 6.0);
            } else {
                o.x = gx[u]; o.y = gy[u]; o.z = gz[u];
                o.w = ec[u] + lj[u] * T(1.0 / 6.0);
            }
            dst[tid + u * NT] = o;
        }
    }
}

// Symmetric FP64 pair kernel: every unordered pair once.  The FP64 pipe
// (2 FMA per clock per SM) is the limit of the FP64 terms, so the row sweep's
// double evaluation of each pair is its largest cost; here an item (i-tile
// I, chunk of j-tiles at or right of I) evaluates each pair (i, j) once,
// adds the force to i's registers and its opposite to j's entry of a
// warp-private shared-memory array (lanes of a warp take distinct j at every
// step: lane t pairs with j = (t + k) mod TJ at step k; the diagonal tile runs
// k = 1 .. TJ/2 and, at k = TJ/2, only its first half of the threads, so
// every pair of the tile appears once).  No atomics: after each j-tile the
// four warps' arrays are summed in warp order into the tile's j-side
// partial rows, and the i-side rows are written once per item; the finalize
// kernel sums an atom's j-side rows (tiles I <= its tile) and i-side rows in
// a fixed order.  Row energies count each pair once.
constexpr int NT_SYM = 128;
// resident blocks per SM: 7 caps the kernel at 72 registers (a few spilled
// stack bytes) and measured 1.5 % faster than 6 (80 registers, no spills)
#ifndef FFMIN_SYM_MINBLOCKS
#define FFMIN_SYM_MINBLOCKS 7
#endif
__global__ void __launch_bounds__(NT_SYM, FFMIN_SYM_MINBLOCKS) k_pair64_sym(Ctx c) {
    __shared__ double4_32a sp[TJ];
    __shared__ double2 sq[TJ];
    __shared__ double jfx[NT_SYM / 32][TJ], jfy[NT_SYM / 32][TJ], jfz[NT_SYM / 32][TJ];
    __shared__ int s_item;
    const int32_t *A = c.act + 1 * (2 * c.n_sys + 2);
    const int n_act = A[0], total = A[1];
    if (total == 0) return;
    const int32_t *aoff = A + 2, *asys = A + 2 + c.n_sys;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (;;) {
        if (tid == 0) {
            const int q = (int)atomicAdd(&c.counters[CNT_PAIR64], 1u);
            if (q < total) {  // last active system whose first item is <= q
                int lo = 0, hi = n_act - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (aoff[mid] <= q) lo = mid;
                    else hi = mid - 1;
                }
                s_item = c.sys_items64[asys[lo]].x + (q - aoff[lo]);
            } else {
                s_item = -1;
            }
        }
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it < 0) break;
        const Item I = c.items64[it];
        if (I.tile < 0) {
            bonded_item(c, I.j0, I.nj, 1);
            continue;
        }
        const Tile tl = c.tiles[I.tile];
        const int kind = c.st[tl.sys].ev_kind;
        if (kind == EV_NONE || c.st[tl.sys].mode != 1) continue;
        const bool grad = kind == EV_EG;
        double4_32a pi;
        double2 ci;
        if (tid < tl.na) {
            pi = c.posd[tl.a0 + tid];
            ci = c.pard[tl.a0 + tid];
        } else {  // padding atom far away with no charge and no LJ
            pi = make_double4_32a(-1e6, -1e6, -1e6, 0.0);
            ci = make_double2(0.0, 0.0);
        }
        double gx = 0.0, gy = 0.0, gz = 0.0, ec = 0.0, lj = 0.0;
        double sc1 = 0.0, s6 = 0.0, s12 = 0.0;  // energy-only factored sums
        const int jend = I.j0 + I.nj;
        for (int jt = I.j0; jt < jend; jt += TJ) {
            const int jl = jt + tid;
            if (jl < jend) {
                sp[tid] = c.posd[jl];
                sq[tid] = c.pard[jl];
            } else {
                sp[tid] = make_double4_32a(1e6, 1e6, 1e6, 0.0);
                sq[tid] = make_double2(0.0, 0.0);
            }
            if (grad) {
#pragma unroll
                for (int q = lane; q < TJ; q += 32) { jfx[w][q] = 0.0; jfy[w][q] = 0.0; jfz[w][q] = 0.0; }
            }
            __syncthreads();
            // the diagonal tile (j-tile == i-tile) pairs t with t + k,
            // k = 1 .. TJ/2 (at k = TJ/2 only t < TJ/2); other tiles every k
            const bool diag = I.diag && jt == I.j0;
            const int k0 = diag ? 1 : 0, k1 = diag ? TJ / 2 : TJ - 1;
            if (!grad) {
                // energy only: the i atom's factors leave the sums,
                // E_i = q'_i sum q'_j / r + (c12_i sum c12_j r^-12 - c6_i sum c6_j r^-6) / 6
                for (int k = k0; k <= k1; k++) {
                    if (diag && k == TJ / 2 && tid >= TJ / 2) break;  // warp-uniform
                    const int j = (tid + k) & (TJ - 1);
                    const double4_32a pj = sp[j];
                    const double2 qj = sq[j];
                    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    const double ri = rsqrt(r2);
                    const double ri2 = ri * ri;
                    const double ri6 = ri2 * ri2 * ri2;
                    sc1 = fma(pj.w, ri, sc1);
                    s6 = fma(qj.x, ri6, s6);
                    s12 = fma(qj.y, ri6 * ri6, s12);
                }
                __syncthreads();
                continue;
            }
            for (int k = k0; k <= k1; k++) {
                if (diag && k == TJ / 2 && tid >= TJ / 2) break;  // warp-uniform
                const int j = (tid + k) & (TJ - 1);
                const double4_32a pj = sp[j];
                const double2 qj = sq[j];
                const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = rsqrt(r2);
                const double ri2 = ri * ri;
                const double e = pi.w * pj.w * ri;
                const double ri6 = ri2 * ri2 * ri2;
                const double c6 = ci.x * qj.x, c12 = ci.y * qj.y;
                const double t1 = c12 * ri6 - c6;
                ec += e;
                lj += ri6 * t1;
                if (grad) {
                    const double t2 = c12 * ri6 + t1;
                    const double f = (ri6 * t2 + e) * ri2;
                    gx += f * dx;
                    gy += f * dy;
                    gz += f * dz;
                    jfx[w][j] -= f * dx;
                    jfy[w][j] -= f * dy;
                    jfz[w][j] -= f * dz;
                }
                __syncwarp();
            }
            __syncthreads();
            if (grad) {  // j-side partial rows of this j-tile, warps summed in order
                double4_32a o;
                o.x = jfx[0][tid]; o.y = jfy[0][tid]; o.z = jfz[0][tid];
#pragma unroll
                for (int v = 1; v < NT_SYM / 32; v++) { o.x += jfx[v][tid]; o.y += jfy[v][tid]; o.z += jfz[v][tid]; }
                o.w = 0.0;
                c.gpd[(int64_t)(I.slot + 1 + (jt - I.j0) / TJ) * TI + tid] = o;
            }
            __syncthreads();
        }
        double4_32a o;
        o.x = gx; o.y = gy; o.z = gz;
        o.w = grad ? ec + lj * (1.0 / 6.0) : pi.w * sc1 + (ci.y * s12 - ci.x * s6) * (1.0 / 6.0);
        c.gpd[(int64_t)I.slot * TI + tid] = o;
    }
}

// FP64 row sweep: one i-atom per thread (the FP64 pipe, not the loads, is
// the limit)
constexpr int NT_F64 = 128;
#define K_F64 k_pair<double, 128, 1>

int pair_grid_size(int mode, int f32_ipt) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool one = f32_ipt == 1;
    if (mode == 0 && one)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<float, TI, 1>, TI, 0);
    else if (mode == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<float, TI / 2, 2>, TI / 2, 0);
    else if (mode == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, K_F64, NT_F64, 0);
    else if (mode == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair64_sym, NT_SYM, 0);
    else if (one)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<float, TI, 1, false, true>, TI, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<float, TI / 2, 2, false, true>, TI / 2, 0);
    if (per < 1) per = 1;
    return sms * per;
}

// the FP32 E + grad and energy-only kernels of one shape
template <int IPT>
static void launch_f32(const Ctx &c, int grid32, int grid32e, cudaStream_t s, cudaStream_t se) {
    constexpr int NT = TI / IPT;
    if (c.xs_off) {
        k_pair<float, NT, IPT, true><<<grid32, NT, 0, s>>>(c);
        k_pair<float, NT, IPT, true, true><<<grid32e, NT, 0, se>>>(c);
    } else {
        k_pair<float, NT, IPT><<<grid32, NT, 0, s>>>(c);
        k_pair<float, NT, IPT, false, true><<<grid32e, NT, 0, se>>>(c);
    }
}

// Active lists for the two pair kernels: for each precision mode, the
// systems with an evaluation request in that mode and the exclusive prefix
// of their item counts, in system order (one block; warp-shuffle scans over
// chunks of 256 systems).  The block also resets both work-queue counters.
__global__ void __launch_bounds__(256) k_activelist(Ctx c) {
    __shared__ int wsum_i[8], wsum_s[8];
    __shared__ int base_items, base_sys;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        c.counters[CNT_PAIR] = 0;
        c.counters[CNT_PAIR64] = 0;
        c.counters[CNT_PAIR32E] = 0;
    }
    for (int L = 0; L < N_LISTS; L++) {
        int32_t *A = c.act + L * (2 * c.n_sys + 2);
        if (threadIdx.x == 0) { base_items = 0; base_sys = 0; }
        __syncthreads();
        for (int b0 = 0; b0 < c.n_sys; b0 += 256) {
            const int b = b0 + threadIdx.x;
            int n = 0;
            if (b < c.n_sys) {
                const SysState &S = c.st[b];
                // queue of the system's evaluation: FP32 E + grad (row list),
                // FP64 terms or FP32 energy only (symmetric list when the
                // object has one)
                const int mine = S.ev_kind == EV_NONE ? -1
                                 : (S.mode == 1 ? LIST_F64 : (S.ev_kind == EV_E ? LIST_F32_E : LIST_F32_EG));
                if (mine == L) n = (c.sym64 && L != LIST_F32_EG ? c.sys_items64 : c.sys_items)[b].y;
            }
            const int f = n > 0 ? 1 : 0;
            int si = n, ss = f;  // inclusive scans within the warp
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int ti = __shfl_up_sync(0xffffffffu, si, o), ts = __shfl_up_sync(0xffffffffu, ss, o);
                if (lane >= o) { si += ti; ss += ts; }
            }
            if (lane == 31) { wsum_i[warp] = si; wsum_s[warp] = ss; }
            __syncthreads();
            int pi = base_items + si - n, ps = base_sys + ss - f;
            for (int w = 0; w < warp; w++) { pi += wsum_i[w]; ps += wsum_s[w]; }
            if (f) {
                A[2 + ps] = pi;
                A[2 + c.n_sys + ps] = b;
            }
            __syncthreads();
            if (threadIdx.x == 255) { base_items = pi + n; base_sys = ps + f; }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            A[0] = base_sys;
            A[1] = base_items;
        }
        __syncthreads();
    }
}

cudaError_t launch_activelist(const Ctx &c, cudaStream_t s) {
    k_activelist<<<1, 256, 0, s>>>(c);  // also gives every pair kernel a fresh work queue
    return cudaGetLastError();
}

// The three pair kernels of a MIXED object take disjoint work queues and
// write disjoint outputs, so with side streams the FP32 energy-only and the
// FP64 kernels run beside the FP32 E + grad kernel (parallel graph branches
// when captured): a round waits for the slowest, not for all three in turn.
cudaError_t launch_pair_kernels(const Ctx &c, int grid32, int grid32e, int grid64, cudaStream_t s,
                                const Branches *br) {
    cudaError_t e;
    if (c.prec != FFMIN_MIXED) {
        if (c.sym64) k_pair64_sym<<<grid64, NT_SYM, 0, s>>>(c);
        else K_F64<<<grid64, NT_F64, 0, s>>>(c);
        return cudaGetLastError();
    }
    cudaStream_t se = s, s64 = s;
    if (br) {
        if ((e = cudaEventRecord(br->fork, s)) != cudaSuccess) return e;
        for (int k = 0; k < 2; k++)
            if ((e = cudaStreamWaitEvent(br->side[k], br->fork, 0)) != cudaSuccess) return e;
        se = br->side[0];
        s64 = br->side[1];
    }
    if (c.f32_ipt == 1) launch_f32<1>(c, grid32, grid32e, s, se);
    else launch_f32<2>(c, grid32, grid32e, s, se);
    if (c.sym64) k_pair64_sym<<<grid64, NT_SYM, 0, s64>>>(c);
    else K_F64<<<grid64, NT_F64, 0, s64>>>(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (br) {
        for (int k = 0; k < 2; k++) {
            if ((e = cudaEventRecord(br->join[k], br->side[k])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, br->join[k], 0)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_pair(const Ctx &c, int grid32, int grid32e, int grid64, cudaStream_t s) {
    cudaError_t e = launch_activelist(c, s);
    return e != cudaSuccess ? e : launch_pair_kernels(c, grid32, grid32e, grid64, s, nullptr);
}

}  // namespace ffm
