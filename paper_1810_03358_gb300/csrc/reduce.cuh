// Deterministic block and per-system reductions shared by the per-tile
// kernels: every block stores its partial sums; the last block to finish
// (atomic ticket, no waiting) sums each system's blocks in a fixed order.
#pragma once

#include "ffmin_internal.cuh"

namespace ffm {

constexpr int NW = TI / 32;

template <int NR>
__device__ inline void block_reduce_store(double (&v)[NR], unsigned maxmask, double *dst) {
    __shared__ double sh[NW][NR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NR; k++) {
        double x = v[k];
        const bool mx = (maxmask >> k) & 1u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = mx ? fmax(x, y) : x + y;
        }
        if (lane == 0) sh[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NR) {
        const int k = threadIdx.x;
        const bool mx = (maxmask >> k) & 1u;
        double x = sh[0][k];
        for (int j = 1; j < NW; j++) x = mx ? fmax(x, sh[j][k]) : x + sh[j][k];
        dst[k] = x;
    }
}

__device__ inline bool last_block(unsigned int *cnt) {
    __shared__ int am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(cnt, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last != 0;
}

// Block reduction of nv <= NV values through shared memory: every thread
// stores its values; column k is summed (or, for the bits of maxmask,
// maximised) in RSTRANDS interleaved strands (strand s: threads s,
// s + RSTRANDS, ... in order), then its strand results in strand order.
// One FP64 operation per thread and value, where a shuffle tree costs five
// (the FP64 pipe is the scarce unit of the kernels that use it), and a
// dependent chain of TI / RSTRANDS + RSTRANDS operations instead of TI (a
// dependent FP64 operation takes hundreds of cycles when the pipe is shared).
constexpr int RSTRANDS = 8;
template <int NV>
__device__ inline double (*columns_buffer())[TI + 1] {
    __shared__ double sh[NV][TI + 1];
    return sh;
}
template <int NV>
__device__ inline void block_reduce_columns(const double (&v)[NV], int nv, unsigned maxmask, double *dst) {
    double (*sh)[TI + 1] = columns_buffer<NV>();
    __shared__ double part[NV][RSTRANDS];
#pragma unroll
    for (int k = 0; k < NV; k++)
        if (k < nv) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int u = threadIdx.x; u < nv * RSTRANDS; u += TI) {
        const int k = u / RSTRANDS, s = u % RSTRANDS;
        const bool mx = (maxmask >> k) & 1u;
        double x = sh[k][s];
#pragma unroll 4
        for (int t = s + RSTRANDS; t < TI; t += RSTRANDS) x = mx ? fmax(x, sh[k][t]) : x + sh[k][t];
        part[k][s] = x;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
        const int k = threadIdx.x;
        const bool mx = (maxmask >> k) & 1u;
        double x = part[k][0];
#pragma unroll
        for (int s = 1; s < RSTRANDS; s++) x = mx ? fmax(x, part[k][s]) : x + part[k][s];
        dst[k] = x;
    }
}

// sum (or max) of one reduction value over a system's tiles, fixed order,
// executed by a whole warp; the result is valid on every lane
__device__ inline double warp_sys_sum(const Ctx &c, const SysState &S, int k, bool mx) {
    const int lane = threadIdx.x & 31;
    double x = 0.0;
    for (int t = S.tile0 + lane; t < S.tile0 + S.ntile; t += 32) {
        const double y = __ldcg(&c.red[(int64_t)t * NRED + k]);
        x = mx ? fmax(x, y) : x + y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, x, o);
        x = mx ? fmax(x, y) : x + y;
    }
    return x;
}

// the same for the first nv reduction values, eight at a time (the same
// order per value, so the same results): lane l takes tiles l, l + 32, ...
// in order with the group's values of a tile loaded together, then a
// butterfly over the lanes; lane 0 stores the results to out
template <int NR>
__device__ inline void warp_sys_sums(const Ctx &c, const SysState &S, int nv, unsigned maxmask, double *out) {
    constexpr int G = NR < 8 ? NR : 8;
    const int lane = threadIdx.x & 31;
    for (int k0 = 0; k0 < nv; k0 += G) {  // nv is the same on every lane
        double x[G];
#pragma unroll
        for (int k = 0; k < G; k++) x[k] = 0.0;
        for (int t = S.tile0 + lane; t < S.tile0 + S.ntile; t += 32) {
            const double *r = &c.red[(int64_t)t * NRED + k0];
            double y[G];
#pragma unroll
            for (int k = 0; k < G; k++) y[k] = k0 + k < nv ? __ldcg(r + k) : 0.0;
#pragma unroll
            for (int k = 0; k < G; k++) x[k] = ((maxmask >> (k0 + k)) & 1u) ? fmax(x[k], y[k]) : x[k] + y[k];
        }
#pragma unroll
        for (int k = 0; k < G; k++) {
            const bool mx = (maxmask >> (k0 + k)) & 1u;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, x[k], o);
                x[k] = mx ? fmax(x[k], y) : x[k] + y;
            }
            if (lane == 0 && k0 + k < nv) out[k0 + k] = x[k];
        }
    }
}

// A system's control state copied by a warp (8-byte words, coalesced), so
// that the control step, one thread's long chain of dependent reads and
// writes of the state, runs on a shared-memory copy instead of global memory
__device__ inline void warp_copy_state(SysState *dst, const SysState *src) {
    static_assert(sizeof(SysState) % 8 == 0, "SysState is copied in 8-byte words");
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    for (int k = threadIdx.x & 31; k < (int)(sizeof(SysState) / 8); k += 32) d[k] = s[k];
    __syncwarp();
}

// The last block's per-system work (fewer than 8 systems; larger batches
// reduce in k_sysreduce): the warps reduce the systems' tiles (warp w takes
// systems w, w + 4, ...), then warp 0 runs fn(S, totals) for every system
// for which pred(S) holds, in system order, each on a shared-memory copy
// of its state that is written back afterwards (the copy lives in the
// buffer of block_reduce_columns<NR>, whose work is done by then).
template <int NR, typename Pred, typename Fn>
__device__ inline void last_block_systems(const Ctx &c, int nv_max, unsigned maxmask, Pred pred,
                                          Fn fn, int (*nv_of)(const SysState &)) {
    static_assert(sizeof(SysState) <= sizeof(double) * NR * (TI + 1), "state copy fits the column buffer");
    __shared__ double wtot[LB_MAX_SYS][NR];
    __shared__ int on[LB_MAX_SYS];
    SysState &sS = *reinterpret_cast<SysState *>(columns_buffer<NR>());
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = c.n_sys < LB_MAX_SYS ? c.n_sys : LB_MAX_SYS;
    for (int b = w; b < n; b += TI / 32) {
        const SysState &S = c.st[b];
        const bool p = pred(S);
        if (lane == 0) on[b] = p ? 1 : 0;
        if (!p) continue;
        warp_sys_sums<NR>(c, S, nv_of ? nv_of(S) : nv_max, maxmask, wtot[b]);
    }
    __syncthreads();
    if (w != 0) return;
    for (int b = 0; b < n; b++) {
        if (!on[b]) continue;
        warp_copy_state(&sS, &c.st[b]);
        if (lane == 0) fn(sS, wtot[b]);
        __syncwarp();
        warp_copy_state(&c.st[b], &sS);
    }
}

}  // namespace ffm
