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
// stores its values, then thread k sums (or, for the bits of maxmask, takes
// the max of) column k over the block's threads in order.  One FP64
// operation per thread and value, where a shuffle tree costs five: the FP64
// pipe is the scarce unit of the kernels that use it.
template <int NV>
__device__ inline void block_reduce_columns(const double (&v)[NV], int nv, unsigned maxmask, double *dst) {
    __shared__ double sh[NV][TI + 1];
#pragma unroll
    for (int k = 0; k < NV; k++)
        if (k < nv) sh[k][threadIdx.x] = v[k];
    __syncthreads();
    if (threadIdx.x < nv) {
        const int k = threadIdx.x;
        const bool mx = (maxmask >> k) & 1u;
        double x = sh[k][0];
        for (int t = 1; t < TI; t++) x = mx ? fmax(x, sh[k][t]) : x + sh[k][t];
        dst[k] = x;
    }
}

// sum (or max) of one reduction value over a system's tiles, in tile order,
// by a single thread (used when the last block spreads systems over threads)
__device__ inline double thread_sys_sum(const Ctx &c, const SysState &S, int k, bool mx) {
    double x = 0.0;
    for (int t = S.tile0; t < S.tile0 + S.ntile; t++) {
        const double y = __ldcg(&c.red[(int64_t)t * NRED + k]);
        x = mx ? fmax(x, y) : x + y;
    }
    return x;
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

// The last block's per-system work: with few systems a warp reduces each
// system's tiles cooperatively; with many, every thread takes whole systems
// (the control steps of different systems then run in parallel).
// fn(S, totals) runs once per system for which pred(S) holds.
template <int NR, typename Pred, typename Fn>
__device__ inline void last_block_systems(const Ctx &c, int nv_max, unsigned maxmask, Pred pred,
                                          Fn fn, int (*nv_of)(const SysState &)) {
    if (c.n_sys >= 8) {
        double tot[NR];
        for (int b = threadIdx.x; b < c.n_sys; b += blockDim.x) {
            SysState &S = c.st[b];
            if (!pred(S)) continue;
            const int nv = nv_of ? nv_of(S) : nv_max;
            for (int k = 0; k < nv; k++) tot[k] = thread_sys_sum(c, S, k, (maxmask >> k) & 1u);
            fn(S, tot);
        }
        return;
    }
    __shared__ double wtot[TI / 32][NR];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = w; b < c.n_sys; b += TI / 32) {
        SysState &S = c.st[b];
        if (!pred(S)) continue;
        const int nv = nv_of ? nv_of(S) : nv_max;
        for (int k = 0; k < nv; k++) {
            const double x = warp_sys_sum(c, S, k, (maxmask >> k) & 1u);
            if (lane == 0) wtot[w][k] = x;
        }
        __syncwarp();
        if (lane == 0) fn(S, wtot[w]);
        __syncwarp();
    }
}

}  // namespace ffm
