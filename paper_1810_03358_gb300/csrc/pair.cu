// Non-bonded pair energy and gradient: the O(N^2) hot loop of the method.
//
// E_cul + E_vdw over all atom pairs (arXiv 1810.03358, Section 2), evaluated
// as a row sweep parallel over the outer sum (Section 3: one inner sum per
// GPU thread).  Every thread owns one i-atom of a 128-atom tile in registers
// and walks a j-chunk staged through shared memory; the pair (i, j) is
// evaluated in row i and again in row j, so no force is ever scattered and
// no atomic touches a force (Newton's third law is not used).
//
// Work items are (i-tile, j-chunk) pairs taken from a device queue by a
// persistent grid; each item writes its partial row sums (gx, gy, gz, row
// energy) to its own slot, and the finalize kernel sums the slots of an
// atom in a fixed order, so results are deterministic for a given chunking.
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

template <typename T, bool GRAD, bool DIAG>
__device__ __forceinline__ void sweep(const typename VT<T>::V4 *__restrict__ sp,
                                      const typename VT<T>::V2 *__restrict__ sq, T xi, T yi,
                                      T zi, T qi, T c6i, T c12i, int diag_k, T &gx, T &gy, T &gz,
                                      T &ec, T &lj) {
#pragma unroll 8
    for (int k = 0; k < TJ; k++) {
        const typename VT<T>::V4 pj = sp[k];
        const typename VT<T>::V2 qj = sq[k];
        const T dx = pj.x - xi, dy = pj.y - yi, dz = pj.z - zi;
        const T r2 = dx * dx + dy * dy + dz * dz;
        T ri = VT<T>::rsq(r2);
        if (DIAG) ri = (k == diag_k) ? T(0) : ri;
        const T ri2 = ri * ri;
        const T e = qi * pj.w * ri;
        const T ri6 = ri2 * ri2 * ri2;
        const T c6 = c6i * qj.x, c12 = c12i * qj.y;
        const T t1 = c12 * ri6 - c6;
        ec += e;
        lj += ri6 * t1;
        if (GRAD) {
            const T t2 = c12 * ri6 + t1;
            const T f = (ri6 * t2 + e) * ri2;
            gx += f * dx;
            gy += f * dy;
            gz += f * dz;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(TI) k_pair(Ctx c) {
    using V4 = typename VT<T>::V4;
    using V2 = typename VT<T>::V2;
    __shared__ V4 sp[TJ];
    __shared__ V2 sq[TJ];
    __shared__ int s_item;
    const V4 *__restrict__ pos;
    const V2 *__restrict__ par;
    V4 *__restrict__ out;
    if constexpr (sizeof(T) == 4) {
        pos = c.posf; par = c.parf; out = c.gpf;
    } else {
        pos = c.posd; par = c.pard; out = c.gpd;
    }
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&c.counters[CNT_PAIR], 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= c.n_items) break;
        const Item I = c.items[it];
        const Tile tl = c.tiles[I.tile];
        const int kind = c.st[tl.sys].ev_kind;
        if (kind == EV_NONE) continue;
        const bool valid = tid < tl.na;
        const int ig = tl.a0 + tid;
        V4 pi;
        V2 ai;
        if (valid) {
            pi = pos[ig];
            ai = par[ig];
        } else {
            pi.x = T(-1e6); pi.y = T(-1e6); pi.z = T(-1e6); pi.w = T(0);
            ai.x = T(0); ai.y = T(0);
        }
        T gx = 0, gy = 0, gz = 0, ec = 0, lj = 0;
        const int jend = I.j0 + I.nj;
        for (int jt = I.j0; jt < jend; jt += TJ) {
            const int jl = jt + tid;
            if (jl < jend) {
                sp[tid] = pos[jl];
                sq[tid] = par[jl];
            } else {
                V4 d; d.x = T(1e6); d.y = T(1e6); d.z = T(1e6); d.w = T(0);
                V2 z; z.x = T(0); z.y = T(0);
                sp[tid] = d;
                sq[tid] = z;
            }
            __syncthreads();
            const int dk = ig - jt;  // position of atom i inside this j tile, if any
            const bool diag = I.diag && dk >= 0 && dk < TJ;
            if (kind == EV_EG) {
                if (diag)
                    sweep<T, true, true>(sp, sq, pi.x, pi.y, pi.z, pi.w, ai.x, ai.y, dk, gx, gy, gz, ec, lj);
                else
                    sweep<T, true, false>(sp, sq, pi.x, pi.y, pi.z, pi.w, ai.x, ai.y, -1, gx, gy, gz, ec, lj);
            } else {
                if (diag)
                    sweep<T, false, true>(sp, sq, pi.x, pi.y, pi.z, pi.w, ai.x, ai.y, dk, gx, gy, gz, ec, lj);
                else
                    sweep<T, false, false>(sp, sq, pi.x, pi.y, pi.z, pi.w, ai.x, ai.y, -1, gx, gy, gz, ec, lj);
            }
            __syncthreads();
        }
        V4 o;
        o.x = gx; o.y = gy; o.z = gz;
        o.w = ec + lj * T(1.0 / 6.0);
        out[(int64_t)it * TI + tid] = o;
    }
    if (tid == 0) {
        __threadfence();
        const unsigned d = atomicAdd(&c.counters[CNT_PAIR_EXIT], 1u);
        if (d == gridDim.x - 1) {  // every block is past its last queue access
            c.counters[CNT_PAIR] = 0;
            c.counters[CNT_PAIR_EXIT] = 0;
            __threadfence();
        }
    }
}

int pair_grid_size(int prec) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (prec == FFMIN_MIXED)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<float>, TI, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pair<double>, TI, 0);
    if (per < 1) per = 1;
    return sms * per;
}

cudaError_t launch_pair(const Ctx &c, int grid, cudaStream_t s) {
    if (c.prec == FFMIN_MIXED)
        k_pair<float><<<grid, TI, 0, s>>>(c);
    else
        k_pair<double><<<grid, TI, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace ffm
