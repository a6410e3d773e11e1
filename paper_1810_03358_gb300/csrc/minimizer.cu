// Per-tile kernels of the minimizer pipeline (one 128-thread block per
// 128-atom tile, one thread per atom) and the bonded terms.
//
//   prepare   trial point XT = base + h * dir * scale (FP64, fused multiply-add
//             per component) and the pair-kernel positions (float4/double4_32a)
//   finalize  per-atom sum of the pair kernel's partial rows in a fixed order,
//             bonded terms of Section 2 gathered per atom (no atomics),
//             energy / gradient reductions, then the control step
//   update    accept a point, push an L-BFGS pair, FGM vector updates
//   dir       search directions: a G + b R + sum c_j S_j + sum c_j Y_j,
//             scaled by gamma (and the learned diagonal), with their dots
//
// Reductions are deterministic: every block writes its partial sums, the
// last block to finish (atomic ticket) sums each system's blocks in a fixed
// order and runs that system's control step.  No thread ever waits.
//
// This file is compiled without contraction of a*b+c into FMA so that the
// scalar control arithmetic and the vector updates round like their
// textbook statements; fused multiply-adds appear only where written.
#include <cmath>

#include "control.cuh"

namespace ffm {

constexpr int NW = TI / 32;

template <int NR>
__device__ void block_reduce_store(double (&v)[NR], unsigned maxmask, double *dst) {
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

__device__ bool last_block(unsigned int *cnt) {
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

// sum (or max) of one reduction value over a system's tiles, fixed order,
// executed by a whole warp; the result is valid on every lane
__device__ double warp_sys_sum(const Ctx &c, const SysState &S, int k, bool mx) {
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

// ---------------------------------------------------------------- bonded
__device__ __forceinline__ void ld3(const double *x, int a, double *o) {
    o[0] = x[3 * a]; o[1] = x[3 * a + 1]; o[2] = x[3 * a + 2];
}
__device__ __forceinline__ double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Energy of one bonded term; when g != nullptr also the gradient of the
// term with respect to the atom at position `pos` of the term.
//   bond     E = K (r - r0)^2
//   angle    E = K (theta - theta0)^2, theta = atan2(|u x v|, u.v)
//   dihedral E = 1/2 [V1(1+cos p) + V2(1-cos 2p) + V3(1+cos 3p) + V4(1-cos 4p)]
// (Section 2).  cos(k phi), sin(k phi) come from cos phi = m.n/(|m||n|) and
// sin phi = |b2| b1.n/(|m||n|) by the multiple-angle identities.
__device__ double bonded_term(const Ctx &c, const double *x, int type, int term, int pos,
                              double *g, int *degenerate) {
    if (type == 0) {
        const int2 ij = c.bidx[term];
        const double2 kp = c.bpar[term];
        double xi[3], xj[3], d[3];
        ld3(x, ij.x, xi);
        ld3(x, ij.y, xj);
        for (int k = 0; k < 3; k++) d[k] = xi[k] - xj[k];
        const double r = sqrt(dot3(d, d));
        const double e = kp.x * (r - kp.y) * (r - kp.y);
        if (g) {
            const double f = 2.0 * kp.x * (r - kp.y) / r * (pos == 0 ? 1.0 : -1.0);
            for (int k = 0; k < 3; k++) g[k] = f * d[k];
        }
        return e;
    }
    if (type == 1) {
        const int4 q = c.aidx[term];
        const double2 kp = c.apar[term];
        double xi[3], xj[3], xk[3], u[3], v[3], w[3];
        ld3(x, q.x, xi);
        ld3(x, q.y, xj);
        ld3(x, q.z, xk);
        for (int k = 0; k < 3; k++) { u[k] = xi[k] - xj[k]; v[k] = xk[k] - xj[k]; }
        cross3(u, v, w);
        const double cr = sqrt(dot3(w, w));
        const double uv = dot3(u, v);
        const double th = atan2(cr, uv);
        const double e = kp.x * (th - kp.y) * (th - kp.y);
        if (g) {
            if (cr > 0.0) {
                const double de = 2.0 * kp.x * (th - kp.y);
                const double uu = dot3(u, u), vv = dot3(v, v);
                for (int k = 0; k < 3; k++) {
                    const double dti = (uv * u[k] / uu - v[k]) / cr;
                    const double dtk = (uv * v[k] / vv - u[k]) / cr;
                    g[k] = pos == 0 ? de * dti : (pos == 2 ? de * dtk : -(de * dti + de * dtk));
                }
            } else {
                g[0] = g[1] = g[2] = 0.0;
            }
        }
        return e;
    }
    const int4 q = c.didx[term];
    const double4_32a V = c.dpar[term];
    double xi[3], xj[3], xk[3], xl[3], b1[3], b2[3], b3[3], m[3], n[3];
    ld3(x, q.x, xi);
    ld3(x, q.y, xj);
    ld3(x, q.z, xk);
    ld3(x, q.w, xl);
    for (int k = 0; k < 3; k++) { b1[k] = xj[k] - xi[k]; b2[k] = xk[k] - xj[k]; b3[k] = xl[k] - xk[k]; }
    cross3(b1, b2, m);
    cross3(b2, b3, n);
    const double mm = dot3(m, m), nn = dot3(n, n), b2n = sqrt(dot3(b2, b2));
    const bool deg = (mm < 1e-12 || nn < 1e-12);
    if (degenerate) *degenerate = deg;
    double cp, sp;
    if (deg) {
        const double phi = atan2(b2n * dot3(b1, n), dot3(m, n));
        cp = cos(phi);
        sp = sin(phi);
    } else {
        const double inv = 1.0 / sqrt(mm * nn);
        cp = dot3(m, n) * inv;
        sp = b2n * dot3(b1, n) * inv;
    }
    const double c2 = 2.0 * cp * cp - 1.0;
    const double c3 = cp * (4.0 * cp * cp - 3.0);
    const double c4 = 2.0 * c2 * c2 - 1.0;
    const double e = 0.5 * (V.x * (1.0 + cp) + V.y * (1.0 - c2) + V.z * (1.0 + c3) + V.w * (1.0 - c4));
    if (g) {
        if (deg) {
            g[0] = g[1] = g[2] = 0.0;
        } else {
            const double s2 = 2.0 * sp * cp;
            const double s3 = sp * (4.0 * cp * cp - 1.0);
            const double s4 = 2.0 * s2 * c2;
            const double dedphi = 0.5 * (-V.x * sp + 2.0 * V.y * s2 - 3.0 * V.z * s3 + 4.0 * V.w * s4);
            const double bb = b2n * b2n;
            const double ca = dot3(b1, b2) / bb, cc = dot3(b3, b2) / bb;
            for (int k = 0; k < 3; k++) {
                const double pi_ = -b2n / mm * m[k];
                const double pl = b2n / nn * n[k];
                double p;
                if (pos == 0) p = pi_;
                else if (pos == 1) p = -(1.0 + ca) * pi_ + cc * pl;
                else if (pos == 2) p = ca * pi_ - (1.0 + cc) * pl;
                else p = pl;
                g[k] = dedphi * p;
            }
        }
    }
    return e;
}

// ---------------------------------------------------------------- prepare
__global__ void __launch_bounds__(TI) k_prepare(Ctx c) {
    const Tile t = c.tiles[blockIdx.x];
    const SysState &S = c.st[t.sys];
    if (S.ev_kind == EV_NONE) return;
    const int i = threadIdx.x;
    if (i >= t.na) return;
    const int a = t.a0 + i;
    const double *base = vslot(c, S.ev_base) + 3 * a;
    double *xt = vslot(c, V_XT) + 3 * a;
    double p[3];
    if (S.ev_dir >= 0) {
        const double *d = vslot(c, S.ev_dir) + 3 * a;
        const double h = S.ev_h, sc = S.ev_scale;
        for (int k = 0; k < 3; k++) p[k] = fma(h, d[k] * sc, base[k]);
    } else {
        for (int k = 0; k < 3; k++) p[k] = base[k];
    }
    for (int k = 0; k < 3; k++) xt[k] = p[k];
    const double q = c.qs[a];
    if (c.prec == FFMIN_MIXED)
        c.posf[a] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)q);
    else
        c.posd[a] = make_double4_32a(p[0], p[1], p[2], q);
}

// ---------------------------------------------------------------- finalize
__global__ void __launch_bounds__(TI) k_finalize(Ctx c) {
    const Tile t = c.tiles[blockIdx.x];
    const int kind = c.st[t.sys].ev_kind;
    double v[RF_N];
#pragma unroll
    for (int k = 0; k < RF_N; k++) v[k] = 0.0;
    const int i = threadIdx.x;
    if (kind != EV_NONE && i < t.na) {
        const int a = t.a0 + i;
        double e = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        if (c.prec == FFMIN_MIXED) {
            for (int it = 0; it < t.nitem; it++) {
                const float4 p = c.gpf[(int64_t)(t.item0 + it) * TI + i];
                e += (double)p.w;
                g0 += (double)p.x; g1 += (double)p.y; g2 += (double)p.z;
            }
        } else {
            for (int it = 0; it < t.nitem; it++) {
                const double4_32a p = c.gpd[(int64_t)(t.item0 + it) * TI + i];
                e += p.w;
                g0 += p.x; g1 += p.y; g2 += p.z;
            }
        }
        e = 0.5 * e;  // every pair was counted in both of its rows
        const double *xt = vslot(c, V_XT);
        const bool grad = kind == EV_EG;
        for (int k = c.inc_off[a]; k < c.inc_off[a + 1]; k++) {
            const int2 in = c.inc[k];
            const int type = in.x >> 2, pos = in.x & 3;
            if (!grad && pos != 0) continue;
            double gb[3];
            const double et = bonded_term(c, xt, type, in.y, pos, grad ? gb : nullptr, nullptr);
            if (pos == 0) e += et;
            if (grad) { g0 += gb[0]; g1 += gb[1]; g2 += gb[2]; }
        }
        v[RF_E] = e;
        bool bad = !isfinite(e);
        if (grad) {
            double *gt = vslot(c, V_GT) + 3 * a;
            gt[0] = g0; gt[1] = g1; gt[2] = g2;
            const double *G = vslot(c, V_G) + 3 * a;
            const double *R = vslot(c, V_R) + 3 * a;
            v[RF_GG] = g0 * g0 + g1 * g1 + g2 * g2;
            v[RF_GINF] = fmax(fabs(g0), fmax(fabs(g1), fabs(g2)));
            v[RF_GTG] = g0 * G[0] + g1 * G[1] + g2 * G[2];
            v[RF_GTR] = g0 * R[0] + g1 * R[1] + g2 * R[2];
            bad = bad || !isfinite(g0) || !isfinite(g1) || !isfinite(g2);
        }
        v[RF_BAD] = bad ? 1.0 : 0.0;
    }
    const unsigned maxmask = (1u << RF_GINF) | (1u << RF_BAD);
    block_reduce_store<RF_N>(v, maxmask, &c.red[(int64_t)blockIdx.x * NRED]);
    if (!last_block(&c.counters[CNT_FIN])) return;
    __shared__ double tot[NW][RF_N];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = w; b < c.n_sys; b += NW) {
        SysState &S = c.st[b];
        if (S.ev_kind == EV_NONE) continue;
        for (int k = 0; k < RF_N; k++) {
            const double x = warp_sys_sum(c, S, k, (maxmask >> k) & 1u);
            if (lane == 0) tot[w][k] = x;
        }
        __syncwarp();
        if (lane == 0) on_eval_done(c, S, tot[w]);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) c.counters[CNT_FIN] = 0;
}

// ---------------------------------------------------------------- update
__global__ void __launch_bounds__(TI) k_update(Ctx c) {
    const Tile t = c.tiles[blockIdx.x];
    const SysState &S = c.st[t.sys];
    const int op = S.upd.op;
    const int i = threadIdx.x;
    if (op == U_PUSH) {
        double v[RU_N];
#pragma unroll
        for (int k = 0; k < RU_N; k++) v[k] = 0.0;
        if (i < t.na) {
            const int64_t off = 3 * (int64_t)(t.a0 + i);
            double *X = vslot(c, V_X) + off, *G = vslot(c, V_G) + off;
            const double *XT = vslot(c, V_XT) + off, *GT = vslot(c, V_GT) + off;
            double *Ss = vslot(c, V_S0 + S.upd.stage) + off, *Ys = vslot(c, V_Y0 + S.upd.stage) + off;
            double s[3], y[3];
            for (int k = 0; k < 3; k++) {
                s[k] = XT[k] - X[k];
                y[k] = GT[k] - G[k];
                Ss[k] = s[k];
                Ys[k] = y[k];
            }
            v[RU_SY] = s[0] * y[0] + s[1] * y[1] + s[2] * y[2];
            v[RU_YY] = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
            v[RU_SG] = s[0] * GT[0] + s[1] * GT[1] + s[2] * GT[2];
            const int nS = S.upd.nS;
#pragma unroll
            for (int j = 0; j < NRING; j++) {
                if (j < nS) {
                    const double *sj = vslot(c, V_S0 + S.upd.sS[j]) + off;
                    v[RU_SJY + j] = sj[0] * y[0] + sj[1] * y[1] + sj[2] * y[2];
                    v[RU_SJG + j] = sj[0] * GT[0] + sj[1] * GT[1] + sj[2] * GT[2];
                }
            }
            for (int k = 0; k < 3; k++) { X[k] = XT[k]; G[k] = GT[k]; }
        }
        block_reduce_store<RU_N>(v, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    } else if (op != U_NONE && i < t.na) {
        const int64_t off = 3 * (int64_t)(t.a0 + i);
        double *X = vslot(c, V_X) + off, *G = vslot(c, V_G) + off, *W = vslot(c, V_W) + off;
        double *P = vslot(c, V_P) + off, *XB = vslot(c, V_XB) + off;
        const double *XT = vslot(c, V_XT) + off, *GT = vslot(c, V_GT) + off;
        switch (op) {
        case U_ACCEPT:
            for (int k = 0; k < 3; k++) { X[k] = XT[k]; G[k] = GT[k]; }
            break;
        case U_FGM_W:
            for (int k = 0; k < 3; k++) { W[k] = XT[k]; G[k] = GT[k]; }
            if (S.upd.best) for (int k = 0; k < 3; k++) XB[k] = XT[k];
            break;
        case U_FGM_ACCEPT: {
            const double *R = vslot(c, V_R) + off;
            const double h = S.upd.h, inv = S.upd.inv;
            for (int k = 0; k < 3; k++) {
                const double xn = fma(h, R[k] * inv, W[k]);
                P[k] = S.upd.restart ? 0.0 : xn - X[k];
                X[k] = xn;
                if (S.upd.best) XB[k] = xn;
            }
            break;
        }
        case U_FGM_RESET:
            for (int k = 0; k < 3; k++) { X[k] = W[k]; P[k] = 0.0; }
            break;
        case U_FGM_BEST_W:
            for (int k = 0; k < 3; k++) XB[k] = W[k];
            break;
        default:
            break;
        }
    }
    if (!last_block(&c.counters[CNT_UPD])) return;
    __shared__ double tot[NW][RU_N];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = w; b < c.n_sys; b += NW) {
        SysState &Sb = c.st[b];
        if (Sb.upd.op == U_NONE) continue;
        if (Sb.upd.op == U_PUSH) {
            for (int k = 0; k < RU_N; k++) {
                const double x = warp_sys_sum(c, Sb, k, false);
                if (lane == 0) tot[w][k] = x;
            }
        }
        __syncwarp();
        if (lane == 0) on_update_done(c, Sb, tot[w]);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) c.counters[CNT_UPD] = 0;
}

// ---------------------------------------------------------------- direction
template <int WHICH>
__global__ void __launch_bounds__(TI) k_dir(Ctx c) {
    const Tile t = c.tiles[blockIdx.x];
    const SysState &S = c.st[t.sys];
    const DirOp &d = S.dir[WHICH];
    const int i = threadIdx.x;
    double v[NRING];
#pragma unroll
    for (int k = 0; k < NRING; k++) v[k] = 0.0;
    const bool on = d.on != 0;
    if (on && i < t.na) {
        const int64_t off = 3 * (int64_t)(t.a0 + i);
        const double *G = vslot(c, V_G) + off;
        double *R = vslot(c, V_R) + off;
        const double *D = vslot(c, V_D) + off;
        double acc[3];
        for (int k = 0; k < 3; k++) {
            double x = 0.0;
            if (d.a != 0.0) x = d.a * G[k];
            if (d.b != 0.0) x = x + d.b * R[k];
            acc[k] = x;
        }
        for (int j = 0; j < d.nY; j++) {
            const double *y = vslot(c, V_Y0 + d.sY[j]) + off;
            const double cy = d.cY[j];
            for (int k = 0; k < 3; k++) acc[k] = acc[k] + cy * y[k];
        }
        for (int j = 0; j < d.nS; j++) {
            const double *s = vslot(c, V_S0 + d.sS[j]) + off;
            const double cs = d.cS[j];
            for (int k = 0; k < 3; k++) acc[k] = acc[k] + cs * s[k];
        }
        for (int k = 0; k < 3; k++) {
            acc[k] = d.use_d ? (d.outer * D[k]) * acc[k] : d.outer * acc[k];
            R[k] = acc[k];
        }
        if (d.dots == 1) {
            v[RD_RR] = acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2];
            v[RD_GR] = G[0] * acc[0] + G[1] * acc[1] + G[2] * acc[2];
        } else if (d.dots == 2) {
#pragma unroll
            for (int j = 0; j < NRING; j++) {
                if (j < d.nY) {
                    const double *y = vslot(c, V_Y0 + d.sY[j]) + off;
                    v[j] = y[0] * acc[0] + y[1] * acc[1] + y[2] * acc[2];
                }
            }
        }
    }
    if (on) block_reduce_store<NRING>(v, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    if (!last_block(&c.counters[WHICH == 0 ? CNT_DIR1 : CNT_DIR2])) return;
    __shared__ double tot[NW][NRING];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int b = w; b < c.n_sys; b += NW) {
        SysState &Sb = c.st[b];
        if (!Sb.dir[WHICH].on) continue;
        const int nv = Sb.dir[WHICH].dots == 2 ? Sb.dir[WHICH].nY : 2;
        for (int k = 0; k < nv; k++) {
            const double x = warp_sys_sum(c, Sb, k, false);
            if (lane == 0) tot[w][k] = x;
        }
        __syncwarp();
        if (lane == 0) on_dir_done(c, Sb, WHICH, tot[w]);
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) c.counters[WHICH == 0 ? CNT_DIR1 : CNT_DIR2] = 0;
}

cudaError_t launch_prepare(const Ctx &c, cudaStream_t s) {
    k_prepare<<<c.n_tiles, TI, 0, s>>>(c);
    return cudaGetLastError();
}
cudaError_t launch_finalize(const Ctx &c, cudaStream_t s) {
    k_finalize<<<c.n_tiles, TI, 0, s>>>(c);
    return cudaGetLastError();
}
cudaError_t launch_update(const Ctx &c, cudaStream_t s) {
    k_update<<<c.n_tiles, TI, 0, s>>>(c);
    return cudaGetLastError();
}
cudaError_t launch_dir(const Ctx &c, int which, cudaStream_t s) {
    if (which == 0) k_dir<0><<<c.n_tiles, TI, 0, s>>>(c);
    else k_dir<1><<<c.n_tiles, TI, 0, s>>>(c);
    return cudaGetLastError();
}

}  // namespace ffm
