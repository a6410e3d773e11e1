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

#include "bonded.cuh"
#include "control.cuh"
#include "mlp.cuh"
#include "reduce.cuh"

namespace ffm {

// <a, b> of two 3-vectors with explicit FMA (this unit is compiled without
// implicit contraction; the vector kernels are FP64-pipe bound)
__device__ __forceinline__ double dot3_fma(const double *a, const double *b) {
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
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
    if (S.mode == 0 && S.ev_delta) {
        // difference trial: base position and the displacement, each rounded
        // once to FP32 (the displacement keeps its full relative precision)
        c.posf[a] = make_float4((float)base[0], (float)base[1], (float)base[2], (float)q);
        c.dispf[a] = make_float4((float)(p[0] - base[0]), (float)(p[1] - base[1]), (float)(p[2] - base[2]), 0.f);
    } else if (S.mode == 0) {
        c.posf[a] = make_float4((float)p[0], (float)p[1], (float)p[2], (float)q);
    } else {
        c.posd[a] = make_double4_32a(p[0], p[1], p[2], q);
    }
}

// ---------------------------------------------------------------- finalize
// sum over q < n of f(q) (a double4; only .x .y .z when XYZ, only .w when
// W) in four interleaved strands (q mod 4), combined as (s0 + s1) + (s2 + s3):
// every group of four loads is issued together and no dependent chain of
// FP64 adds is longer than n / 4 + 2
template <bool XYZ, bool W, typename F>
__device__ __forceinline__ double4 strand_sum(int n, F f) {
    double ax[4] = {0.0, 0.0, 0.0, 0.0}, ay[4] = {0.0, 0.0, 0.0, 0.0};
    double az[4] = {0.0, 0.0, 0.0, 0.0}, aw[4] = {0.0, 0.0, 0.0, 0.0};
    int q = 0;
    for (; q + 4 <= n; q += 4) {
        double4 p[4];
#pragma unroll
        for (int u = 0; u < 4; u++) p[u] = f(q + u);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (XYZ) { ax[u] += p[u].x; ay[u] += p[u].y; az[u] += p[u].z; }
            if (W) aw[u] += p[u].w;
        }
    }
#pragma unroll
    for (int u = 0; u < 3; u++) {
        if (q + u < n) {
            const double4 p = f(q + u);
            if (XYZ) { ax[u] += p.x; ay[u] += p.y; az[u] += p.z; }
            if (W) aw[u] += p.w;
        }
    }
    return make_double4(XYZ ? (ax[0] + ax[1]) + (ax[2] + ax[3]) : 0.0, XYZ ? (ay[0] + ay[1]) + (ay[2] + ay[3]) : 0.0,
                        XYZ ? (az[0] + az[1]) + (az[2] + az[3]) : 0.0, W ? (aw[0] + aw[1]) + (aw[2] + aw[3]) : 0.0);
}

__global__ void __launch_bounds__(TI) k_finalize(Ctx c) {
    const Tile t = c.tiles[blockIdx.x];
    const int kind = c.st[t.sys].ev_kind;
    const int mode = c.st[t.sys].mode;
    double v[RF_N];
#pragma unroll
    for (int k = 0; k < RF_N; k++) v[k] = 0.0;
    const int i = threadIdx.x;
    if (kind != EV_NONE && i < t.na) {
        const int a = t.a0 + i;
        double e, g0 = 0.0, g1 = 0.0, g2 = 0.0;
        if (mode == 0 && c.sym64 && kind == EV_E) {
            // FP32 energy only on the symmetric list: the i-side rows of the
            // tile's own row of items (consecutive slots, 1 + C apart), each
            // pair counted once
            const SysState &S = c.st[t.sys];
            const int T = t.tloc, C = t.chunk64;
            const int nch = (S.ntile - T + C - 1) / C;
            e = strand_sum<false, true>(nch, [&](int q) {
                    const float4 p = c.gpf_sym[((int64_t)t.slot64 + (int64_t)q * (1 + C)) * TI + i];
                    return make_double4(0.0, 0.0, 0.0, (double)p.w);
                }).w;
        } else if (mode == 0) {
            const double4 r = strand_sum<true, true>(t.nitem, [&](int it) {
                const float4 p = c.gpf[(int64_t)(t.item0 + it) * TI + i];
                return make_double4((double)p.x, (double)p.y, (double)p.z, (double)p.w);
            });
            e = 0.5 * r.w;  // every pair was counted in both of its rows
            g0 = r.x; g1 = r.y; g2 = r.z;
        } else if (c.sym64) {
            // symmetric tiles: the j-side rows this tile received from the
            // items of rows I <= T, then its own row's i-side rows; each
            // pair's energy was counted once (the slot of row I's item u is
            // tiles[I].slot64 + u * (1 + C))
            const SysState &S = c.st[t.sys];
            const int T = t.tloc, C = t.chunk64;
            double4 rj = make_double4(0.0, 0.0, 0.0, 0.0);
            if (kind == EV_EG)
                rj = strand_sum<true, false>(T + 1, [&](int I) {
                    const int q = T - I;
                    const int64_t slot = (int64_t)c.tiles[S.tile0 + I].slot64 + (int64_t)(q / C) * (1 + C) + 1 + q % C;
                    const double4_32a p = c.gpd[slot * TI + i];
                    return make_double4(p.x, p.y, p.z, 0.0);
                });
            const int nch = (S.ntile - T + C - 1) / C;
            const double4 ri = strand_sum<true, true>(nch, [&](int q) {
                const double4_32a p = c.gpd[((int64_t)t.slot64 + (int64_t)q * (1 + C)) * TI + i];
                return make_double4(p.x, p.y, p.z, p.w);
            });
            e = ri.w;
            g0 = rj.x + ri.x; g1 = rj.y + ri.y; g2 = rj.z + ri.z;
        } else {
            const double4 r = strand_sum<true, true>(t.nitem, [&](int it) {
                const double4_32a p = c.gpd[(int64_t)(t.item0 + it) * TI + i];
                return make_double4(p.x, p.y, p.z, p.w);
            });
            e = 0.5 * r.w;  // every pair was counted in both of its rows
            g0 = r.x; g1 = r.y; g2 = r.z;
        }
        v[RF_EPAIR] = e;
        // bonded terms: evaluated once per term by the pair kernel's bonded
        // items; every atom gathers its terms' energies (as owner) and
        // position gradients through its incidence list (four entries'
        // loads issued together; entry u of each group to strand u mod 2)
        const bool grad = kind == EV_EG;
        double be[2] = {0.0, 0.0}, bg[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        const int k1 = c.inc_off[a + 1];
        for (int k = c.inc_off[a]; k < k1; k += 4) {
            int2 in[4];
            double te[4], gb[4][3];
#pragma unroll
            for (int u = 0; u < 4; u++) in[u] = k + u < k1 ? c.inc[k + u] : make_int2(-1, 0);
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int type = in[u].x >> 2, pos = in[u].x & 3;
                te[u] = in[u].x >= 0 && pos == 0 ? c.te[bonded_index(c, type, in[u].y)] : 0.0;
                if (grad && in[u].x >= 0) {
                    const double *g = c.tg + 3 * bonded_grad_slot(c, type, in[u].y, pos);
                    gb[u][0] = g[0]; gb[u][1] = g[1]; gb[u][2] = g[2];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (in[u].x < 0) break;
                if ((in[u].x & 3) == 0) be[u & 1] += te[u];
                if (grad) { bg[u & 1][0] += gb[u][0]; bg[u & 1][1] += gb[u][1]; bg[u & 1][2] += gb[u][2]; }
            }
        }
        e += be[0] + be[1];
        if (grad) {
            g0 += bg[0][0] + bg[1][0];
            g1 += bg[0][1] + bg[1][1];
            g2 += bg[0][2] + bg[1][2];
        }
        v[RF_E] = e;
        bool bad = !isfinite(e);
        if (grad) {
            double *gt = vslot(c, V_GT) + 3 * a;
            gt[0] = g0; gt[1] = g1; gt[2] = g2;
            const double *G = vslot(c, V_G) + 3 * a;
            const double *R = vslot(c, V_R) + 3 * a;
            v[RF_GG] = fma(g0, g0, fma(g1, g1, g2 * g2));
            v[RF_GINF] = fmax(fabs(g0), fmax(fabs(g1), fabs(g2)));
            v[RF_GTG] = fma(g0, G[0], fma(g1, G[1], g2 * G[2]));
            v[RF_GTR] = fma(g0, R[0], fma(g1, R[1], g2 * R[2]));
            bad = bad || !isfinite(g0) || !isfinite(g1) || !isfinite(g2);
        }
        v[RF_BAD] = bad ? 1.0 : 0.0;
    }
    const unsigned maxmask = (1u << RF_GINF) | (1u << RF_BAD);
    block_reduce_columns<RF_N>(v, RF_N, maxmask, &c.red[(int64_t)blockIdx.x * NRED]);
    if (c.sep_reduce || !last_block(&c.counters[CNT_FIN])) return;
    last_block_systems<RF_N>(
        c, RF_N, maxmask, [](const SysState &S) { return S.ev_kind != EV_NONE; },
        [&](SysState &S, const double *tot) { on_eval_done(c, S, tot); }, nullptr);
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
            v[RU_SY] = dot3_fma(s, y);
            v[RU_YY] = dot3_fma(y, y);
            if (S.rec_ptr && S.rec_every > 0 && S.iter % S.rec_every == 0) {
                const int slot = S.iter / S.rec_every - 1;
                if (slot < S.rec_slots) {
                    double *r = S.rec_ptr + ((int64_t)slot * c.n_atoms + t.a0 + i) * 4;
                    r[0] = v[RU_SY];
                    r[1] = v[RU_YY];
                    r[2] = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
                    r[3] = 1.0;
                }
            }
            v[RU_SG] = dot3_fma(s, GT);
            const int nS = S.upd.nS;
#pragma unroll
            for (int j = 0; j < NRING; j++) {
                if (j < nS) {
                    const double *sj = vslot(c, V_S0 + S.upd.sS[j]) + off;
                    v[ru_sjy(j)] = dot3_fma(sj, y);
                    v[ru_sjg(j)] = dot3_fma(sj, GT);
                }
            }
            for (int k = 0; k < 3; k++) { X[k] = XT[k]; G[k] = GT[k]; }
        }
        block_reduce_columns<RU_N>(v, ru_count(S.upd.nS), 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    } else if (op == U_OGM) {
        double v[1] = {0.0};
        if (i < t.na) {
            const int64_t off = 3 * (int64_t)(t.a0 + i);
            double *X = vslot(c, V_X) + off, *G = vslot(c, V_G) + off, *W = vslot(c, V_W) + off;
            double *R = vslot(c, V_R) + off, *X0 = vslot(c, V_X0) + off, *DS = vslot(c, V_DS) + off;
            const double *XT = vslot(c, V_XT) + off, *GT = vslot(c, V_GT) + off;
            const UpdOp &u = S.upd;
            double rr[3];
            for (int k = 0; k < 3; k++) {
                double x = X[k], g = G[k];
                if (u.accept) { x = XT[k]; g = GT[k]; X[k] = x; G[k] = g; }
                double x0, ds;
                if (u.restart) {
                    x0 = x;
                    ds = g;
                    X0[k] = x0;
                } else {
                    x0 = X0[k];
                    ds = u.accept ? fma(u.h, g, DS[k]) : DS[k];
                }
                DS[k] = ds;
                W[k] = fma(u.a, x, u.b * x0);
                const double r = -fma(u.a, g, u.inv * ds);
                R[k] = r;
                rr[k] = r;
            }
            v[0] = dot3_fma(rr, rr);
        }
        block_reduce_columns<1>(v, 1, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
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
            if (S.upd.restart)  // a (re)start at XT: x^k = x^{k-1} = XT
                for (int k = 0; k < 3; k++) { X[k] = XT[k]; P[k] = 0.0; }
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
        case U_HB: {  // Eq. 8, formed as the oracle forms it
            // accept the evaluated point (XT, GT): x^{k+1}, or at the start
            // x^0 itself with x^{-1} = x^0; then form the next iterate
            double *XTw = vslot(c, V_XT) + off;
            const double a = S.upd.a, b = S.upd.b;
            for (int k = 0; k < 3; k++) {
                const double x = XT[k], g = GT[k];
                const double xp = S.upd.accept ? X[k] : x;
                X[k] = x;
                G[k] = g;
                P[k] = xp;
                XTw[k] = fma(b, x - xp, fma(-a, g, x));
            }
            break;
        }
        default:
            break;
        }
    }
    if (c.sep_reduce || !last_block(&c.counters[CNT_UPD])) return;
    last_block_systems<RU_N>(
        c, RU_N, 0u, [](const SysState &S) { return S.upd.op != U_NONE; },
        [&](SysState &S, const double *tot) { on_update_done(c, S, tot); },
        [](const SysState &S) { return S.upd.op == U_PUSH ? ru_count(S.upd.nS) : (S.upd.op == U_OGM ? 1 : 0); });
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
    __shared__ float w_mlp[MLP_NW];
    if (on && d.use_d) {  // learned H0 diagonal: FP16 weights -> FP32 in shared memory
        for (int k = threadIdx.x; k < MLP_NW; k += blockDim.x)
            w_mlp[k] = __half2float(__ushort_as_half(c.mlp_w[k]));
        __syncthreads();
    }
    if (on && i < t.na) {
        const int64_t off = 3 * (int64_t)(t.a0 + i);
        const double *G = vslot(c, V_G) + off;
        double *R = vslot(c, V_R) + off;
        double acc[3];
        for (int k = 0; k < 3; k++) {
            double x = 0.0;
            if (d.a != 0.0) x = d.a * G[k];
            if (d.b != 0.0) x = fma(d.b, R[k], x);
            acc[k] = x;
        }
        for (int j = 0; j < d.nY; j++) {
            const double *y = vslot(c, V_Y0 + d.sY[j]) + off;
            const double cy = d.cY[j];
            for (int k = 0; k < 3; k++) acc[k] = fma(cy, y[k], acc[k]);
        }
        for (int j = 0; j < d.nS; j++) {
            const double *s = vslot(c, V_S0 + d.sS[j]) + off;
            const double cs = d.cS[j];
            for (int k = 0; k < 3; k++) acc[k] = fma(cs, s[k], acc[k]);
        }
        double dscale = 1.0;
        if (d.use_d) {
            const int a = t.a0 + i;
            float f[MLP_IN];
            const double gn = sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
            mlp_features(c.feat[3 * a], c.feat[3 * a + 1], c.feat[3 * a + 2], c.ncount[a], (float)gn, f);
            dscale = (double)mlp_scale(w_mlp, f);
        }
        for (int k = 0; k < 3; k++) {
            acc[k] = d.use_d ? (d.outer * dscale) * acc[k] : d.outer * acc[k];
            R[k] = acc[k];
        }
        if (d.dots == 1) {
            v[RD_RR] = dot3_fma(acc, acc);
            v[RD_GR] = dot3_fma(G, acc);
        } else if (d.dots == 2) {
#pragma unroll
            for (int j = 0; j < NRING; j++) {
                if (j < d.nY) {
                    const double *y = vslot(c, V_Y0 + d.sY[j]) + off;
                    v[j] = dot3_fma(y, acc);
                }
            }
        }
    }
    if (on) block_reduce_columns<NRING>(v, d.dots == 2 ? d.nY : 2, 0u, &c.red[(int64_t)blockIdx.x * NRED]);
    if (c.sep_reduce || !last_block(&c.counters[WHICH == 0 ? CNT_DIR1 : CNT_DIR2])) return;
    last_block_systems<NRING>(
        c, 2, 0u, [](const SysState &S) { return S.dir[WHICH].on != 0; },
        [&](SysState &S, const double *tot) { on_dir_done(c, S, WHICH, tot); },
        [](const SysState &S) { return S.dir[WHICH].dots == 2 ? S.dir[WHICH].nY : 2; });
    __syncthreads();
    if (threadIdx.x == 0) c.counters[WHICH == 0 ? CNT_DIR1 : CNT_DIR2] = 0;
}

// one block per system: the system's tile partials of every value are summed
// by the block's warps in tile order, then thread 0 runs the control step
template <int STAGE>
__global__ void __launch_bounds__(TI) k_sysreduce(Ctx c) {
    SysState &S = c.st[blockIdx.x];
    int nv;
    unsigned maxmask = 0u;
    if (STAGE == 0) {
        if (S.upd.op == U_NONE) return;
        nv = S.upd.op == U_PUSH ? ru_count(S.upd.nS) : (S.upd.op == U_OGM ? 1 : 0);
    } else if (STAGE == 1 || STAGE == 2) {
        const DirOp &d = S.dir[STAGE - 1];
        if (!d.on) return;
        nv = d.dots == 2 ? d.nY : 2;
    } else {
        if (S.ev_kind == EV_NONE) return;
        nv = RF_N;
        maxmask = (1u << RF_GINF) | (1u << RF_BAD);
    }
    __shared__ double tot[NRED];
    __shared__ SysState sS;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = w; k < nv; k += NW) {
        const double x = warp_sys_sum(c, S, k, (maxmask >> k) & 1u);
        if (lane == 0) tot[k] = x;
    }
    __syncthreads();
    if (w != 0) return;
    // the control step on a shared-memory copy of the state
    warp_copy_state(&sS, &S);
    if (lane == 0) {
        if (STAGE == 0) on_update_done(c, sS, tot);
        else if (STAGE == 1) on_dir_done(c, sS, 0, tot);
        else if (STAGE == 2) on_dir_done(c, sS, 1, tot);
        else on_eval_done(c, sS, tot);
    }
    __syncwarp();
    warp_copy_state(&S, &sS);
}

cudaError_t launch_sysreduce(const Ctx &c, int stage, cudaStream_t s) {
    switch (stage) {
    case 0: k_sysreduce<0><<<c.n_sys, TI, 0, s>>>(c); break;
    case 1: k_sysreduce<1><<<c.n_sys, TI, 0, s>>>(c); break;
    case 2: k_sysreduce<2><<<c.n_sys, TI, 0, s>>>(c); break;
    default: k_sysreduce<3><<<c.n_sys, TI, 0, s>>>(c); break;
    }
    return cudaGetLastError();
}

// neighbours within 8 A of every atom inside its own system, from X
__global__ void __launch_bounds__(TI) k_ncount(Ctx c, const double *x, int32_t *out) {
    const Tile t = c.tiles[blockIdx.x];
    const SysState &S = c.st[t.sys];
    const int i = threadIdx.x;
    if (i >= t.na) return;
    const int a = t.a0 + i;
    const float xi = (float)x[3 * a], yi = (float)x[3 * a + 1], zi = (float)x[3 * a + 2];
    int n = 0;
    for (int j = S.atom0; j < S.atom0 + S.natoms; j++) {
        const float dx = (float)x[3 * j] - xi, dy = (float)x[3 * j + 1] - yi, dz = (float)x[3 * j + 2] - zi;
        n += (j != a && dx * dx + dy * dy + dz * dz < 64.f) ? 1 : 0;
    }
    out[a] = n;
}

cudaError_t launch_ncount(const Ctx &c, const double *x, int32_t *out, cudaStream_t s) {
    k_ncount<<<c.n_tiles, TI, 0, s>>>(c, x, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- basin hopping
// one block per tile, one thread per atom; the offset is formed as the
// oracle forms it (this unit has no implicit FMA contraction)
__global__ void __launch_bounds__(TI) k_mbh_perturb(Ctx c, const double *best, double *out, double step,
                                                   uint64_t seed, int64_t hop) {
    const Tile t = c.tiles[blockIdx.x];
    const int i = threadIdx.x;
    if (i >= t.na) return;
    const SysState &S = c.st[t.sys];
    const int a = t.a0 + i;
    const uint64_t base = (uint64_t)hop * (uint64_t)(3 * S.natoms) + 3ull * (uint64_t)(a - S.atom0);
    for (int k = 0; k < 3; k++) {
        const double u = (double)(splitmix64(seed + (uint64_t)t.sys, base + k) >> 11) * 0x1.0p-53;
        out[3 * a + k] = best[3 * a + k] + step * (2.0 * u - 1.0);
    }
}

__global__ void __launch_bounds__(TI) k_mbh_accept(Ctx c, const int32_t *flags, const double *x, double *best) {
    const Tile t = c.tiles[blockIdx.x];
    const int i = threadIdx.x;
    if (i >= t.na || !flags[t.sys]) return;
    const int a = t.a0 + i;
    for (int k = 0; k < 3; k++) best[3 * a + k] = x[3 * a + k];
}

cudaError_t launch_mbh_perturb(const Ctx &c, const double *best, double *out, double step, uint64_t seed,
                               int64_t hop, cudaStream_t s) {
    k_mbh_perturb<<<c.n_tiles, TI, 0, s>>>(c, best, out, step, seed, hop);
    return cudaGetLastError();
}
cudaError_t launch_mbh_accept(const Ctx &c, const int32_t *flags, const double *x, double *best, cudaStream_t s) {
    k_mbh_accept<<<c.n_tiles, TI, 0, s>>>(c, flags, x, best);
    return cudaGetLastError();
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
