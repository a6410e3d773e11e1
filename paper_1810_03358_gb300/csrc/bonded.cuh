// Bonded terms of the force field (Section 2): harmonic bonds and angles
// and the four-term torsion, energy and per-position gradient, FP64.
#pragma once

#include "ffmin_internal.cuh"

namespace ffm {

// position of atom a; atom ova (if >= 0) is read from ov instead
__device__ __forceinline__ void ld3(const double *x, int a, double *o, int ova = -1,
                                    const double *ov = nullptr) {
    if (a == ova) {
        o[0] = ov[0]; o[1] = ov[1]; o[2] = ov[2];
    } else {
        o[0] = x[3 * a]; o[1] = x[3 * a + 1]; o[2] = x[3 * a + 2];
    }
}
__device__ __forceinline__ double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Exclusion correction (type 3, a force-field variant outside the paper):
// w times the non-bonded pair term of atoms (i, j), w = s_ij - 1, in FP64:
//   E = w (q'_i q'_j / r + r^-6 (C12 r^-6 - C6) / 6),
//   grad_i E = w (e_cul + r^-6 (2 C12 r^-6 - C6)) r^-2 (x_j - x_i),
// the same pair term the sweep adds, so that the sum is s_ij times it.
__device__ inline double excl_term(const Ctx &c, const double *x, int term, double *gi, int ova,
                                   const double *ov) {
    const int2 ij = c.xidx[term];
    const double w = c.xw[term];
    double xi[3], xj[3], d[3];
    ld3(x, ij.x, xi, ova, ov);
    ld3(x, ij.y, xj, ova, ov);
    for (int k = 0; k < 3; k++) d[k] = xj[k] - xi[k];
    const double r2 = dot3(d, d);
    const double ri = 1.0 / sqrt(r2), ri2 = ri * ri, ri6 = ri2 * ri2 * ri2;
    const double2 pi = c.pard[ij.x], pj = c.pard[ij.y];
    const double C6 = pi.x * pj.x, C12 = pi.y * pj.y;
    const double ec = c.qs[ij.x] * c.qs[ij.y] * ri;
    const double e = w * (ec + ri6 * (C12 * ri6 - C6) * (1.0 / 6.0));
    if (gi) {
        const double f = w * (ec + ri6 * (2.0 * C12 * ri6 - C6)) * ri2;
        for (int k = 0; k < 3; k++) gi[k] = f * d[k];
    }
    return e;
}

// Energy of one bonded term; when g != nullptr also the gradient of the
// term with respect to the atom at position `pos` of the term.
//   bond     E = K (r - r0)^2
//   angle    E = K (theta - theta0)^2, theta = atan2(|u x v|, u.v)
//   dihedral E = 1/2 [V1(1+cos p) + V2(1-cos 2p) + V3(1+cos 3p) + V4(1-cos 4p)]
// (Section 2).  cos(k phi), sin(k phi) come from cos phi = m.n/(|m||n|) and
// sin phi = |b2| b1.n/(|m||n|) by the multiple-angle identities.
__device__ inline double bonded_term(const Ctx &c, const double *x, int type, int term, int pos,
                              double *g, int *degenerate, int ova, const double *ov) {
    if (type == 3) {
        const double e = excl_term(c, x, term, g, ova, ov);
        if (g && pos == 1)
            for (int k = 0; k < 3; k++) g[k] = -g[k];
        return e;
    }
    if (type == 0) {
        const int2 ij = c.bidx[term];
        const double2 kp = c.bpar[term];
        double xi[3], xj[3], d[3];
        ld3(x, ij.x, xi, ova, ov);
        ld3(x, ij.y, xj, ova, ov);
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
        ld3(x, q.x, xi, ova, ov);
        ld3(x, q.y, xj, ova, ov);
        ld3(x, q.z, xk, ova, ov);
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
    ld3(x, q.x, xi, ova, ov);
    ld3(x, q.y, xj, ova, ov);
    ld3(x, q.z, xk, ova, ov);
    ld3(x, q.w, xl, ova, ov);
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

// Energy of one bonded term and its gradient for every position of the
// term (g[p] for atom p of the term), the same formulas as bonded_term.
__device__ inline double bonded_term_all(const Ctx &c, const double *x, int type, int term,
                                         double (*g)[3]) {
    if (type == 3) {
        const double e = excl_term(c, x, term, g ? g[0] : nullptr, -1, nullptr);
        if (g) for (int k = 0; k < 3; k++) g[1][k] = -g[0][k];
        return e;
    }
    if (type == 0) {
        const double e = bonded_term(c, x, 0, term, 0, g ? g[0] : nullptr, nullptr, -1, nullptr);
        if (g) for (int k = 0; k < 3; k++) g[1][k] = -g[0][k];
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
                    g[0][k] = de * dti;
                    g[2][k] = de * dtk;
                    g[1][k] = -(de * dti + de * dtk);
                }
            } else {
                for (int p = 0; p < 3; p++) g[p][0] = g[p][1] = g[p][2] = 0.0;
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
            for (int p = 0; p < 4; p++) g[p][0] = g[p][1] = g[p][2] = 0.0;
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
                g[0][k] = dedphi * pi_;
                g[1][k] = dedphi * (-(1.0 + ca) * pi_ + cc * pl);
                g[2][k] = dedphi * (ca * pi_ - (1.0 + cc) * pl);
                g[3][k] = dedphi * pl;
            }
        }
    }
    return e;
}

// global bonded-term index of (type, term) and the slot of its position
// gradients: bonds first, then angles, dihedrals, exclusion corrections
__device__ __forceinline__ int bonded_index(const Ctx &c, int type, int term) {
    return type == 0 ? term
                     : (type == 1 ? c.n_bonds + term
                                  : (type == 2 ? c.n_bonds + c.n_angles + term
                                               : c.n_bonds + c.n_angles + c.n_dihedrals + term));
}
__device__ __forceinline__ int64_t bonded_grad_slot(const Ctx &c, int type, int term, int pos) {
    return type == 0 ? 2LL * term + pos
                     : (type == 1 ? 2LL * c.n_bonds + 3LL * term + pos
                                  : (type == 2 ? 2LL * c.n_bonds + 3LL * c.n_angles + 4LL * term + pos
                                               : 2LL * c.n_bonds + 3LL * c.n_angles + 4LL * c.n_dihedrals +
                                                     2LL * term + pos));
}

// one bonded work item: every term of [t0, t0 + nt) whose system evaluates
// in precision `mode`, energies to te[], position gradients to tg[]
__device__ inline void bonded_item(const Ctx &c, int t0, int nt, int mode) {
    const double *x = vslot(c, V_XT);
    for (int t = t0 + threadIdx.x; t < t0 + nt; t += blockDim.x) {
        const SysState &S = c.st[c.term_sys[t]];
        if (S.ev_kind == EV_NONE || S.mode != mode) continue;
        int type, term;
        if (t < c.n_bonds) { type = 0; term = t; }
        else if (t < c.n_bonds + c.n_angles) { type = 1; term = t - c.n_bonds; }
        else if (t < c.n_bonds + c.n_angles + c.n_dihedrals) { type = 2; term = t - c.n_bonds - c.n_angles; }
        else { type = 3; term = t - c.n_bonds - c.n_angles - c.n_dihedrals; }
        double g[4][3];
        const bool grad = S.ev_kind == EV_EG;
        if (type == 3 && mode == 0) {  // FP32 sweeps scale the excluded pairs themselves
            c.te[t] = 0.0;
            if (grad)
                for (int p = 0; p < 2; p++)
                    for (int k = 0; k < 3; k++) c.tg[3 * bonded_grad_slot(c, 3, term, p) + k] = 0.0;
            continue;
        }
        c.te[t] = bonded_term_all(c, x, type, term, grad ? g : nullptr);
        if (grad) {
            const int np = type == 3 ? 2 : type + 2;
            double *dst = c.tg + 3 * bonded_grad_slot(c, type, term, 0);
            for (int p = 0; p < np; p++)
                for (int k = 0; k < 3; k++) dst[3 * p + k] = g[p][k];
        }
    }
}

}  // namespace ffm
