/*
 * FP64 oracle: energy and analytic gradient of the OPLS-style potential of
 * arXiv 1810.03358, Section 2 (TEST INFRASTRUCTURE ONLY, see ffmin_oracle.h).
 *
 *   E = E_stretch + E_bend + E_torsion + E_cul + E_vdw           (Section 2)
 *   E_stretch = sum_bonds K (r - r0)^2                            (no 1/2)
 *   E_bend    = sum_angles K_theta (theta - theta0)^2             (no 1/2)
 *   E_torsion = sum_dihedrals 1/2 [V1(1+cos phi) + V2(1-cos 2phi)
 *                                  + V3(1+cos 3phi) + V4(1-cos 4phi)]
 *   E_cul     = C sum_{i<j} q_i q_j / r_ij
 *   E_vdw     = 4 sum_{i<j} sqrt(eps_i eps_j) [(s/r)^12 - (s/r)^6],
 *               s = sqrt(sigma_i sigma_j)
 * Pairs run over ALL i < j: the paper's non-bonded forces act regardless of
 * whether a bond joins the atoms, so there is no exclusion list.  With
 * ff->exclusions (a force-field variant outside the paper) each pair term is
 * multiplied by s_ij: 0 for atoms joined by a bond or the ends of an angle,
 * scale14 for the ends of a dihedral (when not excluded), else 1.
 * Gradients are the explicit formulas (Section 2 prefers them to autodiff).
 */
#include "ffmin_oracle.h"

#include <math.h>
#include <stddef.h>
#include <stdlib.h>

static void sub3(const double *a, const double *b, double *o) {
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ---- the scale s_ij of the pair (i, j) ---- */
typedef struct {
    int64_t key; /* min(i,j) * N + max(i,j) */
    double s;
} pscale_t;

static int cmp_pscale(const void *a, const void *b) {
    const pscale_t *x = (const pscale_t *)a, *y = (const pscale_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);
}

static int64_t pkey(const orc_ff *ff, int32_t i, int32_t j) {
    return i < j ? (int64_t)i * ff->n_atoms + j : (int64_t)j * ff->n_atoms + i;
}

/* Sorted table of the scaled pairs (smallest scale first among duplicates),
 * or NULL when every pair has scale 1.  *m = entries. */
static pscale_t *scale_table(const orc_ff *ff, int32_t *m) {
    *m = 0;
    if (!ff->exclusions) return NULL;
    int32_t cap = ff->n_bonds + ff->n_angles + ff->n_dihedrals;
    pscale_t *t = (pscale_t *)malloc(sizeof(pscale_t) * (size_t)(cap > 0 ? cap : 1));
    int32_t k = 0;
    for (int32_t b = 0; b < ff->n_bonds; b++) {
        t[k].key = pkey(ff, ff->bond_idx[2 * b], ff->bond_idx[2 * b + 1]);
        t[k++].s = 0.0;
    }
    for (int32_t b = 0; b < ff->n_angles; b++) {
        t[k].key = pkey(ff, ff->angle_idx[3 * b], ff->angle_idx[3 * b + 2]);
        t[k++].s = 0.0;
    }
    for (int32_t b = 0; b < ff->n_dihedrals; b++) {
        t[k].key = pkey(ff, ff->dihedral_idx[4 * b], ff->dihedral_idx[4 * b + 3]);
        t[k++].s = ff->scale14;
    }
    qsort(t, (size_t)k, sizeof(pscale_t), cmp_pscale);
    *m = k;
    return t;
}

/* s_ij: the first (smallest) entry of the pair's key, else 1 */
static double pair_scale(const orc_ff *ff, const pscale_t *t, int32_t m, int32_t i, int32_t j) {
    if (!t) return 1.0;
    const int64_t key = pkey(ff, i, j);
    int32_t lo = 0, hi = m;
    while (lo < hi) {
        int32_t mid = (lo + hi) / 2;
        if (t[mid].key < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < m && t[lo].key == key) ? t[lo].s : 1.0;
}

/* Pair term between atoms with the given parameters at separation vector
 * d = x_i - x_j.  Returns E_cul + E_vdw of the pair; *ec, *ev the parts;
 * *dedr_over_r = (dE/dr)/r so that grad_i = dedr_over_r * d. */
static double pair_term(double c, double qi, double qj, double si, double sj,
                        double ei, double ej, const double *d,
                        double *ec, double *ev, double *dedr_over_r) {
    double r2 = dot3(d, d);
    double r = sqrt(r2);
    double sij = sqrt(si * sj);
    double eij = sqrt(ei * ej);
    double sr = sij / r;
    double sr6 = pow(sr, 6.0);
    double sr12 = sr6 * sr6;
    *ec = c * qi * qj / r;
    *ev = 4.0 * eij * (sr12 - sr6);
    /* dE_cul/dr = -C qi qj / r^2 ; dE_vdw/dr = 4 eps (-12 sr^12 + 6 sr^6) / r */
    double dcul = -(*ec) / r;
    double dvdw = 4.0 * eij * (-12.0 * sr12 + 6.0 * sr6) / r;
    *dedr_over_r = (dcul + dvdw) / r;
    return *ec + *ev;
}

/* Bond i-j: E = K (r - r0)^2; grad_i = 2K (r - r0) (x_i - x_j)/r. */
static double bond_term(const double *xi, const double *xj, double k, double r0,
                        double *gi, double *gj) {
    double d[3];
    sub3(xi, xj, d);
    double r = sqrt(dot3(d, d));
    double e = k * (r - r0) * (r - r0);
    if (gi) {
        double f = 2.0 * k * (r - r0) / r;
        for (int a = 0; a < 3; a++) { gi[a] = f * d[a]; gj[a] = -f * d[a]; }
    }
    return e;
}

/* Angle i-j-k (vertex j): theta = atan2(|u x v|, u.v), u = x_i - x_j,
 * v = x_k - x_j; E = K (theta - theta0)^2.
 * d theta/d x_i = [(u.v) u/|u|^2 - v] / |u x v|, likewise for x_k with u, v
 * swapped; d theta/d x_j = -(d/dx_i + d/dx_k).  At |u x v| = 0 the angle is
 * not differentiable; the gradient contribution is then taken as zero. */
static double angle_term(const double *xi, const double *xj, const double *xk,
                         double kth, double th0, double *gi, double *gj, double *gk) {
    double u[3], v[3], w[3];
    sub3(xi, xj, u);
    sub3(xk, xj, v);
    cross3(u, v, w);
    double cr = sqrt(dot3(w, w));
    double uv = dot3(u, v);
    double th = atan2(cr, uv);
    double e = kth * (th - th0) * (th - th0);
    if (gi) {
        if (cr > 0.0) {
            double de = 2.0 * kth * (th - th0);
            double uu = dot3(u, u), vv = dot3(v, v);
            for (int a = 0; a < 3; a++) {
                double dti = (uv * u[a] / uu - v[a]) / cr;
                double dtk = (uv * v[a] / vv - u[a]) / cr;
                gi[a] = de * dti;
                gk[a] = de * dtk;
                gj[a] = -(gi[a] + gk[a]);
            }
        } else {
            for (int a = 0; a < 3; a++) { gi[a] = 0.0; gj[a] = 0.0; gk[a] = 0.0; }
        }
    }
    return e;
}

/* Dihedral i-j-k-l: b1 = x_j - x_i, b2 = x_k - x_j, b3 = x_l - x_k,
 * m = b1 x b2, n = b2 x b3, phi = atan2(|b2| b1.n, m.n) (cis = 0,
 * trans = pi).  E = 1/2 [V1(1+cos phi) + V2(1-cos 2phi) + V3(1+cos 3phi)
 * + V4(1-cos 4phi)].  Gradient of phi (Blondel & Karplus 1996):
 *   dphi/dx_i = -|b2|/|m|^2 m,  dphi/dx_l = |b2|/|n|^2 n,
 *   dphi/dx_j = -(1 + a) dphi/dx_i + c dphi/dx_l,
 *   dphi/dx_k = a dphi/dx_i - (1 + c) dphi/dx_l,
 * with a = b1.b2/|b2|^2 and c = b3.b2/|b2|^2.  When |m|^2 or |n|^2 falls
 * below 1e-12 A^4 (collinear atoms) phi is taken from atan2 as is and the
 * gradient contribution is zero. */
static double dihedral_term(const double *xi, const double *xj, const double *xk,
                            const double *xl, const double *v, double *gi, double *gj,
                            double *gk, double *gl, int *degenerate) {
    double b1[3], b2[3], b3[3], m[3], n[3];
    sub3(xj, xi, b1);
    sub3(xk, xj, b2);
    sub3(xl, xk, b3);
    cross3(b1, b2, m);
    cross3(b2, b3, n);
    double mm = dot3(m, m), nn = dot3(n, n), b2n = sqrt(dot3(b2, b2));
    double phi = atan2(b2n * dot3(b1, n), dot3(m, n));
    double e = 0.5 * (v[0] * (1.0 + cos(phi)) + v[1] * (1.0 - cos(2.0 * phi)) +
                      v[2] * (1.0 + cos(3.0 * phi)) + v[3] * (1.0 - cos(4.0 * phi)));
    int deg = (mm < 1e-12 || nn < 1e-12);
    if (degenerate) *degenerate = deg;
    if (gi) {
        if (deg) {
            for (int a = 0; a < 3; a++) { gi[a] = gj[a] = gk[a] = gl[a] = 0.0; }
        } else {
            double dedphi = 0.5 * (-v[0] * sin(phi) + 2.0 * v[1] * sin(2.0 * phi) -
                                   3.0 * v[2] * sin(3.0 * phi) + 4.0 * v[3] * sin(4.0 * phi));
            double bb = b2n * b2n;
            double ca = dot3(b1, b2) / bb, cc = dot3(b3, b2) / bb;
            for (int a = 0; a < 3; a++) {
                double pi_ = -b2n / mm * m[a];
                double pl = b2n / nn * n[a];
                double pj = -(1.0 + ca) * pi_ + cc * pl;
                double pk = ca * pi_ - (1.0 + cc) * pl;
                gi[a] = dedphi * pi_;
                gj[a] = dedphi * pj;
                gk[a] = dedphi * pk;
                gl[a] = dedphi * pl;
            }
        }
    }
    return e;
}

/* The bonded terms (stretch, bend, torsion of Section 2) added into *t and,
 * when grad != NULL, their gradient into grad. */
static void add_bonded(const orc_ff *ff, const double *x, double *grad, orc_terms *tp) {
    orc_terms t = *tp;
    /* bonds */
    for (int b = 0; b < ff->n_bonds; b++) {
        int i = ff->bond_idx[2 * b], j = ff->bond_idx[2 * b + 1];
        double gi[3] = {0.0}, gj[3] = {0.0};
        double e = bond_term(x + 3 * i, x + 3 * j, ff->bond_k[b], ff->bond_r0[b],
                             grad ? gi : NULL, gj);
        t.stretch += e;
        t.sum_abs += fabs(e);
        if (grad)
            for (int a = 0; a < 3; a++) { grad[3 * i + a] += gi[a]; grad[3 * j + a] += gj[a]; }
    }
    /* angles */
    for (int b = 0; b < ff->n_angles; b++) {
        int i = ff->angle_idx[3 * b], j = ff->angle_idx[3 * b + 1], k = ff->angle_idx[3 * b + 2];
        double gi[3] = {0.0}, gj[3] = {0.0}, gk[3] = {0.0};
        double e = angle_term(x + 3 * i, x + 3 * j, x + 3 * k, ff->angle_k[b],
                              ff->angle_theta0[b], grad ? gi : NULL, gj, gk);
        t.bend += e;
        t.sum_abs += fabs(e);
        if (grad)
            for (int a = 0; a < 3; a++) {
                grad[3 * i + a] += gi[a]; grad[3 * j + a] += gj[a]; grad[3 * k + a] += gk[a];
            }
    }
    /* dihedrals */
    for (int b = 0; b < ff->n_dihedrals; b++) {
        const int32_t *q = ff->dihedral_idx + 4 * b;
        double gi[3] = {0.0}, gj[3] = {0.0}, gk[3] = {0.0}, gl[3] = {0.0};
        int deg = 0;
        double e = dihedral_term(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3],
                                 ff->dihedral_v + 4 * b, grad ? gi : NULL, gj, gk, gl, &deg);
        t.torsion += e;
        t.sum_abs += fabs(e);
        t.degenerate_dihedrals += deg;
        if (grad)
            for (int a = 0; a < 3; a++) {
                grad[3 * q[0] + a] += gi[a]; grad[3 * q[1] + a] += gj[a];
                grad[3 * q[2] + a] += gk[a]; grad[3 * q[3] + a] += gl[a];
            }
    }
    *tp = t;
}

int orc_energy_terms(const orc_ff *ff, const double *x, double *grad, orc_terms *out) {
    const int n = ff->n_atoms;
    orc_terms t = {0};
    int status = ORC_OK;
    if (grad)
        for (int k = 0; k < 3 * n; k++) grad[k] = 0.0;

    /* non-bonded: every unordered pair i < j, times its scale s_ij */
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            sub3(x + 3 * i, x + 3 * j, d);
            if (dot3(d, d) == 0.0) { status = ORC_NONFINITE; continue; }
            const double s = pair_scale(ff, sc, m_sc, i, j);
            if (s == 0.0) continue;
            double ec, ev, f;
            pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                      ff->epsilon[i], ff->epsilon[j], d, &ec, &ev, &f);
            ec *= s;
            ev *= s;
            f *= s;
            t.coulomb += ec;
            t.vdw += ev;
            t.sum_abs += fabs(ec) + fabs(ev);
            if (grad) {
                for (int a = 0; a < 3; a++) {
                    grad[3 * i + a] += f * d[a];
                    grad[3 * j + a] -= f * d[a];
                }
            }
        }
    }
    free(sc);
    add_bonded(ff, x, grad, &t);
    t.total = t.stretch + t.bend + t.torsion + t.coulomb + t.vdw;
    if (!isfinite(t.total)) status = ORC_NONFINITE;
    if (grad)
        for (int k = 0; k < 3 * n; k++)
            if (!isfinite(grad[k])) status = ORC_NONFINITE;
    if (out) *out = t;
    return status;
}

/* orc_energy_terms restricted to the pairs (i, j), i < j, with i in [i0, i1),
 * plus the bonded terms when i0 == 0: the energies of these terms (sum_abs
 * and the parts as in orc_terms) and their gradient added into grad [3N]
 * (rows of both atoms of a pair).  Summing the blocks of a partition of
 * [0, N) gives the whole energy and gradient (in another order). */
int orc_energy_rows(const orc_ff *ff, const double *x, int32_t i0, int32_t i1, double *grad,
                    orc_terms *out) {
    const int n = ff->n_atoms;
    orc_terms t = {0};
    int status = ORC_OK;
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    if (i0 < 0) i0 = 0;
    if (i1 > n) i1 = n;
    for (int i = i0; i < i1; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            sub3(x + 3 * i, x + 3 * j, d);
            if (dot3(d, d) == 0.0) { status = ORC_NONFINITE; continue; }
            const double s = pair_scale(ff, sc, m_sc, i, j);
            if (s == 0.0) continue;
            double ec, ev, f;
            pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                      ff->epsilon[i], ff->epsilon[j], d, &ec, &ev, &f);
            ec *= s;
            ev *= s;
            f *= s;
            t.coulomb += ec;
            t.vdw += ev;
            t.sum_abs += fabs(ec) + fabs(ev);
            if (grad) {
                for (int a = 0; a < 3; a++) {
                    grad[3 * i + a] += f * d[a];
                    grad[3 * j + a] -= f * d[a];
                }
            }
        }
    }
    free(sc);
    if (i0 == 0) add_bonded(ff, x, grad, &t);
    t.total = t.stretch + t.bend + t.torsion + t.coulomb + t.vdw;
    if (!isfinite(t.total)) status = ORC_NONFINITE;
    if (out) *out = t;
    return status;
}

/* E(xp) - E(x) as a sum of per-term differences (every Section 2 term at
 * xp minus the same term at x), with the sum of |difference| over the terms.
 * Pairs (i, j), i < j, with i in [i0, i1) (so that independent callers can
 * split the rows); the bonded terms only when i0 == 0. */
int orc_energy_delta(const orc_ff *ff, const double *x, const double *xp, int32_t i0, int32_t i1,
                     double *delta, double *sum_abs) {
    const int n = ff->n_atoms;
    int status = ORC_OK;
    double dsum = 0.0, asum = 0.0;
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    if (i0 < 0) i0 = 0;
    if (i1 > n) i1 = n;
    for (int i = i0; i < i1; i++) {
        for (int j = i + 1; j < n; j++) {
            double d0[3], d1[3];
            sub3(x + 3 * i, x + 3 * j, d0);
            sub3(xp + 3 * i, xp + 3 * j, d1);
            if (dot3(d0, d0) == 0.0 || dot3(d1, d1) == 0.0) { status = ORC_NONFINITE; continue; }
            const double s = pair_scale(ff, sc, m_sc, i, j);
            if (s == 0.0) continue;
            double ec, ev, f;
            const double e0 = pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i],
                                        ff->sigma[j], ff->epsilon[i], ff->epsilon[j], d0, &ec, &ev, &f);
            const double e1 = pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i],
                                        ff->sigma[j], ff->epsilon[i], ff->epsilon[j], d1, &ec, &ev, &f);
            const double de = s * (e1 - e0);
            dsum += de;
            asum += fabs(de);
        }
    }
    free(sc);
    if (i0 == 0) {
        for (int b = 0; b < ff->n_bonds; b++) {
            int i = ff->bond_idx[2 * b], j = ff->bond_idx[2 * b + 1];
            const double de = bond_term(xp + 3 * i, xp + 3 * j, ff->bond_k[b], ff->bond_r0[b], NULL, NULL) -
                              bond_term(x + 3 * i, x + 3 * j, ff->bond_k[b], ff->bond_r0[b], NULL, NULL);
            dsum += de;
            asum += fabs(de);
        }
        for (int b = 0; b < ff->n_angles; b++) {
            const int32_t *q = ff->angle_idx + 3 * b;
            const double de =
                angle_term(xp + 3 * q[0], xp + 3 * q[1], xp + 3 * q[2], ff->angle_k[b], ff->angle_theta0[b],
                           NULL, NULL, NULL) -
                angle_term(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], ff->angle_k[b], ff->angle_theta0[b],
                           NULL, NULL, NULL);
            dsum += de;
            asum += fabs(de);
        }
        for (int b = 0; b < ff->n_dihedrals; b++) {
            const int32_t *q = ff->dihedral_idx + 4 * b;
            const double *v = ff->dihedral_v + 4 * b;
            const double de =
                dihedral_term(xp + 3 * q[0], xp + 3 * q[1], xp + 3 * q[2], xp + 3 * q[3], v, NULL, NULL, NULL,
                              NULL, NULL) -
                dihedral_term(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3], v, NULL, NULL, NULL,
                              NULL, NULL);
            dsum += de;
            asum += fabs(de);
        }
    }
    if (!isfinite(dsum)) status = ORC_NONFINITE;
    *delta = dsum;
    *sum_abs = asum;
    return status;
}

/* Part of E that depends on atom i, with atom i at p. */
/* e plus every bonded term containing atom i, with atom i at p, added one
 * at a time (bonds, angles, dihedrals) */
static double add_row_bonded(const orc_ff *ff, const double *x, int32_t i, const double p[3], double e) {
#define POS(a) ((a) == i ? p : x + 3 * (a))
    for (int b = 0; b < ff->n_bonds; b++) {
        int a0 = ff->bond_idx[2 * b], a1 = ff->bond_idx[2 * b + 1];
        if (a0 != i && a1 != i) continue;
        e += bond_term(POS(a0), POS(a1), ff->bond_k[b], ff->bond_r0[b], NULL, NULL);
    }
    for (int b = 0; b < ff->n_angles; b++) {
        const int32_t *q = ff->angle_idx + 3 * b;
        if (q[0] != i && q[1] != i && q[2] != i) continue;
        e += angle_term(POS(q[0]), POS(q[1]), POS(q[2]), ff->angle_k[b], ff->angle_theta0[b],
                        NULL, NULL, NULL);
    }
    for (int b = 0; b < ff->n_dihedrals; b++) {
        const int32_t *q = ff->dihedral_idx + 4 * b;
        if (q[0] != i && q[1] != i && q[2] != i && q[3] != i) continue;
        e += dihedral_term(POS(q[0]), POS(q[1]), POS(q[2]), POS(q[3]), ff->dihedral_v + 4 * b,
                           NULL, NULL, NULL, NULL, NULL);
    }
#undef POS
    return e;
}

double orc_row_energy(const orc_ff *ff, const double *x, int32_t i, const double p[3]) {
    const int n = ff->n_atoms;
    double e = 0.0;
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    for (int j = 0; j < n; j++) {
        if (j == i) continue;
        const double s = pair_scale(ff, sc, m_sc, i, j);
        if (s == 0.0) continue;
        double d[3], ec, ev, f;
        sub3(p, x + 3 * j, d);
        e += s * pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                           ff->epsilon[i], ff->epsilon[j], d, &ec, &ev, &f);
    }
    free(sc);
    return add_row_bonded(ff, x, i, p, e);
}

/* The row energy with the far Coulomb terms linearised (Section 3's
 * construction for the gradient-free moves): for every atom j at least r_far
 * from the atom's current position x_i, the Coulomb term at p is replaced by
 * its first-order Taylor expansion about x_i,
 *     e_c(x_i) + grad_i e_c(x_i) . (p - x_i) = e_c0 (1 - d0 . (p - x_i) / r0^2),
 * d0 = x_i - x_j, r0 = |d0|; the Lennard-Jones terms, the near Coulomb terms
 * and the bonded terms stay exact.  r_far = +inf gives orc_row_energy. */
double orc_row_energy_taylor(const orc_ff *ff, const double *x, int32_t i, const double p[3],
                             double r_far) {
    const int n = ff->n_atoms;
    double e = 0.0, delta[3];
    sub3(p, x + 3 * i, delta);
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    for (int j = 0; j < n; j++) {
        if (j == i) continue;
        const double s = pair_scale(ff, sc, m_sc, i, j);
        if (s == 0.0) continue;
        double d0[3], ec, ev, f;
        sub3(x + 3 * i, x + 3 * j, d0);
        const double r02 = dot3(d0, d0);
        if (r02 >= r_far * r_far) {
            double d[3], ec_p;
            sub3(p, x + 3 * j, d);
            pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                      ff->epsilon[i], ff->epsilon[j], d, &ec_p, &ev, &f);
            pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                      ff->epsilon[i], ff->epsilon[j], d0, &ec, &f, &f);
            e += s * (ev + ec * (1.0 - dot3(d0, delta) / r02));
        } else {
            double d[3];
            sub3(p, x + 3 * j, d);
            e += s * pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                               ff->epsilon[i], ff->epsilon[j], d, &ec, &ev, &f);
        }
    }
    free(sc);
    return add_row_bonded(ff, x, i, p, e);
}

int32_t orc_neighbour_count(const orc_ff *ff, const double *x, int32_t i, double rc) {
    int32_t c = 0;
    for (int j = 0; j < ff->n_atoms; j++) {
        if (j == i) continue;
        double d[3];
        sub3(x + 3 * i, x + 3 * j, d);
        if (dot3(d, d) < rc * rc) c++;
    }
    return c;
}

/* Gradient of E with respect to the position of atom i only (g3[3]): the
 * pair terms of row i plus every bonded term containing i. */
int orc_atom_gradient(const orc_ff *ff, const double *x, int32_t i, double *g3) {
    int status = ORC_OK;
    g3[0] = g3[1] = g3[2] = 0.0;
    int32_t m_sc;
    pscale_t *sc = scale_table(ff, &m_sc);
    for (int j = 0; j < ff->n_atoms; j++) {
        if (j == i) continue;
        double d[3], ec, ev, f;
        sub3(x + 3 * i, x + 3 * j, d);
        if (dot3(d, d) == 0.0) { status = ORC_NONFINITE; continue; }
        const double s = pair_scale(ff, sc, m_sc, i, j);
        if (s == 0.0) continue;
        pair_term(ff->coulomb_c, ff->charge[i], ff->charge[j], ff->sigma[i], ff->sigma[j],
                  ff->epsilon[i], ff->epsilon[j], d, &ec, &ev, &f);
        for (int a = 0; a < 3; a++) g3[a] += s * f * d[a];
    }
    free(sc);
    for (int b = 0; b < ff->n_bonds; b++) {
        const int32_t *q = ff->bond_idx + 2 * b;
        if (q[0] != i && q[1] != i) continue;
        double g[2][3];
        bond_term(x + 3 * q[0], x + 3 * q[1], ff->bond_k[b], ff->bond_r0[b], g[0], g[1]);
        for (int p = 0; p < 2; p++)
            if (q[p] == i) for (int a = 0; a < 3; a++) g3[a] += g[p][a];
    }
    for (int b = 0; b < ff->n_angles; b++) {
        const int32_t *q = ff->angle_idx + 3 * b;
        if (q[0] != i && q[1] != i && q[2] != i) continue;
        double g[3][3];
        angle_term(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], ff->angle_k[b], ff->angle_theta0[b],
                   g[0], g[1], g[2]);
        for (int p = 0; p < 3; p++)
            if (q[p] == i) for (int a = 0; a < 3; a++) g3[a] += g[p][a];
    }
    for (int b = 0; b < ff->n_dihedrals; b++) {
        const int32_t *q = ff->dihedral_idx + 4 * b;
        if (q[0] != i && q[1] != i && q[2] != i && q[3] != i) continue;
        double g[4][3];
        dihedral_term(x + 3 * q[0], x + 3 * q[1], x + 3 * q[2], x + 3 * q[3],
                      ff->dihedral_v + 4 * b, g[0], g[1], g[2], g[3], NULL);
        for (int p = 0; p < 4; p++)
            if (q[p] == i) for (int a = 0; a < 3; a++) g3[a] += g[p][a];
    }
    return status;
}
