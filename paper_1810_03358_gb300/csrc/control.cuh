// Per-system control state machine of the minimizers, run on the device by
// one thread per system in the last block of the per-tile kernels.
//
// One "tick" of the device pipeline is
//     update -> direction 1 -> direction 2 -> prepare -> pair -> finalize
// and evaluates at most one energy (E) or energy+gradient (EG) per system.
// After each stage the machine consumes that stage's reductions and writes
// the requests of the following stages, so a whole minimization runs as one
// graph launch of repeated ticks with no host round trip per evaluation.
//
// The machine restates, step for step, Algorithms 1-6 of arXiv 1810.03358
// (Sections 5.1-5.2) and the adaptive gradient descent of Section 3 (Eq. 4),
// with these readings where the paper is silent: normalised directions,
// warm-started steps, one restart after a failed line search, skipped
// L-BFGS pairs with <s, y> <= 0; FGM's function-value momentum restart is
// an option (Algorithm 1 itself has none).  The L-BFGS two-loop recursion (Algorithm 3) is evaluated from
// maintained inner products <s_a, y_b> and <s_a, g> (same alpha and beta as
// the vector recursion) so that it costs two vector passes instead of 2m.
#pragma once

#include "ffmin_internal.cuh"

namespace ffm {

__device__ __forceinline__ double finite_or_inf(double f) { return isfinite(f) ? f : HUGE_VAL; }

__device__ __forceinline__ bool cap_hit(const SysState &S) {
    return S.iter >= S.max_iter || S.ne + S.neg >= S.max_evals;
}

__device__ __forceinline__ void deactivate(const Ctx &c, SysState &S) {
    if (S.active) {
        S.active = 0;
        atomicSub(c.nactive, 1);
        atomicSub(&c.nmode[S.mode], 1);
    }
}

__device__ __forceinline__ void set_eval(SysState &S, int kind, int base, int dir, double h,
                                         double scale) {
    // an FP32 energy-only trial along a direction is taken as a difference
    S.ev_delta = (S.mode == 0 && kind == EV_E && dir >= 0) ? 1 : 0;
    S.ev_kind = kind;
    S.ev_base = base;
    S.ev_dir = dir;
    S.ev_h = h;
    S.ev_scale = scale;
}

__device__ __forceinline__ void set_dir(SysState &S, int which, double a, double b, double outer,
                                        int dots) {
    DirOp &d = S.dir[which];
    d.on = 1;
    d.use_d = 0;
    d.dots = dots;
    d.nS = 0;
    d.nY = 0;
    d.a = a;
    d.b = b;
    d.outer = outer;
}

// finish: the system stops after the pending update op (if any) has run.
// A MIXED run still in its FP32 phase does not stop: a converged or stalled
// FP32 phase hands over to the FP64 phase, which re-evaluates the current
// point (FGM: the best point) with FP64 pair terms and continues the same
// method from there until the FP64 gradient meets the tolerance; an
// iteration cap ends the run where it is (energies then come from the FP32
// pair terms).
__device__ void finish(const Ctx &c, SysState &S, int status, double res_f, double res_ginf) {
    if (S.mixed && S.mode == 0 && S.phase != PH_EVAL_ONLY &&
        (status == FFMIN_OK || status == FFMIN_ERR_LINESEARCH)) {
        S.mode = 1;
        S.iter_fp64_0 = S.iter;
        atomicSub(&c.nmode[0], 1);
        atomicAdd(&c.nmode[1], 1);
        S.dir[0].on = 0;
        S.dir[1].on = 0;
        const int base = S.method == FFMIN_FGM ? V_XB : V_X;
        set_eval(S, EV_EG, base, -1, 0.0, 1.0);
        S.ring_count = 0;
        S.phase = PH_START;
        return;
    }
    S.status = status;
    S.phase = PH_DONE;
    S.ev_kind = EV_NONE;
    S.dir[0].on = 0;
    S.dir[1].on = 0;
    S.res_f = res_f;
    S.res_ginf = res_ginf;
    if (S.upd.op == U_NONE) deactivate(c, S);
}

// ---------------- line searches ----------------
// LS_H (Algorithm 5) and LS_PAR (Algorithm 6) as resumable machines: start
// returns the first trial step; feed consumes phi(trial) and either returns
// the next trial (done = 0) or the result (done = 1, h = 0 on failure).
struct LsOut {
    int done;
    double h, f;
};

__device__ double ls_start(SysState &S, double h0) {
    S.ls_h0v = h0;
    if (S.ls_kind == FFMIN_LS_H) {
        S.ls_step = 0;
        return h0;
    }
    S.lh[0] = 0.0;
    S.lf[0] = S.fstar;
    if (S.g0) {
        S.lh[1] = h0;
        S.ls_step = 1;
    } else {
        S.lh[1] = -0.5 * h0;
        S.ls_step = 11;
    }
    return S.lh[1];
}

__device__ __forceinline__ bool point_less(double ha, double fa, double hb, double fb) {
    if (fa < fb) return true;
    if (fa > fb) return false;
    return fabs(ha) < fabs(hb);
}

__device__ void sort_points(double *h, double *f, int n) {
    for (int a = 1; a < n; a++) {
        double hh = h[a], ff = f[a];
        int b = a - 1;
        while (b >= 0 && point_less(hh, ff, h[b], f[b])) {
            h[b + 1] = h[b];
            f[b + 1] = f[b];
            b--;
        }
        h[b + 1] = hh;
        f[b + 1] = ff;
    }
}

// vertex of the parabola through three points, Newton form
__device__ bool parabola3(const double *h, const double *f, double *vertex) {
    double d1 = (f[1] - f[0]) / (h[1] - h[0]);
    double d2 = (f[2] - f[1]) / (h[2] - h[1]);
    double A = (d2 - d1) / (h[2] - h[0]);
    if (!(A > 0.0) || !isfinite(A)) return false;
    double v = 0.5 * (h[0] + h[1]) - d1 / (2.0 * A);
    if (!isfinite(v)) return false;
    *vertex = v;
    return true;
}

__device__ LsOut ls_par_next(SysState &S) {
    LsOut o;
    if (S.ls_k <= S.K) {
        double v;
        double hmax = fmax(fabs(S.lh[0]), fmax(fabs(S.lh[1]), fabs(S.lh[2])));
        if (!parabola3(S.lh, S.lf, &v)) {
            int ib = 0;
            for (int a = 1; a < 3; a++)
                if (point_less(S.lh[a], S.lf[a], S.lh[ib], S.lf[ib])) ib = a;
            if (S.lh[ib] != 0.0) {
                v = S.kplus * S.lh[ib];
            } else {
                int ic = -1;
                for (int a = 0; a < 3; a++)
                    if (S.lh[a] != 0.0 && (ic < 0 || fabs(S.lh[a]) < fabs(S.lh[ic]))) ic = a;
                v = ic >= 0 ? 0.5 * S.lh[ic] : S.ls_h0v;
            }
        }
        if (fabs(v) > 8.0 * hmax) v = copysign(8.0 * hmax, v);
        S.lh[3] = v;
        S.ls_step = 3;
        o.done = 0;
        o.h = v;
        o.f = 0.0;
        return o;
    }
    if (S.K == 2) sort_points(S.lh, S.lf, 3);
    o.done = 1;
    if (S.lf[0] < S.fstar) {
        o.h = S.lh[0];
        o.f = S.lf[0];
    } else {
        o.h = 0.0;
        o.f = S.fstar;
    }
    return o;
}

__device__ LsOut ls_feed(SysState &S, double f) {
    LsOut o;
    o.done = 0;
    o.f = 0.0;
    if (S.ls_kind == FFMIN_LS_H) {
        if (S.ls_step == 0) {
            S.ls_f0 = f;
            if (f < S.fstar) {
                S.lh[1] = S.kplus * S.ls_h0v;
                S.ls_step = 1;
                o.h = S.lh[1];
            } else {
                S.lh[2] = S.kminus * S.ls_h0v;
                S.ls_step = 2;
                o.h = S.lh[2];
            }
            return o;
        }
        if (S.ls_step == 1) {
            o.done = 1;
            if (f < S.ls_f0) {
                o.h = S.lh[1];
                o.f = f;
            } else {
                o.h = S.ls_h0v;
                o.f = S.ls_f0;
            }
            return o;
        }
        // step 2: shrinking loop
        if (f > S.fstar) {
            S.lh[2] = S.kminus * S.lh[2];
            if (S.lh[2] <= S.eps_h) {
                o.done = 1;
                o.h = 0.0;
                o.f = S.fstar;
                return o;
            }
            o.h = S.lh[2];
            return o;
        }
        o.done = 1;
        o.h = S.lh[2];
        o.f = f;
        return o;
    }
    // LS_PAR
    switch (S.ls_step) {
    case 1: {  // G0: parabola through f(0), f'(0) and (h1, f1)
        S.lf[1] = f;
        double a = (S.lf[1] - S.fstar - S.slope * S.lh[1]) / (S.lh[1] * S.lh[1]);
        double v = -S.slope / (2.0 * a);
        S.lh[2] = (a > 0.0 && isfinite(a) && isfinite(v)) ? v : S.kplus * S.lh[1];
        S.ls_step = 2;
        o.h = S.lh[2];
        return o;
    }
    case 11:
        S.lf[1] = f;
        S.lh[2] = 0.5 * S.ls_h0v;
        S.ls_step = 2;
        o.h = S.lh[2];
        return o;
    case 2:
        S.lf[2] = f;
        S.ls_k = 2;
        return ls_par_next(S);
    default:  // 3
        S.lf[3] = f;
        sort_points(S.lh, S.lf, 4);
        S.ls_k++;
        return ls_par_next(S);
    }
}

// ---------------- minimizer steps ----------------
__device__ void fgm_finish(const Ctx &c, SysState &S, int status);

// FP32 phase of a MIXED run: true when the run should hand over to FP64
// after an accepted point with FP32 |grad|_inf ginf
__device__ bool mixed_handover(const SysState &S, double f, double ginf) {
    (void)f;
    return S.mixed && S.mode == 0 && ginf < MIXED_SWITCH_RATIO * S.gtol;
}

__device__ void lbfgs_pass1(SysState &S, int use_d);

__device__ void ls_begin(const Ctx &c, SysState &S, double rr, double gr) {
    if (S.method == FFMIN_LBFGS && S.dir_used_d && !(gr < 0.0)) {
        // the learned diagonal gave no descent direction: plain L-BFGS for
        // this iteration (the next iteration runs both direction passes again)
        lbfgs_pass1(S, 0);
        return;
    }
    S.dir_used_d = 0;
    if (cap_hit(S)) {
        if (S.method == FFMIN_FGM) fgm_finish(c, S, FFMIN_ERR_MAX_ITER);
        else finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
        return;
    }
    S.rnorm = sqrt(rr);
    const double inv = 1.0 / S.rnorm;
    S.rg = gr;
    S.slope = gr * inv;
    int ls = S.ls;
    if (ls == FFMIN_LS_DEFAULT) ls = (S.method == FFMIN_FGM) ? FFMIN_LS_H : FFMIN_LS_PAR;
    S.ls_kind = ls;
    const bool fgm = S.method == FFMIN_FGM;
    S.fstar = fgm ? S.fw : S.f;
    S.epair_base = S.epair_last;  // the last E + grad evaluation was at the base
    const double h = ls_start(S, S.h0);
    set_eval(S, EV_E, fgm ? V_W : V_X, V_R, h, inv);
    S.phase = PH_LS;
}

__device__ void fgm_finish(const Ctx &c, SysState &S, int status) {
    S.result_slot = V_XB;
    if (S.xb_known || status == FFMIN_ERR_NONFINITE) {
        finish(c, S, status, S.fb, S.xb_ginf);
        return;
    }
    // report the gradient of the returned point: one more evaluation
    S.status = status;
    S.dir[0].on = 0;
    S.dir[1].on = 0;
    set_eval(S, EV_EG, V_XB, -1, 0.0, 1.0);
    S.phase = PH_FINAL;
}

__device__ void fgm_on_w(const Ctx &c, SysState &S, double e, double ginf) {
    S.fw = e;
    if (ginf < S.gtol || mixed_handover(S, e, ginf)) {
        if (e < S.fb) {
            S.upd.best = 1;
            S.fb = e;
            S.xb_ginf = ginf;
            S.xb_known = 1;
        }
        fgm_finish(c, S, FFMIN_OK);
        return;
    }
    if (cap_hit(S)) {
        fgm_finish(c, S, FFMIN_ERR_MAX_ITER);
        return;
    }
    set_dir(S, 1, -1.0, 0.0, 1.0, 1);
    S.phase = PH_DIR;
}

__device__ __forceinline__ double fgm_theta(double tp) {
    return 0.5 * tp * (sqrt(tp * tp + 4.0) - tp);
}

__device__ void fgm_next_w(SysState &S) {
    const double th = fgm_theta(S.th_prev);
    const double beta = S.th_prev * (1.0 - S.th_prev) / (S.th_prev * S.th_prev + th);
    set_eval(S, EV_EG, V_X, V_P, beta, 1.0);
    S.phase = PH_FGM_W;
}

__device__ void fgm_accept(SysState &S, double h, double fnew) {
    const double th = fgm_theta(S.th_prev);
    // Algorithm 1 keeps its momentum (and the best point); the optional
    // function-value restart drops it when the new iterate is worse
    const int restart = S.fgm_restart && fnew > S.fx;
    const int best = fnew < S.fb;
    S.upd.op = U_FGM_ACCEPT;
    S.upd.h = h;
    S.upd.inv = S.ev_scale;
    S.upd.restart = restart;
    S.upd.best = best;
    S.th_prev = restart ? 1.0 : th;
    S.fx = fnew;
    S.h0 = h;
    S.iter++;
    if (best) {
        S.fb = fnew;
        S.xb_known = 0;
    }
    fgm_next_w(S);
}

__device__ double cg_beta(int variant, double gpgp, double gpg, double gpd, double gg, double dg) {
    const double gpy = gpgp - gpg;  // <g+, g+ - g>
    const double dy = gpd - dg;     // <d, g+ - g>
    switch (variant) {
    case FFMIN_CG_HS: return gpy / dy;
    case FFMIN_CG_FR: return gpgp / gg;
    case FFMIN_CG_PRP_PLUS: return fmax(0.0, gpy / gg);
    case FFMIN_CG_CD: return gpgp / (-dg);
    case FFMIN_CG_LS: return gpy / (-dg);
    case FFMIN_CG_DY: return gpgp / dy;
    default: return gpy / gg;
    }
}

// OGM (Section 4, Eq. 11): t_{k+1} = (1 + sqrt(4 t_k^2 + 1)) / 2
__device__ __forceinline__ double ogm_tnext(double t) { return 0.5 * (1.0 + sqrt(4.0 * t * t + 1.0)); }

// the update op of an OGM step: fold the accepted point (and the restart)
// into X, G, X0 and the gradient sum DS, then form the next
// y = (1 - 1/t') X + (1/t') X0 and r = -((1 - 1/t') G + (2/t') DS),
// t' = t_{k+1} from S.ogm_t, and reduce <r, r>
__device__ void ogm_step(SysState &S, int accept, int restart, double wds) {
    const double tn = ogm_tnext(S.ogm_t);
    S.upd.op = U_OGM;
    S.upd.accept = accept;
    S.upd.restart = restart;
    S.upd.h = wds;
    S.upd.a = 1.0 - 1.0 / tn;
    S.upd.b = 1.0 / tn;
    S.upd.inv = 2.0 / tn;
    S.phase = PH_OGM_UPD;
}

// heavy ball (Section 4, Eq. 8): the update kernel accepts the evaluated
// iterate (accept = 1) or starts with x^{-1} = x^0 (accept = 0), then forms
// the next iterate in XT, which the same round's pair kernel evaluates
__device__ void hb_step(SysState &S, int accept) {
    S.upd.op = U_HB;
    S.upd.accept = accept;
    S.upd.restart = !accept;
    S.upd.a = S.hb_alpha;
    S.upd.b = S.hb_beta;
    set_eval(S, EV_EG, V_XT, -1, 0.0, 1.0);
    S.phase = PH_HB;
}

// reductions of the finalize kernel
enum { RF_E = 0, RF_GG, RF_GINF, RF_GTG, RF_GTR, RF_BAD, RF_EPAIR, RF_N };

__device__ void on_eval_done(const Ctx &c, SysState &S, const double *v) {
    const double E = S.ev_delta ? S.epair_base + v[RF_E] : v[RF_E];
    const bool bad = v[RF_BAD] > 0.0 || !isfinite(E);
    const int kind = S.ev_kind;
    if (kind == EV_EG) S.epair_last = v[RF_EPAIR];
    S.ev_kind = EV_NONE;
    S.ev_delta = 0;
    if (kind == EV_E) S.ne++;
    else S.neg++;

    if (S.phase == PH_EVAL_ONLY) {
        S.res_f = E;
        S.res_ginf = v[RF_GINF];
        S.status = bad ? FFMIN_ERR_NONFINITE : FFMIN_OK;
        S.phase = PH_DONE;
        deactivate(c, S);
        return;
    }
    if (S.phase == PH_FINAL) {  // FGM report evaluation of the best point
        finish(c, S, S.status, E, v[RF_GINF]);
        return;
    }
    const bool fgm = S.method == FFMIN_FGM;

    if (S.phase == PH_START) {
        if (bad) {
            finish(c, S, FFMIN_ERR_NONFINITE, E, v[RF_GINF]);
            return;
        }
        S.fresh = 1;
        S.h0 = S.h0_init;
        if (fgm) {
            S.f = S.fx = S.fb = S.fw = E;
            S.xb_known = 1;
            S.xb_ginf = v[RF_GINF];
            S.th_prev = 1.0;
            S.result_slot = V_XB;
            S.upd.op = U_FGM_W;
            S.upd.best = 1;
            S.upd.restart = 1;
            S.ginf = v[RF_GINF];
            S.gg = v[RF_GG];
            fgm_on_w(c, S, E, v[RF_GINF]);
            return;
        }
        S.result_slot = V_X;
        S.f = E;
        S.pc_mark_iter = S.iter;  // the learned-diagonal safeguard's first mark
        S.pc_mark_f = E;
        S.gg = v[RF_GG];
        S.ginf = v[RF_GINF];
        S.upd.op = U_ACCEPT;
        if (S.ginf < S.gtol) {
            finish(c, S, FFMIN_OK, S.f, S.ginf);
            return;
        }
        if (S.method == FFMIN_HB) {
            if (cap_hit(S)) {
                finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
                return;
            }
            hb_step(S, 0);
            return;
        }
        if (S.method == FFMIN_OGM) {  // x^0 = X, t_0 = 1, DS = grad f(x^0)
            if (cap_hit(S)) {
                finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
                return;
            }
            S.ogm_t = 1.0;
            ogm_step(S, 1, 1, 0.0);
            return;
        }
        set_dir(S, 1, -1.0, 0.0, 1.0, 1);
        S.phase = PH_DIR;
        return;
    }

    if (S.phase == PH_HB) {  // x^{k+1} evaluated: accept it (no line search)
        if (bad) {  // the run ends at the last finite iterate, still in X
            finish(c, S, FFMIN_ERR_NONFINITE, S.f, S.ginf);
            return;
        }
        S.iter++;
        S.f = E;
        S.ginf = v[RF_GINF];
        S.gg = v[RF_GG];
        hb_step(S, 1);
        if (S.ginf < S.gtol || mixed_handover(S, E, S.ginf)) {
            finish(c, S, FFMIN_OK, S.f, S.ginf);
            return;
        }
        if (cap_hit(S)) finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
        return;
    }

    const bool ogm = S.method == FFMIN_OGM;
    if (S.phase == PH_OGM_Y) {  // E and grad at y: the base of the line search
        if (bad) {
            finish(c, S, FFMIN_ERR_NONFINITE, S.f, S.ginf);
            return;
        }
        S.fstar = E;
        S.epair_base = S.epair_last;
        S.slope = v[RF_GTR] / S.rnorm;
        S.rg = v[RF_GTR];
        S.ls_kind = S.ls == FFMIN_LS_DEFAULT ? FFMIN_LS_PAR : S.ls;
        const double h = ls_start(S, S.h0);
        set_eval(S, EV_E, V_W, V_R, h, 1.0 / S.rnorm);
        S.phase = PH_LS;
        return;
    }

    if (S.phase == PH_LS) {
        const double f = bad ? HUGE_VAL : finite_or_inf(E);
        LsOut o = ls_feed(S, f);
        const int lsb = (fgm || ogm) ? V_W : V_X;  // base point of the search
        if (!o.done) {
            set_eval(S, EV_E, lsb, V_R, o.h, S.ev_scale);
            return;
        }
        if (o.h != 0.0) {
            S.fresh = 0;
            if (fgm) {
                fgm_accept(S, o.h, o.f);
                return;
            }
            S.h_acc = o.h;
            set_eval(S, EV_EG, lsb, V_R, o.h, S.ev_scale);
            S.phase = PH_ACCEPT;
            return;
        }
        S.lsf++;
        if (S.fresh) {
            if (fgm) fgm_finish(c, S, FFMIN_ERR_LINESEARCH);
            else finish(c, S, FFMIN_ERR_LINESEARCH, S.f, S.ginf);
            return;
        }
        S.fresh = 1;
        S.h0 = S.h0_init;
        if (fgm) {
            S.th_prev = 1.0;
            S.upd.op = U_FGM_RESET;
            S.fx = S.fw;
            fgm_next_w(S);
            return;
        }
        if (ogm) {  // restart from x^k: x^0 = X, t = 1, DS = G
            if (cap_hit(S)) {
                finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
                return;
            }
            S.ogm_t = 1.0;
            ogm_step(S, 0, 1, 0.0);
            return;
        }
        S.ring_count = 0;
        set_dir(S, 1, -1.0, 0.0, 1.0, 1);
        S.phase = PH_DIR;
        return;
    }

    if (S.phase == PH_FGM_W) {
        if (bad) {
            fgm_finish(c, S, FFMIN_ERR_NONFINITE);
            return;
        }
        S.upd.op = U_FGM_W;
        S.upd.best = 0;
        S.upd.restart = 0;
        S.ginf = v[RF_GINF];
        S.gg = v[RF_GG];
        fgm_on_w(c, S, E, v[RF_GINF]);
        return;
    }

    if (S.phase == PH_ACCEPT) {
        S.upd.op = U_ACCEPT;
        if (bad) {
            finish(c, S, FFMIN_ERR_NONFINITE, E, S.ginf);
            return;
        }
        S.iter++;
        S.h0 = fabs(S.h_acc);
        const double gninf = v[RF_GINF];
        if (ogm) {  // x^{k+1} accepted: t = t_{k+1}, DS += t_{k+1} grad f(x^{k+1})
            const double tn = ogm_tnext(S.ogm_t);
            S.ogm_t = tn;
            S.f = E;
            S.ginf = gninf;
            S.gg = v[RF_GG];
            ogm_step(S, 1, 0, tn);
            if (S.ginf < S.gtol || mixed_handover(S, E, gninf)) {
                finish(c, S, FFMIN_OK, S.f, S.ginf);
                return;
            }
            if (cap_hit(S)) finish(c, S, FFMIN_ERR_MAX_ITER, S.f, S.ginf);
            return;
        }
        if (S.method == FFMIN_LBFGS) {
            // stage (s, y) and the inner products with the committed pairs
            int used[NRING];
            for (int a = 0; a < NRING; a++) used[a] = 0;
            for (int k = 0; k < S.ring_count; k++) used[S.ring[k]] = 1;
            int stage = 0;
            while (stage < NRING && used[stage]) stage++;
            S.upd.op = U_PUSH;
            S.upd.stage = stage;
            S.upd.nS = S.ring_count;
            for (int k = 0; k < S.ring_count; k++) S.upd.sS[k] = S.ring[k];
            S.f = E;
            S.ginf = gninf;
            S.gg = v[RF_GG];
            S.phase = PH_DIR;
            return;
        }
        if (S.method == FFMIN_CG && gninf >= S.gtol) {
            if (S.iter % S.restart_every == 0) {
                set_dir(S, 0, -1.0, 0.0, 1.0, 1);
                S.cg_check = 0;
            } else {
                const double beta = cg_beta(S.cg_variant, v[RF_GG], v[RF_GTG], v[RF_GTR], S.gg, S.rg);
                set_dir(S, 0, -1.0, beta, 1.0, 1);
                S.cg_check = 1;
            }
        }
        S.f = E;
        S.ginf = gninf;
        S.gg = v[RF_GG];
        if (S.ginf < S.gtol || mixed_handover(S, E, gninf)) {
            finish(c, S, FFMIN_OK, S.f, S.ginf);
            return;
        }
        if (S.method == FFMIN_GD) set_dir(S, 1, -1.0, 0.0, 1.0, 1);
        S.phase = PH_DIR;
        return;
    }
}

// first pass of the L-BFGS direction: r0 = gamma D (-g - sum alpha_j y_j)
// with D the learned diagonal when use_d (else the identity)
__device__ void lbfgs_pass1(SysState &S, int use_d) {
    const int n = S.ring_count;
    const int nw = S.ring[n - 1];
    const double gamma = S.SY[nw][nw] / S.yy[nw];
    DirOp &d = S.dir[0];
    set_dir(S, 0, -1.0, 0.0, gamma, 2);
    d.use_d = use_d;
    S.dir_used_d = use_d;
    d.nY = n;
    for (int j = 0; j < n; j++) {  // newest first, as the vector recursion
        const int a = S.ring[n - 1 - j];
        d.sY[j] = a;
        d.cY[j] = -S.alpha[a];
    }
}

// reductions of the update kernel (U_PUSH)
// <s,y>, <y,y>, <s,g+>, then (<s_j,y>, <s_j,g+>) interleaved for the nS
// committed pairs, so a push reduces only 3 + 2 nS values
enum { RU_SY = 0, RU_YY, RU_SG, RU_N = 3 + 2 * NRING };
__host__ __device__ constexpr int ru_sjy(int j) { return 3 + 2 * j; }
__host__ __device__ constexpr int ru_sjg(int j) { return 4 + 2 * j; }
__host__ __device__ constexpr int ru_count(int nS) { return 3 + 2 * nS; }

__device__ void on_update_done(const Ctx &c, SysState &S, const double *v) {
    const int op = S.upd.op;
    S.upd.op = U_NONE;
    S.upd.best = 0;
    if (S.phase == PH_DONE) {
        deactivate(c, S);
        return;
    }
    if (op == U_OGM) {  // <r, r> of the new direction: evaluate E and grad at y
        if (S.phase != PH_OGM_UPD) return;
        S.rnorm = sqrt(v[0]);
        set_eval(S, EV_EG, V_W, -1, 0.0, 1.0);
        S.phase = PH_OGM_Y;
        return;
    }
    if (op != U_PUSH) return;
    const int nS = S.upd.nS;
    for (int k = 0; k < nS; k++) S.sg[S.upd.sS[k]] = v[ru_sjg(k)];
    const double sy = v[RU_SY];
    if (sy > 0.0) {
        if (S.ring_count == S.m) {  // drop the oldest pair
            for (int k = 1; k < S.ring_count; k++) S.ring[k - 1] = S.ring[k];
            S.ring_count--;
        }
        const int st = S.upd.stage;
        for (int k = 0; k < nS; k++) {
            const int a = S.upd.sS[k];
            S.SY[a][st] = v[ru_sjy(k)];
        }
        S.rho[st] = 1.0 / sy;
        S.yy[st] = v[RU_YY];
        S.SY[st][st] = sy;
        S.sg[st] = v[RU_SG];
        S.ring[S.ring_count++] = st;
    }
    if (S.ginf < S.gtol || mixed_handover(S, S.f, S.ginf)) {
        finish(c, S, FFMIN_OK, S.f, S.ginf);
        return;
    }
    // learned-diagonal safeguard (not in the paper): a run whose energy
    // stalls far from a stationary point with the diagonal continues as
    // plain L-BFGS, the method's own fallback
    if (S.precond_on && S.pc_window > 0 && S.iter - S.pc_mark_iter >= S.pc_window) {
        if (S.ginf > S.pc_gfar * S.gtol && !(S.pc_mark_f - S.f >= S.pc_rel * fabs(S.pc_mark_f))) S.precond_on = 0;
        S.pc_mark_iter = S.iter;
        S.pc_mark_f = S.f;
    }
    const int n = S.ring_count;
    if (n == 0) {
        set_dir(S, 1, -1.0, 0.0, 1.0, 1);
        return;
    }
    // first loop (newest -> oldest): alpha_i = rho_i <s_i, q_i>,
    // q_i = -g - sum_{j newer} alpha_j y_j
    for (int k = n - 1; k >= 0; k--) {
        const int a = S.ring[k];
        double q = -S.sg[a];
        for (int j = n - 1; j > k; j--) {
            const int b = S.ring[j];
            q = q - S.alpha[b] * S.SY[a][b];
        }
        S.alpha[a] = S.rho[a] * q;
    }
    lbfgs_pass1(S, S.precond_on);
}

// reductions of the direction kernels
enum { RD_RR = 0, RD_GR = 1 };

__device__ void on_dir_done(const Ctx &c, SysState &S, int which, const double *v) {
    S.dir[which].on = 0;
    if (S.phase == PH_DONE) return;
    if (which == 0) {
        if (S.method == FFMIN_LBFGS) {
            // second loop (oldest -> newest): beta_i = rho_i <y_i, r_i>,
            // r_i = r0 + sum_{j older} (alpha_j - beta_j) s_j
            const int n = S.ring_count;
            double beta[NRING];
            DirOp &d = S.dir[1];
            set_dir(S, 1, 0.0, 1.0, 1.0, 1);
            d.nS = n;
            for (int k = 0; k < n; k++) {
                const int a = S.ring[k];
                double yr = v[n - 1 - k];  // <y_a, r0>, dots were newest first
                for (int j = 0; j < k; j++) {
                    const int b = S.ring[j];
                    yr = yr + (S.alpha[b] - beta[j]) * S.SY[b][a];
                }
                beta[k] = S.rho[a] * yr;
                d.sS[k] = a;
                d.cS[k] = S.alpha[a] - beta[k];
            }
            return;
        }
        if (S.method == FFMIN_CG && S.cg_check && v[RD_GR] >= 0.0) {
            set_dir(S, 1, -1.0, 0.0, 1.0, 1);  // not a descent direction: restart
            return;
        }
    }
    ls_begin(c, S, v[RD_RR], v[RD_GR]);
}

}  // namespace ffm
