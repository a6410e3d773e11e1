/*
 * FP64 oracle of the preconditioner network (TEST INFRASTRUCTURE ONLY, see
 * ffmin_oracle.h).  Not in the paper: a per-atom MLP 5 -> 64 (ReLU) -> 1 whose
 * output z scales the L-BFGS initial Hessian by exp(clamp(z, -3, 3)) on the
 * atom's three coordinates.  Weights: W1 [64][5], b1 [64], w2 [64], b2.
 * Features: charge, sigma, epsilon, n(8 A)/64, log(1 + |grad_i|).
 */
#include "ffmin_oracle.h"

#include <math.h>
#include <stdlib.h>

#define NIN 5
#define NH 64
#define OW1 0
#define OB1 (NH * NIN)
#define OW2 (OB1 + NH)
#define OB2 (OW2 + NH)

double orc_mlp_forward(const double *w, const double *f, double *h) {
    double z = w[OB2];
    for (int k = 0; k < NH; k++) {
        double a = w[OB1 + k];
        for (int i = 0; i < NIN; i++) a += w[OW1 + k * NIN + i] * f[i];
        if (a < 0.0) a = 0.0;
        if (h) h[k] = a;
        z += w[OW2 + k] * a;
    }
    return z;
}

/* mean over n rows of (z - t)^2 and its gradient with respect to w */
double orc_mlp_loss_grad(const double *w, const double *feat, const double *target, int64_t n,
                         double *grad) {
    for (int k = 0; k < ORC_MLP_NW; k++) grad[k] = 0.0;
    double loss = 0.0;
    for (int64_t r = 0; r < n; r++) {
        double h[NH];
        const double *f = feat + r * NIN;
        double z = orc_mlp_forward(w, f, h);
        double e = z - target[r];
        loss += e * e;
        double dz = 2.0 * e / (double)n;
        grad[OB2] += dz;
        for (int k = 0; k < NH; k++) {
            grad[OW2 + k] += dz * h[k];
            double dh = h[k] > 0.0 ? dz * w[OW2 + k] : 0.0;
            grad[OB1 + k] += dh;
            for (int i = 0; i < NIN; i++) grad[OW1 + k * NIN + i] += dh * f[i];
        }
    }
    return loss / (double)n;
}

void orc_mlp_features(double q, double sigma, double eps, int32_t n8, double gnorm, double *f) {
    f[0] = q;
    f[1] = sigma;
    f[2] = eps;
    f[3] = (double)n8 / 64.0;
    f[4] = log1p(gnorm);
}

/* per-coordinate diagonal d [3N] from the network at gradient g [3N] */
void orc_precond_diag(const orc_ff *ff, const double *w, const int32_t *n8, const double *g, double *d) {
    for (int i = 0; i < ff->n_atoms; i++) {
        double f[NIN];
        const double *gi = g + 3 * i;
        orc_mlp_features(ff->charge[i], ff->sigma[i], ff->epsilon[i], n8[i],
                         sqrt(gi[0] * gi[0] + gi[1] * gi[1] + gi[2] * gi[2]), f);
        double z = orc_mlp_forward(w, f, NULL);
        if (z < -3.0) z = -3.0;
        if (z > 3.0) z = 3.0;
        const double s = exp(z);
        d[3 * i] = d[3 * i + 1] = d[3 * i + 2] = s;
    }
}
