/*
 * FP64 reference of the glass-slab surrogate network -- TEST INFRASTRUCTURE ONLY
 * (see sddm_oracle.h).
 *
 * The network stands in for the exact absorbing-slab R, T of Sec. 6 (glass
 * from the Fresnel equations) as a function of (cos theta, lambda, s,
 * thickness): 4 inputs -> 64 -> 64 -> 64 SiLU units -> 2 outputs (R, T).
 * Inputs are mapped to [-1, 1]:
 *   x0 = 2 sqrt(cos) - 1, x1 = 2 (lambda - 380) / 400 - 1, x2 = 2 s - 1,
 *   x3 = 2 exp(-(alpha d + A_f)) - 1,
 * where alpha = alpha_clear(lambda) + s dalpha(lambda) is the material's
 * absorption coefficient (1/m) at the coloration state s, so that x3 carries
 * the thickness as the slab's internal transmittance at normal incidence, and
 * A_f = sum_j 4 pi k_j t_j / lambda is the normal-incidence absorbance of any
 * coating films (0 for bare glass).
 * The two outputs y are log(R + 1e-3) and log(T + 1e-3); the served values are
 * R = max(exp(y0) - 1e-3, 0), T = max(exp(y1) - 1e-3, 0) (orc_mlp_rt).
 * Parameters, in this order (8770 floats): W1[64][4], b1[64], W2[64][64], b2[64],
 * W3[64][64], b3[64], W4[2][64], b4[2]; layer l computes z = W h + b.
 * Loss: mean over the batch and both outputs of the squared error.
 * Everything here is plain double-precision backpropagation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "sddm_oracle.h"

#define H 64
#define OFF_W1 0
#define OFF_B1 (OFF_W1 + H * 4)
#define OFF_W2 (OFF_B1 + H)
#define OFF_B2 (OFF_W2 + H * H)
#define OFF_W3 (OFF_B2 + H)
#define OFF_B3 (OFF_W3 + H * H)
#define OFF_W4 (OFF_B3 + H)
#define OFF_B4 (OFF_W4 + 2 * H)
#define N_PARAMS (OFF_B4 + 2)

int orc_mlp_n_params(void) { return N_PARAMS; }

void orc_mlp_features(double c, double lam_nm, double s, double d, double alpha, double film_absorbance,
                      double x[4])
{
    x[0] = 2.0 * sqrt(c > 0.0 ? c : 0.0) - 1.0;
    x[1] = 2.0 * (lam_nm - 380.0) / 400.0 - 1.0;
    x[2] = 2.0 * s - 1.0;
    x[3] = 2.0 * exp(-(alpha * d + film_absorbance)) - 1.0;
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }
static double silu(double z) { return z * sigmoid(z); }
static double dsilu(double z)
{
    double g = sigmoid(z);
    return g * (1.0 + z * (1.0 - g));
}

typedef struct {
    double z1[H], h1[H], z2[H], h2[H], z3[H], h3[H], y[2];
} orc_mlp_acts;

static void forward(const double *p, const double x[4], orc_mlp_acts *a)
{
    for (int o = 0; o < H; ++o) {
        double z = p[OFF_B1 + o];
        for (int k = 0; k < 4; ++k)
            z += (double)p[OFF_W1 + 4 * o + k] * x[k];
        a->z1[o] = z;
        a->h1[o] = silu(z);
    }
    for (int o = 0; o < H; ++o) {
        double z = p[OFF_B2 + o];
        for (int k = 0; k < H; ++k)
            z += (double)p[OFF_W2 + H * o + k] * a->h1[k];
        a->z2[o] = z;
        a->h2[o] = silu(z);
    }
    for (int o = 0; o < H; ++o) {
        double z = p[OFF_B3 + o];
        for (int k = 0; k < H; ++k)
            z += (double)p[OFF_W3 + H * o + k] * a->h2[k];
        a->z3[o] = z;
        a->h3[o] = silu(z);
    }
    for (int o = 0; o < 2; ++o) {
        double z = p[OFF_B4 + o];
        for (int k = 0; k < H; ++k)
            z += (double)p[OFF_W4 + H * o + k] * a->h3[k];
        a->y[o] = z;
    }
}

void orc_mlp_forward_d(const double *params, const double x[4], double y[2])
{
    orc_mlp_acts a;
    forward(params, x, &a);
    y[0] = a.y[0];
    y[1] = a.y[1];
}

/* Loss = mean_{i, o} (y_io - t_io)^2 over n rows; grad (N_PARAMS doubles) = dLoss/dparams. */
double orc_mlp_loss_grad_d(const double *params, int n, const double *X, const double *Tgt, double *grad)
{
    orc_mlp_acts a;
    double loss = 0.0;
    if (grad)
        memset(grad, 0, sizeof(double) * N_PARAMS);
    const double scale = 2.0 / (2.0 * (double)n);
    for (int i = 0; i < n; ++i) {
        const double *x = X + 4 * (size_t)i;
        forward(params, x, &a);
        double dy[2];
        for (int o = 0; o < 2; ++o) {
            double e = a.y[o] - Tgt[2 * (size_t)i + o];
            loss += e * e;
            dy[o] = scale * e;
        }
        if (!grad)
            continue;
        double dz3[H], dz2[H], dz1[H];
        for (int o = 0; o < 2; ++o) {
            grad[OFF_B4 + o] += dy[o];
            for (int k = 0; k < H; ++k)
                grad[OFF_W4 + H * o + k] += dy[o] * a.h3[k];
        }
        for (int k = 0; k < H; ++k) {
            double dh = dy[0] * params[OFF_W4 + k] + dy[1] * params[OFF_W4 + H + k];
            dz3[k] = dh * dsilu(a.z3[k]);
        }
        for (int o = 0; o < H; ++o) {
            grad[OFF_B3 + o] += dz3[o];
            for (int k = 0; k < H; ++k)
                grad[OFF_W3 + H * o + k] += dz3[o] * a.h2[k];
        }
        for (int k = 0; k < H; ++k) {
            double dh = 0.0;
            for (int o = 0; o < H; ++o)
                dh += dz3[o] * params[OFF_W3 + H * o + k];
            dz2[k] = dh * dsilu(a.z2[k]);
        }
        for (int o = 0; o < H; ++o) {
            grad[OFF_B2 + o] += dz2[o];
            for (int k = 0; k < H; ++k)
                grad[OFF_W2 + H * o + k] += dz2[o] * a.h1[k];
        }
        for (int k = 0; k < H; ++k) {
            double dh = 0.0;
            for (int o = 0; o < H; ++o)
                dh += dz2[o] * params[OFF_W2 + H * o + k];
            dz1[k] = dh * dsilu(a.z1[k]);
        }
        for (int o = 0; o < H; ++o) {
            grad[OFF_B1 + o] += dz1[o];
            for (int k = 0; k < 4; ++k)
                grad[OFF_W1 + 4 * o + k] += dz1[o] * x[k];
        }
    }
    return loss / (2.0 * (double)n);
}

static double *widen(const float *p)
{
    double *d = (double *)malloc(sizeof(double) * N_PARAMS);
    if (d)
        for (int i = 0; i < N_PARAMS; ++i)
            d[i] = (double)p[i];
    return d;
}

/* float32 parameters (the layout the CUDA path trains), widened to double. */
void orc_mlp_forward(const float *params, const double x[4], double y[2])
{
    double *d = widen(params);
    if (!d) {
        y[0] = y[1] = NAN;
        return;
    }
    orc_mlp_forward_d(d, x, y);
    free(d);
}

double orc_mlp_loss_grad(const float *params, int n, const double *X, const double *Tgt, double *grad)
{
    double *d = widen(params);
    if (!d)
        return NAN;
    double l = orc_mlp_loss_grad_d(d, n, X, Tgt, grad);
    free(d);
    return l;
}

/* Served (R, T) of the network at inputs x: the output map of the header. */
void orc_mlp_rt(const float *params, const double x[4], double rt[2])
{
    double y[2];
    orc_mlp_forward(params, x, y);
    for (int k = 0; k < 2; ++k) {
        const double v = exp(y[k]) - 1e-3;
        rt[k] = v > 0.0 ? v : 0.0;
    }
}
