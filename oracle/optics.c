/*
 * Material optics of the oracle, in double precision (complex.h).
 *
 * TEST INFRASTRUCTURE ONLY (see sddm_oracle.h).
 *
 * Eq. 1 gives the complex index n~ = n + ik. Sec. 2 describes metals by their
 * optical constants and Sec. 6 evaluates glass "by the Fresnel definition";
 * the photochromic/electrochromic state is an absorption change. Fresnel's
 * amplitude coefficients for a wave arriving from vacuum:
 *     cos_t = sqrt(1 - sin^2(theta_i) / n~^2)   (principal root)
 *     r_s   = (cos_i - n~ cos_t) / (cos_i + n~ cos_t)
 *     r_p   = (n~ cos_i - cos_t) / (n~ cos_i + cos_t)
 * The glass pane is a plane-parallel slab of thickness d whose bulk absorbs
 * with coefficient alpha = alpha_clear + s*dalpha (1/m), k = alpha*lambda/(4 pi).
 * Summing the multiply reflected beams inside the slab (geometric series) per
 * polarisation j with rho_j = |r_j|^2 and internal transmittance
 * tau = exp(-alpha d / cos_t,real):
 *     R_j = rho_j + (1-rho_j)^2 rho_j tau^2 / (1 - rho_j^2 tau^2)
 *     T_j = (1-rho_j)^2 tau / (1 - rho_j^2 tau^2)
 * and unpolarised light averages the two.
 */
#include <complex.h>
#include <math.h>

#include "sddm_oracle.h"

void orc_fresnel(double c, double n, double k, double *Rs, double *Rp)
{
    double complex eta = n + I * k;
    double s2 = 1.0 - c * c;
    double complex ct = csqrt(1.0 - s2 / (eta * eta));
    double complex rs = (c - eta * ct) / (c + eta * ct);
    double complex rp = (eta * c - ct) / (eta * c + ct);
    *Rs = creal(rs) * creal(rs) + cimag(rs) * cimag(rs);
    *Rp = creal(rp) * creal(rp) + cimag(rp) * cimag(rp);
}

double orc_conductor(double c, double n, double k)
{
    double Rs, Rp;
    if (c <= 0.0)
        return 1.0;
    if (c > 1.0)
        c = 1.0;
    orc_fresnel(c, n, k, &Rs, &Rp);
    return 0.5 * (Rs + Rp);
}

void orc_slab(double c, double lam_nm, double n, double alpha_per_m, double thick_m,
              double *R, double *T)
{
    if (c <= 0.0) {
        *R = 1.0;
        *T = 0.0;
        return;
    }
    if (c > 1.0)
        c = 1.0;
    const double pi = 3.14159265358979323846;
    double k = alpha_per_m * lam_nm * 1e-9 / (4.0 * pi);
    double rho[2];
    orc_fresnel(c, n, k, &rho[0], &rho[1]);
    double ctr = sqrt(1.0 - (1.0 - c * c) / (n * n));
    double tau = exp(-alpha_per_m * thick_m / ctr);
    double Rsum = 0.0, Tsum = 0.0;
    for (int j = 0; j < 2; ++j) {
        double p = rho[j];
        double den = 1.0 - p * p * tau * tau;
        Rsum += p + (1.0 - p) * (1.0 - p) * p * tau * tau / den;
        Tsum += (1.0 - p) * (1.0 - p) * tau / den;
    }
    *R = 0.5 * Rsum;
    *T = 0.5 * Tsum;
}

/*
 * Probability of taking the reflected branch at a glass vertex. It must not
 * depend on which slab model (exact or learned) supplies R and T, nor on the
 * arithmetic precision, or the two modes would follow different paths. It is
 * the lossless slab reflectance 2 rho/(1 + rho) of the real index, averaged
 * over polarisations and wavelength bins, clamped to [0.05, 0.95].
 *
 * Because it decides an integer, it is evaluated in float exactly as the
 * kernel evaluates it: same operations, same order, no contraction
 * (this file is compiled with -ffp-contract=off), correctly rounded sqrt/div.
 */
float orc_branch_proxy(float c, int L, const float *n)
{
    float s2 = 1.0f - c * c;
    float acc = 0.0f;
    for (int i = 0; i < L; ++i) {
        float ni = n[i];
        float x = 1.0f - s2 / (ni * ni);
        float rs2, rp2;
        if (x <= 0.0f) {
            rs2 = 1.0f;
            rp2 = 1.0f;
        } else {
            float ct = sqrtf(x);
            float a = c - ni * ct, b = c + ni * ct;
            float e = ni * c - ct, f = ni * c + ct;
            float rs = a / b, rp = e / f;
            rs2 = rs * rs;
            rp2 = rp * rp;
        }
        float ps = (rs2 + rs2) / (1.0f + rs2);
        float pp = (rp2 + rp2) / (1.0f + rp2);
        acc = acc + 0.5f * (ps + pp);
    }
    float m = acc / (float)L;
    if (m < 0.05f)
        m = 0.05f;
    if (m > 0.95f)
        m = 0.95f;
    return m;
}
