/*
 * Material optics of the oracle, in double precision (complex.h).
 *
 * TEST INFRASTRUCTURE ONLY (see sddm_oracle.h).
 *
 * Eq. 1 gives the complex index n~ = n + ik. Sec. 2 describes metals by their
 * optical constants and Sec. 6 evaluates glass with the Fresnel equations;
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
#include <string.h>

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
 * Glass slab coated on both outer faces with the same stack of J thin films
 * (an electrochromic device: e.g. a conductor / absorbing electrochromic layer
 * / conductor sandwich). Each face is a coherent stack, evaluated by the
 * characteristic (transfer) matrix of thin-film optics: per film j, complex
 * index n_j + i k_j, thickness t_j, the Snell invariant sin(theta) carried
 * through, cos(theta_j) = sqrt(1 - sin^2 / n_j^2) on the decaying branch,
 * tilted admittance eta_j = n_j cos(theta_j) (s) or n_j / cos(theta_j) (p),
 * phase delta_j = 2 pi n_j t_j cos(theta_j) / lambda and, for the complex
 * index n + i k (fields ~ exp(i (k z - omega t)), so that Im(delta) > 0 decays),
 *     M_j = [[cos delta_j, -i sin delta_j / eta_j], [-i eta_j sin delta_j, cos delta_j]].
 * From air: [B, C] = M_1 ... M_J [1, eta_sub], r = (eta_0 B - C) / (eta_0 B + C),
 * T = 4 eta_0 Re(eta_sub) / |eta_0 B + C|^2. From inside the glass the films
 * come in reverse order with air beyond. The thick substrate (real index,
 * internal transmittance tau = exp(-alpha d / cos theta_t)) combines the two
 * faces incoherently, as the bare slab does:
 *     R = R_a + T_a T_g R_g tau^2 / (1 - R_g^2 tau^2),  T = T_a T_g tau / (1 - R_g^2 tau^2)
 * (R_a, T_a seen from air, R_g, T_g from the glass), per polarisation, then
 * averaged. With no film the bare slab (orc_slab) is used.
 */
static double complex film_cos(double complex n, double s2)
{
    double complex ct = csqrt(1.0 - s2 / (n * n));
    if (cimag(n * ct) < 0.0)
        ct = -ct;
    return ct;
}

void orc_coated_face(double c, double lam_nm, double n_sub, int J, const double *nf, const double *kf,
                     const double *tf_nm, int pol, double *Ra, double *Ta, double *Rg, double *Tg)
{
    const double pi = 3.14159265358979323846;
    double s2 = 1.0 - c * c;
    double ct_sub = sqrt(1.0 - s2 / (n_sub * n_sub));
    double complex eta0 = pol == 0 ? c : 1.0 / c;
    double complex etas = pol == 0 ? n_sub * ct_sub : n_sub / ct_sub;
    double complex m[2][2] = {{1.0, 0.0}, {0.0, 1.0}};   /* M_1 ... M_J */
    double complex g[2][2] = {{1.0, 0.0}, {0.0, 1.0}};   /* M_J ... M_1 */
    for (int j = 0; j < J; ++j) {
        double complex n = nf[j] + I * kf[j];
        double complex ct = film_cos(n, s2);
        double complex eta = pol == 0 ? n * ct : n / ct;
        double complex delta = 2.0 * pi * n * (tf_nm[j] * 1e-9) * ct / (lam_nm * 1e-9);
        double complex mj[2][2] = {{ccos(delta), -I * csin(delta) / eta}, {-I * eta * csin(delta), ccos(delta)}};
        double complex t[2][2];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                t[a][b] = m[a][0] * mj[0][b] + m[a][1] * mj[1][b];
        memcpy(m, t, sizeof t);
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                t[a][b] = mj[a][0] * g[0][b] + mj[a][1] * g[1][b];
        memcpy(g, t, sizeof t);
    }
    double complex B = m[0][0] + m[0][1] * etas, C = m[1][0] + m[1][1] * etas;
    double complex r = (eta0 * B - C) / (eta0 * B + C);
    double complex den = eta0 * B + C;
    *Ra = creal(r * conj(r));
    *Ta = 4.0 * creal(eta0) * creal(etas) / creal(den * conj(den));
    double complex B2 = g[0][0] + g[0][1] * eta0, C2 = g[1][0] + g[1][1] * eta0;
    double complex r2 = (etas * B2 - C2) / (etas * B2 + C2);
    double complex den2 = etas * B2 + C2;
    *Rg = creal(r2 * conj(r2));
    *Tg = 4.0 * creal(etas) * creal(eta0) / creal(den2 * conj(den2));
}

void orc_coated_slab(double c, double lam_nm, double n_sub, double alpha_per_m, double thick_m, int J,
                     const double *nf, const double *kf, const double *tf_nm, double *R, double *T)
{
    if (J <= 0) {
        orc_slab(c, lam_nm, n_sub, alpha_per_m, thick_m, R, T);
        return;
    }
    if (c <= 0.0) {
        *R = 1.0;
        *T = 0.0;
        return;
    }
    if (c > 1.0)
        c = 1.0;
    double ctr = sqrt(1.0 - (1.0 - c * c) / (n_sub * n_sub));
    double tau = exp(-alpha_per_m * thick_m / ctr);
    double Rsum = 0.0, Tsum = 0.0;
    for (int pol = 0; pol < 2; ++pol) {
        double Ra, Ta, Rg, Tg;
        orc_coated_face(c, lam_nm, n_sub, J, nf, kf, tf_nm, pol, &Ra, &Ta, &Rg, &Tg);
        double den = 1.0 - Rg * Rg * tau * tau;
        Rsum += Ra + Ta * Tg * Rg * tau * tau / den;
        Tsum += Ta * Tg * tau / den;
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
