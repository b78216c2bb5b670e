/*
 * The oracle's estimator: spectral Monte Carlo path tracing, FP64.
 *
 * TEST INFRASTRUCTURE ONLY (see sddm_oracle.h).
 *
 * One camera path per (pixel, sample) carries all L wavelength bins at once
 * (the lambda grid is fixed input, never sampled). Following the rendering
 * algorithm of Sec. 4 and the model of Sec. 3:
 *   - a primary ray leaves each pixel (pinhole, or orthographic as in Sec. 4);
 *   - at each of at most D vertices the closest surface is found;
 *   - an emitter seen directly, or through a chain of specular vertices, adds
 *     its radiance (Eq. 2's L_i at that vertex); with next-event estimation
 *     off every emitter hit counts;
 *   - at a Lambertian vertex Eq. 3's light sum is estimated by one shadow ray
 *     toward a point drawn on the area lights (Sec. 4 casts a ray from each hit
 *     point toward every light source); the shadow ray passes through
 *     glass slabs and is weighted by their transmittance;
 *   - the path continues by the reflection/refraction laws (Sec. 4): a
 *     cosine-distributed direction at a Lambertian vertex, the mirror
 *     direction weighted by Fresnel at a metal (Sec. 2, Eq. 1), and at a glass
 *     slab either the mirror direction weighted by R or straight transmission
 *     weighted by T (Sec. 6: glass from the Fresnel equations);
 *   - it stops after D vertices (the paper's fixed bounce limit), on a
 *     miss or on a black emitter.
 * XYZ = sum_i w_i L(lambda_i) cmf(lambda_i); a pixel is the mean of its spp.
 *
 * Random numbers: Philox4x32-10, counter (pixel, sample, vertex, slot), key
 * (seed, render); the camera uses vertex 0.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "oracle_internal.h"

#define SLOT_CAMERA 0x10000u
#define SLOT_BSDF 0x10001u
#define SLOT_LIGHT 0x10002u
#define SLOT_GLASS 0x10003u

static const double PI = 3.14159265358979323846;
static const double RAY_OFFSET = 1e-4;      /* metres, along the geometric normal */
static const double SHADOW_SHORTEN = 1e-4;  /* shadow rays stop at (1 - 1e-4) * distance */

/* ----------------------------------------------------------- context --- */
static double *dup_d(const float *src, size_t n)
{
    double *d = (double *)malloc(sizeof(double) * (n ? n : 1));
    if (d && src)
        for (size_t i = 0; i < n; ++i)
            d[i] = (double)src[i];
    else if (d)
        memset(d, 0, sizeof(double) * (n ? n : 1));
    return d;
}

void orc_destroy(void *p)
{
    orc_ctx *c = (orc_ctx *)p;
    if (!c)
        return;
    free(c->lam); free(c->w); free(c->cmf);
    free(c->kind); free(c->a); free(c->b); free(c->c); free(c->a_f);
    free(c->thick); free(c->s);
    free(c->nlayers); free(c->ln); free(c->lk); free(c->ldk); free(c->lt);
    free(c->v); free(c->ng); free(c->mat); free(c->obj);
    free(c->nodes); free(c->tri_order);
    free(c->light_tri); free(c->light_cdf);
    free(c);
}

int orc_create(void **out, const orc_scene_desc *d)
{
    *out = NULL;
    if (d->L < 1 || d->L > ORC_MAX_L || d->n_mat < 1 || d->nt < 0 || d->nv < 0)
        return -1;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    if (!c)
        return -2;
    int L = d->L;
    size_t ML = (size_t)d->n_mat * (size_t)L;
    c->L = L;
    c->lam = dup_d(d->lam_nm, (size_t)L);
    c->w = dup_d(d->quad_w, (size_t)L);
    c->cmf = dup_d(d->cmf, (size_t)L * 3);
    c->n_mat = d->n_mat;
    c->kind = (int *)malloc(sizeof(int) * (size_t)d->n_mat);
    c->a = dup_d(d->mat_a, ML);
    c->b = dup_d(d->mat_b, ML);
    c->c = dup_d(d->mat_c, ML);
    c->a_f = (float *)malloc(sizeof(float) * ML);
    c->thick = dup_d(d->mat_thick, (size_t)d->n_mat);
    c->s = dup_d(d->mat_s, (size_t)d->n_mat);
    size_t MF = (size_t)d->n_mat * ORC_MAX_FILMS;
    c->nlayers = (int *)calloc((size_t)d->n_mat, sizeof(int));
    c->ln = dup_d(d->layer_n, MF * (size_t)L);
    c->lk = dup_d(d->layer_k, MF * (size_t)L);
    c->ldk = dup_d(d->layer_dk, MF * (size_t)L);
    c->lt = dup_d(d->layer_t, MF);
    if (!c->nlayers || !c->ln || !c->lk || !c->ldk || !c->lt) {
        orc_destroy(c);
        return -2;
    }
    for (int m = 0; m < d->n_mat; ++m) {
        int nl = d->mat_nlayers ? d->mat_nlayers[m] : 0;
        if (nl < 0 || nl > ORC_MAX_FILMS) {
            orc_destroy(c);
            return -1;
        }
        c->nlayers[m] = nl;
    }
    c->nt = d->nt;
    size_t nt = (size_t)d->nt;
    c->v = (double *)malloc(sizeof(double) * 9 * (nt ? nt : 1));
    c->ng = (double *)malloc(sizeof(double) * 3 * (nt ? nt : 1));
    c->mat = (int *)malloc(sizeof(int) * (nt ? nt : 1));
    c->obj = (int *)malloc(sizeof(int) * (nt ? nt : 1));
    if (!c->kind || !c->a_f || !c->v || !c->ng || !c->mat || !c->obj) {
        orc_destroy(c);
        return -2;
    }
    for (int m = 0; m < d->n_mat; ++m) {
        c->kind[m] = d->mat_kind[m];
        if (c->kind[m] < ORC_LAMBERT || c->kind[m] > ORC_DIFFUSE_EMITTER) {
            orc_destroy(c);
            return -1;
        }
    }
    for (size_t i = 0; i < ML; ++i)
        c->a_f[i] = d->mat_a ? d->mat_a[i] : 0.0f;
    for (size_t t = 0; t < nt; ++t) {
        for (int k = 0; k < 3; ++k) {
            uint32_t vi = d->F[3 * t + k];
            if (vi >= (uint32_t)d->nv) {
                orc_destroy(c);
                return -1;
            }
            for (int a = 0; a < 3; ++a)
                c->v[9 * t + 3 * k + a] = (double)d->V[3 * (size_t)vi + a];
        }
        if (d->mat_id[t] >= (uint32_t)d->n_mat) {
            orc_destroy(c);
            return -1;
        }
        c->mat[t] = (int)d->mat_id[t];
        c->obj[t] = (int)d->obj_id[t];
        const double *v = c->v + 9 * t;
        double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        for (int a = 0; a < 3; ++a)
            c->ng[3 * t + a] = len > 0.0 ? n[a] / len : 0.0;
    }
    /* area lights: every triangle whose material emits */
    c->light_tri = (int *)malloc(sizeof(int) * (nt ? nt : 1));
    c->light_cdf = (float *)malloc(sizeof(float) * (nt ? nt : 1));
    double *cum = (double *)malloc(sizeof(double) * (nt ? nt : 1));
    if (!c->light_tri || !c->light_cdf || !cum) {
        free(cum);
        orc_destroy(c);
        return -2;
    }
    c->n_light = 0;
    double total = 0.0;
    for (size_t t = 0; t < nt; ++t) {
        int k = c->kind[c->mat[t]];
        if (k != ORC_EMITTER && k != ORC_DIFFUSE_EMITTER)
            continue;
        const double *v = c->v + 9 * t;
        double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double area = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        total += area;
        cum[c->n_light] = total;
        c->light_tri[c->n_light++] = (int)t;
    }
    for (int i = 0; i < c->n_light; ++i)
        c->light_cdf[i] = (float)(cum[i] / total);
    c->light_area = total;
    free(cum);
    if (orc_build_bvh(c) != 0) {
        orc_destroy(c);
        return -2;
    }
    *out = c;
    return 0;
}

int orc_num_lights(void *ctx)
{
    return ((orc_ctx *)ctx)->n_light;
}

/* ------------------------------------------------------------ helpers --- */
static void philox_u(uint32_t p, uint32_t j, uint32_t b, uint32_t slot, const orc_render_desc *r,
                     double u[4])
{
    uint32_t ctr[4] = {p, j, b, slot}, key[2] = {r->seed, r->render_id}, x[4];
    orc_philox4x32_10(ctr, key, x);
    for (int i = 0; i < 4; ++i)
        u[i] = orc_u01(x[i]);
}

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void normalize3(double *v)
{
    double l = sqrt(dot3(v, v));
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
}

void orc_camera_ray(const orc_render_desc *r, double px, double py, double o[3], double d[3])
{
    double f[3], rt[3], up[3];
    for (int a = 0; a < 3; ++a)
        f[a] = r->cam_look[a] - r->cam_pos[a];
    normalize3(f);
    rt[0] = f[1] * r->cam_up[2] - f[2] * r->cam_up[1];
    rt[1] = f[2] * r->cam_up[0] - f[0] * r->cam_up[2];
    rt[2] = f[0] * r->cam_up[1] - f[1] * r->cam_up[0];
    normalize3(rt);
    up[0] = rt[1] * f[2] - rt[2] * f[1];
    up[1] = rt[2] * f[0] - rt[0] * f[2];
    up[2] = rt[0] * f[1] - rt[1] * f[0];
    double nx = 2.0 * px / r->width - 1.0;
    double ny = 1.0 - 2.0 * py / r->height;
    double aspect = (double)r->width / (double)r->height;
    if (r->ortho_height > 0.0) {
        double h = 0.5 * r->ortho_height;
        for (int a = 0; a < 3; ++a) {
            o[a] = r->cam_pos[a] + nx * h * aspect * rt[a] + ny * h * up[a];
            d[a] = f[a];
        }
        return;
    }
    double th = tan(0.5 * r->vfov_deg * PI / 180.0);
    for (int a = 0; a < 3; ++a) {
        o[a] = r->cam_pos[a];
        d[a] = f[a] + nx * th * aspect * rt[a] + ny * th * up[a];
    }
    normalize3(d);
}

/* Cosine-distributed direction about the unit normal ns: Malley's method on
 * the Shirley-Chiu concentric disk, frame from Duff et al. (JCGT 2017). */
void orc_cosine_dir(const double ns[3], double u0, double u1, double out[3])
{
    double a = 2.0 * u0 - 1.0, b = 2.0 * u1 - 1.0, r, phi;
    double dx = 0.0, dy = 0.0;
    if (a != 0.0 || b != 0.0) {
        if (fabs(a) > fabs(b)) {
            r = a;
            phi = (PI / 4.0) * (b / a);
        } else {
            r = b;
            phi = PI / 2.0 - (PI / 4.0) * (a / b);
        }
        dx = r * cos(phi);
        dy = r * sin(phi);
    }
    double dz = sqrt(fmax(0.0, 1.0 - dx * dx - dy * dy));
    double sgn = ns[2] >= 0.0 ? 1.0 : -1.0;
    double aa = -1.0 / (sgn + ns[2]);
    double bb = ns[0] * ns[1] * aa;
    double t[3] = {1.0 + sgn * ns[0] * ns[0] * aa, sgn * bb, -sgn * ns[0]};
    double bt[3] = {bb, sgn + ns[1] * ns[1] * aa, -ns[1]};
    for (int k = 0; k < 3; ++k)
        out[k] = dx * t[k] + dy * bt[k] + dz * ns[k];
}

static double state_s(const orc_ctx *c, const orc_render_desc *r, int m)
{
    if (r->s_override && r->s_override[m] >= 0.0f)
        return (double)r->s_override[m];
    return c->s[m];
}

static void slab_rt(const orc_ctx *c, const orc_render_desc *r, int m, double cosv, int i,
                    double *R, double *T)
{
    size_t k = (size_t)m * c->L + i;
    double s = state_s(c, r, m);
    double alpha = c->b[k] + s * c->c[k];
    int J = c->nlayers[m];
    double nf[ORC_MAX_FILMS], kf[ORC_MAX_FILMS], tf[ORC_MAX_FILMS];
    for (int j = 0; j < J; ++j) {
        size_t f = ((size_t)m * ORC_MAX_FILMS + j) * c->L + i;
        nf[j] = c->ln[f];
        kf[j] = c->lk[f] + s * c->ldk[f];
        tf[j] = c->lt[(size_t)m * ORC_MAX_FILMS + j];
    }
    orc_coated_slab(cosv, c->lam[i], c->a[k], alpha, c->thick[m], J, nf, kf, tf, R, T);
}

/* ------------------------------------------------------- photon map --- */
typedef struct {
    int L;
    int64_t n;                 /* stored photons */
    double *pos, *dir, *pow;   /* [n][3], [n][3], [n][L] */
    double radius;
    double lo[3];              /* grid over the stored photons, cell = radius */
    int dims[3];
    int64_t *cell_start;       /* [cells + 1] */
    int64_t *order;            /* photon indices sorted by cell */
} orc_pmap;

static void pm_slot_u(uint32_t i, uint32_t b, uint32_t slot, const orc_render_desc *r, double u[4])
{
    philox_u(i, 0xffffffffu, b, slot, r, u);
}

/* Trace photon i; write its deposits (at most D - 1) into rec[k] = {x, d, valid}, pw[k][L]. */
static void trace_photon(const orc_ctx *c, const orc_render_desc *r, uint32_t i, double phi0_scale,
                         double *rec, double *pw, double *Phi)
{
    const int L = c->L, D = r->max_depth;
    for (int k = 0; k < D - 1; ++k)
        rec[7 * k + 6] = 0.0;
    if (c->n_light == 0 || D < 2)
        return;
    double u[4];
    pm_slot_u(i, 0u, SLOT_LIGHT, r, u);
    int li = c->n_light - 1;
    for (int k = 0; k < c->n_light; ++k)
        if (u[0] < (double)c->light_cdf[k]) {
            li = k;
            break;
        }
    int lt = c->light_tri[li];
    const double *lv = c->v + 9 * (size_t)lt, *nl = c->ng + 3 * (size_t)lt;
    double su = sqrt(u[1]);
    double b0 = 1.0 - su, b1 = u[2] * su, b2 = 1.0 - b0 - b1;
    double o[3], d[3];
    for (int a = 0; a < 3; ++a)
        o[a] = b0 * lv[a] + b1 * lv[3 + a] + b2 * lv[6 + a] + RAY_OFFSET * nl[a];
    pm_slot_u(i, 0u, SLOT_BSDF, r, u);
    orc_cosine_dir(nl, u[0], u[1], d);
    const double *Le = c->a + (size_t)c->mat[lt] * L;
    for (int l = 0; l < L; ++l)
        Phi[l] = Le[l] * PI * c->light_area * phi0_scale;
    int excl_prim = lt, excl_obj = -1, changed = 0, diffuse_seen = 0;
    for (int b = 1; b <= D - 1; ++b) {
        orc_hit h;
        if (!orc_trace_closest(c, o, d, excl_prim, excl_obj, r->brute_force, &h, NULL))
            return;
        int tri = h.prim, mat = c->mat[tri], kind = c->kind[mat];
        const double *ng = c->ng + 3 * (size_t)tri;
        double x[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]};
        double cd = dot3(d, ng);
        double ns[3];
        for (int a = 0; a < 3; ++a)
            ns[a] = cd < 0.0 ? ng[a] : -ng[a];
        const double *mA = c->a + (size_t)mat * L, *mB = c->b + (size_t)mat * L;
        if (kind == ORC_EMITTER)
            return;
        if (kind == ORC_LAMBERT || kind == ORC_DIFFUSE_EMITTER) {
            if (changed) {
                double *q = rec + 7 * (b - 1);
                for (int a = 0; a < 3; ++a) {
                    q[a] = x[a];
                    q[3 + a] = d[a];
                }
                q[6] = diffuse_seen ? 1.0 : 2.0;   /* 1: global, 2: caustic (only specular reflections so far) */
                for (int l = 0; l < L; ++l)
                    pw[(size_t)(b - 1) * L + l] = Phi[l];
            }
            if (b == D - 1)
                return;
            const double *rho = kind == ORC_LAMBERT ? mA : mB;
            pm_slot_u(i, (uint32_t)b, SLOT_BSDF, r, u);
            orc_cosine_dir(ns, u[0], u[1], d);
            for (int l = 0; l < L; ++l)
                Phi[l] *= rho[l];
            for (int a = 0; a < 3; ++a)
                o[a] = x[a] + RAY_OFFSET * ns[a];
            excl_prim = tri;
            excl_obj = -1;
            changed = 1;
            diffuse_seen = 1;
        } else if (kind == ORC_CONDUCTOR) {
            if (b == D - 1)
                return;
            double cosv = fabs(cd);
            for (int l = 0; l < L; ++l)
                Phi[l] *= orc_conductor(cosv, mA[l], mB[l]);
            for (int a = 0; a < 3; ++a) {
                d[a] = d[a] - 2.0 * cd * ng[a];
                o[a] = x[a] + RAY_OFFSET * ns[a];
            }
            excl_prim = tri;
            excl_obj = -1;
            changed = 1;
        } else {
            if (b == D - 1)
                return;
            double cosv = fabs(cd);
            float pr = orc_branch_proxy((float)cosv, L, c->a_f + (size_t)mat * L);
            pm_slot_u(i, (uint32_t)b, SLOT_GLASS, r, u);
            int reflect = u[0] < (double)pr;
            for (int l = 0; l < L; ++l) {
                double Rr, Tt;
                slab_rt(c, r, mat, cosv, l, &Rr, &Tt);
                Phi[l] *= reflect ? Rr / (double)pr : Tt / (1.0 - (double)pr);
            }
            if (reflect) {
                for (int a = 0; a < 3; ++a) {
                    d[a] = d[a] - 2.0 * cd * ng[a];
                    o[a] = x[a] + RAY_OFFSET * ns[a];
                }
                excl_prim = tri;
                excl_obj = -1;
                changed = 1;
            } else {
                for (int a = 0; a < 3; ++a)
                    o[a] = x[a] - RAY_OFFSET * ns[a];
                excl_prim = tri;
                excl_obj = c->obj[tri];
            }
        }
    }
}

typedef struct {
    const orc_ctx *c;
    const orc_render_desc *r;
    int64_t n;
    double scale;
    double *rec, *pw;
    atomic_llong next;
} orc_pjob;

static void *photon_worker(void *arg)
{
    orc_pjob *jb = (orc_pjob *)arg;
    const int L = jb->c->L, D = jb->r->max_depth;
    double *Phi = (double *)malloc(sizeof(double) * (size_t)L);
    if (!Phi)
        return NULL;
    for (;;) {
        int64_t i0 = atomic_fetch_add(&jb->next, 64);
        if (i0 >= jb->n)
            break;
        int64_t i1 = i0 + 64 < jb->n ? i0 + 64 : jb->n;
        for (int64_t i = i0; i < i1; ++i)
            trace_photon(jb->c, jb->r, (uint32_t)i, jb->scale, jb->rec + (size_t)i * 7 * (D - 1),
                         jb->pw + (size_t)i * (D - 1) * L, Phi);
    }
    free(Phi);
    return NULL;
}

void orc_photon_map_free(void *p)
{
    orc_pmap *pm = (orc_pmap *)p;
    if (!pm)
        return;
    free(pm->pos); free(pm->dir); free(pm->pow); free(pm->cell_start); free(pm->order);
    free(pm);
}

static int64_t pm_cell(const orc_pmap *pm, const double *x)
{
    int c[3];
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor((x[a] - pm->lo[a]) / pm->radius);
        c[a] = k < 0 ? 0 : (k >= pm->dims[a] ? pm->dims[a] - 1 : k);
    }
    return ((int64_t)c[2] * pm->dims[1] + c[1]) * pm->dims[0] + c[0];
}

void *orc_photon_map_build(void *ctx, const orc_render_desc *r, int64_t n_photons, double radius, int n_threads)
{
    return orc_photon_map_build_kind(ctx, r, n_photons, radius, 0, n_threads);
}

void *orc_photon_map_build_kind(void *ctx, const orc_render_desc *r, int64_t n_photons, double radius, int kind,
                                int n_threads)
{
    const orc_ctx *c = (const orc_ctx *)ctx;
    if (!c || !r || n_photons < 0 || !(radius > 0.0) || r->max_depth < 2 || kind < 0 || kind > 2)
        return NULL;
    const int L = c->L, D = r->max_depth;
    size_t slots = (size_t)n_photons * (size_t)(D - 1);
    /* no photons: an empty map */
    double *rec = (double *)malloc(sizeof(double) * 7 * (slots ? slots : 1));
    double *pw = (double *)malloc(sizeof(double) * (slots ? slots : 1) * (size_t)L);
    orc_pmap *pm = (orc_pmap *)calloc(1, sizeof(orc_pmap));
    if (!rec || !pw || !pm) {
        free(rec); free(pw); free(pm);
        return NULL;
    }
    orc_pjob jb = {c, r, n_photons, n_photons ? 1.0 / (double)n_photons : 0.0, rec, pw, 0};
    atomic_init(&jb.next, 0);
    if (n_threads <= 0) {
        long nc = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = nc > 0 ? (int)nc : 1;
    }
    if (n_threads > 512)
        n_threads = 512;
    pthread_t th[512];
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, photon_worker, &jb) != 0)
            break;
        ++started;
    }
    if (started == 0)
        photon_worker(&jb);
    for (int t = 0; t < started; ++t)
        pthread_join(th[t], NULL);
    /* compact the stored photons in slot order */
    /* kind 0: every stored photon; 1: global photons only; 2: caustic photons only */
#define PM_KEEP(flag) ((flag) != 0.0 && (kind == 0 || (flag) == (double)kind))
    int64_t n = 0;
    for (size_t s = 0; s < slots; ++s)
        n += PM_KEEP(rec[7 * s + 6]);
    pm->L = L;
    pm->n = n;
    pm->radius = radius;
    pm->pos = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
    pm->dir = (double *)malloc(sizeof(double) * 3 * (size_t)(n ? n : 1));
    pm->pow = (double *)malloc(sizeof(double) * (size_t)L * (size_t)(n ? n : 1));
    if (!pm->pos || !pm->dir || !pm->pow) {
        free(rec); free(pw);
        orc_photon_map_free(pm);
        return NULL;
    }
    int64_t k = 0;
    for (size_t s = 0; s < slots; ++s) {
        if (!PM_KEEP(rec[7 * s + 6]))
            continue;
        for (int a = 0; a < 3; ++a) {
            pm->pos[3 * k + a] = rec[7 * s + a];
            pm->dir[3 * k + a] = rec[7 * s + 3 + a];
        }
        memcpy(pm->pow + (size_t)k * L, pw + s * (size_t)L, sizeof(double) * (size_t)L);
        ++k;
    }
    free(rec);
    free(pw);
    /* uniform grid of cell size = radius over the photons */
    double hi[3];
    for (int a = 0; a < 3; ++a) {
        pm->lo[a] = INFINITY;
        hi[a] = -INFINITY;
    }
    for (int64_t q = 0; q < n; ++q)
        for (int a = 0; a < 3; ++a) {
            pm->lo[a] = fmin(pm->lo[a], pm->pos[3 * q + a]);
            hi[a] = fmax(hi[a], pm->pos[3 * q + a]);
        }
    int64_t cells = 1;
    for (int a = 0; a < 3; ++a) {
        if (n == 0) {
            pm->lo[a] = 0.0;
            hi[a] = 0.0;
        }
        pm->dims[a] = (int)floor((hi[a] - pm->lo[a]) / radius) + 1;
        cells *= pm->dims[a];
    }
    pm->cell_start = (int64_t *)calloc((size_t)cells + 1, sizeof(int64_t));
    pm->order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n ? n : 1));
    if (!pm->cell_start || !pm->order) {
        orc_photon_map_free(pm);
        return NULL;
    }
    for (int64_t q = 0; q < n; ++q)
        pm->cell_start[pm_cell(pm, pm->pos + 3 * q) + 1]++;
    for (int64_t cidx = 0; cidx < cells; ++cidx)
        pm->cell_start[cidx + 1] += pm->cell_start[cidx];
    int64_t *fill = (int64_t *)calloc((size_t)cells, sizeof(int64_t));
    if (!fill) {
        orc_photon_map_free(pm);
        return NULL;
    }
    for (int64_t q = 0; q < n; ++q) {
        int64_t cc = pm_cell(pm, pm->pos + 3 * q);
        pm->order[pm->cell_start[cc] + fill[cc]++] = q;
    }
    free(fill);
    return pm;
}

int64_t orc_photon_map_get(const void *p, double *pos, double *dir, double *power)
{
    const orc_pmap *pm = (const orc_pmap *)p;
    if (!pm)
        return -1;
    if (pos)
        memcpy(pos, pm->pos, sizeof(double) * 3 * (size_t)pm->n);
    if (dir)
        memcpy(dir, pm->dir, sizeof(double) * 3 * (size_t)pm->n);
    if (power)
        memcpy(power, pm->pow, sizeof(double) * (size_t)pm->L * (size_t)pm->n);
    return pm->n;
}

/* Radiance estimate at a diffuse point x seen from the side ns: the power of
 * the photons within the radius that arrived on that side, over pi r^2,
 * times rho / pi (added to Ls with the path throughput T). */
static void pm_gather(const orc_pmap *pm, const double *x, const double *ns, const double *rho, const double *T,
                      double *Ls)
{
    if (pm->n == 0)
        return;
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
        c0[a] = (int)floor((x[a] - pm->radius - pm->lo[a]) / pm->radius);
        c1[a] = (int)floor((x[a] + pm->radius - pm->lo[a]) / pm->radius);
        c0[a] = c0[a] < 0 ? 0 : c0[a];
        c1[a] = c1[a] >= pm->dims[a] ? pm->dims[a] - 1 : c1[a];
    }
    const int L = pm->L;
    const double r2 = pm->radius * pm->radius, norm = 1.0 / (PI * r2);
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy)
            for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                int64_t cc = ((int64_t)cz * pm->dims[1] + cy) * pm->dims[0] + cx;
                for (int64_t s = pm->cell_start[cc]; s < pm->cell_start[cc + 1]; ++s) {
                    int64_t q = pm->order[s];
                    const double *xp = pm->pos + 3 * q;
                    double dx = xp[0] - x[0], dy = xp[1] - x[1], dz = xp[2] - x[2];
                    if (dx * dx + dy * dy + dz * dz >= r2)
                        continue;
                    if (dot3(pm->dir + 3 * q, ns) >= 0.0)
                        continue;
                    const double *pw = pm->pow + (size_t)q * L;
                    for (int l = 0; l < L; ++l)
                        Ls[l] += T[l] * rho[l] / PI * pw[l] * norm;
                }
            }
}

/* ----------------------------------------------------------- one path --- */
typedef struct {
    double *T, *Lsum;     /* [L] */
    int64_t seg_ext, seg_shadow;
} orc_scratch;

static void trace_path(const orc_ctx *c, const orc_render_desc *r, int px, int py, int j,
                       orc_scratch *ws, int32_t *first_prim, double *margin_out, double *cos_min_out)
{
    const int L = c->L;
    const int brute = r->brute_force;
    double *T = ws->T, *Ls = ws->Lsum;
    double margin = INFINITY, m, cos_min = INFINITY;
    for (int i = 0; i < L; ++i) {
        T[i] = 1.0;
        Ls[i] = 0.0;
    }
    uint32_t p = (uint32_t)py * (uint32_t)r->width + (uint32_t)px;
    double u[4];
    philox_u(p, (uint32_t)j, 0u, SLOT_CAMERA, r, u);
    double o[3], d[3];
    orc_camera_ray(r, px + u[0], py + u[1], o, d);
    int excl_prim = -1, excl_obj = -1, prev_specular = 1;
    if (first_prim)
        *first_prim = -1;

    for (int b = 1; b <= r->max_depth; ++b) {
        orc_hit h;
        ws->seg_ext++;
        int hit = orc_trace_closest(c, o, d, excl_prim, excl_obj, brute, &h, brute ? &m : NULL);
        if (brute)
            margin = fmin(margin, m);
        if (b == 1 && first_prim)
            *first_prim = hit ? h.prim : -1;
        if (!hit)
            break;
        int tri = h.prim, mat = c->mat[tri], kind = c->kind[mat];
        const double *ng = c->ng + 3 * (size_t)tri;
        double x[3] = {o[0] + h.t * d[0], o[1] + h.t * d[1], o[2] + h.t * d[2]};
        double cd = dot3(d, ng);
        double ns[3];
        for (int a = 0; a < 3; ++a)
            ns[a] = cd < 0.0 ? ng[a] : -ng[a];
        const double *mA = c->a + (size_t)mat * L, *mB = c->b + (size_t)mat * L;

        /* emission seen from the front */
        if ((kind == ORC_EMITTER || kind == ORC_DIFFUSE_EMITTER) && cd < 0.0 &&
            (!r->nee || b == 1 || prev_specular))
            for (int i = 0; i < L; ++i)
                Ls[i] += T[i] * mA[i];
        if (kind == ORC_EMITTER)
            break;

        if (kind == ORC_LAMBERT || kind == ORC_DIFFUSE_EMITTER) {
            const double *rho = kind == ORC_LAMBERT ? mA : mB;
            if (r->nee && c->n_light > 0) {
                philox_u(p, (uint32_t)j, (uint32_t)b, SLOT_LIGHT, r, u);
                int li = c->n_light - 1;
                for (int k = 0; k < c->n_light; ++k)
                    if (u[0] < (double)c->light_cdf[k]) {
                        li = k;
                        break;
                    }
                if (brute)
                    for (int k = 0; k < c->n_light; ++k)
                        margin = fmin(margin, fabs(u[0] - (double)c->light_cdf[k]));
                int lt = c->light_tri[li];
                const double *lv = c->v + 9 * (size_t)lt;
                double su = sqrt(u[1]);
                double b0 = 1.0 - su, b1 = u[2] * su, b2 = 1.0 - b0 - b1;
                double y[3], xo[3], w[3];
                for (int a = 0; a < 3; ++a) {
                    y[a] = b0 * lv[a] + b1 * lv[3 + a] + b2 * lv[6 + a];
                    xo[a] = x[a] + RAY_OFFSET * ns[a];
                    w[a] = y[a] - xo[a];
                }
                double dist = sqrt(dot3(w, w));
                for (int a = 0; a < 3; ++a)
                    w[a] /= dist;
                const double *nl = c->ng + 3 * (size_t)lt;
                double cx = dot3(ns, w), cy = -dot3(nl, w);
                if (brute)
                    margin = fmin(margin, fmin(fabs(cx), fabs(cy)));
                if (cx > 0.0 && cy > 0.0) {
                    int ncr;
                    int32_t cobj[ORC_MAX_CROSS], ctri[ORC_MAX_CROSS];
                    ws->seg_shadow++;
                    int occ = orc_trace_shadow(c, xo, w, (1.0 - SHADOW_SHORTEN) * dist, tri, brute,
                                               &ncr, cobj, ctri, brute ? &m : NULL);
                    if (brute)
                        margin = fmin(margin, m);
                    if (!occ) {
                        cos_min = fmin(cos_min, fmin(cx, cy));
                        double G = cx * cy / (dist * dist) * c->light_area;
                        const double *Le = c->a + (size_t)c->mat[lt] * L;
                        for (int i = 0; i < L; ++i) {
                            double tr = 1.0;
                            for (int q = 0; q < ncr; ++q) {
                                double R, Tt;
                                double cc = -dot3(w, c->ng + 3 * (size_t)ctri[q]);
                                slab_rt(c, r, c->mat[ctri[q]], cc, i, &R, &Tt);
                                tr *= Tt;
                            }
                            Ls[i] += T[i] * rho[i] / PI * Le[i] * G * tr;
                        }
                    }
                }
            }
            if (r->photon_map) {   /* photon mapping: indirect and caustic light from the map(s), then stop */
                pm_gather((const orc_pmap *)r->photon_map, x, ns, rho, T, Ls);
                if (r->caustic_map)
                    pm_gather((const orc_pmap *)r->caustic_map, x, ns, rho, T, Ls);
                break;
            }
            if (b == r->max_depth)
                break;
            philox_u(p, (uint32_t)j, (uint32_t)b, SLOT_BSDF, r, u);
            orc_cosine_dir(ns, u[0], u[1], d);
            for (int i = 0; i < L; ++i)
                T[i] *= rho[i];
            for (int a = 0; a < 3; ++a)
                o[a] = x[a] + RAY_OFFSET * ns[a];
            excl_prim = tri;
            excl_obj = -1;
            prev_specular = 0;
        } else if (kind == ORC_CONDUCTOR) {
            if (b == r->max_depth)
                break;
            double cosv = fabs(cd);
            for (int i = 0; i < L; ++i)
                T[i] *= orc_conductor(cosv, mA[i], mB[i]);
            for (int a = 0; a < 3; ++a) {
                d[a] = d[a] - 2.0 * cd * ng[a];
                o[a] = x[a] + RAY_OFFSET * ns[a];
            }
            excl_prim = tri;
            excl_obj = -1;
            prev_specular = 1;
        } else { /* glass slab */
            if (b == r->max_depth)
                break;
            double cosv = fabs(cd);
            float pr = orc_branch_proxy((float)cosv, L, c->a_f + (size_t)mat * L);
            philox_u(p, (uint32_t)j, (uint32_t)b, SLOT_GLASS, r, u);
            if (brute)
                margin = fmin(margin, fabs(u[0] - (double)pr));
            int reflect = u[0] < (double)pr;
            for (int i = 0; i < L; ++i) {
                double R, Tt;
                slab_rt(c, r, mat, cosv, i, &R, &Tt);
                T[i] *= reflect ? R / (double)pr : Tt / (1.0 - (double)pr);
            }
            if (reflect) {
                for (int a = 0; a < 3; ++a) {
                    d[a] = d[a] - 2.0 * cd * ng[a];
                    o[a] = x[a] + RAY_OFFSET * ns[a];
                }
                excl_prim = tri;
                excl_obj = -1;
            } else {
                for (int a = 0; a < 3; ++a)
                    o[a] = x[a] - RAY_OFFSET * ns[a];
                excl_prim = tri;
                excl_obj = c->obj[tri];
            }
            prev_specular = 1;
        }
    }
    if (margin_out)
        *margin_out = brute ? margin : NAN;
    if (cos_min_out)
        *cos_min_out = cos_min;
}

/* --------------------------------------------------------- the driver --- */
typedef struct {
    const orc_ctx *c;
    const orc_render_desc *r;
    int64_t n_pix;
    const int64_t *pix;
    double *xyz, *sample_xyz, *margin, *cos_min;
    int32_t *first_prim;
    atomic_llong next;
    atomic_llong seg_ext, seg_shadow;
    atomic_int error;
} orc_job;

static void *worker(void *arg)
{
    orc_job *jb = (orc_job *)arg;
    const orc_ctx *c = jb->c;
    const orc_render_desc *r = jb->r;
    const int L = c->L;
    orc_scratch ws;
    ws.T = (double *)malloc(sizeof(double) * (size_t)L);
    ws.Lsum = (double *)malloc(sizeof(double) * (size_t)L);
    ws.seg_ext = ws.seg_shadow = 0;
    if (!ws.T || !ws.Lsum) {
        atomic_store(&jb->error, 1);
        free(ws.T);
        free(ws.Lsum);
        return NULL;
    }
    for (;;) {
        int64_t k0 = atomic_fetch_add(&jb->next, 8);
        if (k0 >= jb->n_pix)
            break;
        int64_t k1 = k0 + 8 < jb->n_pix ? k0 + 8 : jb->n_pix;
        for (int64_t k = k0; k < k1; ++k) {
            int64_t pidx = jb->pix[k];
            int px = (int)(pidx % r->width), py = (int)(pidx / r->width);
            double acc[3] = {0.0, 0.0, 0.0};
            for (int j = 0; j < r->spp; ++j) {
                size_t si = (size_t)k * (size_t)r->spp + (size_t)j;
                int32_t fp;
                double mg, cm;
                trace_path(c, r, px, py, j, &ws, &fp, &mg, &cm);
                double X = 0.0, Y = 0.0, Z = 0.0;
                for (int i = 0; i < L; ++i) {
                    double e = c->w[i] * ws.Lsum[i];
                    X += e * c->cmf[3 * i];
                    Y += e * c->cmf[3 * i + 1];
                    Z += e * c->cmf[3 * i + 2];
                }
                acc[0] += X;
                acc[1] += Y;
                acc[2] += Z;
                if (jb->sample_xyz) {
                    jb->sample_xyz[3 * si] = X;
                    jb->sample_xyz[3 * si + 1] = Y;
                    jb->sample_xyz[3 * si + 2] = Z;
                }
                if (jb->first_prim)
                    jb->first_prim[si] = fp;
                if (jb->margin)
                    jb->margin[si] = mg;
                if (jb->cos_min)
                    jb->cos_min[si] = cm;
            }
            for (int a = 0; a < 3; ++a)
                jb->xyz[3 * k + a] = acc[a] / (double)r->spp;
        }
    }
    atomic_fetch_add(&jb->seg_ext, ws.seg_ext);
    atomic_fetch_add(&jb->seg_shadow, ws.seg_shadow);
    free(ws.T);
    free(ws.Lsum);
    return NULL;
}

int orc_render_pixels(void *ctx, const orc_render_desc *r, int64_t n_pix, const int64_t *pix,
                      double *xyz_out, double *sample_xyz, int32_t *first_prim, double *margin,
                      double *cos_min, int n_threads, int64_t *seg_out)
{
    const orc_ctx *c = (const orc_ctx *)ctx;
    if (!c || !r || r->width <= 0 || r->height <= 0 || r->spp <= 0 || r->max_depth <= 0 || n_pix < 0)
        return -1;
    for (int64_t k = 0; k < n_pix; ++k)
        if (pix[k] < 0 || pix[k] >= (int64_t)r->width * r->height)
            return -1;
    if (n_threads <= 0) {
        long nc = sysconf(_SC_NPROCESSORS_ONLN);
        n_threads = nc > 0 ? (int)nc : 1;
    }
    if (n_threads > 512)
        n_threads = 512;
    orc_job jb;
    jb.c = c;
    jb.r = r;
    jb.n_pix = n_pix;
    jb.pix = pix;
    jb.xyz = xyz_out;
    jb.sample_xyz = sample_xyz;
    jb.first_prim = first_prim;
    jb.margin = margin;
    jb.cos_min = cos_min;
    atomic_init(&jb.next, 0);
    atomic_init(&jb.seg_ext, 0);
    atomic_init(&jb.seg_shadow, 0);
    atomic_init(&jb.error, 0);
    pthread_t th[512];
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, worker, &jb) != 0)
            break;
        ++started;
    }
    if (started == 0)
        worker(&jb);
    for (int t = 0; t < started; ++t)
        pthread_join(th[t], NULL);
    if (seg_out) {
        seg_out[0] += atomic_load(&jb.seg_ext);
        seg_out[1] += atomic_load(&jb.seg_shadow);
    }
    return atomic_load(&jb.error) ? -2 : 0;
}

/* ------------------------------------------------------ query hooks --- */
int orc_closest_hit(void *ctx, const double o[3], const double d[3], int brute_force,
                    double *t_out, double b_out[3])
{
    orc_hit h;
    int hit = orc_trace_closest((const orc_ctx *)ctx, o, d, -1, -1, brute_force, &h, NULL);
    if (!hit)
        return -1;
    *t_out = h.t;
    for (int a = 0; a < 3; ++a)
        b_out[a] = h.b[a];
    return h.prim;
}

int orc_shadow(void *ctx, const double o[3], const double d[3], double tmax, int excl_prim,
               int brute_force, int *n_cross, int32_t cross_obj[4], double cross_cos[4])
{
    const orc_ctx *c = (const orc_ctx *)ctx;
    int32_t ctri[ORC_MAX_CROSS];
    int occ = orc_trace_shadow(c, o, d, tmax, excl_prim, brute_force, n_cross, cross_obj, ctri, NULL);
    for (int q = 0; q < *n_cross; ++q)
        cross_cos[q] = -dot3(d, c->ng + 3 * (size_t)ctri[q]);
    return occ;
}
