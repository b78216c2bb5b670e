/*
 * FP64 CPU oracle of the spectral domain-decomposition path tracer
 * (Gbikpi-Benissan, Callet, Magoules, arXiv:1912.06474).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this code: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no source, header, table or helper with the
 * CUDA path; the two meet only in the seeded input arrays.
 *
 * What it computes, in the paper's terms:
 *   - Eq. 1: complex index n + ik feeding Fresnel's equations for metals and
 *     glass (Sec. 2), the glass as an absorbing slab with multiple internal
 *     reflections; coloration state s sets the absorption alpha + s*dalpha.
 *   - Eq. 2 estimated by Monte Carlo path tracing (Sec. 4), Eq. 3's light sum
 *     as next-event estimation toward area lights, shadow rays to the light
 *     (Sec. 4, local illumination), reflection/refraction continuation and a
 *     bounce limit (same passage).
 *   - The domain decomposition of Sec. 5 hands a ray on across interfaces with
 *     its properties unchanged, so its closest hit is that of a single global
 *     domain: the oracle traces against one global structure (FP64 median-split
 *     BVH, or brute force over all triangles).
 *
 * Every floating-point quantity is double except the glass branch proxy, which
 * decides an integer (reflect or transmit) and is therefore evaluated in the
 * kernel's precision (float, no contraction), and the inputs, which are the
 * caller's float32 arrays widened to double.
 *
 * The random stream is pinned by Philox4x32-10's published known-answer
 * vectors and statistically (tests/test_oracle_geometry.py).
 */
#ifndef SDDM_ORACLE_H
#define SDDM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_LAMBERT = 0, ORC_CONDUCTOR = 1, ORC_GLASS = 2, ORC_EMITTER = 3, ORC_DIFFUSE_EMITTER = 4 };

/* Scene as plain arrays (the caller keeps ownership; everything is copied). */
typedef struct {
    int L;
    const float *lam_nm;      /* [L] */
    const float *quad_w;      /* [L] nm */
    const float *cmf;         /* [L][3] */
    int n_mat;
    const int32_t *mat_kind;  /* [n_mat] */
    const float *mat_a;       /* [n_mat][L]: rho | n | n (glass) | Le (emitters) */
    const float *mat_b;       /* [n_mat][L]: -   | k | alpha_clear | rho (diffuse emitter) */
    const float *mat_c;       /* [n_mat][L]: -   | - | dalpha      | - */
    const float *mat_thick;   /* [n_mat] slab thickness, m */
    const float *mat_s;       /* [n_mat] default coloration state */
    int nv;
    const float *V;           /* [nv][3] */
    int nt;
    const uint32_t *F;        /* [nt][3] */
    const uint32_t *mat_id;   /* [nt] */
    const uint32_t *obj_id;   /* [nt] */
    /* thin-film coating of glass materials (both faces); NULL = none */
    const int32_t *mat_nlayers; /* [n_mat] films per face, 0..10 */
    const float *layer_n;     /* [n_mat][ORC_MAX_FILMS][L] film real index */
    const float *layer_k;     /* [n_mat][ORC_MAX_FILMS][L] film extinction at s = 0 */
    const float *layer_dk;    /* [n_mat][ORC_MAX_FILMS][L] extinction added at s = 1 (k = k + s dk) */
    const float *layer_t;     /* [n_mat][ORC_MAX_FILMS] film thickness, nm */
} orc_scene_desc;

typedef struct {
    int width, height, spp, max_depth;
    uint32_t seed, render_id;
    int nee;                  /* 1: next-event estimation on; 0: emission counted at every vertex */
    double cam_pos[3], cam_look[3], cam_up[3];
    double vfov_deg;
    double ortho_height;      /* > 0: orthographic camera of this height */
    const float *s_override;  /* [n_mat] or NULL; a negative entry keeps the default */
    int brute_force;          /* 1: test every triangle and compute decision margins */
    const void *photon_map;   /* NULL, or a photon map (orc_photon_map_build): at the first diffuse
                                 vertex the path adds next-event light and the photons' radiance
                                 estimate, then stops */
    const void *caustic_map;  /* NULL, or a second map gathered there too (with photon_map set): the
                                 caustic photons when photon_map holds the global ones */
} orc_render_desc;

/* Photon map (Sec. 4, global illumination by photon mapping). Photons leave
 * the lights (triangle by area, uniform point, cosine direction from the front
 * face, power pi Le A / N each), follow the same interactions as paths (diffuse
 * bounce, conductor mirror, glass branch) for at most max_depth - 1 hits, and
 * are stored at every diffuse hit once their direction has been changed by a
 * diffuse bounce or a reflection (light reaching a surface straight, through
 * glass or not, is next-event light). Random numbers: Philox counter (photon,
 * 0xffffffff, hit, slot), key (seed, render id). */
void *orc_photon_map_build(void *ctx, const orc_render_desc *r, int64_t n_photons, double radius, int n_threads);
/* The same photons split in two maps (Sec. 4 names global and caustic maps): a
 * stored photon is caustic when only reflections (metal, glass), no diffuse
 * bounce, changed its direction since the light; kind 0 keeps every stored
 * photon, 1 the global ones, 2 the caustic ones. */
void *orc_photon_map_build_kind(void *ctx, const orc_render_desc *r, int64_t n_photons, double radius, int kind,
                                int n_threads);
void orc_photon_map_free(void *pm);
/* Stored photons: count, and optionally positions [n][3], directions [n][3], power [n][L]. */
int64_t orc_photon_map_get(const void *pm, double *pos, double *dir, double *power);

int  orc_create(void **out, const orc_scene_desc *d);
void orc_destroy(void *ctx);

/* Mean XYZ over spp for each listed pixel (linear index y*W+x).
 * xyz_out [n_pix][3]; optional per-sample outputs (NULL to skip):
 *   sample_xyz [n_pix][spp][3], first_prim [n_pix][spp] (-1 = miss),
 *   margin [n_pix][spp] (smallest decision margin on the path; brute_force only),
 *   cos_min [n_pix][spp] (smallest cosine of a contributing shadow ray, +inf if none:
 *   the conditioning of the sample, a cosine c carrying ~1e-7/c relative error in float).
 * seg_out[0] += extension segments, seg_out[1] += shadow segments. */
int orc_render_pixels(void *ctx, const orc_render_desc *r, int64_t n_pix, const int64_t *pix,
                      double *xyz_out, double *sample_xyz, int32_t *first_prim, double *margin,
                      double *cos_min, int n_threads, int64_t *seg_out);

/* Test hooks ------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);
void orc_fresnel(double c, double n, double k, double *Rs, double *Rp);
void orc_slab(double c, double lam_nm, double n, double alpha_per_m, double thick_m,
              double *R, double *T);
/* Slab coated on both faces with J thin films (n, k, thickness in nm each):
 * one face seen from air (Ra, Ta) and from the glass (Rg, Tg), polarisation 0 = s, 1 = p. */
void orc_coated_face(double c, double lam_nm, double n_sub, int J, const double *nf, const double *kf,
                     const double *tf_nm, int pol, double *Ra, double *Ta, double *Rg, double *Tg);
void orc_coated_slab(double c, double lam_nm, double n_sub, double alpha_per_m, double thick_m, int J,
                     const double *nf, const double *kf, const double *tf_nm, double *R, double *T);
double orc_conductor(double c, double n, double k);
float orc_branch_proxy(float c, int L, const float *n);
void orc_cosine_dir(const double ns[3], double u0, double u1, double out[3]);
void orc_camera_ray(const orc_render_desc *r, double px, double py, double o[3], double d[3]);
/* Closest hit of one ray; returns the triangle id or -1; t_out, b_out[3] barycentrics. */
int orc_closest_hit(void *ctx, const double o[3], const double d[3], int brute_force,
                    double *t_out, double b_out[3]);
/* Shadow query: returns 1 if occluded; crossings (object, cos) written to cross_obj/cross_cos. */
int orc_shadow(void *ctx, const double o[3], const double d[3], double tmax, int excl_prim,
               int brute_force, int *n_cross, int32_t cross_obj[4], double cross_cos[4]);
int orc_num_lights(void *ctx);
/* Watertight ray/triangle test (Woop, Benthin, Wald 2013) in double precision:
 * 1 and *t when the line of the ray (o, d) meets triangle v[9], else 0. Pins only. */
int orc_watertight(const double *v, const double o[3], const double d[3], double *t);
/* Moller-Trumbore parameters of the same ray and triangle: 0 when parallel,
 * else 1 with t and the barycentrics (u, w) of vertices 1 and 2. */
int orc_plane(const double *v, const double o[3], const double d[3], double *t, double *u, double *w);

/* Glass surrogate network (mlp.c): 4 -> 64 -> 64 -> 64 (SiLU) -> 2, 8770 parameters. */
int orc_mlp_n_params(void);
void orc_mlp_features(double c, double lam_nm, double s, double d, double alpha, double film_absorbance,
                      double x[4]);
void orc_mlp_forward(const float *params, const double x[4], double y[2]);
void orc_mlp_rt(const float *params, const double x[4], double rt[2]);
void orc_mlp_forward_d(const double *params, const double x[4], double y[2]);
double orc_mlp_loss_grad(const float *params, int n, const double *X, const double *Tgt, double *grad);
double orc_mlp_loss_grad_d(const double *params, int n, const double *X, const double *Tgt, double *grad);

#ifdef __cplusplus
}
#endif
#endif
