/* Internal declarations shared by the oracle's own C files.
 * TEST INFRASTRUCTURE ONLY (see sddm_oracle.h). */
#ifndef SDDM_ORACLE_INTERNAL_H
#define SDDM_ORACLE_INTERNAL_H

#include "sddm_oracle.h"

#define ORC_MAX_L 256
#define ORC_MAX_CROSS 4
#define ORC_MAX_FILMS 10

typedef struct {
    double lo[3], hi[3];
    int left, right;   /* children, or -1 for a leaf */
    int first, count;  /* leaf range in tri_order */
} orc_node;

typedef struct {
    int L;
    double *lam, *w, *cmf;           /* [L], [L], [L*3] */
    int n_mat;
    int *kind;
    double *a, *b, *c;               /* [n_mat*L] */
    float *a_f;                      /* float copy of mat_a (glass real index for the proxy) */
    double *thick, *s;
    int *nlayers;                    /* [n_mat] coating films per face */
    double *ln, *lk, *ldk;           /* [n_mat*4*L] film n, k, dk */
    double *lt;                      /* [n_mat*4] film thickness, nm */
    int nt;
    double *v;                       /* [nt*9]: v0, v1, v2 */
    double *ng;                      /* [nt*3] unit geometric normal, CCW */
    int *mat, *obj;
    orc_node *nodes;
    int n_nodes;
    int *tri_order;
    int n_light;
    int *light_tri;
    float *light_cdf;                /* cumulative area fraction, rounded to float */
    double light_area;               /* total emitting area */
} orc_ctx;

/* geometry (geom.c) */
typedef struct {
    double t;
    int prim;
    double b[3];
} orc_hit;

int orc_plane(const double *v, const double o[3], const double d[3], double *t, double *u, double *w);
int orc_trace_closest(const orc_ctx *c, const double o[3], const double d[3], int excl_prim,
                      int excl_obj, int brute, orc_hit *h, double *margin);
int orc_trace_shadow(const orc_ctx *c, const double o[3], const double d[3], double tmax,
                     int excl_prim, int brute, int *n_cross, int32_t cross_obj[ORC_MAX_CROSS],
                     int32_t cross_tri[ORC_MAX_CROSS], double *margin);
int orc_build_bvh(orc_ctx *c);

#endif
