/*
 * Ray/triangle geometry of the oracle, double precision.
 *
 * TEST INFRASTRUCTURE ONLY (see sddm_oracle.h).
 *
 * Sec. 4 and Sec. 5 of the paper place the cost in computing how rays interact
 * with the objects: finding the closest surface a ray meets and, for
 * the rays shot toward the lights, whether anything lies in between. The
 * oracle answers both by the plain definition:
 *   - Moller-Trumbore intersection, double sided, a hit needs t > 0 and
 *     barycentrics u >= 0, v >= 0, u + v <= 1;
 *   - closest hit = smallest t, ties to the lower triangle id, skipping the
 *     triangle the ray leaves (or the whole slab object after a transmission);
 *   - shadow query over (0, tmax]: any opaque triangle occludes; a glass
 *     triangle hit from its front (entering the convex slab) records one
 *     crossing per slab object; more than ORC_MAX_CROSS distinct slabs
 *     occlude.
 * The same answers come from brute force over every triangle or from a
 * median-split BVH; brute force also reports decision margins (how far the
 * ray is from changing its answer), used to filter rays whose answer float
 * arithmetic may legitimately flip.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle_internal.h"

static void sub3(const double *a, const double *b, double *r)
{
    r[0] = a[0] - b[0];
    r[1] = a[1] - b[1];
    r[2] = a[2] - b[2];
}

static void cross3(const double *a, const double *b, double *r)
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Ray/plane parameters of the Moller-Trumbore test: t and the barycentrics
 * (u, w) of the point where the ray meets the triangle's plane. Returns 0 when
 * the ray is parallel to the plane. */
int orc_plane(const double *v, const double o[3], const double d[3], double *t, double *u, double *w)
{
    double e1[3], e2[3], p[3], s[3], q[3];
    sub3(v + 3, v, e1);
    sub3(v + 6, v, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0)
        return 0;
    double inv = 1.0 / det;
    sub3(o, v, s);
    *u = dot3(s, p) * inv;
    cross3(s, e1, q);
    *w = dot3(d, q) * inv;
    *t = dot3(e2, q) * inv;
    return 1;
}

/* Watertight ray/triangle test of Woop, Benthin and Wald (JCGT 2013), double
 * sided, in double precision. The vertices are taken relative to the ray
 * origin and sheared so that the ray runs along +z (kz = the axis of the
 * largest |d|, kx and ky the next two in cyclic order, swapped when d[kz] < 0
 * to keep the winding); the projected triangle's signed edge functions
 * U, V, W decide: a hit needs all three >= 0 or all three <= 0 and a nonzero
 * sum, and then t = (U z_a + V z_b + W z_c) / (U + V + W) with z the sheared
 * depths. Two triangles that share an edge compute its edge function from the
 * same two projected vertices with opposite signs, so a ray cannot pass
 * between them. Returns 1 with *t for a hit of the ray's line (t of either
 * sign), else 0. The pins compare it with orc_plane; the renderer itself
 * uses orc_plane. */
int orc_watertight(const double *v, const double o[3], const double d[3], double *t)
{
    const double ad[3] = {fabs(d[0]), fabs(d[1]), fabs(d[2])};
    int kz = ad[0] >= ad[1] ? (ad[0] >= ad[2] ? 0 : 2) : (ad[1] >= ad[2] ? 1 : 2);
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) {
        int tmp = kx;
        kx = ky;
        ky = tmp;
    }
    const double sx = d[kx] / d[kz], sy = d[ky] / d[kz], sz = 1.0 / d[kz];
    double px[3], py[3], pz[3];
    for (int i = 0; i < 3; ++i) {
        double rel[3];
        sub3(v + 3 * i, o, rel);
        px[i] = rel[kx] - sx * rel[kz];
        py[i] = rel[ky] - sy * rel[kz];
        pz[i] = sz * rel[kz];
    }
    /* edge functions: U opposite vertex 0 (edge 1-2), V opposite 1, W opposite 2 */
    const double U = px[2] * py[1] - py[2] * px[1];
    const double V = px[0] * py[2] - py[0] * px[2];
    const double W = px[1] * py[0] - py[1] * px[0];
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0))
        return 0;
    const double det = U + V + W;
    if (det == 0.0)
        return 0;
    *t = (U * pz[0] + V * pz[1] + W * pz[2]) / det;
    return 1;
}

static int excluded(const orc_ctx *c, int tri, int excl_prim, int excl_obj)
{
    return tri == excl_prim || (excl_obj >= 0 && c->obj[tri] == excl_obj);
}

static int tri_hit(const orc_ctx *c, int tri, const double o[3], const double d[3], double tmax,
                   orc_hit *h)
{
    double t, u, w;
    if (!orc_plane(c->v + 9 * (size_t)tri, o, d, &t, &u, &w))
        return 0;
    if (!(t > 0.0) || t > tmax || u < 0.0 || w < 0.0 || u + w > 1.0)
        return 0;
    h->t = t;
    h->prim = tri;
    h->b[0] = 1.0 - u - w;
    h->b[1] = u;
    h->b[2] = w;
    return 1;
}

static int better(const orc_hit *a, const orc_hit *b)
{
    return a->t < b->t || (a->t == b->t && a->prim < b->prim);
}

/* ---------------------------------------------------------------- BVH --- */
typedef struct {
    double key;
    int idx;
} keyed;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key < b->key)
        return -1;
    if (a->key > b->key)
        return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static void tri_bounds(const orc_ctx *c, int tri, double lo[3], double hi[3])
{
    const double *v = c->v + 9 * (size_t)tri;
    for (int a = 0; a < 3; ++a) {
        lo[a] = fmin(v[a], fmin(v[3 + a], v[6 + a]));
        hi[a] = fmax(v[a], fmax(v[3 + a], v[6 + a]));
    }
}

static int build_rec(orc_ctx *c, keyed *scratch, int first, int count, int *n_nodes)
{
    int id = (*n_nodes)++;
    orc_node *nd = &c->nodes[id];
    for (int a = 0; a < 3; ++a) {
        nd->lo[a] = INFINITY;
        nd->hi[a] = -INFINITY;
    }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = first; i < first + count; ++i) {
        double lo[3], hi[3];
        tri_bounds(c, c->tri_order[i], lo, hi);
        for (int a = 0; a < 3; ++a) {
            nd->lo[a] = fmin(nd->lo[a], lo[a]);
            nd->hi[a] = fmax(nd->hi[a], hi[a]);
            double cen = 0.5 * (lo[a] + hi[a]);
            clo[a] = fmin(clo[a], cen);
            chi[a] = fmax(chi[a], cen);
        }
    }
    /* pad so that a ray touching the triangle set always enters the box */
    for (int a = 0; a < 3; ++a) {
        double pad = 1e-9 * (1.0 + fabs(nd->lo[a]) + fabs(nd->hi[a]));
        nd->lo[a] -= pad;
        nd->hi[a] += pad;
    }
    nd->first = first;
    nd->count = count;
    nd->left = nd->right = -1;
    if (count <= 4)
        return id;
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis])
            axis = a;
    for (int i = 0; i < count; ++i) {
        double lo[3], hi[3];
        int tri = c->tri_order[first + i];
        tri_bounds(c, tri, lo, hi);
        scratch[i].key = 0.5 * (lo[axis] + hi[axis]);
        scratch[i].idx = tri;
    }
    qsort(scratch, (size_t)count, sizeof(keyed), cmp_keyed);
    for (int i = 0; i < count; ++i)
        c->tri_order[first + i] = scratch[i].idx;
    int half = count / 2;
    int l = build_rec(c, scratch, first, half, n_nodes);
    int r = build_rec(c, scratch, first + half, count - half, n_nodes);
    nd = &c->nodes[id];
    nd->left = l;
    nd->right = r;
    return id;
}

int orc_build_bvh(orc_ctx *c)
{
    int nt = c->nt;
    c->tri_order = (int *)malloc(sizeof(int) * (size_t)(nt > 0 ? nt : 1));
    c->nodes = (orc_node *)malloc(sizeof(orc_node) * (size_t)(2 * nt + 1));
    keyed *scratch = (keyed *)malloc(sizeof(keyed) * (size_t)(nt > 0 ? nt : 1));
    if (!c->tri_order || !c->nodes || !scratch) {
        free(scratch);
        return -1;
    }
    for (int i = 0; i < nt; ++i)
        c->tri_order[i] = i;
    c->n_nodes = 0;
    if (nt > 0)
        build_rec(c, scratch, 0, nt, &c->n_nodes);
    free(scratch);
    return 0;
}

/* Slab test of the ray segment [0, tmax] against a box; *tnear = entry. */
static int box_hit(const orc_node *nd, const double o[3], const double d[3], double tmax, double *tnear)
{
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < nd->lo[a] || o[a] > nd->hi[a])
                return 0;
            continue;
        }
        double ta = (nd->lo[a] - o[a]) / d[a];
        double tb = (nd->hi[a] - o[a]) / d[a];
        if (ta > tb) {
            double x = ta;
            ta = tb;
            tb = x;
        }
        if (ta > t0)
            t0 = ta;
        if (tb < t1)
            t1 = tb;
        if (t0 > t1)
            return 0;
    }
    *tnear = t0;
    return 1;
}

/* -------------------------------------------------------- closest hit --- */
static int closest_bvh(const orc_ctx *c, const double o[3], const double d[3], int excl_prim,
                       int excl_obj, orc_hit *best)
{
    int found = 0;
    best->t = INFINITY;
    best->prim = -1;
    if (c->n_nodes == 0)
        return 0;
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_node *nd = &c->nodes[stack[--sp]];
        double tn;
        if (!box_hit(nd, o, d, found ? best->t : INFINITY, &tn))
            continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; ++i) {
                int tri = c->tri_order[i];
                orc_hit h;
                if (excluded(c, tri, excl_prim, excl_obj))
                    continue;
                if (tri_hit(c, tri, o, d, INFINITY, &h) && (!found || better(&h, best))) {
                    *best = h;
                    found = 1;
                }
            }
            continue;
        }
        double tl, tr;
        double lim = found ? best->t : INFINITY;
        int hl = box_hit(&c->nodes[nd->left], o, d, lim, &tl);
        int hr = box_hit(&c->nodes[nd->right], o, d, lim, &tr);
        if (hl && hr) {
            /* push the far child first so the near one is visited first */
            if (tl <= tr) {
                stack[sp++] = nd->right;
                stack[sp++] = nd->left;
            } else {
                stack[sp++] = nd->left;
                stack[sp++] = nd->right;
            }
        } else if (hl) {
            stack[sp++] = nd->left;
        } else if (hr) {
            stack[sp++] = nd->right;
        }
    }
    return found;
}

static int closest_brute(const orc_ctx *c, const double o[3], const double d[3], int excl_prim,
                         int excl_obj, orc_hit *best, double *margin)
{
    int found = 0;
    best->t = INFINITY;
    best->prim = -1;
    for (int tri = 0; tri < c->nt; ++tri) {
        orc_hit h;
        if (excluded(c, tri, excl_prim, excl_obj))
            continue;
        if (tri_hit(c, tri, o, d, INFINITY, &h) && (!found || better(&h, best))) {
            *best = h;
            found = 1;
        }
    }
    if (margin) {
        /* margin: barycentric distance to an edge of every triangle the ray
         * meets (or nearly meets) up to the hit, the relative gap to the next
         * hit, and the hit distance itself. */
        double m = INFINITY, t2 = INFINITY;
        for (int tri = 0; tri < c->nt; ++tri) {
            double t, u, w;
            if (excluded(c, tri, excl_prim, excl_obj))
                continue;
            if (!orc_plane(c->v + 9 * (size_t)tri, o, d, &t, &u, &w) || !(t > 0.0))
                continue;
            double beta = fmin(1.0 - u - w, fmin(u, w));
            if (!found || t <= best->t * (1.0 + 1e-6))
                m = fmin(m, fabs(beta));
            if (found && beta >= 0.0 && tri != best->prim && t < t2)
                t2 = t;
        }
        if (found) {
            m = fmin(m, best->t);
            if (t2 < INFINITY)
                m = fmin(m, (t2 - best->t) / best->t);
        }
        *margin = m;
    }
    return found;
}

int orc_trace_closest(const orc_ctx *c, const double o[3], const double d[3], int excl_prim,
                      int excl_obj, int brute, orc_hit *h, double *margin)
{
    if (brute)
        return closest_brute(c, o, d, excl_prim, excl_obj, h, margin);
    if (margin)
        *margin = NAN;
    return closest_bvh(c, o, d, excl_prim, excl_obj, h);
}

/* ------------------------------------------------------------ shadow --- */
/* Handle one triangle hit by a shadow ray. Returns 1 if it occludes. */
static int shadow_visit(const orc_ctx *c, int tri, const double d[3], int *n_cross,
                        int32_t cross_obj[ORC_MAX_CROSS], int32_t cross_tri[ORC_MAX_CROSS])
{
    if (c->kind[c->mat[tri]] != ORC_GLASS)
        return 1;
    if (dot3(d, c->ng + 3 * (size_t)tri) >= 0.0)
        return 0;                      /* leaving face of a slab: ignored */
    int ob = c->obj[tri];
    for (int i = 0; i < *n_cross; ++i)
        if (cross_obj[i] == ob)
            return 0;                  /* this slab already counted */
    if (*n_cross >= ORC_MAX_CROSS)
        return 1;
    cross_obj[*n_cross] = ob;
    cross_tri[*n_cross] = tri;
    ++*n_cross;
    return 0;
}

int orc_trace_shadow(const orc_ctx *c, const double o[3], const double d[3], double tmax,
                     int excl_prim, int brute, int *n_cross, int32_t cross_obj[ORC_MAX_CROSS],
                     int32_t cross_tri[ORC_MAX_CROSS], double *margin)
{
    *n_cross = 0;
    if (brute) {
        int occluded = 0;
        for (int tri = 0; tri < c->nt && !occluded; ++tri) {
            orc_hit h;
            if (tri == excl_prim)
                continue;
            if (tri_hit(c, tri, o, d, tmax, &h))
                occluded = shadow_visit(c, tri, d, n_cross, cross_obj, cross_tri);
        }
        if (margin) {
            double m = INFINITY;
            for (int tri = 0; tri < c->nt; ++tri) {
                double t, u, w;
                if (tri == excl_prim)
                    continue;
                if (!orc_plane(c->v + 9 * (size_t)tri, o, d, &t, &u, &w) || !(t > 0.0))
                    continue;
                if (t > tmax * (1.0 + 1e-6))
                    continue;
                double beta = fmin(1.0 - u - w, fmin(u, w));
                m = fmin(m, fabs(beta));
                if (beta >= 0.0)
                    m = fmin(m, fmin(t, fabs(t - tmax) / tmax));
            }
            *margin = m;
        }
        return occluded;
    }
    if (margin)
        *margin = NAN;
    if (c->n_nodes == 0)
        return 0;
    int stack[256];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const orc_node *nd = &c->nodes[stack[--sp]];
        double tn;
        if (!box_hit(nd, o, d, tmax, &tn))
            continue;
        if (nd->left < 0) {
            for (int i = nd->first; i < nd->first + nd->count; ++i) {
                int tri = c->tri_order[i];
                orc_hit h;
                if (tri == excl_prim)
                    continue;
                if (tri_hit(c, tri, o, d, tmax, &h) &&
                    shadow_visit(c, tri, d, n_cross, cross_obj, cross_tri))
                    return 1;
            }
            continue;
        }
        stack[sp++] = nd->left;
        stack[sp++] = nd->right;
    }
    return 0;
}
