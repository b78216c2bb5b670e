// Device building blocks of the path tracer: random stream, ray/box and
// ray/triangle tests, BVH traversal, spectral optics, sampling, compensated sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sddm_internal.h"

namespace sddm {

// ----------------------------------------------------------- vector helpers
struct V3 {
    float x, y, z;
};
__device__ __forceinline__ V3 v3(float x, float y, float z) { return V3{x, y, z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ V3 operator*(float s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ V3 normalize(V3 a) {
    float inv = 1.0f / sqrtf(dot(a, a));
    return inv * a;
}
__device__ __forceinline__ V3 xyz(float4 f) { return v3(f.x, f.y, f.z); }

// ------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two
// 32x32->64 products whose high halves are xored with the other counter words
// and the round key; the key advances by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}
// Top 24 bits as a uniform in [0, 1): exact in float.
__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------- BVH nodes
// Node = 4 float4: (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y) (c1 same) (c0.lo.z, c0.hi.z,
// c1.lo.z, c1.hi.z) (child0, child1 as int bits). child >= 0: node index;
// child < 0: leaf, ~child = (first triangle << 4) | count.
// Triangle = 3 float4: (v0, id) (v1, obj) (v2, flags): the vertices
// themselves, so that triangles sharing an edge see bit-identical endpoints.

// A ray with what its box and triangle tests need: reciprocal direction and
// origin times it (boxes), and the set-up of the watertight triangle test of
// Woop, Benthin and Wald (JCGT 2013): the axis kz along which the direction is
// largest, the other two kx, ky (swapped when d[kz] < 0, which keeps the
// winding), and the shear (sx, sy) = (d[kx], d[ky]) / d[kz] that maps the
// ray onto the +z axis of a frame centred on its origin; the scale 1 / d[kz]
// is inv[kz] (|d[kz]| >= 1/sqrt(3) for a unit direction, never clamped).
struct Ray {
    V3 o, d, inv, oi;   // oi = o * inv
    float sx, sy;
    int k;              // kx | ky << 2 | kz << 4
};
__device__ __forceinline__ float safe_inv(float d) {
    return 1.0f / (fabsf(d) > 1e-20f ? d : copysignf(1e-20f, d));
}
__device__ __forceinline__ float comp(V3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ Ray make_ray(V3 o, V3 d) {
    Ray r;
    r.o = o;
    r.d = d;
    r.inv = v3(safe_inv(d.x), safe_inv(d.y), safe_inv(d.z));
    r.oi = v3(o.x * r.inv.x, o.y * r.inv.y, o.z * r.inv.z);
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    const int kz = ax >= ay ? (ax >= az ? 0 : 2) : (ay >= az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1, ky = kx == 2 ? 0 : kx + 1;
    const float dz = comp(d, kz);
    if (dz < 0.0f) {
        const int t = kx;
        kx = ky;
        ky = t;
    }
    r.sx = comp(d, kx) / dz;
    r.sy = comp(d, ky) / dz;
    r.k = kx | (ky << 2) | (kz << 4);
    return r;
}

// Watertight ray/triangle test (Woop, Benthin, Wald 2013), double sided:
// the vertices are taken relative to the ray origin and sheared so that the
// ray runs along +z; the signed edge functions U, V, W of the projected
// triangle decide inside/outside. Each is a difference of two correctly
// rounded products, so a shared edge gives its two triangles edge functions
// of exactly opposite sign and a ray through it cannot slip between them;
// an exact zero is re-evaluated in double precision. Returns the hit
// distance, or +inf.
__device__ __forceinline__ float wt_intersect(const Ray &r, V3 p0, V3 p1, V3 p2) {
    const int kx = r.k & 3, ky = (r.k >> 2) & 3, kz = r.k >> 4;
    const V3 A = p0 - r.o, B = p1 - r.o, C = p2 - r.o;
    const float Az = comp(A, kz), Bz = comp(B, kz), Cz = comp(C, kz);
    const float Ax = fmaf(-r.sx, Az, comp(A, kx)), Ay = fmaf(-r.sy, Az, comp(A, ky));
    const float Bx = fmaf(-r.sx, Bz, comp(B, kx)), By = fmaf(-r.sy, Bz, comp(B, ky));
    const float Cx = fmaf(-r.sx, Cz, comp(C, kx)), Cy = fmaf(-r.sy, Cz, comp(C, ky));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if (fminf(U, fminf(V, W)) < 0.0f && fmaxf(U, fmaxf(V, W)) > 0.0f) return __int_as_float(0x7f800000);
    const float det = U + V + W;
    if (det == 0.0f) return __int_as_float(0x7f800000);
    const float sz = comp(r.inv, kz);
    const float T = fmaf(U, sz * Az, fmaf(V, sz * Bz, W * (sz * Cz)));
    return T / det;
}

// Slab test of both children of a node against [tmin, tmax]: hit flags and entry distances.
__device__ __forceinline__ void child_boxes(const Ray &r, float4 n0, float4 n1, float4 n2, float tmin, float tmax,
                                            float &t0, float &t1, bool &h0, bool &h1) {
    float ax0 = fmaf(n0.x, r.inv.x, -r.oi.x), ax1 = fmaf(n0.y, r.inv.x, -r.oi.x);
    float ay0 = fmaf(n0.z, r.inv.y, -r.oi.y), ay1 = fmaf(n0.w, r.inv.y, -r.oi.y);
    float az0 = fmaf(n2.x, r.inv.z, -r.oi.z), az1 = fmaf(n2.y, r.inv.z, -r.oi.z);
    float bx0 = fmaf(n1.x, r.inv.x, -r.oi.x), bx1 = fmaf(n1.y, r.inv.x, -r.oi.x);
    float by0 = fmaf(n1.z, r.inv.y, -r.oi.y), by1 = fmaf(n1.w, r.inv.y, -r.oi.y);
    float bz0 = fmaf(n2.z, r.inv.z, -r.oi.z), bz1 = fmaf(n2.w, r.inv.z, -r.oi.z);
    float alo = fmaxf(fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)), fmaxf(fminf(az0, az1), tmin));
    float ahi = fminf(fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)), fminf(fmaxf(az0, az1), tmax));
    float blo = fmaxf(fmaxf(fminf(bx0, bx1), fminf(by0, by1)), fmaxf(fminf(bz0, bz1), tmin));
    float bhi = fminf(fminf(fmaxf(bx0, bx1), fmaxf(by0, by1)), fminf(fmaxf(bz0, bz1), tmax));
    h0 = alo <= ahi;
    h1 = blo <= bhi;
    t0 = alo;
    t1 = blo;
}

struct Hit {
    float t;
    int prim;   // original triangle id, -1 = none
};

// Closest hit with t in (tmin, tmax]; ties on t go to the lower triangle id.
// excl_prim: triangle skipped; excl_obj >= 0: every triangle of that object skipped.
// The hierarchy starts at node `root` (0 for the global one).
// With COUNT, interior nodes visited and triangles tested are added to *cnt.
struct TravCount {
    unsigned long long nodes = 0, tris = 0;
};
template <bool COUNT = false>
__device__ __forceinline__ Hit trace_closest(const float4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                             int root, const Ray &r, float tmin, float tmax, int excl_prim,
                                             int excl_obj, TravCount *cnt = nullptr) {
    Hit h;
    h.t = tmax;
    h.prim = -1;
    int stack[kStackSize];
    int sp = 0;
    int node = root;
    for (;;) {
        if (node >= 0) {
            if (COUNT) ++cnt->nodes;
            float4 n0 = __ldg(nodes + 4 * node + 0);
            float4 n1 = __ldg(nodes + 4 * node + 1);
            float4 n2 = __ldg(nodes + 4 * node + 2);
            float4 n3 = __ldg(nodes + 4 * node + 3);
            float ta, tb;
            bool ha, hb;
            child_boxes(r, n0, n1, n2, tmin, h.t, ta, tb, ha, hb);
            int ca = __float_as_int(n3.x), cb = __float_as_int(n3.y);
            if (ha && hb) {
                int near = ta <= tb ? ca : cb, far = ta <= tb ? cb : ca;
                if (sp < kStackSize) stack[sp++] = far;
                node = near;
                continue;
            }
            if (ha) { node = ca; continue; }
            if (hb) { node = cb; continue; }
        } else {
            int v = ~node;
            int first = v >> kLeafBits, count = v & ((1 << kLeafBits) - 1);
            for (int i = 0; i < count; ++i) {
                const float4 *tp = tris + 3 * (first + i);
                float4 a = __ldg(tp), b = __ldg(tp + 1), c = __ldg(tp + 2);
                int id = __float_as_int(a.w);
                if (id == excl_prim || (excl_obj >= 0 && __float_as_int(b.w) == excl_obj)) continue;
                if (COUNT) ++cnt->tris;
                float t = wt_intersect(r, xyz(a), xyz(b), xyz(c));
                if (t > tmin && (t < h.t || (t == h.t && (h.prim < 0 || id < h.prim)))) {
                    h.t = t;
                    h.prim = id;
                }
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return h;
}

// Shadow query over (tmin, tmax]. Returns true if occluded. Glass triangles
// hit from their front (the ray enters the convex slab) are recorded once per
// slab object in cross_obj/cross_tri (up to kMaxCross; one more occludes);
// glass leaving faces are ignored; any other triangle occludes.
struct Crossings {
    int n;
    int obj[kMaxCross];
    int tri[kMaxCross];
};
template <bool COUNT = false>
__device__ __forceinline__ bool trace_shadow(const float4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                             int root, const Ray &r, float tmin, float tmax, int excl_prim,
                                             Crossings &cr, TravCount *cnt = nullptr) {
    int stack[kStackSize];
    int sp = 0;
    int node = root;
    for (;;) {
        if (node >= 0) {
            if (COUNT) ++cnt->nodes;
            float4 n0 = __ldg(nodes + 4 * node + 0);
            float4 n1 = __ldg(nodes + 4 * node + 1);
            float4 n2 = __ldg(nodes + 4 * node + 2);
            float4 n3 = __ldg(nodes + 4 * node + 3);
            float ta, tb;
            bool ha, hb;
            child_boxes(r, n0, n1, n2, tmin, tmax, ta, tb, ha, hb);
            int ca = __float_as_int(n3.x), cb = __float_as_int(n3.y);
            if (ha && hb) {
                if (sp < kStackSize) stack[sp++] = cb;
                node = ca;
                continue;
            }
            if (ha) { node = ca; continue; }
            if (hb) { node = cb; continue; }
        } else {
            int v = ~node;
            int first = v >> kLeafBits, count = v & ((1 << kLeafBits) - 1);
            for (int i = 0; i < count; ++i) {
                const float4 *tp = tris + 3 * (first + i);
                float4 a = __ldg(tp), b = __ldg(tp + 1), c = __ldg(tp + 2);
                int id = __float_as_int(a.w);
                if (id == excl_prim) continue;
                if (COUNT) ++cnt->tris;
                float t = wt_intersect(r, xyz(a), xyz(b), xyz(c));
                if (!(t > tmin && t <= tmax)) continue;
                if (!(__float_as_uint(c.w) & kTriGlass)) return true;
                if (dot(r.d, cross(xyz(b) - xyz(a), xyz(c) - xyz(a))) >= 0.0f) continue;   // leaving face
                int ob = __float_as_int(b.w);
                bool seen = false;
                for (int q = 0; q < cr.n; ++q) seen |= cr.obj[q] == ob;
                if (seen) continue;
                if (cr.n >= kMaxCross) return true;
                cr.obj[cr.n] = ob;
                cr.tri[cr.n] = id;
                ++cr.n;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return false;
}

// ------------------------------------------------------------------- optics
// Fresnel reflectances |r_s|^2, |r_p|^2 for light arriving from vacuum onto a
// medium of complex index n + ik (Eq. 1), cos_i = c in (0, 1], in real
// arithmetic: with a + ib = n~ cos_t, (a + ib)^2 = n^2 - k^2 - sin^2 + 2ink, so
// a b = n k, and
//   Rs = ((a - c)^2 + b^2) / ((a + c)^2 + b^2),
//   Rp = Rs ((a - q)^2 + b^2) / ((a + q)^2 + b^2),  q = sin^2 / cos.
// a or b is taken from the larger-magnitude side of the square root so that
// neither suffers cancellation (k is ~1e-5 for glass, ~1..8 for metals).
__device__ __forceinline__ void fresnel_rs_rp(float c, float n, float k, float &Rs, float &Rp) {
    const float s2 = fmaf(-c, c, 1.0f);
    const float t0 = fmaf(n, n, -fmaf(k, k, s2));
    const float nk = n * k;
    const float r = sqrtf(fmaf(t0, t0, 4.0f * nk * nk));
    float a, b;
    if (t0 >= 0.0f) {
        a = sqrtf(0.5f * (r + t0));
        b = a > 0.0f ? __fdividef(nk, a) : 0.0f;
    } else {
        b = sqrtf(0.5f * (r - t0));
        a = __fdividef(nk, b);
    }
    const float b2 = b * b;
    const float am = a - c, ap = a + c;
    Rs = __fdividef(fmaf(am, am, b2), fmaf(ap, ap, b2));
    const float q = __fdividef(s2, c);
    const float qm = a - q, qp = a + q;
    Rp = Rs * __fdividef(fmaf(qm, qm, b2), fmaf(qp, qp, b2));
}

__device__ __forceinline__ float conductor_F(float c, float n, float k) {
    if (c <= 0.0f) return 1.0f;
    c = fminf(fmaxf(c, 1e-8f), 1.0f);
    float Rs, Rp;
    fresnel_rs_rp(c, n, k, Rs, Rp);
    return 0.5f * (Rs + Rp);
}

// Absorbing plane-parallel slab (Sec. 6 evaluates glass with the Fresnel
// equations; Eq. 1 with k = alpha lambda / 4 pi): interface reflectance rho_j per
// polarisation, internal transmittance tau = exp(-alpha d / cos_t) with the
// real-index refraction angle, and the multiple-reflection sums
//   R_j = rho_j + (1 - rho_j)^2 rho_j tau^2 / (1 - rho_j^2 tau^2)
//   T_j = (1 - rho_j)^2 tau / (1 - rho_j^2 tau^2),   R, T = mean over j.
__device__ __forceinline__ void slab_RT(float c, float lam_nm, float n, float alpha, float thick, float &R,
                                        float &T) {
    if (c <= 0.0f) {
        R = 1.0f;
        T = 0.0f;
        return;
    }
    c = fminf(fmaxf(c, 1e-8f), 1.0f);
    const float k = alpha * lam_nm * (1e-9f / (4.0f * 3.14159265358979f));
    float Rs, Rp;
    fresnel_rs_rp(c, n, k, Rs, Rp);
    const float s2 = fmaf(-c, c, 1.0f);
    const float ctr = __fdividef(sqrtf(fmaf(n, n, -s2)), n);
    const float tau = __expf(-__fdividef(alpha * thick, ctr));
    const float t2 = tau * tau;
    const float ds = __frcp_rn(fmaf(-Rs * Rs, t2, 1.0f)), dp = __frcp_rn(fmaf(-Rp * Rp, t2, 1.0f));
    const float qs = (1.0f - Rs) * (1.0f - Rs), qp = (1.0f - Rp) * (1.0f - Rp);
    R = 0.5f * (fmaf(qs * Rs * t2, ds, Rs) + fmaf(qp * Rp * t2, dp, Rp));
    T = 0.5f * tau * (qs * ds + qp * dp);
}

// ---------------------------------------------------- coated glass (thin films)
// Complex numbers for the thin-film characteristic matrices.
struct Cx {
    float r, i;
};
__device__ __forceinline__ Cx cx(float r, float i = 0.0f) { return Cx{r, i}; }
__device__ __forceinline__ Cx operator+(Cx a, Cx b) { return Cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Cx operator-(Cx a, Cx b) { return Cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Cx operator*(Cx a, Cx b) { return Cx{fmaf(a.r, b.r, -a.i * b.i), fmaf(a.r, b.i, a.i * b.r)}; }
__device__ __forceinline__ Cx operator*(float s, Cx a) { return Cx{s * a.r, s * a.i}; }
__device__ __forceinline__ float cx_abs2(Cx a) { return fmaf(a.r, a.r, a.i * a.i); }
__device__ __forceinline__ Cx cx_div(Cx a, Cx b) {
    const float d = __frcp_rn(cx_abs2(b));
    return Cx{d * fmaf(a.r, b.r, a.i * b.i), d * fmaf(a.i, b.r, -a.r * b.i)};
}
__device__ __forceinline__ Cx cx_sqrt(Cx z) {   // principal root
    const float m = sqrtf(sqrtf(cx_abs2(z)));
    const float h = 0.5f * atan2f(z.i, z.r);
    float sh, ch;
    sincosf(h, &sh, &ch);
    return Cx{m * ch, m * sh};
}

// Up to kMaxFilms films per face.
constexpr int kMaxFilms = SDDM_MAX_FILMS;

// Glass coated on both faces with the same stack of J thin films (outermost
// first): each face is a coherent stack evaluated by its characteristic
// matrix (per film: complex index n + i k, cos theta = sqrt(1 - sin^2 / n^2)
// on the decaying branch, tilted admittance n cos (s) or n / cos (p), phase
// delta = 2 pi n t cos / lambda, M = [[cos d, -i sin d / eta], [-i eta sin d, cos d]]),
// from air onto the glass and from the glass out to air (films reversed);
// the thick substrate (real index, tau = exp(-alpha d / cos_t)) combines the
// faces incoherently:
//   R = R_a + T_a T_g R_g tau^2 / (1 - R_g^2 tau^2),  T = T_a T_g tau / (1 - R_g^2 tau^2),
// per polarisation, averaged.
static __device__ __noinline__ void coated_RT(float c, float lam_nm, float n_sub, float alpha, float thick, int J,
                                       const float *nf, const float *kf, const float *tf_nm, float &R, float &T) {
    if (c <= 0.0f) {
        R = 1.0f;
        T = 0.0f;
        return;
    }
    c = fminf(fmaxf(c, 1e-8f), 1.0f);
    const float s2 = fmaf(-c, c, 1.0f);
    const float ct_sub = sqrtf(fmaf(-s2, __frcp_rn(n_sub * n_sub), 1.0f));
    const float tau = expf(-alpha * thick / ct_sub), t2 = tau * tau;
    Cx N[kMaxFilms], CT[kMaxFilms], CD[kMaxFilms], SD[kMaxFilms];
    for (int j = 0; j < J; ++j) {
        N[j] = cx(nf[j], kf[j]);
        const Cx n2 = N[j] * N[j];
        Cx ct = cx_sqrt(cx(1.0f) - cx_div(cx(s2), n2));
        if ((N[j] * ct).i < 0.0f) ct = (-1.0f) * ct;
        CT[j] = ct;
        const Cx delta = (6.283185307179586f * tf_nm[j] / lam_nm) * (N[j] * ct);
        float sa, ca;
        sincosf(delta.r, &sa, &ca);
        const float ep = expf(delta.i), em = expf(-delta.i);
        const float chb = 0.5f * (ep + em), shb = 0.5f * (ep - em);
        CD[j] = cx(ca * chb, -sa * shb);   // cos(a + ib)
        SD[j] = cx(sa * chb, ca * shb);    // sin(a + ib)
    }
    float Rsum = 0.0f, Tsum = 0.0f;
    for (int pol = 0; pol < 2; ++pol) {
        const float eta0 = pol == 0 ? c : __frcp_rn(c);
        const float etas = pol == 0 ? n_sub * ct_sub : n_sub / ct_sub;
        Cx m00 = cx(1.0f), m01 = cx(0.0f), m10 = cx(0.0f), m11 = cx(1.0f);   // M_1 ... M_J
        Cx g00 = cx(1.0f), g01 = cx(0.0f), g10 = cx(0.0f), g11 = cx(1.0f);   // M_J ... M_1
        for (int j = 0; j < J; ++j) {
            const Cx eta = pol == 0 ? N[j] * CT[j] : cx_div(N[j], CT[j]);
            const Cx a = CD[j];
            const Cx b = cx_div(cx(SD[j].i, -SD[j].r), eta);   // -i sin / eta
            const Cx d = eta * cx(SD[j].i, -SD[j].r);          // -i eta sin
            Cx t00 = m00 * a + m01 * d, t01 = m00 * b + m01 * a, t10 = m10 * a + m11 * d, t11 = m10 * b + m11 * a;
            m00 = t00;
            m01 = t01;
            m10 = t10;
            m11 = t11;
            t00 = a * g00 + b * g10;
            t01 = a * g01 + b * g11;
            t10 = d * g00 + a * g10;
            t11 = d * g01 + a * g11;
            g00 = t00;
            g01 = t01;
            g10 = t10;
            g11 = t11;
        }
        const Cx B = m00 + etas * m01, C = m10 + etas * m11;
        const Cx dn = eta0 * B + C, nu = eta0 * B - C;
        const float id = __frcp_rn(cx_abs2(dn));
        const float Ra = cx_abs2(nu) * id, Ta = 4.0f * eta0 * etas * id;
        const Cx B2 = g00 + eta0 * g01, C2 = g10 + eta0 * g11;
        const Cx dn2 = etas * B2 + C2, nu2 = etas * B2 - C2;
        const float id2 = __frcp_rn(cx_abs2(dn2));
        const float Rg = cx_abs2(nu2) * id2, Tg = 4.0f * etas * eta0 * id2;
        const float den = __frcp_rn(fmaf(-Rg * Rg, t2, 1.0f));
        Rsum += fmaf(Ta * Tg * Rg * t2, den, Ra);
        Tsum += Ta * Tg * tau * den;
    }
    R = 0.5f * Rsum;
    T = 0.5f * Tsum;
}

// R, T of glass material m at wavelength bin i: the bare absorbing slab, or
// the coated slab when the material carries films (film k = k + s dk).
// Kernels are instantiated with FILMS = false for scenes without coated glass,
// which keeps the film code (and its call) out of them entirely.
template <bool FILMS = true>
__device__ __forceinline__ void glass_rt(const DevScene &sc, int m, int i, float c, float s, float thick, float &R,
                                         float &T) {
    const size_t k = (size_t)m * sc.L + i;
    const float alpha = __ldg(sc.mat_b + k) + s * __ldg(sc.mat_c + k);
    if constexpr (!FILMS) {
        slab_RT(c, __ldg(sc.lam + i), __ldg(sc.mat_a + k), alpha, thick, R, T);
    } else {
        const int J = sc.mat_nfilm ? __ldg(sc.mat_nfilm + m) : 0;
        if (J == 0) {
            slab_RT(c, __ldg(sc.lam + i), __ldg(sc.mat_a + k), alpha, thick, R, T);
            return;
        }
        float nf[kMaxFilms], kf[kMaxFilms], tf[kMaxFilms];
        for (int j = 0; j < J; ++j) {
            const size_t f = ((size_t)m * kMaxFilms + j) * sc.L + i;
            nf[j] = __ldg(sc.film_n + f);
            kf[j] = __ldg(sc.film_k + f) + s * __ldg(sc.film_dk + f);
            tf[j] = __ldg(sc.film_t + (size_t)m * kMaxFilms + j);
        }
        coated_RT(c, __ldg(sc.lam + i), __ldg(sc.mat_a + k), alpha, thick, J, nf, kf, tf, R, T);
    }
}

// Glass branch probability: clamp(mean over bins of the lossless slab
// reflectance 2 rho / (1 + rho), averaged over polarisations, 0.05, 0.95).
// It decides an integer, so it is evaluated with explicitly rounded
// operations in a fixed order (no contraction), matching a plain float
// evaluation of the same formula.
static __device__ __noinline__ float branch_proxy(float c, int L, const float *__restrict__ n) {
    float s2 = __fsub_rn(1.0f, __fmul_rn(c, c));
    float acc = 0.0f;
    for (int i = 0; i < L; ++i) {
        float ni = __ldg(n + i);
        float x = __fsub_rn(1.0f, __fdiv_rn(s2, __fmul_rn(ni, ni)));
        float rs2, rp2;
        if (x <= 0.0f) {
            rs2 = 1.0f;
            rp2 = 1.0f;
        } else {
            float ct = __fsqrt_rn(x);
            float a = __fsub_rn(c, __fmul_rn(ni, ct)), b = __fadd_rn(c, __fmul_rn(ni, ct));
            float e = __fsub_rn(__fmul_rn(ni, c), ct), f = __fadd_rn(__fmul_rn(ni, c), ct);
            float rs = __fdiv_rn(a, b), rp = __fdiv_rn(e, f);
            rs2 = __fmul_rn(rs, rs);
            rp2 = __fmul_rn(rp, rp);
        }
        float ps = __fdiv_rn(__fadd_rn(rs2, rs2), __fadd_rn(1.0f, rs2));
        float pp = __fdiv_rn(__fadd_rn(rp2, rp2), __fadd_rn(1.0f, rp2));
        acc = __fadd_rn(acc, __fmul_rn(0.5f, __fadd_rn(ps, pp)));
    }
    float m = __fdiv_rn(acc, (float)L);
    return fminf(fmaxf(m, 0.05f), 0.95f);
}

// -------------------------------------------------------------- sampling
// Cosine-distributed direction about unit ns: Malley's method on the
// Shirley-Chiu concentric disk; tangent frame of Duff et al. (JCGT 2017).
__device__ __forceinline__ V3 cosine_dir(V3 ns, float u0, float u1) {
    float a = 2.0f * u0 - 1.0f, b = 2.0f * u1 - 1.0f;
    float dx = 0.0f, dy = 0.0f;
    if (a != 0.0f || b != 0.0f) {
        float r, phi;
        if (fabsf(a) > fabsf(b)) {
            r = a;
            phi = 0.78539816339744831f * (b / a);
        } else {
            r = b;
            phi = 1.57079632679489662f - 0.78539816339744831f * (a / b);
        }
        float sp, cp;
        sincosf(phi, &sp, &cp);
        dx = r * cp;
        dy = r * sp;
    }
    float dz = sqrtf(fmaxf(0.0f, 1.0f - dx * dx - dy * dy));
    float sgn = ns.z >= 0.0f ? 1.0f : -1.0f;
    float aa = -1.0f / (sgn + ns.z);
    float bb = ns.x * ns.y * aa;
    V3 t = v3(1.0f + sgn * ns.x * ns.x * aa, sgn * bb, -sgn * ns.x);
    V3 bt = v3(bb, sgn + ns.y * ns.y * aa, -ns.y);
    return dx * t + dy * bt + dz * ns;
}

// ----------------------------------------------------- compensated sums
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};
struct Kahan3 {
    Kahan x, y, z;
    __device__ __forceinline__ void add(float a, float b, float c) {
        x.add(a);
        y.add(b);
        z.add(c);
    }
};

// ------------------------------------------------------------------ camera
__device__ __forceinline__ void camera_ray(const RenderInfo &ri, float px, float py, V3 &o, V3 &d) {
    float nx = 2.0f * px / (float)ri.width - 1.0f;
    float ny = 1.0f - 2.0f * py / (float)ri.height;
    V3 f = v3(ri.cam_f[0], ri.cam_f[1], ri.cam_f[2]);
    V3 X = v3(ri.cam_x[0], ri.cam_x[1], ri.cam_x[2]);
    V3 Y = v3(ri.cam_y[0], ri.cam_y[1], ri.cam_y[2]);
    V3 c = v3(ri.cam_o[0], ri.cam_o[1], ri.cam_o[2]);
    if (ri.ortho) {
        o = c + nx * X + ny * Y;
        d = f;
    } else {
        o = c;
        d = normalize(f + nx * X + ny * Y);
    }
}

// Render of a global path index (binary search over the batch table).
__device__ __forceinline__ int find_render(const RenderBatch &rb, int64_t g) {
    int lo = 0, hi = rb.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (rb.info[mid].path_begin <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int find_render_pixel(const RenderBatch &rb, int64_t gp) {
    int lo = 0, hi = rb.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (rb.info[mid].pixel_begin <= gp) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace sddm
