// Plain baseline: one thread per camera path over the global BVH -- the
// classical parallelisation of Sec. 5 (split the pixels, every worker sees
// the whole scene) -- computing the same estimator as the DDM path.
//
// Per path (pixel p, sample j, render r), following Sec. 4's algorithm and
// Eq. 2-3: a primary ray per pixel; at each of at most D vertices the closest
// surface; emission seen directly or through specular vertices; at Lambertian
// vertices one shadow ray toward a point on the area lights (Eq. 3's light
// sum), through glass slabs weighted by their transmittance; continuation by
// the reflection/refraction laws (cosine-distributed diffuse, Fresnel-weighted
// mirror for metals, R- or T-weighted mirror/straight branch for glass).
// Spectral values over the L bins are turned into XYZ with a compensated sum.
// With a photon map (PM) the path ends at its first diffuse vertex, after the
// emission and the next-event light there, with the photons' radiance estimate
// (Sec. 4's photon mapping for global illumination): rho / pi times the power
// of the photons within radius r that arrived on the visible side, over pi r^2.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "photon.cuh"

namespace sddm {

// Spectral throughput storage: registers for a compile-time L, local memory otherwise.
template <int LT>
struct Spectrum {
    float v[LT > 0 ? LT : kMaxL];
};

__device__ __forceinline__ float state_of(const RenderBatch &rb, int r, int mat, int n_mat) {
    return __ldg(rb.state_s + (size_t)r * n_mat + mat);
}

// Loop over the L bins: unrolled (throughput in registers) for a small
// compile-time L, a plain loop over local memory otherwise.
template <int LT, typename F>
__device__ __forceinline__ void for_bins(int L, F &&f) {
    if constexpr (LT > 0) {
#pragma unroll
        for (int i = 0; i < LT; ++i) f(i);
    } else {
#pragma unroll 1
        for (int i = 0; i < L; ++i) f(i);
    }
}

// Add sum_i wcmf_i * f(i) to acc (compensated over i).
template <int LT, typename F>
__device__ __forceinline__ void add_xyz(const DevScene &sc, int L, Kahan3 &acc, F &&f) {
    Kahan X, Y, Z;
    for_bins<LT>(L, [&](int i) {
        float e = f(i);
        const float4 w4 = __ldg(sc.wcmf + i);
        X.add(e * w4.x);
        Y.add(e * w4.y);
        Z.add(e * w4.z);
    });
    acc.add(X.s, Y.s, Z.s);
}

template <int LT, bool COUNT, bool FILMS, bool PM>
__global__ void __launch_bounds__(128) k_megakernel(MegaArgs a) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.path_count) return;
    const DevScene &sc = a.sc;
    const int L = LT > 0 ? LT : sc.L;
    const int64_t gp = a.path_begin + g;
    const int r = find_render(a.rb, gp);
    const RenderInfo &ri = a.rb.info[r];
    const int64_t local = gp - ri.path_begin;
    const uint32_t p = (uint32_t)(local / ri.spp), j = (uint32_t)(local % ri.spp);
    const int px = (int)(p % (uint32_t)ri.width), py = (int)(p / (uint32_t)ri.width);
    const uint32_t k0 = ri.seed, k1 = ri.render_id;

    uint4 x = philox4x32_10(make_uint4(p, j, 0u, kSlotCamera), k0, k1);
    V3 o, d;
    camera_ray(ri, (float)px + u01(x.x), (float)py + u01(x.y), o, d);

    Spectrum<LT> T;
    for_bins<LT>(L, [&](int i) {
        T.v[i] = 1.0f;
    });
    Kahan3 acc;
    int excl_prim = -1, excl_obj = -1;
    bool prev_specular = true;
    unsigned long long n_ext = 0, n_sh = 0, n_glass = 0;
    TravCount tc;
    int first = -1;

    for (int b = 1; b <= ri.max_depth; ++b) {
        Ray ray = make_ray(o, d);
        ++n_ext;
        Hit h = trace_closest<COUNT>(sc.g_nodes, sc.g_tris, 0, ray, 0.0f, __int_as_float(0x7f800000), excl_prim,
                                           excl_obj, &tc);
        if (b == 1) first = h.prim;
        if (h.prim < 0) break;
        const float4 tn = __ldg(sc.tri_n + h.prim);
        const V3 ng = xyz(tn);
        const int mat = __float_as_int(tn.w);
        const int kind = __ldg(sc.mat_kind + mat);
        const V3 xh = o + h.t * d;
        const float cd = dot(d, ng);
        const V3 ns = cd < 0.0f ? ng : (-1.0f) * ng;
        const float *mA = sc.mat_a + (size_t)mat * L;
        const float *mB = sc.mat_b + (size_t)mat * L;

        if ((kind == kEmitter || kind == kDiffuseEmitter) && cd < 0.0f && (!ri.nee || b == 1 || prev_specular))
            add_xyz<LT>(sc, L, acc, [&](int i) { return T.v[i] * __ldg(mA + i); });
        if (kind == kEmitter) break;

        if (kind == kLambert || kind == kDiffuseEmitter) {
            const float *rho = kind == kLambert ? mA : mB;
            if (ri.nee && sc.n_light > 0) {
                uint4 xl = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotLight), k0, k1);
                float ua = u01(xl.x), su = sqrtf(u01(xl.y)), u2 = u01(xl.z);
                int li = sc.n_light - 1;
                for (int q = 0; q < sc.n_light; ++q)
                    if (ua < __ldg(sc.light_cdf + q)) { li = q; break; }
                const float4 lv0 = __ldg(sc.light_v + 3 * li), lv1 = __ldg(sc.light_v + 3 * li + 1),
                             lv2 = __ldg(sc.light_v + 3 * li + 2);
                const float b0 = 1.0f - su, b1 = u2 * su, b2 = 1.0f - b0 - b1;
                const V3 y = b0 * xyz(lv0) + b1 * xyz(lv1) + b2 * xyz(lv2);
                const V3 xo = xh + kRayOffset * ns;
                V3 w = y - xo;
                const float dist = sqrtf(dot(w, w));
                w = (1.0f / dist) * w;
                const int lt = __float_as_int(lv0.w);
                const float4 ln = __ldg(sc.tri_n + lt);
                const float cx = dot(ns, w), cy = -dot(xyz(ln), w);
                if (cx > 0.0f && cy > 0.0f) {
                    ++n_sh;
                    Crossings cr;
                    cr.n = 0;
                    Ray sray = make_ray(xo, w);
                    bool occ = trace_shadow<COUNT>(sc.g_nodes, sc.g_tris, 0, sray, 0.0f,
                                                   (1.0f - kShadowShorten) * dist, h.prim, cr, &tc);
                    if (!occ) {
                        const float G = cx * cy / (dist * dist) * sc.light_area * (1.0f / 3.14159265358979f);
                        const float *Le = sc.mat_a + (size_t)__float_as_int(ln.w) * L;
                        float ccos[kMaxCross];
                        int cmat[kMaxCross];
                        for (int q = 0; q < cr.n; ++q) {
                            const float4 cn = __ldg(sc.tri_n + cr.tri[q]);
                            ccos[q] = -dot(w, xyz(cn));
                            cmat[q] = __float_as_int(cn.w);
                        }
                        n_glass += cr.n;
                        add_xyz<LT>(sc, L, acc, [&](int i) {
                            float tr = 1.0f;
                            for (int q = 0; q < cr.n; ++q) {
                                const int m = cmat[q];
                                float R_, T_;
                                glass_rt<FILMS>(sc, m, i, ccos[q], state_of(a.rb, r, m, sc.n_mat), __ldg(sc.mat_thick + m), R_,
                                         T_);
                                tr *= T_;
                            }
                            return T.v[i] * __ldg(rho + i) * __ldg(Le + i) * G * tr;
                        });
                    }
                }
            }
            if constexpr (PM) {
                pm_radiance_xyz(a.pm, a.pmc, xh, ns, L, rho, sc.wcmf, [&](int i) { return T.v[i]; }, acc);
                break;
            }
            if (b == ri.max_depth) break;
            uint4 xb = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotBsdf), k0, k1);
            d = cosine_dir(ns, u01(xb.x), u01(xb.y));
            for_bins<LT>(L, [&](int i) {
                T.v[i] *= __ldg(rho + i);
            });
            o = xh + kRayOffset * ns;
            excl_prim = h.prim;
            excl_obj = -1;
            prev_specular = false;
        } else if (kind == kConductor) {
            if (b == ri.max_depth) break;
            const float c = fabsf(cd);
            for_bins<LT>(L, [&](int i) {
                T.v[i] *= conductor_F(c, __ldg(mA + i), __ldg(mB + i));
            });
            d = d - (2.0f * cd) * ng;
            o = xh + kRayOffset * ns;
            excl_prim = h.prim;
            excl_obj = -1;
            prev_specular = true;
        } else {  // glass slab
            if (b == ri.max_depth) break;
            const float c = fabsf(cd);
            const float pr = branch_proxy(c, L, mA);
            uint4 xg = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotGlass), k0, k1);
            const bool reflect = u01(xg.x) < pr;
            const float s = state_of(a.rb, r, mat, sc.n_mat);
            const float th = __ldg(sc.mat_thick + mat);
            const float wsel = reflect ? 1.0f / pr : 1.0f / (1.0f - pr);
            ++n_glass;
            for_bins<LT>(L, [&](int i) {
                float R_, T_;
                glass_rt<FILMS>(sc, mat, i, c, s, th, R_, T_);
                T.v[i] *= (reflect ? R_ : T_) * wsel;
            });
            if (reflect) {
                d = d - (2.0f * cd) * ng;
                o = xh + kRayOffset * ns;
                excl_obj = -1;
            } else {
                o = xh - kRayOffset * ns;
                excl_obj = __ldg(sc.tri_obj + h.prim);
            }
            excl_prim = h.prim;
            prev_specular = true;
        }
    }
    a.sample_xyz[3 * g + 0] = acc.x.s;
    a.sample_xyz[3 * g + 1] = acc.y.s;
    a.sample_xyz[3 * g + 2] = acc.z.s;
    if (a.first_prim) a.first_prim[g] = first;
    // counters: warp-aggregated when the whole warp is here, per thread otherwise
    if (!a.counters) return;
    unsigned long long v[6] = {n_ext, n_sh, n_glass, tc.nodes, tc.tris, n_ext + n_sh};
    const int nv = COUNT ? 6 : 3;
    if (__activemask() == 0xffffffffu) {
        for (int k = 0; k < nv; ++k)
            for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
        if ((threadIdx.x & 31) != 0) return;
    }
    atomicAdd(a.counters + 0, v[0]);
    atomicAdd(a.counters + 1, v[1]);
    atomicAdd(a.counters + 2, v[2]);
    if (COUNT) {
        atomicAdd(a.counters + 5, v[3]);
        atomicAdd(a.counters + 6, v[4]);
        atomicAdd(a.counters + 7, v[5]);
    }
}

template <bool COUNT, bool FILMS, bool PM = false>
static void launch_mk(const MegaArgs &a, unsigned nb, int threads, cudaStream_t stream) {
    switch (a.sc.L) {
        case 8: k_megakernel<8, COUNT, FILMS, PM><<<nb, threads, 0, stream>>>(a); break;
        case 16: k_megakernel<16, COUNT, FILMS, PM><<<nb, threads, 0, stream>>>(a); break;
        default: k_megakernel<0, COUNT, FILMS, PM><<<nb, threads, 0, stream>>>(a); break;
    }
}

cudaError_t launch_megakernel(const MegaArgs &a, cudaStream_t stream) {
    if (a.path_count <= 0) return cudaSuccess;
    const int threads = 128;
    const int64_t blocks = (a.path_count + threads - 1) / threads;
    const unsigned nb = (unsigned)blocks;
    const bool films = a.sc.mat_nfilm != nullptr;
    if (a.pm.on)
        films ? launch_mk<false, true, true>(a, nb, threads, stream) : launch_mk<false, false, true>(a, nb, threads, stream);
    else if (a.count_traversal)
        films ? launch_mk<true, true>(a, nb, threads, stream) : launch_mk<true, false>(a, nb, threads, stream);
    else
        films ? launch_mk<false, true>(a, nb, threads, stream) : launch_mk<false, false>(a, nb, threads, stream);
    return cudaGetLastError();
}

}  // namespace sddm
