// Photon pass of photon mapping (Sec. 4: photons launched from the light
// sources are stored where they hit objects, then the indirect light at a
// camera vertex is estimated from the stored photons). Photons leave the area
// lights (triangle by area, uniform point, cosine direction from the front
// face, power pi Le A / N each), follow the interactions paths follow
// (diffuse bounce, conductor mirror, glass branch with the same branch
// probability and weights) for at most max_depth - 1 hits over the global
// BVH, and are stored at each diffuse hit once a diffuse bounce or a
// reflection has changed their direction: light arriving straight, through
// glass or not, is the camera pass's next-event light. Random numbers:
// Philox counter (photon, 0xffffffff, hit, slot), key (seed, render id).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "photon.cuh"
#include "sddm_photon.h"

namespace sddm {
namespace {

template <bool FILMS>
__global__ void __launch_bounds__(128) k_photon_trace(DevScene sc, PhotonTraceArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_photons || sc.n_light == 0) return;
    const int L = sc.L, D = a.max_depth;
    const uint32_t pi = (uint32_t)i, pj = 0xffffffffu;
    uint4 xl = philox4x32_10(make_uint4(pi, pj, 0u, kSlotLight), a.seed, a.render_id);
    const float ua = u01(xl.x), su = sqrtf(u01(xl.y)), u2 = u01(xl.z);
    int li = sc.n_light - 1;
    for (int q = 0; q < sc.n_light; ++q)
        if (ua < __ldg(sc.light_cdf + q)) { li = q; break; }
    const float4 lv0 = __ldg(sc.light_v + 3 * li), lv1 = __ldg(sc.light_v + 3 * li + 1),
                 lv2 = __ldg(sc.light_v + 3 * li + 2);
    const int lt = __float_as_int(lv0.w);
    const float4 ln = __ldg(sc.tri_n + lt);
    const V3 nl = xyz(ln);
    const float b0 = 1.0f - su, b1 = u2 * su, b2 = 1.0f - b0 - b1;
    V3 o = b0 * xyz(lv0) + b1 * xyz(lv1) + b2 * xyz(lv2) + kRayOffset * nl;
    uint4 xd = philox4x32_10(make_uint4(pi, pj, 0u, kSlotBsdf), a.seed, a.render_id);
    V3 d = cosine_dir(nl, u01(xd.x), u01(xd.y));
    float *Phi = a.scratch + (size_t)i * L;   // the photon's power, [L]
    const float *Le = sc.mat_a + (size_t)__float_as_int(ln.w) * L;
    const float scale = 3.14159265358979f * sc.light_area / (float)a.n_photons;
    for (int l = 0; l < L; ++l) Phi[l] = __ldg(Le + l) * scale;
    int excl_prim = lt, excl_obj = -1;
    bool changed = false, diffuse = false;   // turned at all / by a diffuse bounce
    unsigned long long segs = 0;
    for (int b = 1; b <= D - 1; ++b) {
        const Ray ray = make_ray(o, d);
        ++segs;
        const Hit h = trace_closest(sc.g_nodes, sc.g_tris, 0, ray, 0.0f, __int_as_float(0x7f800000), excl_prim,
                                    excl_obj);
        if (h.prim < 0) break;
        const float4 tn = __ldg(sc.tri_n + h.prim);
        const V3 ng = xyz(tn);
        const int mat = __float_as_int(tn.w), kind = __ldg(sc.mat_kind + mat);
        const V3 x = o + h.t * d;
        const float cd = dot(d, ng);
        const V3 ns = cd < 0.0f ? ng : (-1.0f) * ng;
        const float *mA = sc.mat_a + (size_t)mat * L, *mB = sc.mat_b + (size_t)mat * L;
        if (kind == kEmitter) break;
        if (kind == kLambert || kind == kDiffuseEmitter) {
            if (changed) {
                const size_t slot = (size_t)i * (D - 1) + (b - 1);
                // w: 1 global photon, 2 caustic photon (only reflections turned it)
                a.pos[slot] = make_float4(x.x, x.y, x.z, diffuse ? 1.0f : 2.0f);
                a.dir[slot] = make_float4(d.x, d.y, d.z, 0.0f);
                float *pw = a.pow + slot * L;
                for (int l = 0; l < L; ++l) pw[l] = Phi[l];
            }
            if (b == D - 1) break;
            const float *rho = kind == kLambert ? mA : mB;
            uint4 xb = philox4x32_10(make_uint4(pi, pj, (uint32_t)b, kSlotBsdf), a.seed, a.render_id);
            d = cosine_dir(ns, u01(xb.x), u01(xb.y));
            for (int l = 0; l < L; ++l) Phi[l] *= __ldg(rho + l);
            o = x + kRayOffset * ns;
            excl_prim = h.prim;
            excl_obj = -1;
            changed = true;
            diffuse = true;
        } else if (kind == kConductor) {
            if (b == D - 1) break;
            const float c = fabsf(cd);
            for (int l = 0; l < L; ++l) Phi[l] *= conductor_F(c, __ldg(mA + l), __ldg(mB + l));
            d = d - (2.0f * cd) * ng;
            o = x + kRayOffset * ns;
            excl_prim = h.prim;
            excl_obj = -1;
            changed = true;
        } else {   // glass slab
            if (b == D - 1) break;
            const float c = fabsf(cd);
            const float pr = branch_proxy(c, L, mA);
            uint4 xg = philox4x32_10(make_uint4(pi, pj, (uint32_t)b, kSlotGlass), a.seed, a.render_id);
            const bool reflect = u01(xg.x) < pr;
            const float s = a.state_s ? __ldg(a.state_s + mat) : 0.0f;
            const float th = __ldg(sc.mat_thick + mat);
            const float wsel = reflect ? 1.0f / pr : 1.0f / (1.0f - pr);
            for (int l = 0; l < L; ++l) {
                float R_, T_;
                glass_rt<FILMS>(sc, mat, l, c, s, th, R_, T_);
                Phi[l] *= (reflect ? R_ : T_) * wsel;
            }
            if (reflect) {
                d = d - (2.0f * cd) * ng;
                o = x + kRayOffset * ns;
                excl_obj = -1;
                changed = true;
            } else {
                o = x - kRayOffset * ns;
                excl_obj = __ldg(sc.tri_obj + h.prim);
            }
            excl_prim = h.prim;
        }
    }
    for (int off = 16; off > 0; off >>= 1) segs += __shfl_down_sync(__activemask(), segs, off);
    if ((threadIdx.x & 31) == 0 && a.segments) atomicAdd(a.segments, segs);
}

__device__ __forceinline__ int pm_cell_of(const PhotonGridView &g, float4 p) {
    const float xx[3] = {p.x, p.y, p.z};
    int c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = min(g.dims[k] - 1, max(0, (int)floorf((xx[k] - g.lo[k]) / g.cell)));
    return (c[2] * g.dims[1] + c[1]) * g.dims[0] + c[0];
}

// Stored photons of the wanted kind: 0 any, 1 global, 2 caustic.
__device__ __forceinline__ bool pm_keep(float w, int kind) { return w != 0.0f && (kind == 0 || w == (float)kind); }

__global__ void k_pm_count(PhotonGridView g, int64_t slots, int kind, int *cnt, unsigned long long *stored) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = false;
    if (s < slots) {
        const float4 p = g.pos[s];
        if (pm_keep(p.w, kind)) {
            atomicAdd(cnt + pm_cell_of(g, p), 1);
            ok = true;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, ok);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(stored, (unsigned long long)__popc(m));
}

__global__ void k_pm_scatter(PhotonGridView g, int64_t slots, int kind, const int *start, int *fill, int *order) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= slots) return;
    const float4 p = g.pos[s];
    if (!pm_keep(p.w, kind)) return;
    const int c = pm_cell_of(g, p);
    order[start[c] + atomicAdd(fill + c, 1)] = (int)s;
}

// Exclusive scan of n ints in three passes: per-block sums of 1024 entries,
// one block scanning those sums, then each block's entries.
constexpr int kScanTile = 1024;
__global__ void k_scan_sums(const int *in, int64_t n, int *sums) {
    __shared__ int s_w[8];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int v = 0;
    for (int k = threadIdx.x; k < kScanTile; k += 256)
        if (base + k < n) v += in[base + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_top(int *sums, int nb, int *total) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int b = 0; b < nb; ++b) {
        const int v = sums[b];
        sums[b] = run;
        run += v;
    }
    *total = run;
}

__global__ void k_scan_apply(const int *in, int64_t n, const int *sums, int *out) {
    __shared__ int s_v[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int k = threadIdx.x; k < kScanTile; k += 256) s_v[k] = base + k < n ? in[base + k] : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = sums[blockIdx.x];
        for (int k = 0; k < kScanTile; ++k) {
            const int v = s_v[k];
            s_v[k] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kScanTile; k += 256)
        if (base + k < n) out[base + k] = s_v[k];
}

}  // namespace

cudaError_t launch_photon_trace(const DevScene &sc, const PhotonTraceArgs &a, cudaStream_t s) {
    const unsigned nb = (unsigned)((a.n_photons + 127) / 128);
    if (sc.mat_nfilm)
        k_photon_trace<true><<<nb, 128, 0, s>>>(sc, a);
    else
        k_photon_trace<false><<<nb, 128, 0, s>>>(sc, a);
    return cudaGetLastError();
}

cudaError_t build_photon_grid(PhotonGridView &g, int64_t slots, int kind, int *cnt, int *start, int *fill, int *order,
                              int *scan_sums, unsigned long long *stored, cudaStream_t s) {
    const int64_t cells = (int64_t)g.dims[0] * g.dims[1] * g.dims[2];
    const unsigned ns = (unsigned)((slots + 255) / 256);
    cudaError_t e;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)cells, s)) ||
        (e = cudaMemsetAsync(fill, 0, sizeof(int) * (size_t)cells, s)) ||
        (e = cudaMemsetAsync(stored, 0, sizeof(unsigned long long), s)))
        return e;
    if (ns > 0) k_pm_count<<<ns, 256, 0, s>>>(g, slots, kind, cnt, stored);
    const int nb = (int)((cells + kScanTile - 1) / kScanTile);
    k_scan_sums<<<nb, 256, 0, s>>>(cnt, cells, scan_sums);
    k_scan_top<<<1, 32, 0, s>>>(scan_sums, nb, start + cells);
    k_scan_apply<<<nb, 256, 0, s>>>(cnt, cells, scan_sums, start);
    if (ns > 0) k_pm_scatter<<<ns, 256, 0, s>>>(g, slots, kind, start, fill, order);
    return cudaGetLastError();
}

}  // namespace sddm
