// Photon map on the device (Sec. 4, global illumination by photon mapping):
// the radiance estimate at a diffuse point from the stored photons in their
// uniform grid (PhotonGridView). Built by photon.cu, read by the camera pass
// (megakernel.cu).
#pragma once

#include "device_common.cuh"

namespace sddm {

// Calls f(slot) for every stored photon within the
// radius of x that arrived on the side ns faces; returns how many.
template <typename F>
__device__ __forceinline__ int pm_gather_visit(const PhotonGridView &pm, V3 x, V3 ns, F &&f) {
    const float xx[3] = {x.x, x.y, x.z};
    int c0[3], c1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        c0[a] = max(0, (int)floorf((xx[a] - pm.radius - pm.lo[a]) / pm.cell));
        c1[a] = min(pm.dims[a] - 1, (int)floorf((xx[a] + pm.radius - pm.lo[a]) / pm.cell));
    }
    const float r2 = pm.radius * pm.radius;
    int n = 0;
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy)
            for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                const int c = (cz * pm.dims[1] + cy) * pm.dims[0] + cx;
                const int k1 = __ldg(pm.cell_start + c + 1);
                for (int k = __ldg(pm.cell_start + c); k < k1; ++k) {
                    const int s = __ldg(pm.order + k);
                    const float4 p = __ldg(pm.pos + s);
                    const float dx = p.x - x.x, dy = p.y - x.y, dz = p.z - x.z;
                    if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) >= r2) continue;
                    const float4 dd = __ldg(pm.dir + s);
                    if (fmaf(dd.x, ns.x, fmaf(dd.y, ns.y, dd.z * ns.z)) >= 0.0f) continue;
                    f(s);
                    ++n;
                }
            }
    return n;
}

// Bins summed per walk over the gathered photons: their sums stay in registers.
constexpr int kPmChunk = 32;

// Photon-map radiance at a diffuse point (the megakernel's camera pass),
// added to acc as XYZ: per bin i,
// T(i) rho_i / pi times the power of the global map's photons within its radius
// over pi r^2, plus the caustic map's (pmc.on) over its own pi r^2. The bins
// are taken kPmChunk at a time, each chunk with its own walk over the photons,
// so that the per-bin sums live in registers rather than in a local array.
template <typename TF>
__device__ __forceinline__ void pm_radiance_xyz(const PhotonGridView &pm, const PhotonGridView &pmc, V3 x, V3 ns,
                                                int L, const float *rho, const float4 *wcmf, TF &&Tof, Kahan3 &acc) {
    const float inv_g = 1.0f / (3.14159265358979f * pm.radius * pm.radius);
    const float inv_c = pmc.on ? 1.0f / (3.14159265358979f * pmc.radius * pmc.radius) : 0.0f;
    const float norm = 1.0f / 3.14159265358979f;
    Kahan X, Y, Z;
    for (int c0 = 0; c0 < L; c0 += kPmChunk) {
        const int n = min(kPmChunk, L - c0);
        float S[kPmChunk];
#pragma unroll
        for (int k = 0; k < kPmChunk; ++k) S[k] = 0.0f;
        pm_gather_visit(pm, x, ns, [&](int slot) {
            const float *pw = pm.pow + (size_t)slot * L + c0;
#pragma unroll
            for (int k = 0; k < kPmChunk; ++k)
                if (k < n) S[k] += __ldg(pw + k);
        });
#pragma unroll
        for (int k = 0; k < kPmChunk; ++k) S[k] *= inv_g;
        if (pmc.on)
            pm_gather_visit(pmc, x, ns, [&](int slot) {
                const float *pw = pmc.pow + (size_t)slot * L + c0;
#pragma unroll
                for (int k = 0; k < kPmChunk; ++k)
                    if (k < n) S[k] = fmaf(__ldg(pw + k), inv_c, S[k]);
            });
#pragma unroll
        for (int k = 0; k < kPmChunk; ++k) {
            if (k < n) {
                const int i = c0 + k;
                const float e = Tof(i) * __ldg(rho + i) * S[k] * norm;
                const float4 w4 = __ldg(wcmf + i);
                X.add(e * w4.x);
                Y.add(e * w4.y);
                Z.add(e * w4.z);
            }
        }
    }
    acc.add(X.s, Y.s, Z.s);
}

}  // namespace sddm
