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

}  // namespace sddm
