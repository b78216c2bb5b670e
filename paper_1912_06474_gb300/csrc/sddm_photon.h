// Photon map construction (photon.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sddm_internal.h"

namespace sddm {

struct PhotonTraceArgs {
    int64_t n_photons;
    int max_depth;              // photons take at most max_depth - 1 hits
    uint32_t seed, render_id;
    const float *state_s;       // [n_mat] coloration state of this render
    float *scratch;             // [n_photons][L] power in flight
    float4 *pos, *dir;          // [n_photons * (max_depth - 1)]
    float *pow;                 // [n_photons * (max_depth - 1)][L]
    unsigned long long *segments;
};
cudaError_t launch_photon_trace(const DevScene &sc, const PhotonTraceArgs &a, cudaStream_t stream);
// Sort the stored slots of one kind (0 any, 1 global, 2 caustic: pos.w) into
// the grid g (dims, lo, cell set by the caller) from the given buffers
// ([cells] counts and cursors, [cells + 1] starts, [slots] order).
cudaError_t build_photon_grid(PhotonGridView &g, int64_t slots, int kind, int *cnt, int *start, int *fill, int *order,
                              int *scan_sums, unsigned long long *stored, cudaStream_t stream);

}  // namespace sddm
