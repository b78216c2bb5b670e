// Photon mapping through the domain decomposition (ddm.cu, ddm_photon.cuh):
// the photon pass runs through the same per-subdomain ray queues, waves and
// trace kernel as camera paths; the camera pass gathers the map at the first
// diffuse vertex.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sddm_ddm.h"

namespace sddm {

struct DDMPhotonRun {
    DevScene sc;
    DDMScene g;
    int64_t begin, count;       // photons [begin, begin + count) of n_total
    int64_t n_total;
    int max_depth;              // photons take at most max_depth - 1 hits
    uint32_t seed, render_id;
    const float *state_s;       // [n_mat] coloration state of this render
    float4 *pos, *dir;          // [n_total * (max_depth - 1)] stored photons (pos.w = 1)
    float *pow;                 // [n_total * (max_depth - 1)][L]
    unsigned long long *counters;   // [8]: photon segments at 0, crossings at 3
    int *error_flag;
    int sm_count, blocks_per_sm;
    int64_t *launches;
};

// Trace one chunk of photons through the subdomain queues and store them.
int ddm_photon_pass(const DDMPhotonRun &run, DDMBuffers &buf, cudaStream_t stream);
// ddm_trace_chunk with a photon map (and optionally a caustic map, pmc.on)
// gathered at each path's first diffuse vertex.
int ddm_trace_chunk_pm(const DDMRun &run, const PhotonGridView &pm, const PhotonGridView &pmc, DDMBuffers &buf,
                       cudaStream_t stream);

}  // namespace sddm
