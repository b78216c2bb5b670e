// Domain-decomposition (DDM) wavefront path: data layout and launchers.
//
// Sec. 5 of the paper: the scene is split into subdomains; a ray is traced
// inside one subdomain and, when it leaves through an interface, its
// properties (origin, direction, distance travelled, what it must skip) are
// handed unchanged to the neighbouring subdomain. Here the subdomains are the
// cells of a regular grid, each with its own BVH; rays wait in per-cell queues
// and persistent thread blocks drain the queues cell by cell, so that the
// blocks working at one time share one cell's nodes and triangles in L1/L2.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sddm_internal.h"

namespace sddm {

struct CellCache;

constexpr int kMaxCells = 2048;
constexpr int kMaxBins = 2 * kMaxCells;   // queue sort key: (cell, ray kind[, direction octant])

struct DDMScene {
    int dims[3];
    float lo[3], hi[3], cell[3], inv_cell[3];
    float eps;            // slack of the per-cell acceptance window, metres
    int n_cells;
    int n_oct;            // sub-bins per (cell, kind): 64 (direction octant x entry half-cell), 8 (octant) or 1,
                          // the largest that keeps 2 n_cells n_oct <= kMaxBins
    int n_bins;           // 2 n_cells n_oct queue bins
    const float4 *nodes;  // all cells' BVH nodes
    const float4 *tris;   // all cells' triangle references
    const int *root;      // [n_cells] root node of each cell
    int64_t node_cap, tri_cap;   // node and triangle records addressable from nodes / tris
    int continue_cells;   // 1: a ray leaving a cell is carried on by the same lane (one wave per bounce)
    int handoff_waves;    // > 0: waves of neighbour-queue hand-off per bounce before a last wave in which the
                          // lane carries every remaining ray on (continue_cells 0)
    // per cell: bounding planes (x-, x+, y-, y+), (z-, z+, -, -) and the
    // neighbours across those faces (-1 outside the grid), 2 entries each
    const float4 *cell_planes;
    const int4 *cell_next;
};

// Path state of one chunk of np path slots (structure of arrays).
struct PathState {
    int64_t np;
    float *T;             // [L][np] spectral throughput
    float *acc;           // [6][np] XYZ compensated sums (s, c) x 3
    int *flags;           // [np] kFl* bits
    int *pend_mat;        // [np] material of the last vertex (weight still to apply)
    float *pend_cos;      // [np] |cos| at that vertex
    float *pend_w;        // [np] branch weight 1/P (glass), sign: + transmit, - reflect
    float *nee_G;         // [np] geometry factor of the shadow ray in flight
    int *nee_lmat;        // [np] light material of the shadow ray in flight
    int *sh_status;       // [np] 1 unoccluded, 2 occluded (written by the trace)
    int *cross_obj;       // [kMaxCross][np]
    int *cross_mat;       // [kMaxCross][np]
    float *cross_cos;     // [kMaxCross][np]
    float4 *hit0;         // [np] (x, prim)
    float4 *hit1;         // [np] (d, t)
};

constexpr int kFlExt = 1;        // extension ray in flight (hit record will be written)
constexpr int kFlShadow = 2;     // shadow ray in flight
constexpr int kFlPrevSpec = 4;   // previous vertex specular (or camera)
constexpr int kFlPend = 8;       // pend_* holds a weight to apply
constexpr int kRayShadow = 1;    // ray record flag bit
constexpr int kShadowOccluded = 2, kShadowClear = 1;

// Ray queues: rays of a wave sorted by cell (in), and the staging area the
// trace and shade kernels append to (unsorted, cell in r2.w).
struct Queues {
    int64_t cap;          // rays per buffer
    float4 *in;           // [cap][3]
    float4 *stage;        // [cap][3]
    int *cnt;             // [n_bins] rays staged per (cell, kind, octant) bin
    int *fill;            // [n_bins] scatter cursors
    int *off;             // [n_bins + 1] offsets of the sorted `in`
    unsigned long long *ctl;   // [4]: stage count, claim cursor, -, -
};

struct DDMBuffers {
    void *mem = nullptr;
    size_t bytes = 0;
    std::vector<cudaEvent_t> events;   // start/stop pairs of timed trace launches
    int events_used = 0;
    std::vector<cudaEvent_t> mlp_events;   // start/stop pairs of timed surrogate-network launches
    int mlp_events_used = 0;
    ~DDMBuffers();
    cudaError_t event_pair(cudaEvent_t &a, cudaEvent_t &b);
    cudaError_t mlp_event_pair(cudaEvent_t &a, cudaEvent_t &b);
};

struct DDMRun {
    DevScene sc;
    DDMScene g;
    RenderBatch rb;
    int64_t path_begin, path_count;
    int max_depth;
    float *sample_xyz;
    int32_t *first_prim;
    unsigned long long *counters;   // ext, shadow, glass, crossings, fallbacks, nodes, tris, visits, mlp batches,
                                    // mlp rows
    int *error_flag;
    int sm_count, blocks_per_sm;
    int64_t queue_capacity;
    int bsdf_mode;
    int time_trace, count_traversal;
    int64_t *launches;
    // learned glass model (bsdf_mode == SDDM_BSDF_MLP)
    const float *mlp_params;
    float mlp_dmin, mlp_dmax;
    uint32_t probe_key;
    // subdomain BVHs cached in device memory under a byte budget (NULL: all resident)
    CellCache *cache = nullptr;
};

// Run every bounce of one chunk of paths (asynchronous on `stream`).
int ddm_trace_chunk(const DDMRun &run, DDMBuffers &buf, cudaStream_t stream);
// Fill g.cell_planes / g.cell_next (2 * n_cells entries each, device memory
// the caller owns) from the grid's dims, lo and cell size.
cudaError_t build_cell_table(const DDMScene &g, float4 *planes, int4 *next, cudaStream_t stream);
cudaError_t check_kernel_image();

}  // namespace sddm
