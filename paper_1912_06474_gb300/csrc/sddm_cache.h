// Device cache of subdomain BVHs under a byte budget (Sec. 5: each process
// loads subdomains up to its memory limit and unloads one when its rays have
// run out). The subdomain BVHs stay in pinned host memory; before each wave of
// the domain-decomposition trace the cells that hold rays are brought into a
// fixed device buffer, fullest cells first, least recently used cells are
// evicted, and the wave is traced in groups of cells that fit at once. Copies
// run on a stream of their own, so the loads of the next group overlap the
// trace of the current one.
//
// CellPlanner is the residency bookkeeping (host only, no CUDA calls; a CPU
// check drives it); CellCache carries out its plans on the device.
#pragma once

#include <stdint.h>

#include <functional>
#include <map>
#include <string>
#include <vector>

#include "sddm_internal.h"

#if defined(__CUDACC__)
#define SDDM_HD __host__ __device__
#else
#define SDDM_HD
#endif

namespace sddm {

// A node's child entry moved from the host arrays' numbering to the cache's:
// interior children by node_delta nodes, leaves by tri_delta triangle records.
SDDM_HD inline int relocate_child(int ch, int node_delta, int tri_delta) {
    if (ch >= 0) return ch + node_delta;
    const int v = ~ch;
    return ~((((v >> kLeafBits) + tri_delta) << kLeafBits) | (v & ((1 << kLeafBits) - 1)));
}

struct CellPlanner {
    static constexpr int64_t kUnit = 192;   // lcm of the node (64 B) and triangle (48 B) records
    struct Load {
        int cell;
        int64_t where;                       // byte offset in the cache
        std::vector<int> evicted;            // cells whose space it takes
    };
    struct Group {
        std::vector<int> cells;              // traced together, in queue order
        std::vector<int64_t> where;          // byte offset of each of them while the group is traced
        std::vector<Load> loads;             // the group's cells that were not resident
        int64_t begin, end;                  // the group's range of the wave's sorted queue
    };
    std::vector<int64_t> node_cnt, tri_cnt;  // per cell
    int n_cells = 0;
    int64_t budget = 0;
    std::vector<int64_t> off;                // per cell: byte offset in the cache, -1 = not resident
    std::vector<int64_t> stamp;              // per cell: last use (LRU)
    std::map<int64_t, int64_t> free_;        // free ranges: offset -> bytes
    int64_t clock = 0;
    int64_t hits = 0;

    // Returns "" or the reason the budget cannot serve these cells.
    std::string init(const std::vector<int64_t> &node_cnt, const std::vector<int64_t> &tri_cnt, int64_t bytes);
    int64_t cell_bytes(int c) const;
    // Groups of one wave: cells with rays, fullest first; each group the cells
    // already resident plus every further cell that fits after evicting least
    // recently used cells outside the group. perm[0..n_cells): the order of the
    // cells in the sorted queue (group by group, cells without rays last).
    std::vector<Group> plan_wave(const std::vector<int64_t> &cell_rays, int *perm);

   private:
    bool allocate(int c, const std::vector<char> &in_group, int64_t &where, std::vector<int> &evicted);
};

}  // namespace sddm

#include <cuda_runtime.h>

namespace sddm {

struct CellCache {
    CellPlanner plan;
    // the BVHs as built: per cell a run of nodes (4 float4 each) and of
    // triangle references (3 float4 each) in the pinned host arrays, with child
    // and leaf indices absolute in those arrays
    const float4 *h_nodes = nullptr, *h_tris = nullptr;
    std::vector<int64_t> node_base, tri_base;
    float4 *d_cache = nullptr;         // the cache; a resident cell holds [off, off + bytes) of it
    int *d_root = nullptr;             // root node of each cell, relocated on load
    cudaStream_t copy_stream = nullptr;
    std::vector<int> last_use_ev;      // per cell: event after the last trace launch that read it, -1 = none
    std::vector<cudaEvent_t> events;   // pool, reused after each wave's host synchronisation
    int events_used = 0;
    // per-wave exchange with the host: bin counts in, cell order out
    int *h_cnt = nullptr;              // pinned [n_bins]
    int *h_perm = nullptr;             // pinned [n_cells]
    int *d_perm = nullptr;             // [n_cells]
    int *h_err = nullptr;              // pinned [4]: the device error word, read each wave
    // statistics of the current call
    int64_t loads = 0, bytes_loaded = 0, groups = 0;

    ~CellCache();
    void release();
    int init(const float4 *h_nodes, const float4 *h_tris, const std::vector<int64_t> &node_base,
             const std::vector<int64_t> &node_cnt, const std::vector<int64_t> &tri_base,
             const std::vector<int64_t> &tri_cnt, int64_t budget, int *d_root, int n_bins);
    // One wave: `cell_rays[c]` rays wait in cell c. Plans the groups, writes
    // the cell order to h_perm, calls before() (which sorts the wave's queue
    // in that order), then for each group loads its missing cells on the copy
    // stream and calls launch(begin, end) with the group's range of the
    // queue, on `stream` after those loads.
    int run_wave(const std::vector<int64_t> &cell_rays, cudaStream_t stream, const std::function<int()> &before,
                 const std::function<int(int64_t, int64_t)> &launch);

   private:
    int load(const CellPlanner::Load &ld);
    cudaError_t next_event(cudaEvent_t &ev, int &index);
};

}  // namespace sddm
