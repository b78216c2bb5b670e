// Device side of the subdomain cache (see sddm_cache.h): the planner's loads
// carried out on a copy stream (copy, then index relocation), and each
// group's trace launched after its loads.
#include <algorithm>
#include <cstdio>

#include "sddm_cache.h"
#include "sddm_ddm.h"

namespace sddm {
namespace {

// Rewrite the child and leaf indices of one cell's nodes, just copied into the
// cache, from the host arrays' numbering to the cache's, and point the cell's
// root at its first node there.
__global__ void k_relocate_cell(float4 *nodes, int n_nodes, int node_delta, int tri_delta, int *root, int cell,
                                int new_root) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) root[cell] = new_root;
    if (i >= n_nodes) return;
    float4 n3 = nodes[4 * (size_t)i + 3];
    n3.x = __int_as_float(relocate_child(__float_as_int(n3.x), node_delta, tri_delta));
    n3.y = __int_as_float(relocate_child(__float_as_int(n3.y), node_delta, tri_delta));
    nodes[4 * (size_t)i + 3] = n3;
}

int64_t round_up(int64_t x, int64_t u) { return (x + u - 1) / u * u; }

}  // namespace

CellCache::~CellCache() { release(); }

void CellCache::release() {
    if (d_cache) cudaFree(d_cache);
    d_cache = nullptr;
    if (d_perm) cudaFree(d_perm);
    d_perm = nullptr;
    if (h_cnt) cudaFreeHost(h_cnt);
    h_cnt = nullptr;
    if (h_perm) cudaFreeHost(h_perm);
    h_perm = nullptr;
    if (h_err) cudaFreeHost(h_err);
    h_err = nullptr;
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    events.clear();
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    plan = CellPlanner();
}

int CellCache::init(const float4 *hn, const float4 *ht, const std::vector<int64_t> &nb,
                    const std::vector<int64_t> &nc, const std::vector<int64_t> &tb, const std::vector<int64_t> &tc,
                    int64_t bytes, int *root, int n_bins) {
    release();
    const std::string why = plan.init(nc, tc, bytes);
    if (!why.empty()) {
        set_error(why);
        return SDDM_ERR_INVALID_ARG;
    }
    h_nodes = hn;
    h_tris = ht;
    node_base = nb;
    tri_base = tb;
    d_root = root;
    cudaError_t e = cudaMalloc(&d_cache, (size_t)plan.budget);
    if (e != cudaSuccess) {
        d_cache = nullptr;
        set_error("sddm_build: allocation of the subdomain cache failed");
        return SDDM_ERR_OOM;
    }
    if ((e = cudaStreamCreateWithFlags(&copy_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaMallocHost(&h_cnt, sizeof(int) * (size_t)std::max(n_bins, 1))) != cudaSuccess ||
        (e = cudaMallocHost(&h_perm, sizeof(int) * (size_t)plan.n_cells)) != cudaSuccess ||
        (e = cudaMallocHost(&h_err, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&d_perm, sizeof(int) * (size_t)plan.n_cells)) != cudaSuccess)
        return cuda_fail(e, "sddm_build: cache set-up");
    last_use_ev.assign(plan.n_cells, -1);
    return SDDM_OK;
}

cudaError_t CellCache::next_event(cudaEvent_t &ev, int &index) {
    if (events_used == (int)events.size()) {
        cudaEvent_t x;
        cudaError_t e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
        events.push_back(x);
    }
    index = events_used++;
    ev = events[index];
    return cudaSuccess;
}

int CellCache::load(const CellPlanner::Load &ld) {
    cudaError_t e;
    // the space may still be read by the trace of an earlier group
    for (int y : ld.evicted)
        if (last_use_ev[y] >= 0 && (e = cudaStreamWaitEvent(copy_stream, events[last_use_ev[y]], 0)) != cudaSuccess)
            return cuda_fail(e, "sddm_render: cache wait");
    const int c = ld.cell;
    char *base = reinterpret_cast<char *>(d_cache) + ld.where;
    const int64_t nn = plan.node_cnt[c], nt = plan.tri_cnt[c];
    const int64_t node_bytes = round_up(64 * nn, CellPlanner::kUnit);
    if ((e = cudaMemcpyAsync(base, h_nodes + 4 * node_base[c], (size_t)(64 * nn), cudaMemcpyHostToDevice,
                             copy_stream)) != cudaSuccess)
        return cuda_fail(e, "sddm_render: cache load (nodes)");
    if (nt > 0 && (e = cudaMemcpyAsync(base + node_bytes, h_tris + 3 * tri_base[c], (size_t)(48 * nt),
                                       cudaMemcpyHostToDevice, copy_stream)) != cudaSuccess)
        return cuda_fail(e, "sddm_render: cache load (triangles)");
    const int new_node = (int)(ld.where / 64), new_tri = (int)((ld.where + node_bytes) / 48);
    k_relocate_cell<<<(unsigned)std::max<int64_t>(1, (nn + 255) / 256), 256, 0, copy_stream>>>(
        reinterpret_cast<float4 *>(base), (int)nn, new_node - (int)node_base[c], new_tri - (int)tri_base[c], d_root,
        c, new_node);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "sddm_render: cache relocation");
    bytes_loaded += 64 * nn + 48 * nt;
    ++loads;
    return SDDM_OK;
}

int CellCache::run_wave(const std::vector<int64_t> &cell_rays, cudaStream_t stream, const std::function<int()> &before,
                        const std::function<int(int64_t, int64_t)> &launch) {
    // everything launched before this wave has finished (the caller synchronised)
    events_used = 0;
    std::fill(last_use_ev.begin(), last_use_ev.end(), -1);
    const std::vector<CellPlanner::Group> groups_ = plan.plan_wave(cell_rays, h_perm);
    bool any = false;
    for (int64_t r : cell_rays) any |= r > 0;
    if (any && groups_.empty()) {
        set_error("sddm_render: a subdomain does not fit the cell cache");
        return SDDM_ERR_INVALID_ARG;
    }
    const int rc0 = before();
    if (rc0 != SDDM_OK) return rc0;
    cudaError_t e;
    for (const CellPlanner::Group &gp : groups_) {
        ++groups;
        if (!gp.loads.empty()) {
            for (const CellPlanner::Load &ld : gp.loads) {
                const int rc = load(ld);
                if (rc != SDDM_OK) return rc;
            }
            cudaEvent_t ev;
            int idx;
            if ((e = next_event(ev, idx)) || (e = cudaEventRecord(ev, copy_stream)) ||
                (e = cudaStreamWaitEvent(stream, ev, 0)))
                return cuda_fail(e, "sddm_render: cache hand-off");
        }
        const int rc = launch(gp.begin, gp.end);
        if (rc != SDDM_OK) return rc;
        cudaEvent_t ev;
        int idx;
        if ((e = next_event(ev, idx)) || (e = cudaEventRecord(ev, stream)))
            return cuda_fail(e, "sddm_render: cache event");
        for (int c : gp.cells) last_use_ev[c] = idx;
    }
    return SDDM_OK;
}

}  // namespace sddm
