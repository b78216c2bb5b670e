// Domain-decomposition wavefront path tracer.
//
// Sec. 5 of the paper parallelises ray tracing by splitting the scene into
// subdomains; a ray handed across an interface keeps its properties
// (its direction, amplitude and angle) and the subdomain that receives it carries
// on. Each processor works on the subdomains whose rays are waiting, keeping
// their data loaded (Sec. 5, last paragraph). On one GB300 this becomes:
//
//   camera / shade kernels  --append-->  staging area (ray + destination cell)
//   scatter kernel          --sort by cell-->  queue of the wave
//   trace kernel (ddm_trace.cuh; persistent warps take runs of consecutive
//   rays, i.e. they drain the queues cell by cell): traverse the cell's own
//   BVH; a hit inside the cell's [t_cur - eps, t_exit + eps] window is final;
//   otherwise the ray is appended, with t_cur = t_exit, for the neighbouring
//   cell, through a per-warp shared-memory buffer flushed with one atomic.
//   Waves repeat until no ray is left; a ray only ever moves forward along
//   each axis, so dims.x + dims.y + dims.z - 2 waves always suffice.
//
// The closest hit found this way is the global closest hit (up to eps), so
// the estimator is the same one the megakernel computes (Sec. 4 algorithm,
// Eq. 2-3); shading is split into a per-bounce kernel over path slots whose
// spectral throughput lives in HBM as [L][paths].
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "sddm_ddm.h"
#include "sddm_cache.h"
#include "sddm_mlp.h"
#include "sddm_ddm_photon.h"
#include "photon.cuh"

namespace sddm {

DDMBuffers::~DDMBuffers() {
    if (mem) cudaFree(mem);
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaEvent_t e : mlp_events) cudaEventDestroy(e);
}

static cudaError_t next_event_pair(std::vector<cudaEvent_t> &pool, int &used, cudaEvent_t &a, cudaEvent_t &b) {
    while (pool.size() < (size_t)used + 2) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        pool.push_back(e);
    }
    a = pool[used];
    b = pool[used + 1];
    used += 2;
    return cudaSuccess;
}
cudaError_t DDMBuffers::event_pair(cudaEvent_t &a, cudaEvent_t &b) { return next_event_pair(events, events_used, a, b); }
cudaError_t DDMBuffers::mlp_event_pair(cudaEvent_t &a, cudaEvent_t &b) {
    return next_event_pair(mlp_events, mlp_events_used, a, b);
}

struct KArgs {
    DevScene sc;
    DDMScene g;
    RenderBatch rb;
    PathState ps;
    Queues Q;
    int64_t path_begin;
    int b;
    int last_wave;        // rays still moving after this wave are an error
    float *sample_xyz;
    int32_t *first_prim;
    unsigned long long *counters;
    int *err;
    // glass queries gathered per bounce and evaluated (exact or learned) before shading
    int use_queries;
    float4 *queries;
    unsigned long long *n_queries;
    int64_t q_cap;
    int *pend_query;      // [np]
    int *cross_query;     // [kMaxCross][np]
    const float2 *glass_res;
    int *block_cnt;       // [gridDim] glass queries per block of path slots (count pass)
    PhotonGridView pm;    // photon map: gather at the first diffuse vertex, no continuation there
    PhotonGridView pmc;   // caustic map gathered with it (pmc.on)
    // subdomain cache: the wave's queue is sorted with the cells in this order
    // (NULL: cell order), and a trace launch takes queue range [q_begin, q_end)
    // (q_end = 0: the whole wave)
    const int *cell_perm;
    int64_t q_begin, q_end;
};

// Queue bin of a ray: its cell, its kind (extension / shadow) and, as far as
// the bin table allows, the octant of its direction and the half of the cell
// (per axis) where it enters, so that the warps draining a cell hold rays that
// descend the cell's BVH alike. r0 = (origin, t_cur), r1 = (direction, t_max).
__device__ __forceinline__ int ray_bin(const DDMScene &g, int cell, int flags, float4 r0, float4 r1) {
    const int kb = 2 * cell + (flags & kRayShadow);
    if (g.n_oct == 1) return kb;
    const int oct = (r1.x < 0.0f ? 1 : 0) + (r1.y < 0.0f ? 2 : 0) + (r1.z < 0.0f ? 4 : 0);
    if (g.n_oct == 8) return kb * 8 + oct;
    const float px = fmaf(r0.w, r1.x, r0.x), py = fmaf(r0.w, r1.y, r0.y), pz = fmaf(r0.w, r1.z, r0.z);
    const int hx = (int)floorf((px - g.lo[0]) * (2.0f * g.inv_cell[0])) & 1;
    const int hy = (int)floorf((py - g.lo[1]) * (2.0f * g.inv_cell[1])) & 1;
    const int hz = (int)floorf((pz - g.lo[2]) * (2.0f * g.inv_cell[2])) & 1;
    return (kb * 8 + oct) * 8 + hx + 2 * hy + 4 * hz;
}

// ---------------------------------------------------------------- grid
__device__ __forceinline__ bool grid_enter(const DDMScene &g, V3 o, V3 d, float tmax, float &t0, int &cell) {
    float tn = 0.0f, tf = tmax;
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0.0f) {
            if (oo[a] < g.lo[a] || oo[a] > g.hi[a]) return false;
            continue;
        }
        float inv = 1.0f / dd[a];
        float ta = (g.lo[a] - oo[a]) * inv, tb = (g.hi[a] - oo[a]) * inv;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    if (tn > tf) return false;
    int c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float p = oo[a] + tn * dd[a];
        int k = (int)floorf((p - g.lo[a]) * g.inv_cell[a]);
        c[a] = min(max(k, 0), g.dims[a] - 1);
    }
    cell = (c[2] * g.dims[1] + c[1]) * g.dims[0] + c[0];
    t0 = tn;
    return true;
}

#include "ddm_trace.cuh"

// Per-cell planes and face neighbours (one thread per cell).
__global__ void k_cell_table(DDMScene g, float4 *planes, int4 *next) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= g.n_cells) return;
    const int c[3] = {cell % g.dims[0], (cell / g.dims[0]) % g.dims[1], cell / (g.dims[0] * g.dims[1])};
    float lo[3], hi[3];
    int nb[3][2];
    for (int a = 0; a < 3; ++a) {
        lo[a] = g.lo[a] + (float)c[a] * g.cell[a];
        hi[a] = g.lo[a] + (float)(c[a] + 1) * g.cell[a];
        for (int s = 0; s < 2; ++s) {
            int cc[3] = {c[0], c[1], c[2]};
            cc[a] += s ? 1 : -1;
            nb[a][s] = (cc[a] >= 0 && cc[a] < g.dims[a]) ? (cc[2] * g.dims[1] + cc[1]) * g.dims[0] + cc[0] : -1;
        }
    }
    planes[2 * cell] = make_float4(lo[0], hi[0], lo[1], hi[1]);
    planes[2 * cell + 1] = make_float4(lo[2], hi[2], 0.0f, 0.0f);
    next[2 * cell] = make_int4(nb[0][0], nb[0][1], nb[1][0], nb[1][1]);
    next[2 * cell + 1] = make_int4(nb[2][0], nb[2][1], -1, -1);
}


// Block-aggregated append of up to two rays per thread (an extension ray e
// and a shadow ray s): one global atomic per block and call on the staging
// cursor instead of one per warp and ray, so that thousands of warps do not
// serialise on one counter. All threads of the block call it together.
struct PushSmem {
    int warp_off[32];
    unsigned long long base;
};

__device__ __forceinline__ void put_ray(const Queues &Q, unsigned long long slot, float4 r0, float4 r1, int4 r2,
                                        int *err) {
    if (slot < (unsigned long long)Q.cap) {
        float4 *dst = Q.stage + 3 * slot;
        dst[0] = r0;
        dst[1] = r1;
        dst[2] = make_float4(__int_as_float(r2.x), __int_as_float(r2.y), __int_as_float(r2.z), __int_as_float(r2.w));
    } else {
        atomicCAS(err, 0, 1);
    }
}

__device__ __forceinline__ void block_stage_push2(const Queues &Q, const DDMScene &g, PushSmem &sm, int *bins, bool we,
                                                  int ce, float4 e0,
                                                  float4 e1, int4 e2, bool ws, int cs, float4 s0, float4 s1, int4 s2,
                                                  int *err) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned me = __ballot_sync(full, we), ms = __ballot_sync(full, ws);
    if (lane == 0) sm.warp_off[w] = __popc(me) + __popc(ms);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            const int c = sm.warp_off[k];
            sm.warp_off[k] = tot;
            tot += c;
        }
        sm.base = tot ? atomicAdd(Q.ctl + 0, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
    const unsigned long long base = sm.base + (unsigned long long)sm.warp_off[w];
    __syncthreads();   // the next call rewrites warp_off and base
    if (we) {
        put_ray(Q, base + __popc(me & lt), e0, e1, e2, err);
        const int bin = ray_bin(g, ce, e2.z, e0, e1);
        const unsigned peers = __match_any_sync(me, bin);
        if (lane == __ffs(peers) - 1) atomicAdd(bins + bin, __popc(peers));
    }
    if (ws) {
        put_ray(Q, base + __popc(me) + __popc(ms & lt), s0, s1, s2, err);
        const int bin = ray_bin(g, cs, s2.z, s0, s1);
        const unsigned peers = __match_any_sync(ms, bin);
        if (lane == __ffs(peers) - 1) atomicAdd(bins + bin, __popc(peers));
    }
}

// Per-block queue-bin ray counts in shared memory (n_bins ints of
// dynamic shared memory), added to the global counts once per block.
__device__ __forceinline__ int *block_bins_init(int n_bins) {
    extern __shared__ int s_bins[];
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x) s_bins[i] = 0;
    __syncthreads();
    return s_bins;
}

__device__ __forceinline__ void block_bins_flush(const Queues &Q, const int *bins, int n_bins) {
    __syncthreads();
    for (int i = threadIdx.x; i < n_bins; i += blockDim.x)
        if (bins[i]) atomicAdd(Q.cnt + i, bins[i]);
}

// --------------------------------------------------------- camera rays
__global__ void __launch_bounds__(256) k_camera(KArgs a) {
    const int64_t np = a.ps.np;
    const int L = a.sc.L;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long n_ext = 0;
    __shared__ PushSmem psm;
    int *bins = block_bins_init(a.g.n_bins);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += stride) {   // block-uniform trips
        const int64_t q = base + threadIdx.x;
        bool want = false;
        int cell = 0;
        float4 r0 = make_float4(0, 0, 0, 0), r1 = r0;
        int4 r2 = make_int4(0, 0, 0, 0);
        if (q < np) {
            const int64_t gp = a.path_begin + q;
            const int r = find_render(a.rb, gp);
            const RenderInfo &ri = a.rb.info[r];
            const int64_t local = gp - ri.path_begin;
            const uint32_t p = (uint32_t)(local / ri.spp), j = (uint32_t)(local % ri.spp);
            const int px = (int)(p % (uint32_t)ri.width), py = (int)(p / (uint32_t)ri.width);
            uint4 x = philox4x32_10(make_uint4(p, j, 0u, kSlotCamera), ri.seed, ri.render_id);
            V3 o, d;
            camera_ray(ri, (float)px + u01(x.x), (float)py + u01(x.y), o, d);
            for (int i = 0; i < L; ++i) a.ps.T[(size_t)i * np + q] = 1.0f;
#pragma unroll
            for (int k = 0; k < 6; ++k) a.ps.acc[k * np + q] = 0.0f;
            a.ps.flags[q] = kFlExt | kFlPrevSpec;
            a.ps.sh_status[q] = 0;
            if (a.first_prim) a.first_prim[q] = -1;
            ++n_ext;
            float t0;
            if (grid_enter(a.g, o, d, __int_as_float(0x7f800000), t0, cell)) {
                want = true;
                r0 = make_float4(o.x, o.y, o.z, t0);
                r1 = make_float4(d.x, d.y, d.z, __int_as_float(0x7f800000));
                r2 = make_int4((int)q, -1, 0, cell);
            } else {
                a.ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                a.ps.hit1[q] = make_float4(d.x, d.y, d.z, 0.f);
            }
        }
        block_stage_push2(a.Q, a.g, psm, bins, want, cell, r0, r1, r2, false, 0, r0, r1, r2, a.err);
    }
    block_bins_flush(a.Q, bins, a.g.n_bins);
    block_count3(a.counters + 0, n_ext, nullptr, 0, nullptr, 0);
}

// ------------------------------------------------------ sort by cell
// Exclusive prefix of the per-cell counts into s_off (every block computes it).
// Exclusive prefix sums of the n bin counts in s_off (and the total in
// s_off[n]), the bins taken in the order of `perm` over groups of `per_cell`
// bins (NULL: index order).
__device__ void block_prefix(const int *cnt, int n, int *s_off, int *s_tmp, const int *perm = nullptr,
                             int per_cell = 1) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int per = (n + nt - 1) / nt;
    const int b0 = min(n, t * per), b1 = min(n, b0 + per);
    auto bin = [&](int i) { return perm ? __ldg(perm + i / per_cell) * per_cell + i % per_cell : i; };
    int sum = 0;
    for (int i = b0; i < b1; ++i) sum += cnt[bin(i)];
    s_tmp[t] = sum;
    __syncthreads();
    for (int off = 1; off < nt; off <<= 1) {
        int v = t >= off ? s_tmp[t - off] : 0;
        __syncthreads();
        s_tmp[t] += v;
        __syncthreads();
    }
    int run = s_tmp[t] - sum;
    for (int i = b0; i < b1; ++i) {
        const int b = bin(i);
        s_off[b] = run;
        run += cnt[b];
    }
    if (t == nt - 1) s_off[n] = s_tmp[t];
    __syncthreads();
}

// Sort the staged rays by cell. Each block bins a tile of 1024 rays in shared
// memory and reserves one range per (tile, cell) with a single global atomic.
constexpr int kScatterRaysPerThread = 4;
#ifndef SDDM_SCATTER_MINB
#define SDDM_SCATTER_MINB 4  // resident 256-thread blocks per SM the scatter is compiled for (64
                             // registers, no spills, 4 blocks instead of 3)
#endif
__global__ void __launch_bounds__(256, SDDM_SCATTER_MINB) k_scatter(KArgs a) {
    __shared__ int s_off[kMaxBins + 1];
    __shared__ int s_bin[kMaxBins];
    __shared__ int s_tmp[256];
    const Queues &Q = a.Q;
    const int n_cells = a.g.n_bins;   // bins: (cell, ray kind, octant)
    block_prefix(Q.cnt, n_cells, s_off, s_tmp, a.cell_perm, 2 * a.g.n_oct);
    int total = s_off[n_cells];
    // the per-cell counts must add up to the staged rays, within capacity
    const bool bad = (unsigned long long)total != Q.ctl[0] || (int64_t)total > Q.cap;
    if (bad) total = 0;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < n_cells; i += blockDim.x) Q.off[i] = bad ? 0 : s_off[i];
        if (threadIdx.x == 0) {
            Q.off[n_cells] = total;
            if (bad) atomicCAS(a.err, 0, 3);
        }
    }
    if (total == 0) return;
    const int tile = blockDim.x * kScatterRaysPerThread;
    for (int base = blockIdx.x * tile; base < total; base += gridDim.x * tile) {
        for (int c = threadIdx.x; c < n_cells; c += blockDim.x) s_bin[c] = 0;
        __syncthreads();
        float4 r0[kScatterRaysPerThread], r1[kScatterRaysPerThread], r2[kScatterRaysPerThread];
        int cell[kScatterRaysPerThread], rank[kScatterRaysPerThread];
#pragma unroll
        for (int k = 0; k < kScatterRaysPerThread; ++k) {
            const int i = base + k * blockDim.x + threadIdx.x;
            cell[k] = -1;
            if (i < total) {
                const float4 *src = Q.stage + 3 * (size_t)i;
                r0[k] = src[0];
                r1[k] = src[1];
                r2[k] = src[2];
                cell[k] = ray_bin(a.g, __float_as_int(r2[k].w), __float_as_int(r2[k].z), r0[k], r1[k]);
            }
            // lanes of a warp with the same bin take consecutive ranks with one
            // shared-memory atomic (neighbouring rays mostly share their bin)
            const unsigned peers = __match_any_sync(0xffffffffu, cell[k]);
            const int leader = __ffs(peers) - 1, lane = threadIdx.x & 31;
            int r = 0;
            if (lane == leader && cell[k] >= 0) r = atomicAdd(s_bin + cell[k], __popc(peers));
            r = __shfl_sync(0xffffffffu, r, leader);
            rank[k] = r + __popc(peers & ((1u << lane) - 1u));
        }
        __syncthreads();
        for (int c = threadIdx.x; c < n_cells; c += blockDim.x)
            if (s_bin[c] > 0) s_bin[c] = s_off[c] + atomicAdd(Q.fill + c, s_bin[c]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScatterRaysPerThread; ++k) {
            if (cell[k] < 0) continue;
            const int at = s_bin[cell[k]] + rank[k];
            if (at < 0 || at >= total) {   // the bin offsets must place every ray inside the wave
                if (atomicCAS(a.err, 0, 11) == 0) {
                    a.err[1] = cell[k];
                    a.err[2] = at;
                }
                continue;
            }
            float4 *dst = Q.in + 3 * (size_t)at;
            dst[0] = r0[k];
            dst[1] = r1[k];
            dst[2] = r2[k];
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- shading
__device__ __forceinline__ float st_of(const RenderBatch &rb, int r, int m, int n_mat) {
    return __ldg(rb.state_s + (size_t)r * n_mat + m);
}

// Glass evaluations of this bounce (the weight of a glass vertex pending from
// the last vertex, the slabs an unoccluded shadow ray crossed), compacted into
// a query list in path-slot order, so that the list and everything computed
// from it are the same on every run. Block i owns the contiguous slot range
// [i*chunk, (i+1)*chunk): a count pass stores each block's total, the gather
// pass offsets each block by the totals of the blocks before it. A query index
// of -1 (list full) makes the shading pass use the exact slab.
__device__ __forceinline__ int glass_query_count(const KArgs &a, int64_t q, int &pm) {
    const PathState &ps = a.ps;
    const int fl = q < ps.np ? ps.flags[q] : 0;
    int n = 0;
    pm = 0;
    if (fl & (kFlExt | kFlShadow)) {
        if (fl & kFlPend) {
            pm = ps.pend_mat[q];
            n = __ldg(a.sc.mat_kind + pm) == kGlass;
        }
        if (fl & kFlShadow) {
            const int st = ps.sh_status[q];
            if ((st & 3) == kShadowClear) n += st >> 4;
        }
    }
    return n;
}

__device__ __forceinline__ int64_t glass_chunk(int64_t np) {
    const int64_t per = (np + gridDim.x - 1) / gridDim.x;
    return (per + 255) & ~(int64_t)255;
}

// Block-wide exclusive scan of one int per thread (256 threads); returns the
// thread's exclusive prefix and the block total in *total.
__device__ __forceinline__ int block_scan256(int v, int *s_w, int *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int k = 0; k < 8; ++k) {
        const int t = s_w[k];
        before += k < w ? t : 0;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void __launch_bounds__(256) k_glass_count(KArgs a) {
    __shared__ int s_w[8];
    const int64_t np = a.ps.np, chunk = glass_chunk(np);
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < np ? lo + chunk : np;
    int sum = 0;
    for (int64_t q = lo + threadIdx.x; q < hi; q += 256) {
        int pm;
        sum += glass_query_count(a, q, pm);
    }
    int total;
    block_scan256(sum, s_w, &total);
    if (threadIdx.x == 0) a.block_cnt[blockIdx.x] = total;
}

__global__ void __launch_bounds__(256) k_glass_gather(KArgs a) {
    __shared__ int s_w[8];
    const PathState &ps = a.ps;
    const DevScene &sc = a.sc;
    const int64_t np = ps.np, chunk = glass_chunk(np);
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < np ? lo + chunk : np;
    // this block's offset: the totals of the blocks before it
    int part = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += 256) part += a.block_cnt[k];
    int before_all;
    block_scan256(part, s_w, &before_all);
    int64_t base = before_all;
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        *a.n_queries = (unsigned long long)(base + a.block_cnt[blockIdx.x]);
    for (int64_t t0 = lo; t0 < hi; t0 += 256) {
        const int64_t q = t0 + threadIdx.x;
        int pm = 0;
        const int cnt = q < hi ? glass_query_count(a, q, pm) : 0;
        int tile_total;
        const int excl = block_scan256(cnt, s_w, &tile_total);
        if (cnt > 0) {
            const int fl = ps.flags[q];
            const int n_pend = (fl & kFlPend) && __ldg(sc.mat_kind + pm) == kGlass;
            const int n_cr = cnt - n_pend;
            const int64_t gp = a.path_begin + q;
            const int r = find_render(a.rb, gp);
            int64_t idx = base + excl;
            if (n_pend) {
                const int my = idx < a.q_cap ? (int)idx : -1;
                if (my >= 0)
                    a.queries[my] = make_float4(ps.pend_cos[q], st_of(a.rb, r, pm, sc.n_mat), __ldg(sc.mat_thick + pm),
                                                __int_as_float(pm));
                a.pend_query[q] = my;
                ++idx;
            }
            for (int k = 0; k < n_cr; ++k, ++idx) {
                const int cm = ps.cross_mat[k * np + q];
                const int my = idx < a.q_cap ? (int)idx : -1;
                if (my >= 0)
                    a.queries[my] = make_float4(ps.cross_cos[k * np + q], st_of(a.rb, r, cm, sc.n_mat),
                                                __ldg(sc.mat_thick + cm), __int_as_float(cm));
                a.cross_query[k * np + q] = my;
            }
        }
        base += tile_total;
    }
}

// Spectral half of shading: resolve the previous vertex's shadow ray, apply its
// weight, add this vertex's emission, per bin, with compensated sums.
#ifndef SDDM_SHS_MINB
#define SDDM_SHS_MINB 6      // resident 256-thread blocks per SM the spectral pass is compiled for (40
                             // registers with some spills: 48 warps hide the per-bin load latency; +1.7%
                             // on the hotel bench against 4 blocks, 8 blocks -1.6%)
#endif
#ifndef SDDM_SHS_UNROLL
#define SDDM_SHS_UNROLL 2    // bins in flight per thread (8: -6%)
#endif
constexpr int kShsUnroll = SDDM_SHS_UNROLL;
template <bool FILMS>
__global__ void __launch_bounds__(256, SDDM_SHS_MINB) k_shade_spectral(KArgs a) {
    const int64_t np = a.ps.np;
    const DevScene &sc = a.sc;
    const int L = sc.L;
    const int b = a.b;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long n_glass = 0;
    const PathState &ps = a.ps;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += stride) {   // block-uniform trips
        const int64_t q = base + threadIdx.x;
        int fl = q < np ? ps.flags[q] : 0;
        if (fl & (kFlExt | kFlShadow)) {
            const int64_t gp = a.path_begin + q;
            const int r = find_render(a.rb, gp);
            const RenderInfo &ri = a.rb.info[r];

            // (1) shadow ray of the previous vertex
            bool resolve = false;
            float G = 0.f;
            const float *rho_prev = nullptr, *Le_l = nullptr;
            int ncr = 0;
            int cmat[kMaxCross];
            float ccos[kMaxCross];
            if (fl & kFlShadow) {
                const int stt = ps.sh_status[q];
                if ((stt & 3) == kShadowClear) {
                    resolve = true;
                    ncr = stt >> 4;
                    G = ps.nee_G[q];
                    Le_l = sc.mat_a + (size_t)ps.nee_lmat[q] * L;
                    const int pm = ps.pend_mat[q];
                    rho_prev = (__ldg(sc.mat_kind + pm) == kLambert ? sc.mat_a : sc.mat_b) + (size_t)pm * L;
                    for (int k = 0; k < ncr; ++k) {
                        cmat[k] = ps.cross_mat[k * np + q];
                        ccos[k] = ps.cross_cos[k * np + q];
                    }
                    n_glass += ncr;
                }
            }
            // (2) weight of the previous vertex
            const bool pend = (fl & kFlPend) != 0;
            int pm = -1, pkind = 0;
            float pcos = 0.f, pw = 0.f;
            if (pend) {
                pm = ps.pend_mat[q];
                pkind = __ldg(sc.mat_kind + pm);
                pcos = ps.pend_cos[q];
                pw = ps.pend_w[q];
            }
            // (3) the hit of this vertex
            bool emit = false;
            int prim = -1, mat = 0, kind = 0;
            V3 d = v3(0, 0, 0), ng = d;
            float cd = 0.f;
            if ((fl & kFlExt) && b <= ri.max_depth) {
                const float4 h0 = ps.hit0[q], h1 = ps.hit1[q];
                prim = __float_as_int(h0.w);
                if (prim >= 0) {
                    d = xyz(h1);
                    const float4 tn = __ldg(sc.tri_n + prim);
                    ng = xyz(tn);
                    mat = __float_as_int(tn.w);
                    kind = __ldg(sc.mat_kind + mat);
                    cd = dot(d, ng);
                    emit = (kind == kEmitter || kind == kDiffuseEmitter) && cd < 0.0f &&
                           (!ri.nee || b == 1 || (fl & kFlPrevSpec));
                }
            }
            // spectral pass over the bins: resolve, weight, emit
            const float *Le_b = sc.mat_a + (size_t)mat * L;
            const float *pA = sc.mat_a + (size_t)(pm < 0 ? 0 : pm) * L;
            const float *pB = sc.mat_b + (size_t)(pm < 0 ? 0 : pm) * L;
            const float ps_state = (pend && pkind == kGlass) ? st_of(a.rb, r, pm, sc.n_mat) : 0.f;
            const float pthick = (pend && pkind == kGlass) ? __ldg(sc.mat_thick + pm) : 0.f;
            const float pwabs = fabsf(pw);
            const bool preflect = pw < 0.0f;
            float cst[kMaxCross], cth[kMaxCross];
            int cq[kMaxCross];
            for (int k = 0; k < ncr; ++k) {
                cst[k] = st_of(a.rb, r, cmat[k], sc.n_mat);
                cth[k] = __ldg(sc.mat_thick + cmat[k]);
                cq[k] = a.use_queries ? a.cross_query[k * np + q] : -1;
            }
            const int pq = (a.use_queries && pend && pkind == kGlass) ? a.pend_query[q] : -1;
            const bool need_T = resolve || pend || emit;
            if (need_T) {
                Kahan NX, NY, NZ, EX, EY, EZ;
#pragma unroll kShsUnroll
                for (int i = 0; i < L; ++i) {
                    float t = ps.T[(size_t)i * np + q];
                    const float4 w4 = __ldg(sc.wcmf + i);
                    const float wx = w4.x, wy = w4.y, wz = w4.z;
                    if (resolve) {
                        float tr = 1.0f;
                        for (int k = 0; k < ncr; ++k) {
                            if (cq[k] >= 0) {
                                tr *= a.glass_res[(size_t)cq[k] * L + i].y;
                                continue;
                            }
                            float R_, T_;
                            glass_rt<FILMS>(sc, cmat[k], i, ccos[k], cst[k], cth[k], R_, T_);
                            tr *= T_;
                        }
                        const float c = t * __ldg(rho_prev + i) * __ldg(Le_l + i) * G * tr;
                        NX.add(c * wx);
                        NY.add(c * wy);
                        NZ.add(c * wz);
                    }
                    if (pend) {
                        float w;
                        if (pkind == kLambert) {
                            w = __ldg(pA + i);
                        } else if (pkind == kDiffuseEmitter) {
                            w = __ldg(pB + i);
                        } else if (pkind == kConductor) {
                            w = conductor_F(pcos, __ldg(pA + i), __ldg(pB + i));
                        } else if (pq >= 0) {
                            const float2 rt = a.glass_res[(size_t)pq * L + i];
                            w = (preflect ? rt.x : rt.y) * pwabs;
                        } else {
                            float R_, T_;
                            glass_rt<FILMS>(sc, pm, i, pcos, ps_state, pthick, R_, T_);
                            w = (preflect ? R_ : T_) * pwabs;
                        }
                        t *= w;
                    }
                    if (emit) {
                        const float e = t * __ldg(Le_b + i);
                        EX.add(e * wx);
                        EY.add(e * wy);
                        EZ.add(e * wz);
                    }
                    ps.T[(size_t)i * np + q] = t;
                }
                Kahan3 acc;
                acc.x.s = ps.acc[0 * np + q];
                acc.y.s = ps.acc[1 * np + q];
                acc.z.s = ps.acc[2 * np + q];
                acc.x.c = ps.acc[3 * np + q];
                acc.y.c = ps.acc[4 * np + q];
                acc.z.c = ps.acc[5 * np + q];
                if (resolve) acc.add(NX.s, NY.s, NZ.s);
                if (emit) acc.add(EX.s, EY.s, EZ.s);
                ps.acc[0 * np + q] = acc.x.s;
                ps.acc[1 * np + q] = acc.y.s;
                ps.acc[2 * np + q] = acc.z.s;
                ps.acc[3 * np + q] = acc.x.c;
                ps.acc[4 * np + q] = acc.y.c;
                ps.acc[5 * np + q] = acc.z.c;
            }
        }
    }
    // counted per warp (no block barrier at the end: warps whose paths had less
    // work leave at once instead of waiting for the block's slowest warp)
    for (int off = 16; off > 0; off >>= 1) n_glass += __shfl_down_sync(0xffffffffu, n_glass, off);
    if ((threadIdx.x & 31) == 0 && n_glass) atomicAdd(a.counters + 2, n_glass);
}

// Continuation half of shading: next-event sample toward the lights and the
// next direction at this vertex, appended to the ray staging area.
#ifndef SDDM_SHC_MINB
#define SDDM_SHC_MINB 4      // resident 256-thread blocks per SM the continuation pass is compiled for
                             // (64 registers instead of 77, 4 blocks instead of 3)
#endif
__global__ void __launch_bounds__(256, SDDM_SHC_MINB) k_shade_continue(KArgs a) {
    const int64_t np = a.ps.np;
    const DevScene &sc = a.sc;
    const int L = sc.L;
    const int b = a.b;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long n_ext = 0, n_sh = 0, n_glass = 0;
    const PathState &ps = a.ps;
    __shared__ PushSmem psm;
    int *bins = block_bins_init(a.g.n_bins);
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < np; base += stride) {   // block-uniform trips
        const int64_t q = base + threadIdx.x;
        bool want_e = false, want_s = false;
        int cell_e = 0, cell_s = 0;
        float4 e0 = make_float4(0, 0, 0, 0), e1 = e0, s0 = e0, s1 = e0;
        int4 e2 = make_int4(0, 0, 0, 0), s2 = e2;
        int fl = q < np ? ps.flags[q] : 0;
        if (fl & (kFlExt | kFlShadow)) {
            const int64_t gp = a.path_begin + q;
            const int r = find_render(a.rb, gp);
            const RenderInfo &ri = a.rb.info[r];
            const int64_t local = gp - ri.path_begin;
            const uint32_t p = (uint32_t)(local / ri.spp), j = (uint32_t)(local % ri.spp);

            // (3) the hit of this vertex
            bool has_hit = false;
            int prim = -1, mat = 0, kind = 0;
            V3 x = v3(0, 0, 0), d = x, ng = x, ns = x;
            float cd = 0.f;
            if ((fl & kFlExt) && b <= ri.max_depth) {
                const float4 h0 = ps.hit0[q], h1 = ps.hit1[q];
                prim = __float_as_int(h0.w);
                if (b == 1 && a.first_prim) a.first_prim[q] = prim;
                if (prim >= 0) {
                    has_hit = true;
                    x = xyz(h0);
                    d = xyz(h1);
                    const float4 tn = __ldg(sc.tri_n + prim);
                    ng = xyz(tn);
                    mat = __float_as_int(tn.w);
                    kind = __ldg(sc.mat_kind + mat);
                    cd = dot(d, ng);
                    ns = cd < 0.0f ? ng : (-1.0f) * ng;
                }
            }
            // (4) continue the path from this vertex
            int nfl = fl & kFlPrevSpec;
            nfl &= ~(kFlExt | kFlShadow | kFlPend);
            if (has_hit && kind != kEmitter) {
                const uint32_t k0 = ri.seed, k1 = ri.render_id;
                if (kind == kLambert || kind == kDiffuseEmitter) {
                    if (ri.nee && sc.n_light > 0) {
                        uint4 xl = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotLight), k0, k1);
                        const float ua = u01(xl.x), su = sqrtf(u01(xl.y)), u2 = u01(xl.z);
                        int li = sc.n_light - 1;
                        for (int k = 0; k < sc.n_light; ++k)
                            if (ua < __ldg(sc.light_cdf + k)) { li = k; break; }
                        const float4 lv0 = __ldg(sc.light_v + 3 * li), lv1 = __ldg(sc.light_v + 3 * li + 1),
                                     lv2 = __ldg(sc.light_v + 3 * li + 2);
                        const float b0 = 1.0f - su, b1 = u2 * su, b2 = 1.0f - b0 - b1;
                        const V3 y = b0 * xyz(lv0) + b1 * xyz(lv1) + b2 * xyz(lv2);
                        const V3 xo = x + kRayOffset * ns;
                        V3 w = y - xo;
                        const float dist = sqrtf(dot(w, w));
                        w = (1.0f / dist) * w;
                        const float4 ln = __ldg(sc.tri_n + __float_as_int(lv0.w));
                        const float cx = dot(ns, w), cy = -dot(xyz(ln), w);
                        if (cx > 0.0f && cy > 0.0f) {
                            ++n_sh;
                            ps.nee_G[q] = cx * cy / (dist * dist) * sc.light_area * (1.0f / 3.14159265358979f);
                            ps.nee_lmat[q] = __float_as_int(ln.w);
                            const float tmax = (1.0f - kShadowShorten) * dist;
                            float t0;
                            nfl |= kFlShadow;
                            if (grid_enter(a.g, xo, w, tmax, t0, cell_s)) {
                                ps.sh_status[q] = 0;
                                want_s = true;
                                s0 = make_float4(xo.x, xo.y, xo.z, t0);
                                s1 = make_float4(w.x, w.y, w.z, tmax);
                                s2 = make_int4((int)q, prim, kRayShadow, cell_s);
                            } else {
                                ps.sh_status[q] = kShadowClear;
                            }
                        }
                    }
                    ps.pend_mat[q] = mat;
                    nfl |= kFlPend;
                    nfl &= ~kFlPrevSpec;
                    if (b < ri.max_depth && !a.pm.on) {
                        uint4 xb = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotBsdf), k0, k1);
                        const V3 dn = cosine_dir(ns, u01(xb.x), u01(xb.y));
                        const V3 on = x + kRayOffset * ns;
                        ++n_ext;
                        nfl |= kFlExt;
                        float t0;
                        if (grid_enter(a.g, on, dn, __int_as_float(0x7f800000), t0, cell_e)) {
                            want_e = true;
                            e0 = make_float4(on.x, on.y, on.z, t0);
                            e1 = make_float4(dn.x, dn.y, dn.z, __int_as_float(0x7f800000));
                            e2 = make_int4((int)q, prim, 0, cell_e);
                        } else {
                            ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                        }
                    }
                } else if (b < ri.max_depth) {
                    const float c = fabsf(cd);
                    V3 dn = d, on;
                    int excl = prim;
                    ps.pend_mat[q] = mat;
                    ps.pend_cos[q] = c;
                    if (kind == kConductor) {
                        dn = d - (2.0f * cd) * ng;
                        on = x + kRayOffset * ns;
                        ps.pend_w[q] = 1.0f;
                    } else {
                        const float pr = branch_proxy(c, L, sc.mat_a + (size_t)mat * L);
                        uint4 xg = philox4x32_10(make_uint4(p, j, (uint32_t)b, kSlotGlass), k0, k1);
                        const bool refl = u01(xg.x) < pr;
                        ++n_glass;
                        if (refl) {
                            dn = d - (2.0f * cd) * ng;
                            on = x + kRayOffset * ns;
                            ps.pend_w[q] = -1.0f / pr;
                        } else {
                            on = x - kRayOffset * ns;
                            excl = -__ldg(sc.tri_obj + prim) - 2;
                            ps.pend_w[q] = 1.0f / (1.0f - pr);
                        }
                    }
                    nfl |= kFlPend | kFlPrevSpec | kFlExt;
                    ++n_ext;
                    float t0;
                    if (grid_enter(a.g, on, dn, __int_as_float(0x7f800000), t0, cell_e)) {
                        want_e = true;
                        e0 = make_float4(on.x, on.y, on.z, t0);
                        e1 = make_float4(dn.x, dn.y, dn.z, __int_as_float(0x7f800000));
                        e2 = make_int4((int)q, excl, 0, cell_e);
                    } else {
                        ps.hit0[q] = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
                    }
                }
            }
            ps.flags[q] = nfl;
        }
        block_stage_push2(a.Q, a.g, psm, bins, want_e, cell_e, e0, e1, e2, want_s, cell_s, s0, s1, s2, a.err);
    }
    block_bins_flush(a.Q, bins, a.g.n_bins);
    block_count3(a.counters + 0, n_ext, a.counters + 1, n_sh, a.counters + 2, n_glass);
}

__global__ void k_finalize(KArgs a) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = a.ps.np;
    if (q >= np) return;
    a.sample_xyz[3 * q + 0] = a.ps.acc[0 * np + q];
    a.sample_xyz[3 * q + 1] = a.ps.acc[1 * np + q];
    a.sample_xyz[3 * q + 2] = a.ps.acc[2 * np + q];
}

// Waves of one bounce: dims x + y + z - 2 with the neighbour-queue hand-off
// (each wave moves every ray at least one cell along a monotone axis), one
// when the lane carries rays across faces, handoff_waves + 1 for the mixed
// schedule (hand-off waves, then one wave that carries the rest).
static int ddm_waves(const DDMScene &g) {
    const int full = std::max(1, g.dims[0] + g.dims[1] + g.dims[2] - 2);
    if (g.continue_cells) return 1;
    return g.handoff_waves > 0 ? std::min(g.handoff_waves + 1, full) : full;
}
// Whether the lane carries rays across faces in wave w of `waves`.
static int ddm_wave_continues(const DDMScene &g, int w, int waves) {
    return g.continue_cells || (g.handoff_waves > 0 && w == waves - 1);
}

#include "ddm_photon.cuh"

__global__ void k_image_probe() {}

cudaError_t check_kernel_image() {
    cudaFuncAttributes attr;
    return cudaFuncGetAttributes(&attr, k_image_probe);
}

// ------------------------------------------------------------- host side
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static int trace_chunk(const DDMRun &run, const PhotonGridView &pmv, const PhotonGridView &pmcv, DDMBuffers &buf,
                       cudaStream_t s);

// Blocks for a grid-stride kernel: at most `want`, rounded down to whole waves
// of the blocks that fit on the SMs at once, so that no partial last wave runs
// on a fraction of the machine.
template <typename K>
static unsigned whole_waves(K kernel, int threads, size_t smem, int sm, unsigned want) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        return want;
    const unsigned wave = (unsigned)(per_sm * sm);
    return want <= wave ? want : want / wave * wave;
}

int ddm_trace_chunk(const DDMRun &run, DDMBuffers &buf, cudaStream_t s) {
    return trace_chunk(run, PhotonGridView{}, PhotonGridView{}, buf, s);
}

int ddm_trace_chunk_pm(const DDMRun &run, const PhotonGridView &pm, const PhotonGridView &pmc, DDMBuffers &buf,
                       cudaStream_t s) {
    return trace_chunk(run, pm, pmc, buf, s);
}

static int trace_chunk(const DDMRun &run, const PhotonGridView &pmv, const PhotonGridView &pmcv, DDMBuffers &buf,
                       cudaStream_t s) {
    const int64_t np = run.path_count;
    const int L = run.sc.L;
    const int nc = run.g.n_cells, nb = run.g.n_bins;
    if (nc > kMaxCells || nb > kMaxBins) {
        set_error("sddm_render: the DDM method supports at most 2048 subdomains");
        return SDDM_ERR_INVALID_ARG;
    }
    const int64_t cap = 2 * np;
    // carve one allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    const size_t oT = take(sizeof(float) * (size_t)L * np), oAcc = take(sizeof(float) * 6 * np),
                 oFl = take(4 * np), oPm = take(4 * np), oPc = take(4 * np), oPw = take(4 * np), oG = take(4 * np),
                 oLm = take(4 * np), oSh = take(4 * np), oCo = take(4 * kMaxCross * np), oCm = take(4 * kMaxCross * np),
                 oCc = take(4 * kMaxCross * np), oH0 = take(16 * np), oH1 = take(16 * np), oIn = take(48 * cap),
                 oSt = take(48 * cap), oCtl = take(32 + 4 * (size_t)nb), oFill = take(4 * (size_t)nb),
                 oOff = take(4 * ((size_t)nb + 1));
    // glass evaluations of each bounce go through a query list, evaluated by the
    // exact slab or the learned model in a dense pass before shading
    const bool use_mlp = run.bsdf_mode == SDDM_BSDF_MLP;
    const bool use_queries = true;
    const int64_t q_cap = use_queries ? 2 * np : 0;
    const int sm = std::max(1, run.sm_count);
    const unsigned path_blocks = (unsigned)std::min<int64_t>((np + 255) / 256, (int64_t)sm * 16);
    const size_t oQ = take(16 * (size_t)q_cap + 16), oNq = take(16), oPq = take(use_queries ? 4 * np : 4),
                 oCq = take(use_queries ? 4 * kMaxCross * np : 4), oRes = take(8 * (size_t)q_cap * L + 16),
                 oBc = take(4 * (size_t)path_blocks + 16);
    if (off > buf.bytes) {
        if (buf.mem) cudaFree(buf.mem);
        buf.mem = nullptr;
        buf.bytes = 0;
        cudaError_t e = cudaMalloc(&buf.mem, off);
        if (e != cudaSuccess) {
            buf.mem = nullptr;
            set_error("sddm_render: DDM path-state allocation failed (reduce paths_in_flight)");
            return SDDM_ERR_OOM;
        }
        buf.bytes = off;
    }
    char *m = (char *)buf.mem;
    KArgs a;
    a.sc = run.sc;
    a.g = run.g;
    a.rb = run.rb;
    a.path_begin = run.path_begin;
    a.sample_xyz = run.sample_xyz;
    a.first_prim = run.first_prim;
    a.counters = run.counters;
    a.err = run.error_flag;
    PathState &ps = a.ps;
    ps.np = np;
    ps.T = (float *)(m + oT);
    ps.acc = (float *)(m + oAcc);
    ps.flags = (int *)(m + oFl);
    ps.pend_mat = (int *)(m + oPm);
    ps.pend_cos = (float *)(m + oPc);
    ps.pend_w = (float *)(m + oPw);
    ps.nee_G = (float *)(m + oG);
    ps.nee_lmat = (int *)(m + oLm);
    ps.sh_status = (int *)(m + oSh);
    ps.cross_obj = (int *)(m + oCo);
    ps.cross_mat = (int *)(m + oCm);
    ps.cross_cos = (float *)(m + oCc);
    ps.hit0 = (float4 *)(m + oH0);
    ps.hit1 = (float4 *)(m + oH1);
    Queues &Q = a.Q;
    Q.cap = cap;
    Q.in = (float4 *)(m + oIn);
    Q.stage = (float4 *)(m + oSt);
    Q.ctl = (unsigned long long *)(m + oCtl);
    Q.cnt = (int *)(m + oCtl + 32);
    Q.fill = (int *)(m + oFill);
    Q.off = (int *)(m + oOff);
    a.use_queries = use_queries;
    a.queries = (float4 *)(m + oQ);
    a.n_queries = (unsigned long long *)(m + oNq);
    a.q_cap = q_cap;
    a.pend_query = (int *)(m + oPq);
    a.cross_query = (int *)(m + oCq);
    a.glass_res = (const float2 *)(m + oRes);
    a.block_cnt = (int *)(m + oBc);
    a.pm = pmv;
    a.cell_perm = nullptr;
    a.q_begin = 0;
    a.q_end = 0;
    a.pmc = pmcv;
    MlpRows mr{};
    if (use_queries) {
        mr.params = run.mlp_params;
        mr.sc = run.sc;
        mr.thick_min = run.mlp_dmin;
        mr.thick_max = run.mlp_dmax;
        mr.probe_key = run.probe_key;
        mr.queries = a.queries;
        mr.n_queries = a.n_queries;
        mr.q_cap = q_cap;
        mr.results = (float2 *)(m + oRes);
        mr.mode = 1;
        mr.raw = 0;
        mr.fallbacks = run.counters + 4;
        mr.batches = run.counters + 8;
        mr.rows = run.counters + 9;
        mr.err = run.error_flag;
    }

    const int trace_blocks = sm * (run.blocks_per_sm > 0 ? run.blocks_per_sm : 8);
    const unsigned scatter_blocks = whole_waves(k_scatter, 256, 0, sm, (unsigned)sm * 4);
    const int waves = ddm_waves(run.g);
    const size_t ctl_bytes = 32 + 4 * (size_t)nb;
    const unsigned cont_blocks = whole_waves(k_shade_continue, 256, sizeof(int) * (size_t)nb, sm, path_blocks);
    // the glass count and gather passes share one partition of the path slots
    const unsigned glass_blocks = whole_waves(k_glass_gather, 256, 0, sm, path_blocks);
    cudaError_t e;
#define DDM_CHECK(x)                                                     \
    do {                                                                 \
        if ((e = (x)) != cudaSuccess) return cuda_fail(e, "sddm_render: " #x); \
    } while (0)
    DDM_CHECK(cudaMemsetAsync(Q.ctl, 0, ctl_bytes, s));
    a.b = 0;
    a.last_wave = 0;
    const size_t bins_smem = sizeof(int) * (size_t)nb;
    k_camera<<<path_blocks, 256, bins_smem, s>>>(a);
    DDM_CHECK(cudaGetLastError());
    auto trace_launch = [&]() -> int {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (run.time_trace) {
            if ((e = buf.event_pair(e0, e1)) != cudaSuccess) return cuda_fail(e, "sddm_render: events");
            DDM_CHECK(cudaEventRecord(e0, s));
        }
        if (run.cache)
            k_trace_wave<false, true><<<trace_blocks, 128, 0, s>>>(a);
        else if (run.count_traversal)
            k_trace_wave<true><<<trace_blocks, 128, 0, s>>>(a);
        else
            k_trace_wave<false><<<trace_blocks, 128, 0, s>>>(a);
        DDM_CHECK(cudaGetLastError());
        if (run.time_trace) DDM_CHECK(cudaEventRecord(e1, s));
        *run.launches += 1;
        return SDDM_OK;
    };
    CellCache *cache = run.cache;
    std::vector<int64_t> cell_rays(cache ? (size_t)run.g.n_cells : 0);
    for (int b = 1; b <= run.max_depth + 1; ++b) {
        for (int w = 0; w < waves; ++w) {
            a.last_wave = w == waves - 1;
            a.g.continue_cells = ddm_wave_continues(run.g, w, waves);
            DDM_CHECK(cudaMemsetAsync(Q.fill, 0, 4 * (size_t)nb, s));
            if (!cache) {
                k_scatter<<<scatter_blocks, 256, 0, s>>>(a);
                DDM_CHECK(cudaGetLastError());
                DDM_CHECK(cudaMemsetAsync(Q.ctl, 0, ctl_bytes, s));
                const int rc = trace_launch();
                if (rc != SDDM_OK) return rc;
                *run.launches += 1;
                continue;
            }
            // subdomain cache (Sec. 5's loading and unloading of subdomains):
            // the rays waiting per cell decide which cells are loaded, in
            // which groups the wave is traced, and the order of its queue
            DDM_CHECK(cudaMemcpyAsync(cache->h_cnt, Q.cnt, 4 * (size_t)nb, cudaMemcpyDeviceToHost, s));
            DDM_CHECK(cudaMemcpyAsync(cache->h_err, run.error_flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
            DDM_CHECK(cudaStreamSynchronize(s));
            if (cache->h_err[0] != 0) return SDDM_OK;   // reported by the caller's error-word check
            const int per_cell = 2 * run.g.n_oct;
            for (int c = 0; c < run.g.n_cells; ++c) {
                int64_t r = 0;
                for (int k = 0; k < per_cell; ++k) r += cache->h_cnt[c * per_cell + k];
                cell_rays[c] = r;
            }
            auto sort_queue = [&]() -> int {
                DDM_CHECK(cudaMemcpyAsync(cache->d_perm, cache->h_perm, 4 * (size_t)run.g.n_cells,
                                          cudaMemcpyHostToDevice, s));
                a.cell_perm = cache->d_perm;
                k_scatter<<<scatter_blocks, 256, 0, s>>>(a);
                DDM_CHECK(cudaGetLastError());
                a.cell_perm = nullptr;
                DDM_CHECK(cudaMemsetAsync(Q.ctl, 0, ctl_bytes, s));
                *run.launches += 1;
                return SDDM_OK;
            };
            auto group_launch = [&](int64_t q_begin, int64_t q_end) -> int {
                DDM_CHECK(cudaMemsetAsync(Q.ctl + 1, 0, sizeof(unsigned long long), s));
                a.q_begin = q_begin;
                a.q_end = q_end;
                const int rc = trace_launch();
                a.q_begin = 0;
                a.q_end = 0;
                return rc;
            };
            const int rc = cache->run_wave(cell_rays, s, sort_queue, group_launch);
            if (rc != SDDM_OK) return rc;
        }
        a.b = b;
        if (use_queries && b >= 2) {
            k_glass_count<<<glass_blocks, 256, 0, s>>>(a);
            DDM_CHECK(cudaGetLastError());
            k_glass_gather<<<glass_blocks, 256, 0, s>>>(a);
            DDM_CHECK(cudaGetLastError());
            *run.launches += 1;
            if (use_mlp) {
                cudaEvent_t m0 = nullptr, m1 = nullptr;
                if (run.time_trace && (e = buf.mlp_event_pair(m0, m1)) != cudaSuccess)
                    return cuda_fail(e, "sddm_render: events");
                DDM_CHECK(launch_mlp_rows(mr, run.sm_count, s, m0, m1));
                *run.launches += mr.raw ? 0 : 1;   // the probe pass
            } else
                DDM_CHECK(launch_slab_rows(mr, run.sm_count, s));
            *run.launches += 2;
        }
        if (run.sc.mat_nfilm)
            k_shade_spectral<true><<<path_blocks, 256, 0, s>>>(a);
        else
            k_shade_spectral<false><<<path_blocks, 256, 0, s>>>(a);
        DDM_CHECK(cudaGetLastError());
        if (a.pm.on) {
            // one path slot per thread: the gather is latency-bound and gains from the most blocks in flight
            k_ddm_gather<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(a);
            DDM_CHECK(cudaGetLastError());
            *run.launches += 1;
        }
        k_shade_continue<<<cont_blocks, 256, bins_smem, s>>>(a);
        DDM_CHECK(cudaGetLastError());
        *run.launches += 2;
    }
    k_finalize<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(a);
    DDM_CHECK(cudaGetLastError());
    *run.launches += 2;   // camera + finalize
#undef DDM_CHECK
    return SDDM_OK;
}

cudaError_t build_cell_table(const DDMScene &g, float4 *planes, int4 *next, cudaStream_t stream) {
    k_cell_table<<<(g.n_cells + 127) / 128, 128, 0, stream>>>(g, planes, next);
    return cudaGetLastError();
}

}  // namespace sddm
