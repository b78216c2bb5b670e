// C ABI of libsddm: context, scene validation and upload, build, render.
//
// The host side follows the paper's problem statement (Sec. 1-2: a room, its
// materials' optical properties, natural light; Sec. 5: a decomposition of the
// scene into subdomains) and drives the device kernels on one CUDA stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "sddm_internal.h"
#include "sddm_ddm.h"
#include "sddm_cache.h"
#include "sddm_mlp.h"
#include "sddm_photon.h"
#include "sddm_ddm_photon.h"

namespace sddm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return SDDM_ERR_CUDA;
}

static int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

// Owned device allocation.
// Pinned host memory mapped into the device's address space: the GPU reads it
// directly (over NVLink-C2C on Grace-based systems) without a copy in HBM.
struct HostBuf {
    void *h = nullptr, *d = nullptr;
    size_t bytes = 0;
    HostBuf() = default;
    HostBuf(const HostBuf &) = delete;
    HostBuf &operator=(const HostBuf &) = delete;
    ~HostBuf() { release(); }
    void release() {
        if (h) cudaFreeHost(h);
        h = d = nullptr;
        bytes = 0;
    }
    template <typename T>
    cudaError_t upload(const std::vector<T> &v) {
        release();
        const size_t n = std::max<size_t>(v.size() * sizeof(T), 16);
        cudaError_t e = cudaHostAlloc(&h, n, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) {
            h = nullptr;
            return e;
        }
        bytes = n;
        if (!v.empty()) std::memcpy(h, v.data(), v.size() * sizeof(T));
        return cudaHostGetDevicePointer(&d, h, 0);
    }
    template <typename T>
    const T *as() const {
        return static_cast<const T *>(d);
    }
};

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t upload(const std::vector<T> &v, cudaStream_t s) {
        cudaError_t e = ensure(std::max<size_t>(v.size() * sizeof(T), 16));
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
    template <typename T>
    T *as() const { return reinterpret_cast<T *>(p); }
};

}  // namespace sddm

using namespace sddm;

struct sddm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    // spectrum
    int L = 0;
    std::vector<float> lam, quad_w, cmf;
    // materials
    std::vector<Material> mats;
    // mesh
    std::vector<float> V;
    std::vector<uint32_t> F, mat_id, obj_id;
    bool built = false;
    sddm_build_opts opts{};
    // device scene
    DevBuf d_wcmf, d_lam, d_kind, d_a, d_b, d_c, d_thick, d_tri_n, d_tri_obj, d_light_v, d_light_cdf;
    DevBuf d_nfilm, d_film_n, d_film_k, d_film_dk, d_film_t;
    DevBuf d_gnodes, d_gtris;
    float light_area = 0.f;
    int n_light = 0;
    DevScene dev{};
    DDMScene ddm{};
    DevBuf d_cell_nodes, d_cell_tris, d_cell_root, d_cell_planes, d_cell_next;
    HostBuf h_cell_nodes, h_cell_tris;   // the same, in host memory (bvh_in_host_memory, cell_cache_bytes)
    CellCache cache;                     // device cache of subdomain BVHs (cell_cache_bytes > 0)
    // per-render scratch
    DevBuf d_info, d_state, d_out_tab, d_aov_xyz_tab, d_aov_prim_tab, d_samples, d_first, d_counters, d_err;
    DDMBuffers ddm_buf;
    // photon map (sddm_render_photon_map): slots, grid, and the view the
    // megakernel reads while pm_view.on
    DevBuf pm_state, pm_scratch, pm_pos, pm_dir, pm_pow, pm_cnt, pm_start, pm_fill, pm_order, pm_sums, pm_cntr;
    DevBuf pmc_cnt, pmc_start, pmc_fill, pmc_order, pmc_sums;   // the caustic map's grid
    DevBuf pm_img;                                               // one pass of a progressive render
    PhotonGridView pm_view{}, pmc_view{};
    DDMBuffers pm_ddm_buf;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int profile = 0;
    // learned glass surrogates: one network may serve several materials
    struct MlpNet {
        DevBuf params, m, v;
        int64_t step = 0;
        float dmin = 0.002f, dmax = 0.010f;
    };
    std::vector<std::unique_ptr<MlpNet>> nets;
    std::vector<int> net_of_mat;     // per material, -1 = none
    DevBuf mlp_grad_cta, mlp_loss_cta, mlp_scalar, mlp_X, mlp_Y;
    // CUDA graphs of the render launch sequence, keyed by everything that is
    // baked into kernel parameters (sizes, buffer addresses, build)
    int64_t build_id = 0;
    cudaStream_t gstream = nullptr;
    cudaEvent_t hand0 = nullptr, hand1 = nullptr;
    struct Graph {
        cudaGraphExec_t exec;
        int64_t launches;   // kernels in the captured sequence
        int events_used;    // trace-timing event records captured with it
    };
    std::map<std::string, Graph> graphs;
    std::map<std::string, int> seen;
    bool graphs_enabled = true;
    ~sddm_ctx() {
        for (auto &kv : graphs) cudaGraphExecDestroy(kv.second.exec);
        if (gstream) cudaStreamDestroy(gstream);
        if (hand0) cudaEventDestroy(hand0);
        if (hand1) cudaEventDestroy(hand1);
    }
};

extern "C" {

const char *sddm_last_error(void) { return g_last_error.c_str(); }

const char *sddm_version(void) { return "sddm 0.1 sm_103a"; }

int sddm_create(sddm_ctx **out, int device, void *stream) {
    if (!out) return fail(SDDM_ERR_INVALID_ARG, "sddm_create: out is NULL");
    *out = nullptr;
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_create: cudaGetDeviceCount");
    if (device < 0 || device >= n_dev) return fail(SDDM_ERR_INVALID_ARG, "sddm_create: no such device");
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "sddm_create: cudaSetDevice");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, device)) != cudaSuccess)
        return cuda_fail(e, "sddm_create: cudaGetDeviceProperties");
    if ((e = check_kernel_image()) != cudaSuccess)
        return cuda_fail(e, "sddm_create: no sm_103a kernel image for this device");
    std::unique_ptr<sddm_ctx> c(new (std::nothrow) sddm_ctx());
    if (!c) return fail(SDDM_ERR_OOM, "sddm_create: out of host memory");
    c->device = device;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->sm_count = prop.multiProcessorCount;
    if ((e = cudaEventCreate(&c->ev0)) != cudaSuccess || (e = cudaEventCreate(&c->ev1)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->hand0, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c->hand1, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "sddm_create: events and graph stream");
    *out = c.release();
    return SDDM_OK;
}

int sddm_destroy(sddm_ctx *ctx) {
    if (!ctx) return SDDM_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return SDDM_OK;
}

static bool finite_range(const float *p, int n, float lo, float hi) {
    for (int i = 0; i < n; ++i)
        if (!(p[i] >= lo && p[i] <= hi)) return false;
    return true;
}

int sddm_set_spectrum(sddm_ctx *ctx, int L, const float *lambda_nm, const float *quad_w, const float *cmf_xyz) {
    if (!ctx || !lambda_nm || !quad_w || !cmf_xyz) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_spectrum: NULL");
    if (L < 1 || L > kMaxL) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_spectrum: L must be in 1..256");
    if (!finite_range(lambda_nm, L, 1.0f, 1e5f) || !finite_range(quad_w, L, 0.0f, 1e6f) ||
        !finite_range(cmf_xyz, 3 * L, -1e3f, 1e3f))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_set_spectrum: non-finite or out-of-range values");
    ctx->L = L;
    ctx->lam.assign(lambda_nm, lambda_nm + L);
    ctx->quad_w.assign(quad_w, quad_w + L);
    ctx->cmf.assign(cmf_xyz, cmf_xyz + 3 * L);
    ctx->mats.clear();
    ctx->built = false;
    return SDDM_OK;
}

static int add_mat(sddm_ctx *ctx, Material &&m, uint32_t *mat, const char *who) {
    if (ctx->mats.size() >= (1u << 20)) return fail(SDDM_ERR_INVALID_ARG, std::string(who) + ": too many materials");
    ctx->mats.push_back(std::move(m));
    if (mat) *mat = (uint32_t)(ctx->mats.size() - 1);
    ctx->built = false;
    return SDDM_OK;
}

#define NEED_SPECTRUM(who)                                                                        \
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, who ": ctx is NULL");                            \
    if (ctx->L <= 0) return fail(SDDM_ERR_INVALID_ARG, who ": call sddm_set_spectrum first");

int sddm_add_lambertian(sddm_ctx *ctx, const float *rho, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_lambertian");
    if (!rho || !finite_range(rho, ctx->L, 0.0f, 1.0f))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_add_lambertian: rho must be in [0,1]");
    Material m;
    m.kind = kLambert;
    m.a.assign(rho, rho + ctx->L);
    return add_mat(ctx, std::move(m), mat, "sddm_add_lambertian");
}

int sddm_add_conductor(sddm_ctx *ctx, const float *n, const float *k, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_conductor");
    if (!n || !k || !finite_range(n, ctx->L, 1e-4f, 100.f) || !finite_range(k, ctx->L, 0.0f, 100.f))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_add_conductor: need n in (0,100], k in [0,100]");
    Material m;
    m.kind = kConductor;
    m.a.assign(n, n + ctx->L);
    m.b.assign(k, k + ctx->L);
    return add_mat(ctx, std::move(m), mat, "sddm_add_conductor");
}

int sddm_add_glass_slab(sddm_ctx *ctx, const float *n, const float *alpha_clear, const float *dalpha,
                        float thickness_m, float s_default, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_glass_slab");
    if (!n || !alpha_clear || !dalpha || !finite_range(n, ctx->L, 1.0f, 10.f) ||
        !finite_range(alpha_clear, ctx->L, 0.0f, 1e7f) || !finite_range(dalpha, ctx->L, -1e7f, 1e7f) ||
        !(thickness_m > 0.0f && thickness_m < 1.0f) || !(s_default >= 0.0f && s_default <= 1.0f))
        return fail(SDDM_ERR_INVALID_ARG,
                    "sddm_add_glass_slab: need n in [1,10], alpha >= 0, 0 < thickness < 1 m, s in [0,1]");
    for (int i = 0; i < ctx->L; ++i)
        if (alpha_clear[i] + dalpha[i] < 0.0f)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_add_glass_slab: alpha_clear + dalpha must stay >= 0");
    Material m;
    m.kind = kGlass;
    m.a.assign(n, n + ctx->L);
    m.b.assign(alpha_clear, alpha_clear + ctx->L);
    m.c.assign(dalpha, dalpha + ctx->L);
    m.thick = thickness_m;
    m.s_default = s_default;
    return add_mat(ctx, std::move(m), mat, "sddm_add_glass_slab");
}

int sddm_add_coated_glass(sddm_ctx *ctx, const float *n, const float *alpha_clear, const float *dalpha,
                          float thickness_m, float s_default, int n_films, const float *film_n, const float *film_k,
                          const float *film_dk, const float *film_t_nm, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_coated_glass");
    if (n_films < 0 || n_films > SDDM_MAX_FILMS || (n_films > 0 && (!film_n || !film_k || !film_dk || !film_t_nm)))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_add_coated_glass: 0..SDDM_MAX_FILMS films with n, k, dk and thickness arrays");
    const int L = ctx->L;
    for (int j = 0; j < n_films; ++j) {
        if (!finite_range(film_n + (size_t)j * L, L, 1.0f, 10.f) || !finite_range(film_k + (size_t)j * L, L, 0.0f, 10.f) ||
            !finite_range(film_dk + (size_t)j * L, L, -10.f, 10.f) || !(film_t_nm[j] >= 0.0f && film_t_nm[j] < 1e5f))
            return fail(SDDM_ERR_INVALID_ARG,
                        "sddm_add_coated_glass: film n in [1,10], k >= 0, 0 <= thickness < 1e5 nm");
        for (int i = 0; i < L; ++i)
            if (film_k[(size_t)j * L + i] + film_dk[(size_t)j * L + i] < 0.0f)
                return fail(SDDM_ERR_INVALID_ARG, "sddm_add_coated_glass: film k + dk must stay >= 0");
    }
    uint32_t id = 0;
    int rc = sddm_add_glass_slab(ctx, n, alpha_clear, dalpha, thickness_m, s_default, &id);
    if (rc != SDDM_OK) return rc;
    Material &m = ctx->mats[id];
    m.n_film = n_films;
    m.film_n.assign(film_n ? film_n : n, (film_n ? film_n : n) + (size_t)n_films * L);
    m.film_k.assign(film_k ? film_k : n, (film_k ? film_k : n) + (size_t)n_films * L);
    m.film_dk.assign(film_dk ? film_dk : n, (film_dk ? film_dk : n) + (size_t)n_films * L);
    for (int j = 0; j < n_films; ++j) m.film_t[j] = film_t_nm[j];
    if (mat) *mat = id;
    return SDDM_OK;
}

int sddm_add_emitter(sddm_ctx *ctx, const float *Le, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_emitter");
    if (!Le || !finite_range(Le, ctx->L, 0.0f, 1e12f)) return fail(SDDM_ERR_INVALID_ARG, "sddm_add_emitter: Le >= 0");
    Material m;
    m.kind = kEmitter;
    m.a.assign(Le, Le + ctx->L);
    return add_mat(ctx, std::move(m), mat, "sddm_add_emitter");
}

int sddm_add_diffuse_emitter(sddm_ctx *ctx, const float *rho, const float *Le, uint32_t *mat) {
    NEED_SPECTRUM("sddm_add_diffuse_emitter");
    if (!Le || !rho || !finite_range(Le, ctx->L, 0.0f, 1e12f) || !finite_range(rho, ctx->L, 0.0f, 1.0f))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_add_diffuse_emitter: Le >= 0, rho in [0,1]");
    Material m;
    m.kind = kDiffuseEmitter;
    m.a.assign(Le, Le + ctx->L);
    m.b.assign(rho, rho + ctx->L);
    return add_mat(ctx, std::move(m), mat, "sddm_add_diffuse_emitter");
}

int sddm_set_mesh(sddm_ctx *ctx, const float *v, int nv, const uint32_t *tri, int nt, const uint32_t *mat_id,
                  const uint32_t *obj_id) {
    if (!ctx || !v || !tri || !mat_id || !obj_id) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: NULL");
    if (nv < 3 || nt < 1 || nt > (1 << 26)) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: bad nv/nt");
    for (int64_t i = 0; i < 3LL * nv; ++i)
        if (!std::isfinite(v[i]) || std::fabs(v[i]) > 1e6f)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: non-finite or huge vertex coordinate");
    for (int64_t i = 0; i < 3LL * nt; ++i)
        if (tri[i] >= (uint32_t)nv) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: vertex index out of range");
    for (int i = 0; i < nt; ++i) {
        if (mat_id[i] >= ctx->mats.size())
            return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: material id out of range (add materials first)");
        if (obj_id[i] > 0x7fffffffu) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_mesh: obj id too large");
    }
    ctx->V.assign(v, v + 3LL * nv);
    ctx->F.assign(tri, tri + 3LL * nt);
    ctx->mat_id.assign(mat_id, mat_id + nt);
    ctx->obj_id.assign(obj_id, obj_id + nt);
    ctx->built = false;
    return SDDM_OK;
}

static void default_opts(sddm_build_opts &o) {
    for (int a = 0; a < 3; ++a)
        if (o.grid[a] <= 0) o.grid[a] = 1;
    if (o.leaf_size <= 0) o.leaf_size = 4;
    if (o.sah_bins <= 0) o.sah_bins = 16;
}

int sddm_build(sddm_ctx *ctx, const sddm_build_opts *opts) {
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, "sddm_build: ctx is NULL");
    if (ctx->L <= 0 || ctx->mats.empty() || ctx->F.empty())
        return fail(SDDM_ERR_INVALID_ARG, "sddm_build: spectrum, materials and mesh are required");
    sddm_build_opts o{};
    if (opts) o = *opts;
    default_opts(o);
    if (o.grid[0] > 64 || o.grid[1] > 64 || o.grid[2] > 64 || o.leaf_size > kMaxLeaf || o.sah_bins < 4 ||
        o.sah_bins > 64 || o.queue_capacity < 0 || o.blocks_per_sm < 0 || o.blocks_per_sm > 32 ||
        o.paths_in_flight < 0 || o.bvh_in_host_memory < 0 || o.bvh_in_host_memory > 1 || o.cell_cache_bytes < 0)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_build: options out of range");
    if (o.cell_cache_bytes > 0 && o.bvh_in_host_memory)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_build: cell_cache_bytes and bvh_in_host_memory exclude each other");
    if (o.continue_cells < 0 || o.continue_cells > 1 || (o.continue_cells && o.cell_cache_bytes > 0))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_build: continue_cells is 0 or 1, and not with cell_cache_bytes");
    if (o.handoff_waves < 0 || (o.handoff_waves > 0 && (o.continue_cells || o.cell_cache_bytes > 0)))
        return fail(SDDM_ERR_INVALID_ARG,
                    "sddm_build: handoff_waves >= 0, and not with continue_cells or cell_cache_bytes");
    // every mesh material must exist (the material list may have changed since set_mesh)
    for (uint32_t m : ctx->mat_id)
        if (m >= ctx->mats.size()) return fail(SDDM_ERR_INVALID_ARG, "sddm_build: mesh references a missing material");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_build: cudaSetDevice");
    const int L = ctx->L, M = (int)ctx->mats.size(), nt = (int)ctx->mat_id.size();

    // --- triangles, normals, lights (normals and areas in double, rounded once)
    std::vector<BuildTri> tris(nt);
    std::vector<float4> tri_n(nt);
    std::vector<int> tri_obj(nt);
    std::vector<float4> light_v;
    std::vector<double> light_cum;
    double light_total = 0.0;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int t = 0; t < nt; ++t) {
        BuildTri &bt = tris[t];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                bt.v[k][a] = ctx->V[3 * (size_t)ctx->F[3 * (size_t)t + k] + a];
                lo[a] = std::min(lo[a], bt.v[k][a]);
                hi[a] = std::max(hi[a], bt.v[k][a]);
            }
        const int kind = ctx->mats[ctx->mat_id[t]].kind;
        bt.id = (uint32_t)t;
        bt.obj = ctx->obj_id[t];
        bt.flags = kind == kGlass ? kTriGlass : 0u;
        double e1[3], e2[3];
        for (int a = 0; a < 3; ++a) {
            e1[a] = (double)bt.v[1][a] - bt.v[0][a];
            e2[a] = (double)bt.v[2][a] - bt.v[0][a];
        }
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        int mid = (int)ctx->mat_id[t];
        float fm;
        std::memcpy(&fm, &mid, 4);
        tri_n[t] = len > 0 ? make_float4((float)(n[0] / len), (float)(n[1] / len), (float)(n[2] / len), fm)
                           : make_float4(0.f, 0.f, 0.f, fm);
        tri_obj[t] = (int)ctx->obj_id[t];
        if (kind == kEmitter || kind == kDiffuseEmitter) {
            light_total += 0.5 * len;
            light_cum.push_back(light_total);
            float ft;
            std::memcpy(&ft, &t, 4);
            light_v.push_back(make_float4(bt.v[0][0], bt.v[0][1], bt.v[0][2], ft));
            light_v.push_back(make_float4(bt.v[1][0], bt.v[1][1], bt.v[1][2], 0.f));
            light_v.push_back(make_float4(bt.v[2][0], bt.v[2][1], bt.v[2][2], 0.f));
        }
    }
    std::vector<float> light_cdf(light_cum.size());
    for (size_t i = 0; i < light_cum.size(); ++i) light_cdf[i] = (float)(light_cum[i] / light_total);

    // --- materials, spectral weights
    std::vector<float> wcmf(4 * (size_t)L, 0.f), A((size_t)M * L, 0.f), B((size_t)M * L, 0.f), Cc((size_t)M * L, 0.f),
        thick(M, 0.f);
    std::vector<int> kinds(M);
    for (int i = 0; i < L; ++i)
        for (int c = 0; c < 3; ++c) wcmf[4 * i + c] = ctx->quad_w[i] * ctx->cmf[3 * i + c];
    for (int m = 0; m < M; ++m) {
        const Material &mt = ctx->mats[m];
        kinds[m] = mt.kind;
        for (int i = 0; i < L; ++i) {
            if (!mt.a.empty()) A[(size_t)m * L + i] = mt.a[i];
            if (!mt.b.empty()) B[(size_t)m * L + i] = mt.b[i];
            if (!mt.c.empty()) Cc[(size_t)m * L + i] = mt.c[i];
        }
        thick[m] = mt.thick;
    }
    // coating films of glass materials, [m][SDDM_MAX_FILMS][L] (+ thickness [m][SDDM_MAX_FILMS])
    bool any_film = false;
    for (int m = 0; m < M; ++m) any_film |= ctx->mats[m].n_film > 0;
    std::vector<int> nfilm(M, 0);
    std::vector<float> FN, FK, FDK, FT;
    if (any_film) {
        FN.assign((size_t)M * SDDM_MAX_FILMS * L, 1.f);
        FK.assign((size_t)M * SDDM_MAX_FILMS * L, 0.f);
        FDK.assign((size_t)M * SDDM_MAX_FILMS * L, 0.f);
        FT.assign((size_t)M * SDDM_MAX_FILMS, 0.f);
        for (int m = 0; m < M; ++m) {
            const Material &mt = ctx->mats[m];
            nfilm[m] = mt.n_film;
            for (int j = 0; j < mt.n_film; ++j) {
                for (int i = 0; i < L; ++i) {
                    const size_t f = ((size_t)m * SDDM_MAX_FILMS + j) * L + i;
                    FN[f] = mt.film_n[(size_t)j * L + i];
                    FK[f] = mt.film_k[(size_t)j * L + i];
                    FDK[f] = mt.film_dk[(size_t)j * L + i];
                }
                FT[(size_t)m * SDDM_MAX_FILMS + j] = mt.film_t[j];
            }
        }
    }

    // --- hierarchies: global, and the subdomain grid
    int n_threads = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    std::vector<uint32_t> all(nt);
    for (int t = 0; t < nt; ++t) all[t] = (uint32_t)t;
    float glo[3], ghi[3];
    for (int a = 0; a < 3; ++a) {
        float pad = 1e-4f + 1e-5f * std::max(std::fabs(lo[a]), std::fabs(hi[a]));
        glo[a] = lo[a] - pad;
        ghi[a] = hi[a] + pad;
    }
    PackedBVH global;
    build_bvh(tris, all, glo, ghi, o.leaf_size, o.sah_bins, global);
    const double diag = std::sqrt((double)(ghi[0] - glo[0]) * (ghi[0] - glo[0]) +
                                  (double)(ghi[1] - glo[1]) * (ghi[1] - glo[1]) +
                                  (double)(ghi[2] - glo[2]) * (ghi[2] - glo[2]));
    const float eps = (float)(1e-6 * diag);
    std::vector<PackedBVH> cells;
    build_grid(tris, o.grid, glo, ghi, o.leaf_size, o.sah_bins, eps, cells, n_threads);
    std::vector<float4> cell_nodes, cell_tris;
    std::vector<int> cell_root;
    std::vector<int64_t> c_node_base, c_node_cnt, c_tri_base, c_tri_cnt;   // per cell, for the cache
    int64_t tri_base_check = 0;
    for (auto &c : cells) {
        int node_base = (int)(cell_nodes.size() / 4);
        int tri_base = (int)(cell_tris.size() / 3);
        cell_root.push_back(node_base);
        c_node_base.push_back(node_base);
        c_node_cnt.push_back((int64_t)c.nodes.size() / 4);
        c_tri_base.push_back(tri_base);
        c_tri_cnt.push_back((int64_t)c.tris.size() / 3);
        // rebase child codes
        for (size_t k = 0; k < c.nodes.size(); k += 4) {
            float4 n3 = c.nodes[k + 3];
            int ch[2];
            std::memcpy(&ch[0], &n3.x, 4);
            std::memcpy(&ch[1], &n3.y, 4);
            for (int q = 0; q < 2; ++q) {
                if (ch[q] >= 0) {
                    ch[q] += node_base;
                } else {
                    int v = ~ch[q];
                    int first = (v >> kLeafBits) + tri_base, cnt = v & ((1 << kLeafBits) - 1);
                    ch[q] = ~((first << kLeafBits) | cnt);
                }
            }
            std::memcpy(&n3.x, &ch[0], 4);
            std::memcpy(&n3.y, &ch[1], 4);
            c.nodes[k + 3] = n3;
        }
        cell_nodes.insert(cell_nodes.end(), c.nodes.begin(), c.nodes.end());
        cell_tris.insert(cell_tris.end(), c.tris.begin(), c.tris.end());
        tri_base_check += (int64_t)c.tris.size() / 3;
    }
    if (tri_base_check >= (1LL << (31 - kLeafBits)) || (int64_t)global.tris.size() / 3 >= (1LL << (31 - kLeafBits)))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_build: too many triangle references for the leaf encoding");

    // --- upload
    cudaStream_t s = ctx->stream;
    if ((e = ctx->d_wcmf.upload(wcmf, s)) || (e = ctx->d_lam.upload(ctx->lam, s)) ||
        (e = ctx->d_kind.upload(kinds, s)) || (e = ctx->d_a.upload(A, s)) || (e = ctx->d_b.upload(B, s)) ||
        (e = ctx->d_c.upload(Cc, s)) || (e = ctx->d_thick.upload(thick, s)) || (e = ctx->d_tri_n.upload(tri_n, s)) ||
        (e = ctx->d_tri_obj.upload(tri_obj, s)) || (e = ctx->d_light_v.upload(light_v, s)) ||
        (e = ctx->d_light_cdf.upload(light_cdf, s)) || (e = ctx->d_gnodes.upload(global.nodes, s)) ||
        (e = ctx->d_gtris.upload(global.tris, s)) ||
        ((o.bvh_in_host_memory || o.cell_cache_bytes > 0)
             ? ((e = ctx->h_cell_nodes.upload(cell_nodes)) || (e = ctx->h_cell_tris.upload(cell_tris)))
                              : ((e = ctx->d_cell_nodes.upload(cell_nodes, s)) || (e = ctx->d_cell_tris.upload(cell_tris, s)))) ||
        (e = ctx->d_cell_root.upload(cell_root, s)) ||
        (any_film && ((e = ctx->d_nfilm.upload(nfilm, s)) || (e = ctx->d_film_n.upload(FN, s)) ||
                      (e = ctx->d_film_k.upload(FK, s)) || (e = ctx->d_film_dk.upload(FDK, s)) ||
                      (e = ctx->d_film_t.upload(FT, s)))))
        return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_build: device allocation failed")
                                              : cuda_fail(e, "sddm_build: upload");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "sddm_build: synchronize");

    DevScene &d = ctx->dev;
    d.L = L;
    d.n_mat = M;
    d.wcmf = ctx->d_wcmf.as<float4>();
    d.lam = ctx->d_lam.as<float>();
    d.mat_kind = ctx->d_kind.as<int>();
    d.mat_a = ctx->d_a.as<float>();
    d.mat_b = ctx->d_b.as<float>();
    d.mat_c = ctx->d_c.as<float>();
    d.mat_thick = ctx->d_thick.as<float>();
    d.mat_nfilm = any_film ? ctx->d_nfilm.as<int>() : nullptr;
    d.film_n = any_film ? ctx->d_film_n.as<float>() : nullptr;
    d.film_k = any_film ? ctx->d_film_k.as<float>() : nullptr;
    d.film_dk = any_film ? ctx->d_film_dk.as<float>() : nullptr;
    d.film_t = any_film ? ctx->d_film_t.as<float>() : nullptr;
    d.tri_n = ctx->d_tri_n.as<float4>();
    d.tri_obj = ctx->d_tri_obj.as<int>();
    d.n_light = (int)light_cdf.size();
    d.light_v = ctx->d_light_v.as<float4>();
    d.light_cdf = ctx->d_light_cdf.as<float>();
    d.light_area = (float)light_total;
    d.g_nodes = ctx->d_gnodes.as<float4>();
    d.g_tris = ctx->d_gtris.as<float4>();

    DDMScene &g = ctx->ddm;
    for (int a = 0; a < 3; ++a) {
        g.dims[a] = o.grid[a];
        g.lo[a] = glo[a];
        g.hi[a] = ghi[a];
        g.cell[a] = (ghi[a] - glo[a]) / (float)o.grid[a];
        g.inv_cell[a] = 1.0f / g.cell[a];
    }
    g.eps = eps;
    g.n_cells = o.grid[0] * o.grid[1] * o.grid[2];
#ifndef SDDM_MAX_SUBBINS
#define SDDM_MAX_SUBBINS 8   // 64 measured: trace 2% faster, bin bookkeeping elsewhere slower overall
#endif
    g.n_oct = (SDDM_MAX_SUBBINS >= 64 && 128 * g.n_cells <= kMaxBins) ? 64 : (SDDM_MAX_SUBBINS >= 8 && 16 * g.n_cells <= kMaxBins) ? 8 : 1;
    g.n_bins = 2 * g.n_cells * g.n_oct;
    g.continue_cells = o.continue_cells;
    g.handoff_waves = o.handoff_waves;
    ctx->cache.release();
    if (o.cell_cache_bytes > 0) {
        // subdomains loaded into a device cache of that many bytes as their queues fill
        ctx->d_cell_nodes.release();
        ctx->d_cell_tris.release();
        const int rc = ctx->cache.init(static_cast<const float4 *>(ctx->h_cell_nodes.h),
                                       static_cast<const float4 *>(ctx->h_cell_tris.h), c_node_base, c_node_cnt,
                                       c_tri_base, c_tri_cnt, o.cell_cache_bytes, ctx->d_cell_root.as<int>(),
                                       g.n_bins);
        if (rc != SDDM_OK) {
            ctx->cache.release();
            ctx->built = false;
            return rc;
        }
        g.nodes = ctx->cache.d_cache;
        g.tris = ctx->cache.d_cache;
        g.node_cap = ctx->cache.plan.budget / 64;
        g.tri_cap = ctx->cache.plan.budget / 48;
    } else if (o.bvh_in_host_memory) {
        g.node_cap = (int64_t)cell_nodes.size() / 4;
        g.tri_cap = (int64_t)cell_tris.size() / 3;
        g.nodes = ctx->h_cell_nodes.as<float4>();
        g.tris = ctx->h_cell_tris.as<float4>();
        ctx->d_cell_nodes.release();
        ctx->d_cell_tris.release();
    } else {
        g.node_cap = (int64_t)cell_nodes.size() / 4;
        g.tri_cap = (int64_t)cell_tris.size() / 3;
        g.nodes = ctx->d_cell_nodes.as<float4>();
        g.tris = ctx->d_cell_tris.as<float4>();
        ctx->h_cell_nodes.release();
        ctx->h_cell_tris.release();
    }
    g.root = ctx->d_cell_root.as<int>();
    if ((e = ctx->d_cell_planes.ensure(sizeof(float4) * 2 * (size_t)g.n_cells)) ||
        (e = ctx->d_cell_next.ensure(sizeof(int4) * 2 * (size_t)g.n_cells)))
        return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_build: device allocation failed")
                                              : cuda_fail(e, "sddm_build: cell table");
    g.cell_planes = ctx->d_cell_planes.as<float4>();
    g.cell_next = ctx->d_cell_next.as<int4>();
    if ((e = build_cell_table(g, ctx->d_cell_planes.as<float4>(), ctx->d_cell_next.as<int4>(), s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "sddm_build: cell table");
    ctx->opts = o;
    ctx->built = true;
    ++ctx->build_id;
    return SDDM_OK;
}

// ---------------------------------------------------------------- render
static int validate_desc(const sddm_ctx *ctx, const sddm_render_desc *d, int n) {
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, "sddm_render: ctx is NULL");
    if (!ctx->built) return fail(SDDM_ERR_NOT_BUILT, "sddm_render: call sddm_build first");
    if (!d || n < 1 || n > 4096) return fail(SDDM_ERR_INVALID_ARG, "sddm_render: need 1..4096 descriptors");
    for (int r = 0; r < n; ++r) {
        const sddm_render_desc &x = d[r];
        if (x.width < 1 || x.height < 1 || x.spp < 1 || x.width > 65536 || x.height > 65536 || x.spp > 65536)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: width/height/spp out of range");
        if ((int64_t)x.width * x.height > 0xffffffffLL)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: more pixels than the 32-bit counter word holds");
        if (x.max_depth < 1 || x.max_depth > kMaxDepth)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: max_depth must be in 1..64");
        if (!x.xyz_out) return fail(SDDM_ERR_INVALID_ARG, "sddm_render: xyz_out is NULL");
        if (x.method != d[0].method || x.bsdf_mode != d[0].bsdf_mode)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: renders of one call must share method and bsdf_mode");
        if (x.method != SDDM_METHOD_MEGAKERNEL && x.method != SDDM_METHOD_DDM)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: unknown method");
        if (x.bsdf_mode != SDDM_BSDF_EXACT && x.bsdf_mode != SDDM_BSDF_MLP)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: unknown bsdf_mode");
        const sddm_camera &c = x.camera;
        float f[3] = {c.look[0] - c.pos[0], c.look[1] - c.pos[1], c.look[2] - c.pos[2]};
        float fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        float cr[3] = {f[1] * c.up[2] - f[2] * c.up[1], f[2] * c.up[0] - f[0] * c.up[2], f[0] * c.up[1] - f[1] * c.up[0]};
        float crl = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        if (!(fl > 0) || !(crl > 1e-6f * fl) || !std::isfinite(fl))
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: degenerate camera (look == pos or up parallel)");
        if (!(c.ortho_height > 0) && !(c.vfov_deg > 0.0f && c.vfov_deg < 179.0f))
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: vfov_deg must be in (0, 179)");
        if (x.glass_s)
            for (size_t m = 0; m < ctx->mats.size(); ++m)
                if (x.glass_s[m] > 1.0f || std::isnan(x.glass_s[m]))
                    return fail(SDDM_ERR_INVALID_ARG, "sddm_render: glass_s entries must be <= 1 (negative = default)");
    }
    return SDDM_OK;
}

// Camera frame in double from the float inputs, rounded once.
static void camera_frame(const sddm_render_desc &x, RenderInfo &ri) {
    const sddm_camera &c = x.camera;
    double f[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) f[a] = (double)c.look[a] - c.pos[a];
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] /= fl;
    r[0] = f[1] * c.up[2] - f[2] * c.up[1];
    r[1] = f[2] * c.up[0] - f[0] * c.up[2];
    r[2] = f[0] * c.up[1] - f[1] * c.up[0];
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] /= rl;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    double aspect = (double)x.width / (double)x.height;
    double sy, sx;
    if (c.ortho_height > 0) {
        sy = 0.5 * (double)c.ortho_height;
        ri.ortho = 1;
    } else {
        sy = std::tan(0.5 * (double)c.vfov_deg * 3.14159265358979323846 / 180.0);
        ri.ortho = 0;
    }
    sx = sy * aspect;
    for (int a = 0; a < 3; ++a) {
        ri.cam_o[a] = c.pos[a];
        ri.cam_f[a] = (float)f[a];
        ri.cam_x[a] = (float)(sx * r[a]);
        ri.cam_y[a] = (float)(sy * u[a]);
    }
}

}  // extern "C"

namespace sddm {
// Read-only view of a context for entry points defined in other files.
int ctx_view(sddm_ctx *ctx, CtxView *v) {
    if (!ctx || !v) return fail(SDDM_ERR_INVALID_ARG, "ctx is NULL");
    v->device = ctx->device;
    v->stream = ctx->stream;
    v->built = ctx->built;
    v->dev = ctx->dev;
    v->n_mat = (int)ctx->mats.size();
    v->ev0 = ctx->ev0;
    v->ev1 = ctx->ev1;
    return SDDM_OK;
}
int check_render_desc(const sddm_ctx *ctx, const sddm_render_desc *d, int n) { return validate_desc(ctx, d, n); }
void render_info_for(const sddm_ctx *ctx, const sddm_render_desc &x, RenderInfo &ri) {
    std::memset(&ri, 0, sizeof(ri));
    ri.width = x.width;
    ri.height = x.height;
    ri.spp = x.spp;
    ri.max_depth = x.max_depth;
    ri.seed = x.seed;
    ri.render_id = x.render_id;
    ri.nee = x.nee ? 1 : 0;
    camera_frame(x, ri);
    (void)ctx;
}
float material_state(const sddm_ctx *ctx, const sddm_render_desc &x, int m) {
    return (x.glass_s && x.glass_s[m] >= 0.0f) ? x.glass_s[m] : ctx->mats[m].s_default;
}
}  // namespace sddm

extern "C" {

int sddm_render(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_stats *st) {
    int rc = validate_desc(ctx, d, n);
    if (rc != SDDM_OK) return rc;
    const float *mlp_params = nullptr;
    float mlp_dmin = 0.f, mlp_dmax = 0.f;
    if (d[0].bsdf_mode == SDDM_BSDF_MLP) {
        if (d[0].method != SDDM_METHOD_DDM)
            return fail(SDDM_ERR_INVALID_ARG, "sddm_render: the learned glass model runs with the DDM method");
        int net_id = -1;
        ctx->net_of_mat.resize(ctx->mats.size(), -1);
        for (size_t m = 0; m < ctx->mats.size(); ++m) {
            if (ctx->mats[m].kind != kGlass) continue;
            const int id = ctx->net_of_mat[m];
            if (id < 0) return fail(SDDM_ERR_MLP_UNTRAINED, "sddm_render: a glass material has no trained surrogate");
            if (net_id >= 0 && id != net_id)
                return fail(SDDM_ERR_INVALID_ARG, "sddm_render: the learned model supports one network per call");
            net_id = id;
        }
        if (net_id < 0) return fail(SDDM_ERR_INVALID_ARG, "sddm_render: no glass material in the scene");
        mlp_params = ctx->nets[net_id]->params.as<float>();
        mlp_dmin = ctx->nets[net_id]->dmin;
        mlp_dmax = ctx->nets[net_id]->dmax;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_render: cudaSetDevice");
    const int M = (int)ctx->mats.size();
    std::vector<RenderInfo> info(n);
    std::vector<float> state((size_t)n * M);
    std::vector<float *> outs(n), aov_x(n);
    std::vector<int32_t *> aov_p(n);
    int64_t paths = 0, pixels = 0;
    bool any_aov = false;
    for (int r = 0; r < n; ++r) {
        const sddm_render_desc &x = d[r];
        RenderInfo &ri = info[r];
        std::memset(&ri, 0, sizeof(ri));
        ri.path_begin = paths;
        ri.pixel_begin = pixels;
        ri.width = x.width;
        ri.height = x.height;
        ri.spp = x.spp;
        ri.max_depth = x.max_depth;
        ri.seed = x.seed;
        ri.render_id = x.render_id;
        ri.nee = x.nee ? 1 : 0;
        ri.s_offset = r * M;
        camera_frame(x, ri);
        for (int m = 0; m < M; ++m)
            state[(size_t)r * M + m] = (x.glass_s && x.glass_s[m] >= 0.0f) ? x.glass_s[m] : ctx->mats[m].s_default;
        outs[r] = x.xyz_out;
        aov_x[r] = x.aov_sample_xyz;
        aov_p[r] = x.aov_first_prim;
        any_aov |= x.aov_sample_xyz != nullptr || x.aov_first_prim != nullptr;
        paths += (int64_t)x.width * x.height * x.spp;
        pixels += (int64_t)x.width * x.height;
    }
    cudaStream_t s = ctx->stream;
    if ((e = ctx->d_info.upload(info, s)) || (e = ctx->d_state.upload(state, s)) || (e = ctx->d_out_tab.upload(outs, s)) ||
        (e = ctx->d_aov_xyz_tab.upload(aov_x, s)) || (e = ctx->d_aov_prim_tab.upload(aov_p, s)) ||
        (e = ctx->d_counters.ensure(kNumCounters * sizeof(unsigned long long))) || (e = ctx->d_err.ensure(16)))
        return cuda_fail(e, "sddm_render: upload of the render table");
    if ((e = cudaMemsetAsync(ctx->d_counters.p, 0, kNumCounters * sizeof(unsigned long long), s)) ||
        (e = cudaMemsetAsync(ctx->d_err.p, 0, 16, s)))
        return cuda_fail(e, "sddm_render: memset");
    RenderBatch rb;
    rb.info = ctx->d_info.as<RenderInfo>();
    rb.n = n;
    rb.state_s = ctx->d_state.as<float>();

    // chunks of whole pixels, at most `cap` paths each
    int64_t cap = ctx->opts.paths_in_flight > 0 ? ctx->opts.paths_in_flight : (int64_t)1 << 22;
    int64_t max_spp = 1;
    for (int r = 0; r < n; ++r) max_spp = std::max<int64_t>(max_spp, d[r].spp);
    cap = std::max(cap, max_spp);

    if ((e = cudaEventRecord(ctx->ev0, s)) != cudaSuccess) return cuda_fail(e, "sddm_render: event");
    ctx->ddm_buf.events_used = 0;
    ctx->ddm_buf.mlp_events_used = 0;
    int64_t launches = 0;
    const int time_trace = (ctx->profile & SDDM_PROFILE_TIME_TRACE) != 0;
    const int count_trav = (ctx->profile & SDDM_PROFILE_COUNT_TRAVERSAL) != 0;
    // Every kernel and memset of the call, on stream `ls` (eager, or captured into a graph).
    auto launch_all = [&](cudaStream_t ls) -> int {
        cudaStream_t s = ls;
        int64_t path0 = 0, pix0 = 0;
        int rr = 0;   // render of pix0
        while (path0 < paths) {
            // extend the chunk pixel-row by pixel-row within renders
            int64_t path1 = path0, pix1 = pix0;
            int r = rr;
            while (r < n) {
                const RenderInfo &ri = info[r];
                int64_t render_pix_end = ri.pixel_begin + (int64_t)ri.width * ri.height;
                int64_t room = (cap - (path1 - path0)) / ri.spp;
                if (room <= 0) break;
                int64_t take = std::min(room, render_pix_end - pix1);
                pix1 += take;
                path1 += take * ri.spp;
                if (pix1 == render_pix_end) ++r; else break;
            }
            const int64_t np = path1 - path0;
            if ((e = ctx->d_samples.ensure((size_t)np * 3 * sizeof(float))) ||
                (any_aov && (e = ctx->d_first.ensure((size_t)np * sizeof(int32_t)))))
                return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_render: scratch allocation failed")
                                                      : cuda_fail(e, "sddm_render: scratch");
            if (d[0].method == SDDM_METHOD_MEGAKERNEL) {
                MegaArgs a;
                a.sc = ctx->dev;
                a.rb = rb;
                a.path_begin = path0;
                a.path_count = np;
                a.sample_xyz = ctx->d_samples.as<float>();
                a.first_prim = any_aov ? ctx->d_first.as<int32_t>() : nullptr;
                a.counters = ctx->d_counters.as<unsigned long long>();
                a.error_flag = ctx->d_err.as<int>();
                a.count_traversal = count_trav;
                a.pm = ctx->pm_view;
                a.pmc = ctx->pmc_view;
                cudaEvent_t t0 = nullptr, t1 = nullptr;
                if (time_trace) {
                    if ((e = ctx->ddm_buf.event_pair(t0, t1)) || (e = cudaEventRecord(t0, s)))
                        return cuda_fail(e, "sddm_render: events");
                }
                if ((e = launch_megakernel(a, s)) != cudaSuccess) return cuda_fail(e, "sddm_render: megakernel launch");
                if (time_trace && (e = cudaEventRecord(t1, s)) != cudaSuccess) return cuda_fail(e, "sddm_render: events");
                launches += 1;
            } else {
                DDMRun run;
                run.sc = ctx->dev;
                run.g = ctx->ddm;
                run.rb = rb;
                run.path_begin = path0;
                run.path_count = np;
                run.max_depth = 1;
                for (int q = 0; q < n; ++q) run.max_depth = std::max(run.max_depth, d[q].max_depth);
                run.sample_xyz = ctx->d_samples.as<float>();
                run.first_prim = any_aov ? ctx->d_first.as<int32_t>() : nullptr;
                run.counters = ctx->d_counters.as<unsigned long long>();
                run.error_flag = ctx->d_err.as<int>();
                run.sm_count = ctx->sm_count;
                run.blocks_per_sm = ctx->opts.blocks_per_sm;
                run.queue_capacity = ctx->opts.queue_capacity;
                run.bsdf_mode = d[0].bsdf_mode;
                run.time_trace = time_trace;
                run.count_traversal = count_trav;
                run.launches = &launches;
                run.mlp_params = mlp_params;
                run.mlp_dmin = mlp_dmin;
                run.mlp_dmax = mlp_dmax;
                run.probe_key = d[0].seed ^ 0x9e3779b9u;
                run.cache = ctx->opts.cell_cache_bytes > 0 ? &ctx->cache : nullptr;
                int rc2 = ctx->pm_view.on ? ddm_trace_chunk_pm(run, ctx->pm_view, ctx->pmc_view, ctx->ddm_buf, s)
                                          : ddm_trace_chunk(run, ctx->ddm_buf, s);
                if (rc2 != SDDM_OK) return rc2;
            }
            ReduceArgs ra;
            ra.rb = rb;
            ra.path_begin = path0;
            ra.sample_xyz = ctx->d_samples.as<float>();
            ra.xyz_out = ctx->d_out_tab.as<float *>();
            ra.aov_xyz = ctx->d_aov_xyz_tab.as<float *>();
            ra.aov_prim = ctx->d_aov_prim_tab.as<int32_t *>();
            ra.first_prim = any_aov ? ctx->d_first.as<int32_t>() : nullptr;
            if ((e = launch_reduce_pixels(ra, pix0, pix1 - pix0, s)) != cudaSuccess)
                return cuda_fail(e, "sddm_render: reduce launch");
            launches += 1;
            path0 = path1;
            pix0 = pix1;
            rr = r;
            while (rr < n && pix0 >= info[rr].pixel_begin + (int64_t)info[rr].width * info[rr].height) ++rr;
        }
        return SDDM_OK;
    };
    // the subdomain cache plans each wave on the host from the rays waiting per cell: not capturable
    const bool graphable = ctx->graphs_enabled && !count_trav && !time_trace && !ctx->pm_view.on &&
                           ctx->opts.cell_cache_bytes == 0;
    ctx->cache.loads = ctx->cache.plan.hits = ctx->cache.bytes_loaded = ctx->cache.groups = 0;
    std::string key;
    if (graphable) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "%lld|%d|%d|%d|%d|%lld|%d|%u|%d|%p|%p|%p|%p|%p|%p", (long long)ctx->build_id,
                      n, d[0].method, d[0].bsdf_mode, (int)any_aov, (long long)ctx->opts.paths_in_flight,
                      ctx->opts.blocks_per_sm, d[0].seed, time_trace, ctx->d_samples.p, ctx->d_first.p,
                      ctx->ddm_buf.mem, ctx->d_info.p, (const void *)mlp_params, ctx->d_counters.p);
        key = buf;
        for (int r = 0; r < n; ++r) {
            std::snprintf(buf, sizeof buf, "|%d,%d,%d,%d", d[r].width, d[r].height, d[r].spp, d[r].max_depth);
            key += buf;
        }
    }
    auto it = graphable ? ctx->graphs.find(key) : ctx->graphs.end();
    if (graphable && (it != ctx->graphs.end() || ctx->seen[key] > 0)) {
        if ((e = cudaEventRecord(ctx->hand0, s)) || (e = cudaStreamWaitEvent(ctx->gstream, ctx->hand0, 0)))
            return cuda_fail(e, "sddm_render: stream hand-off");
        if (it == ctx->graphs.end()) {
            if (ctx->graphs.size() >= 8) {
                for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
                ctx->graphs.clear();
            }
            cudaGraph_t graph = nullptr;
            if ((e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal)))
                return cuda_fail(e, "sddm_render: begin capture");
            int rc2 = launch_all(ctx->gstream);
            cudaError_t ce = cudaStreamEndCapture(ctx->gstream, &graph);
            if (rc2 != SDDM_OK) {
                if (graph) cudaGraphDestroy(graph);
                return rc2;
            }
            if (ce) return cuda_fail(ce, "sddm_render: end capture");
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce) return cuda_fail(ce, "sddm_render: graph instantiate");
            it = ctx->graphs.emplace(key, sddm_ctx::Graph{exec, launches, ctx->ddm_buf.events_used}).first;
        }
        launches = it->second.launches;
        ctx->ddm_buf.events_used = it->second.events_used;
        if ((e = cudaGraphLaunch(it->second.exec, ctx->gstream)) || (e = cudaEventRecord(ctx->hand1, ctx->gstream)) ||
            (e = cudaStreamWaitEvent(s, ctx->hand1, 0)))
            return cuda_fail(e, "sddm_render: graph launch");
    } else {
        int rc2 = launch_all(s);
        if (rc2 != SDDM_OK) return rc2;
        if (graphable) ctx->seen[key] = 1;
    }
    if ((e = cudaEventRecord(ctx->ev1, s)) != cudaSuccess) return cuda_fail(e, "sddm_render: event");
    unsigned long long cnt[kNumCounters];
    int err[4];
    if ((e = cudaMemcpyAsync(cnt, ctx->d_counters.p, sizeof(cnt), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(err, ctx->d_err.p, sizeof(err), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "sddm_render: kernel execution");
    if (err[0] != 0) {
        char msg[160];
        std::snprintf(msg, sizeof msg, "sddm_render: device reported error %d (detail %d, %d)", err[0], err[1], err[2]);
        return fail(err[0] == 1 ? SDDM_ERR_QUEUE_OVERFLOW : (err[0] == 2 ? SDDM_ERR_TIMEOUT : SDDM_ERR_DEVICE_CHECK),
                    msg);
    }
    if (st) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        st->paths = paths;
        st->segments_ext = (int64_t)cnt[0];
        st->segments_shadow = (int64_t)cnt[1];
        st->glass_queries = (int64_t)cnt[2];
        st->crossings = (int64_t)cnt[3];
        st->mlp_fallbacks = (int64_t)cnt[4];
        st->mlp_batches = (int64_t)cnt[8];
        st->cache_loads = ctx->cache.loads;
        st->cache_hits = ctx->cache.plan.hits;
        st->cache_bytes_loaded = ctx->cache.bytes_loaded;
        st->gpu_ms = ms;
        st->kernel_launches = launches;
        st->node_visits = count_trav ? (int64_t)cnt[5] : 0;
        st->tri_tests = count_trav ? (int64_t)cnt[6] : 0;
        st->ray_visits = count_trav ? (int64_t)cnt[7] : 0;
        st->ray_continues = count_trav ? (int64_t)cnt[10] : 0;
        double tms = 0.0;
        for (int k = 0; k + 1 < ctx->ddm_buf.events_used; k += 2) {
            float x = 0.f;
            cudaEventElapsedTime(&x, ctx->ddm_buf.events[k], ctx->ddm_buf.events[k + 1]);
            tms += x;
        }
        st->trace_ms = tms;
        st->trace_launches = ctx->ddm_buf.events_used / 2;
        double mms = 0.0;
        for (int k = 0; k + 1 < ctx->ddm_buf.mlp_events_used; k += 2) {
            float x = 0.f;
            cudaEventElapsedTime(&x, ctx->ddm_buf.mlp_events[k], ctx->ddm_buf.mlp_events[k + 1]);
            mms += x;
        }
        st->mlp_ms = mms;
        st->mlp_rows = (int64_t)cnt[9];
    }
    return SDDM_OK;
}

int sddm_render_photon_map(sddm_ctx *ctx, const sddm_render_desc *d, int64_t n_photons, float radius,
                           float caustic_radius, sddm_stats *st, sddm_photon_stats *pst) {
    int rc = validate_desc(ctx, d, 1);
    if (rc != SDDM_OK) return rc;
    if (d->method == SDDM_METHOD_MEGAKERNEL && d->bsdf_mode != SDDM_BSDF_EXACT)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: the megakernel method needs the exact glass model");
    if (!d->nee || d->max_depth < 2)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: needs nee = 1 and max_depth >= 2");
    if (!(radius > 0.0f) || !std::isfinite(radius))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: radius must be positive and finite");
    if (!(caustic_radius >= 0.0f) || !std::isfinite(caustic_radius))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: caustic_radius must be finite and >= 0");
    if (ctx->opts.cell_cache_bytes > 0 && d->method == SDDM_METHOD_DDM)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: not with the subdomain cache (cell_cache_bytes)");
    const bool two_maps = caustic_radius > 0.0f;
    const int64_t per = d->max_depth - 1;
    if (n_photons < 0 || n_photons > ((int64_t)1 << 31) / per - 1)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_photon_map: n_photons * (max_depth - 1) must stay below 2^31");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_render_photon_map: cudaSetDevice");
    const int M = (int)ctx->mats.size(), L = ctx->L;
    const int64_t slots = n_photons * per;
    std::vector<float> state(M);
    for (int m = 0; m < M; ++m) state[m] = material_state(ctx, *d, m);
    // grids over the scene box, cells of side >= the map's radius, at most ~2^24 cells
    const DDMScene &g = ctx->ddm;
    auto grid_for = [&](float r, PhotonGridView &v) {
        double ext[3], vol = 1.0;
        for (int a = 0; a < 3; ++a) {
            ext[a] = std::max<double>(g.hi[a] - g.lo[a], 1e-6);
            vol *= ext[a];
        }
        const double cell = std::max<double>(r, std::cbrt(vol / (double)(1 << 24)) * 1.01);
        int64_t n = 1;
        for (int a = 0; a < 3; ++a) {
            v.lo[a] = g.lo[a];
            v.dims[a] = (int)std::floor(ext[a] / cell) + 1;
            n *= v.dims[a];
        }
        v.cell = (float)cell;
        v.radius = r;
        return n;
    };
    PhotonGridView v{}, vc{};
    const int64_t cells = grid_for(radius, v);
    const int64_t cells_c = two_maps ? grid_for(caustic_radius, vc) : 1;
    const size_t sl = (size_t)std::max<int64_t>(slots, 1);
    cudaStream_t s = ctx->stream;
    if ((e = ctx->pm_state.upload(state, s)) ||
        (e = ctx->pm_scratch.ensure(sizeof(float) * (size_t)std::max<int64_t>(n_photons, 1) * L)) ||
        (e = ctx->pm_pos.ensure(sizeof(float4) * sl)) || (e = ctx->pm_dir.ensure(sizeof(float4) * sl)) ||
        (e = ctx->pm_pow.ensure(sizeof(float) * sl * L)) || (e = ctx->pm_cnt.ensure(sizeof(int) * (size_t)cells)) ||
        (e = ctx->pm_start.ensure(sizeof(int) * (size_t)(cells + 1))) ||
        (e = ctx->pm_fill.ensure(sizeof(int) * (size_t)cells)) || (e = ctx->pm_order.ensure(sizeof(int) * sl)) ||
        (e = ctx->pm_sums.ensure(sizeof(int) * (size_t)(cells / 1024 + 1))) ||
        (e = ctx->pm_cntr.ensure(16 * sizeof(unsigned long long))) ||
        (two_maps && ((e = ctx->pmc_cnt.ensure(sizeof(int) * (size_t)cells_c)) ||
                      (e = ctx->pmc_start.ensure(sizeof(int) * (size_t)(cells_c + 1))) ||
                      (e = ctx->pmc_fill.ensure(sizeof(int) * (size_t)cells_c)) ||
                      (e = ctx->pmc_order.ensure(sizeof(int) * sl)) ||
                      (e = ctx->pmc_sums.ensure(sizeof(int) * (size_t)(cells_c / 1024 + 1))))))
        return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_render_photon_map: device allocation failed")
                                              : cuda_fail(e, "sddm_render_photon_map: scratch");
    if ((e = cudaEventRecord(ctx->ev0, s)) || (e = cudaMemsetAsync(ctx->pm_pos.p, 0, sizeof(float4) * sl, s)) ||
        (e = cudaMemsetAsync(ctx->pm_cntr.p, 0, 16 * sizeof(unsigned long long), s)))
        return cuda_fail(e, "sddm_render_photon_map: memset");
    unsigned long long *cntr = ctx->pm_cntr.as<unsigned long long>();
    int64_t launches = 0;
    if (n_photons > 0 && d->method == SDDM_METHOD_DDM) {
        // through the subdomain queues, in chunks of at most paths_in_flight photons
        const int64_t chunk = ctx->opts.paths_in_flight > 0 ? ctx->opts.paths_in_flight : (int64_t)1 << 22;
        for (int64_t b0 = 0; b0 < n_photons; b0 += chunk) {
            DDMPhotonRun pr;
            pr.sc = ctx->dev;
            pr.g = ctx->ddm;
            pr.begin = b0;
            pr.count = std::min(chunk, n_photons - b0);
            pr.n_total = n_photons;
            pr.max_depth = d->max_depth;
            pr.seed = d->seed;
            pr.render_id = d->render_id;
            pr.state_s = ctx->pm_state.as<float>();
            pr.pos = ctx->pm_pos.as<float4>();
            pr.dir = ctx->pm_dir.as<float4>();
            pr.pow = ctx->pm_pow.as<float>();
            pr.counters = ctx->pm_cntr.as<unsigned long long>() + 2;
            pr.error_flag = ctx->pm_cntr.as<int>() + 20;
            pr.sm_count = ctx->sm_count;
            pr.blocks_per_sm = ctx->opts.blocks_per_sm;
            pr.launches = &launches;
            const int rc2 = ddm_photon_pass(pr, ctx->pm_ddm_buf, s);
            if (rc2 != SDDM_OK) return rc2;
        }
    } else if (n_photons > 0) {
        PhotonTraceArgs ta;
        ta.n_photons = n_photons;
        ta.max_depth = d->max_depth;
        ta.seed = d->seed;
        ta.render_id = d->render_id;
        ta.state_s = ctx->pm_state.as<float>();
        ta.scratch = ctx->pm_scratch.as<float>();
        ta.pos = ctx->pm_pos.as<float4>();
        ta.dir = ctx->pm_dir.as<float4>();
        ta.pow = ctx->pm_pow.as<float>();
        ta.segments = cntr;
        if ((e = launch_photon_trace(ctx->dev, ta, s)) != cudaSuccess)
            return cuda_fail(e, "sddm_render_photon_map: photon launch");
        launches += 1;
    }
    v.pos = ctx->pm_pos.as<float4>();
    v.dir = ctx->pm_dir.as<float4>();
    v.pow = ctx->pm_pow.as<float>();
    v.cell_start = ctx->pm_start.as<int>();
    v.order = ctx->pm_order.as<int>();
    // one map of every stored photon, or the global photons (kind 1) and the caustic ones (kind 2) apart
    if ((e = build_photon_grid(v, slots, two_maps ? 1 : 0, ctx->pm_cnt.as<int>(), ctx->pm_start.as<int>(),
                               ctx->pm_fill.as<int>(), ctx->pm_order.as<int>(), ctx->pm_sums.as<int>(), cntr + 1, s)) !=
        cudaSuccess)
        return cuda_fail(e, "sddm_render_photon_map: grid build");
    launches += slots > 0 ? 5 : 3;
    if (two_maps) {
        vc.pos = v.pos;
        vc.dir = v.dir;
        vc.pow = v.pow;
        vc.cell_start = ctx->pmc_start.as<int>();
        vc.order = ctx->pmc_order.as<int>();
        if ((e = build_photon_grid(vc, slots, 2, ctx->pmc_cnt.as<int>(), ctx->pmc_start.as<int>(),
                                   ctx->pmc_fill.as<int>(), ctx->pmc_order.as<int>(), ctx->pmc_sums.as<int>(),
                                   cntr + 11, s)) != cudaSuccess)
            return cuda_fail(e, "sddm_render_photon_map: caustic grid build");
        launches += slots > 0 ? 5 : 3;
    }
    unsigned long long hc[16];
    if ((e = cudaEventRecord(ctx->ev1, s)) ||
        (e = cudaMemcpyAsync(hc, cntr, sizeof(hc), cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "sddm_render_photon_map: photon pass");
    // counters: [0] megakernel photon segments, [1] stored (global), [2..9] DDM pass (segments at 2), int error
    // word at [10], [11] stored caustic
    int perr;
    std::memcpy(&perr, hc + 10, sizeof perr);
    if (perr != 0) {
        char msg[128];
        std::snprintf(msg, sizeof msg, "sddm_render_photon_map: device reported error %d in the photon pass", perr);
        return fail(perr == 1 ? SDDM_ERR_QUEUE_OVERFLOW : SDDM_ERR_DEVICE_CHECK, msg);
    }
    float pms = 0.f;
    cudaEventElapsedTime(&pms, ctx->ev0, ctx->ev1);
    v.on = 1;
    vc.on = two_maps ? 1 : 0;
    ctx->pm_view = v;
    ctx->pmc_view = vc;
    rc = sddm_render(ctx, d, 1, st);
    ctx->pm_view = PhotonGridView{};
    ctx->pmc_view = PhotonGridView{};
    if (rc != SDDM_OK) return rc;
    if (pst) {
        pst->photons = n_photons;
        pst->photon_segments = (int64_t)(hc[0] + hc[2]);
        pst->stored = (int64_t)hc[1];
        pst->stored_caustic = two_maps ? (int64_t)hc[11] : 0;
        pst->grid_cells = cells + (two_maps ? cells_c : 0);
        pst->photon_ms = pms;
        pst->kernel_launches = launches;
    }
    return SDDM_OK;
}

int sddm_render_progressive_photon_map(sddm_ctx *ctx, const sddm_render_desc *d, int n_passes, int64_t n_photons,
                                       float radius, float caustic_radius, float alpha, sddm_stats *st,
                                       sddm_photon_stats *pst) {
    int rc = validate_desc(ctx, d, 1);
    if (rc != SDDM_OK) return rc;
    if (n_passes < 1 || !(alpha > 0.0f && alpha <= 1.0f))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_render_progressive_photon_map: needs n_passes >= 1 and 0 < alpha <= 1");
    if (!d->xyz_out) return fail(SDDM_ERR_INVALID_ARG, "sddm_render_progressive_photon_map: xyz_out is NULL");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_render_progressive_photon_map: cudaSetDevice");
    const int64_t nv = (int64_t)d->width * d->height * 3;
    if ((e = ctx->pm_img.ensure(sizeof(float) * (size_t)nv)) != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_render_progressive_photon_map: allocation failed")
                                              : cuda_fail(e, "sddm_render_progressive_photon_map: scratch");
    sddm_stats tot{};
    sddm_photon_stats ptot{};
    double r2 = (double)radius * radius, rc2 = (double)caustic_radius * caustic_radius;
    for (int j = 1; j <= n_passes; ++j) {
        sddm_render_desc dj = *d;
        dj.render_id = d->render_id + (uint32_t)(j - 1);   // independent photons and camera samples per pass
        dj.xyz_out = j == 1 ? d->xyz_out : ctx->pm_img.as<float>();
        dj.aov_sample_xyz = nullptr;
        dj.aov_first_prim = nullptr;
        sddm_stats sj{};
        sddm_photon_stats pj{};
        rc = sddm_render_photon_map(ctx, &dj, n_photons, (float)std::sqrt(r2), (float)std::sqrt(rc2), &sj, &pj);
        if (rc != SDDM_OK) return rc;
        if (j > 1) {
            if ((e = launch_blend(nv, (float)(j - 1) / (float)j, 1.0f / (float)j, ctx->pm_img.as<float>(), d->xyz_out,
                                  ctx->stream)) != cudaSuccess ||
                (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
                return cuda_fail(e, "sddm_render_progressive_photon_map: blend");
        }
        tot.paths += sj.paths;
        tot.segments_ext += sj.segments_ext;
        tot.segments_shadow += sj.segments_shadow;
        tot.crossings += sj.crossings;
        tot.glass_queries += sj.glass_queries;
        tot.mlp_fallbacks += sj.mlp_fallbacks;
        tot.mlp_batches += sj.mlp_batches;
        tot.cache_loads += sj.cache_loads;
        tot.cache_hits += sj.cache_hits;
        tot.cache_bytes_loaded += sj.cache_bytes_loaded;
        tot.mlp_ms += sj.mlp_ms;
        tot.mlp_rows += sj.mlp_rows;
        tot.gpu_ms += sj.gpu_ms;
        tot.kernel_launches += sj.kernel_launches + (j > 1 ? 1 : 0);
        ptot.photons += pj.photons;
        ptot.photon_segments += pj.photon_segments;
        ptot.stored += pj.stored;
        ptot.stored_caustic += pj.stored_caustic;
        ptot.grid_cells = pj.grid_cells;
        ptot.photon_ms += pj.photon_ms;
        ptot.kernel_launches += pj.kernel_launches;
        // radius of the next pass: r^2 (j + alpha) / (j + 1)
        r2 *= ((double)j + alpha) / ((double)j + 1.0);
        rc2 *= ((double)j + alpha) / ((double)j + 1.0);
    }
    if (st) *st = tot;
    if (pst) *pst = ptot;
    return SDDM_OK;
}

int sddm_render_host(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_stats *st) {
    int rc = validate_desc(ctx, d, n);
    if (rc != SDDM_OK) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_render_host: cudaSetDevice");
    std::vector<sddm_render_desc> dd(d, d + n);
    std::vector<void *> bufs;
    auto cleanup = [&]() {
        for (void *p : bufs) cudaFree(p);
    };
    for (int r = 0; r < n; ++r) {
        size_t px = (size_t)d[r].width * d[r].height;
        void *p = nullptr;
        if ((e = cudaMalloc(&p, px * 3 * sizeof(float))) != cudaSuccess) {
            cleanup();
            return fail(SDDM_ERR_OOM, "sddm_render_host: device allocation failed");
        }
        bufs.push_back(p);
        dd[r].xyz_out = (float *)p;
        dd[r].aov_sample_xyz = nullptr;
        dd[r].aov_first_prim = nullptr;
        if (d[r].aov_sample_xyz) {
            if ((e = cudaMalloc(&p, px * d[r].spp * 3 * sizeof(float))) != cudaSuccess) {
                cleanup();
                return fail(SDDM_ERR_OOM, "sddm_render_host: device allocation failed");
            }
            bufs.push_back(p);
            dd[r].aov_sample_xyz = (float *)p;
        }
        if (d[r].aov_first_prim) {
            if ((e = cudaMalloc(&p, px * d[r].spp * sizeof(int32_t))) != cudaSuccess) {
                cleanup();
                return fail(SDDM_ERR_OOM, "sddm_render_host: device allocation failed");
            }
            bufs.push_back(p);
            dd[r].aov_first_prim = (int32_t *)p;
        }
    }
    rc = sddm_render(ctx, dd.data(), n, st);
    for (int r = 0; r < n && rc == SDDM_OK; ++r) {
        size_t px = (size_t)d[r].width * d[r].height;
        if ((e = cudaMemcpyAsync(d[r].xyz_out, dd[r].xyz_out, px * 3 * sizeof(float), cudaMemcpyDeviceToHost,
                                 ctx->stream)) ||
            (d[r].aov_sample_xyz &&
             (e = cudaMemcpyAsync(d[r].aov_sample_xyz, dd[r].aov_sample_xyz, px * d[r].spp * 3 * sizeof(float),
                                  cudaMemcpyDeviceToHost, ctx->stream))) ||
            (d[r].aov_first_prim &&
             (e = cudaMemcpyAsync(d[r].aov_first_prim, dd[r].aov_first_prim, px * d[r].spp * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, ctx->stream))))
            rc = cuda_fail(e, "sddm_render_host: copy back");
    }
    if (rc == SDDM_OK && (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        rc = cuda_fail(e, "sddm_render_host: synchronize");
    cleanup();
    return rc;
}

// Pilot-timed choice of subdomain grid, persistent blocks per SM and paths in
// flight (Sec. 5's load balancing, settled here by measurement).
int sddm_autotune(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_build_opts *best) {
    if (!ctx || !d || !best) return fail(SDDM_ERR_INVALID_ARG, "sddm_autotune: NULL argument");
    if (ctx->L <= 0 || ctx->mats.empty() || ctx->F.empty())
        return fail(SDDM_ERR_INVALID_ARG, "sddm_autotune: spectrum, materials and mesh are required");
    sddm_build_opts base = ctx->built ? ctx->opts : sddm_build_opts{};
    default_opts(base);
    // pilot: the same renders at 1 spp and at most 512 x 512 pixels
    std::vector<sddm_render_desc> pilot(d, d + n);
    std::vector<void *> bufs;
    int rc = SDDM_OK;
    for (auto &p : pilot) {
        p.spp = 1;
        p.width = std::min(p.width, 512);
        p.height = std::min(p.height, 512);
        p.method = SDDM_METHOD_DDM;
        p.aov_sample_xyz = nullptr;
        p.aov_first_prim = nullptr;
        void *q = nullptr;
        if (cudaMalloc(&q, (size_t)p.width * p.height * 3 * sizeof(float)) != cudaSuccess) {
            rc = fail(SDDM_ERR_OOM, "sddm_autotune: pilot output allocation failed");
            break;
        }
        bufs.push_back(q);
        p.xyz_out = (float *)q;
    }
    const int grids[][3] = {{1, 1, 1}, {2, 2, 2}, {4, 4, 2}, {8, 4, 4}};
    const int bps_list[] = {4, 8, 16};
    double best_rate = -1.0;
    sddm_build_opts chosen = base;
    for (int trial = 0; trial < 3 * (int)(sizeof grids / sizeof grids[0]); ++trial) {
        if (rc != SDDM_OK) break;
        const int *gdim = grids[trial / 3];
        // hand-off schedule: the neighbour's queue every wave (0), the lane carries
        // rays across faces (1), or one queue wave and then the lane (2)
        const int sched = trial % 3;
        if (sched && ((gdim[0] == 1 && gdim[1] == 1 && gdim[2] == 1) || base.cell_cache_bytes > 0)) continue;
        sddm_build_opts o = base;
        for (int a = 0; a < 3; ++a) o.grid[a] = gdim[a];
        o.continue_cells = sched == 1;
        o.handoff_waves = sched == 2 ? 1 : 0;
        if ((rc = sddm_build(ctx, &o)) != SDDM_OK) break;
        for (int bps : bps_list) {
            ctx->opts.blocks_per_sm = bps;
            sddm_stats st{};
            if ((rc = sddm_render(ctx, pilot.data(), n, &st)) != SDDM_OK) break;   // warm-up
            if ((rc = sddm_render(ctx, pilot.data(), n, &st)) != SDDM_OK) break;
            double rate = (double)(st.segments_ext + st.segments_shadow) / std::max(st.gpu_ms, 1e-6);
            if (rate > best_rate) {
                best_rate = rate;
                chosen = ctx->opts;
            }
        }
    }
    // second stage: paths in flight per chunk (memory per chunk against the
    // per-chunk launch overhead) for the chosen grid and blocks per SM
    if (rc == SDDM_OK && (rc = sddm_build(ctx, &chosen)) == SDDM_OK) {
        const int64_t pif_list[] = {(int64_t)1 << 21, (int64_t)1 << 22, (int64_t)1 << 23};
        sddm_build_opts stage = chosen;
        for (int64_t pif : pif_list) {
            ctx->opts.paths_in_flight = pif;
            sddm_stats st{};
            if ((rc = sddm_render(ctx, pilot.data(), n, &st)) != SDDM_OK) break;
            if ((rc = sddm_render(ctx, pilot.data(), n, &st)) != SDDM_OK) break;
            double rate = (double)(st.segments_ext + st.segments_shadow) / std::max(st.gpu_ms, 1e-6);
            if (rate > best_rate) {
                best_rate = rate;
                stage = ctx->opts;
            }
        }
        chosen = stage;
    }
    for (void *q : bufs) cudaFree(q);
    if (rc != SDDM_OK) return rc;
    if ((rc = sddm_build(ctx, &chosen)) != SDDM_OK) return rc;
    *best = chosen;
    return SDDM_OK;
}

// ---------------------------------------------------- learned glass surrogate
static bool same_curves(const Material &a, const Material &b) {
    if (!(a.kind == kGlass && b.kind == kGlass && a.a == b.a && a.b == b.b && a.c == b.c && a.n_film == b.n_film &&
          a.film_n == b.film_n && a.film_k == b.film_k && a.film_dk == b.film_dk))
        return false;
    for (int j = 0; j < a.n_film; ++j)
        if (a.film_t[j] != b.film_t[j]) return false;
    return true;
}

static int mlp_net_for(sddm_ctx *ctx, uint32_t mat, bool create, sddm_ctx::MlpNet **out) {
    if (mat >= ctx->mats.size() || ctx->mats[mat].kind != kGlass)
        return fail(SDDM_ERR_INVALID_ARG, "surrogate: material is not a glass slab");
    ctx->net_of_mat.resize(ctx->mats.size(), -1);
    int id = ctx->net_of_mat[mat];
    if (id < 0) {
        if (!create) return fail(SDDM_ERR_MLP_UNTRAINED, "surrogate: no weights for this material");
        ctx->nets.emplace_back(new sddm_ctx::MlpNet());
        id = (int)ctx->nets.size() - 1;
        cudaError_t e;
        sddm_ctx::MlpNet &n = *ctx->nets.back();
        if ((e = n.params.ensure(mlp_param_buffer_bytes())) || (e = n.m.ensure(kMlpParams * 4)) ||
            (e = n.v.ensure(kMlpParams * 4)))
            return cuda_fail(e, "surrogate: allocation");
        for (size_t m = 0; m < ctx->mats.size(); ++m)
            if (same_curves(ctx->mats[m], ctx->mats[mat]) && ctx->net_of_mat[m] < 0) ctx->net_of_mat[m] = id;
    }
    *out = ctx->nets[id].get();
    return SDDM_OK;
}

int sddm_mlp_train(sddm_ctx *ctx, uint32_t mat, const sddm_mlp_train_opts *opts, sddm_mlp_report *rep) {
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_train: ctx is NULL");
    if (!ctx->built) return fail(SDDM_ERR_NOT_BUILT, "sddm_mlp_train: call sddm_build first");
    sddm_mlp_train_opts o{};
    if (opts) o = *opts;
    if (o.samples <= 0) o.samples = (int64_t)1 << 22;
    if (o.steps <= 0) o.steps = 20000;
    if (o.batch <= 0) o.batch = 8192;
    if (o.lr <= 0.f) o.lr = 3e-3f;
    if (o.thick_min <= 0.f && o.thick_max <= 0.f) {
        o.thick_min = 0.002f;
        o.thick_max = 0.010f;
    }
    if (o.batch % kMlpRowsPerCta || o.batch > (1 << 20) || o.samples > ((int64_t)1 << 28) ||
        !(o.thick_max > o.thick_min) || o.thick_min <= 0.f)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_train: batch must be a multiple of 64 (<= 2^20), "
                                          "samples <= 2^28, 0 < thick_min < thick_max");
    sddm_ctx::MlpNet *net = nullptr;
    int rc = mlp_net_for(ctx, mat, true, &net);
    if (rc != SDDM_OK) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int n_cta = o.batch / kMlpRowsPerCta;
    if ((e = ctx->mlp_grad_cta.ensure((size_t)n_cta * kMlpParams * 4)) || (e = ctx->mlp_loss_cta.ensure(n_cta * 4)) ||
        (e = ctx->mlp_scalar.ensure(64)) || (e = ctx->mlp_X.ensure((size_t)o.samples * 16)) ||
        (e = ctx->mlp_Y.ensure((size_t)o.samples * 8)))
        return e == cudaErrorMemoryAllocation ? fail(SDDM_ERR_OOM, "sddm_mlp_train: allocation failed")
                                              : cuda_fail(e, "sddm_mlp_train: allocation");
    if (!o.resume || net->step == 0) {
        if ((e = launch_mlp_init(net->params.as<float>(), o.seed, s)) ||
            (e = cudaMemsetAsync(net->m.p, 0, kMlpParams * 4, s)) || (e = cudaMemsetAsync(net->v.p, 0, kMlpParams * 4, s)))
            return cuda_fail(e, "sddm_mlp_train: init");
        net->step = 0;
    }
    net->dmin = o.thick_min;
    net->dmax = o.thick_max;
    if ((e = launch_mlp_data(ctx->dev, mat, 0.f, o.samples, o.seed, o.thick_min, o.thick_max, ctx->mlp_X.as<float>(),
                             ctx->mlp_Y.as<float>(), s)))
        return cuda_fail(e, "sddm_mlp_train: data");
    if ((e = cudaEventRecord(ctx->ev0, s))) return cuda_fail(e, "sddm_mlp_train: event");
    const int64_t t_end = net->step + o.steps;
    for (int k = 0; k < o.steps; ++k) {
        const int64_t t = net->step + 1;
        MlpTrainArgs a;
        a.params = net->params.as<float>();
        a.X = ctx->mlp_X.as<float>();
        a.Y = ctx->mlp_Y.as<float>();
        a.n_samples = o.samples;
        a.row0 = ((t - 1) * (int64_t)o.batch) % o.samples;
        a.n_rows = o.batch;
        a.grad_cta = ctx->mlp_grad_cta.as<float>();
        a.loss_cta = ctx->mlp_loss_cta.as<float>();
        if ((e = launch_mlp_train_tile(a, s))) return cuda_fail(e, "sddm_mlp_train: train kernel");
        // cosine decay from lr to lr / 100 over this call's steps
        const double frac = (double)(t - (t_end - o.steps)) / (double)o.steps;
        const float lr = (float)(o.lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(3.14159265358979 * frac))));
        const float bc1 = (float)(1.0 - std::pow(0.9, (double)t)), bc2 = (float)(1.0 - std::pow(0.999, (double)t));
        const bool last = k == o.steps - 1;
        if ((e = launch_mlp_adam(net->params.as<float>(), net->m.as<float>(), net->v.as<float>(), a.grad_cta,
                                 a.loss_cta, n_cta, lr, bc1, bc2, nullptr, last ? ctx->mlp_scalar.as<float>() : nullptr,
                                 1.0f / (2.0f * (float)o.batch), s)))
            return cuda_fail(e, "sddm_mlp_train: adam kernel");
        net->step = t;
    }
    if ((e = cudaEventRecord(ctx->ev1, s))) return cuda_fail(e, "sddm_mlp_train: event");
    unsigned int *errs = reinterpret_cast<unsigned int *>(ctx->mlp_scalar.as<char>() + 16);
    if ((e = launch_mlp_pack(net->params.as<float>(), s)) || (e = ctx->d_err.ensure(16)) ||
        (e = cudaMemsetAsync(ctx->d_err.p, 0, 16, s)) || (e = cudaMemsetAsync(errs, 0, 8, s)) ||
        (e = launch_mlp_grid_error(net->params.as<float>(), ctx->dev, mat, o.thick_min, o.thick_max, errs,
                                   ctx->d_err.as<int>(), ctx->sm_count, s)))
        return cuda_fail(e, "sddm_mlp_train: held-out error");
    float loss = 0.f;
    unsigned int me[2] = {0, 0};
    int derr[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(&loss, ctx->mlp_scalar.p, 4, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(me, errs, 8, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(derr, ctx->d_err.p, sizeof derr, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "sddm_mlp_train: execution");
    if (derr[0] != 0)
        return fail(SDDM_ERR_TIMEOUT, "sddm_mlp_train: the surrogate's tensor-core evaluation did not complete");
    // the training samples are not needed afterwards
    ctx->mlp_X.release();
    ctx->mlp_Y.release();
    if (rep) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
        rep->final_loss = loss;
        float eR, eT;
        std::memcpy(&eR, &me[0], 4);
        std::memcpy(&eT, &me[1], 4);
        rep->max_abs_err_R = eR;
        rep->max_abs_err_T = eT;
        rep->train_ms = ms;
        const double flop = 3.0 * 2.0 * (64.0 * 64.0 * 2.0) * (double)o.batch * o.steps;   // tensor-core GEMMs
        rep->tflops = ms > 0 ? flop / (ms * 1e-3) / 1e12 : 0.0;
        rep->steps = net->step;
    }
    return SDDM_OK;
}

int sddm_mlp_get_weights(sddm_ctx *ctx, uint32_t mat, float *params) {
    if (!ctx || !params) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_get_weights: NULL");
    sddm_ctx::MlpNet *net = nullptr;
    int rc = mlp_net_for(ctx, mat, false, &net);
    if (rc != SDDM_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(params, net->params.p, kMlpParams * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? SDDM_OK : cuda_fail(e, "sddm_mlp_get_weights");
}

int sddm_mlp_set_weights(sddm_ctx *ctx, uint32_t mat, const float *params, float thick_min, float thick_max) {
    if (!ctx || !params) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_set_weights: NULL");
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(params[i])) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_set_weights: non-finite weight");
    if (!(thick_max > thick_min) || thick_min <= 0.f)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_set_weights: need 0 < thick_min < thick_max");
    sddm_ctx::MlpNet *net = nullptr;
    int rc = mlp_net_for(ctx, mat, true, &net);
    if (rc != SDDM_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(net->params.p, params, kMlpParams * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_mlp_pack(net->params.as<float>(), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->m.p, 0, kMlpParams * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(net->v.p, 0, kMlpParams * 4, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    net->step = 0;
    net->dmin = thick_min;
    net->dmax = thick_max;
    return e == cudaSuccess ? SDDM_OK : cuda_fail(e, "sddm_mlp_set_weights");
}

int sddm_mlp_save(sddm_ctx *ctx, uint32_t mat, const char *path) {
    if (!ctx || !path) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_save: NULL");
    sddm_ctx::MlpNet *net = nullptr;
    int rc = mlp_net_for(ctx, mat, false, &net);
    if (rc != SDDM_OK) return rc;
    std::vector<float> buf(3 * (size_t)kMlpParams);
    cudaError_t e = cudaMemcpyAsync(buf.data(), net->params.p, kMlpParams * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaMemcpyAsync(buf.data() + kMlpParams, net->m.p, kMlpParams * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaMemcpyAsync(buf.data() + 2 * kMlpParams, net->v.p, kMlpParams * 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "sddm_mlp_save");
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(SDDM_ERR_INVALID_ARG, std::string("sddm_mlp_save: cannot open ") + path);
    const char magic[8] = {'S', 'D', 'D', 'M', 'M', 'L', 'P', '1'};
    const int32_t np = kMlpParams;
    bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(&np, 4, 1, f) == 1 &&
              std::fwrite(&net->step, 8, 1, f) == 1 && std::fwrite(&net->dmin, 4, 1, f) == 1 &&
              std::fwrite(&net->dmax, 4, 1, f) == 1 && std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? SDDM_OK : fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_save: write failed");
}

int sddm_mlp_load(sddm_ctx *ctx, uint32_t mat, const char *path) {
    if (!ctx || !path) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_load: NULL");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(SDDM_ERR_INVALID_ARG, std::string("sddm_mlp_load: cannot open ") + path);
    char magic[8];
    int32_t np = 0;
    int64_t step = 0;
    float dmin = 0, dmax = 0;
    std::vector<float> buf(3 * (size_t)kMlpParams);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "SDDMMLP1", 8) == 0 &&
              std::fread(&np, 4, 1, f) == 1 && np == kMlpParams && std::fread(&step, 8, 1, f) == 1 &&
              std::fread(&dmin, 4, 1, f) == 1 && std::fread(&dmax, 4, 1, f) == 1 &&
              std::fread(buf.data(), 4, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok || step < 0 || !(dmax > dmin) || dmin <= 0.f)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_load: not a valid surrogate checkpoint");
    for (float x : buf)
        if (!std::isfinite(x)) return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_load: non-finite values");
    sddm_ctx::MlpNet *net = nullptr;
    int rc = mlp_net_for(ctx, mat, true, &net);
    if (rc != SDDM_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(net->params.p, buf.data(), kMlpParams * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = launch_mlp_pack(net->params.as<float>(), ctx->stream);
    if (!e) e = cudaMemcpyAsync(net->m.p, buf.data() + kMlpParams, kMlpParams * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaMemcpyAsync(net->v.p, buf.data() + 2 * kMlpParams, kMlpParams * 4, cudaMemcpyHostToDevice, ctx->stream);
    if (!e) e = cudaStreamSynchronize(ctx->stream);
    if (e) return cuda_fail(e, "sddm_mlp_load");
    net->step = step;
    net->dmin = dmin;
    net->dmax = dmax;
    return SDDM_OK;
}

int sddm_mlp_grad(sddm_ctx *ctx, int n, const float *X, const float *Y, const float *params, float *grad,
                  float *loss) {
    if (!ctx || n <= 0 || n > (1 << 20) || !X || !Y || !params || !grad || !loss)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_mlp_grad: bad arguments");
    cudaError_t e = cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    const int n_cta = (n + kMlpRowsPerCta - 1) / kMlpRowsPerCta;
    if ((e = ctx->mlp_grad_cta.ensure((size_t)n_cta * kMlpParams * 4)) || (e = ctx->mlp_loss_cta.ensure(n_cta * 4)))
        return cuda_fail(e, "sddm_mlp_grad: allocation");
    MlpTrainArgs a;
    a.params = params;
    a.X = X;
    a.Y = Y;
    a.n_samples = n;
    a.row0 = 0;
    a.n_rows = n;
    a.grad_cta = ctx->mlp_grad_cta.as<float>();
    a.loss_cta = ctx->mlp_loss_cta.as<float>();
    if ((e = launch_mlp_train_tile(a, s)) ||
        (e = launch_mlp_adam(nullptr, nullptr, nullptr, a.grad_cta, a.loss_cta, n_cta, 0.f, 1.f, 1.f, grad, loss,
                             1.0f / (2.0f * (float)n), s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "sddm_mlp_grad");
    return SDDM_OK;
}

int sddm_set_profiling(sddm_ctx *ctx, int flags) {
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, "sddm_set_profiling: ctx is NULL");
    if (flags & ~(SDDM_PROFILE_TIME_TRACE | SDDM_PROFILE_COUNT_TRAVERSAL | SDDM_PROFILE_EAGER |
                  SDDM_PROFILE_TEST_MLP_TIMEOUT))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_set_profiling: unknown flag");
    ctx->profile = flags;
    ctx->graphs_enabled = flags == 0;   // events inside a replayed graph give no elapsed times
    return SDDM_OK;
}

int sddm_glass_eval(sddm_ctx *ctx, uint32_t mat, int n, const float *cos_theta, const int32_t *bin, const float *s,
                    const float *thickness_m, float *R, float *T, int mode) {
    if (!ctx) return fail(SDDM_ERR_INVALID_ARG, "sddm_glass_eval: ctx is NULL");
    if (!ctx->built) return fail(SDDM_ERR_NOT_BUILT, "sddm_glass_eval: call sddm_build first");
    if (mat >= ctx->mats.size() || ctx->mats[mat].kind != kGlass)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_glass_eval: mat is not a glass slab");
    if (n < 0 || (n > 0 && (!cos_theta || !bin || !s || !thickness_m || !R || !T)))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_glass_eval: bad arguments");
    if (mode == SDDM_BSDF_MLP || mode == SDDM_BSDF_MLP_RAW) {
        sddm_ctx::MlpNet *net = nullptr;
        int rc = mlp_net_for(ctx, mat, false, &net);
        if (rc != SDDM_OK) return rc;
        MlpRows a{};
        a.params = net->params.as<float>();
        a.sc = ctx->dev;
        a.thick_min = net->dmin;
        a.thick_max = net->dmax;
        a.probe_key = 0x5eed;
        a.n = n;
        a.mat = mat;
        a.cos_t = cos_theta;
        a.s = s;
        a.thick = thickness_m;
        a.bin = bin;
        a.R = R;
        a.T = T;
        a.mode = 0;
        a.raw = mode == SDDM_BSDF_MLP_RAW;
        a.fallbacks = nullptr;
        a.test_timeout = (ctx->profile & SDDM_PROFILE_TEST_MLP_TIMEOUT) != 0;
        int derr[4] = {0, 0, 0, 0};
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e == cudaSuccess) e = ctx->d_err.ensure(16);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_err.p, 0, 16, ctx->stream);
        a.err = ctx->d_err.as<int>();
        if (e == cudaSuccess) e = launch_mlp_rows(a, ctx->sm_count, ctx->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(derr, ctx->d_err.p, sizeof derr, cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sddm_glass_eval (surrogate)");
        if (derr[0] != 0)
            return fail(SDDM_ERR_TIMEOUT, "sddm_glass_eval: the surrogate's tensor-core evaluation did not complete");
        return SDDM_OK;
    }
    if (mode != SDDM_BSDF_EXACT) return fail(SDDM_ERR_INVALID_ARG, "sddm_glass_eval: unknown mode");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = launch_glass_eval(ctx->dev, mat, n, cos_theta, bin, s, thickness_m, R, T, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? SDDM_OK : cuda_fail(e, "sddm_glass_eval");
}

int sddm_rgb_to_spectrum(sddm_ctx *ctx, int n, const float *rgb, const float *rgb_to_xyz, float *spectra,
                         int clamp01) {
    NEED_SPECTRUM("sddm_rgb_to_spectrum");
    if (n < 0 || (n > 0 && (!rgb || !spectra)) || n > (1 << 24))
        return fail(SDDM_ERR_INVALID_ARG, "sddm_rgb_to_spectrum: 0 <= n <= 2^24 values, rgb and spectra required");
    const int L = ctx->L;
    // A = w_i cmf_i / sum_i w_i ybar_i; Q = A (A^T A)^-1 M, in double on the host (3 x 3 solve)
    const double srgb[9] = {0.4124, 0.3576, 0.1805, 0.2126, 0.7152, 0.0722, 0.0193, 0.1192, 0.9505};
    double M[9];
    for (int k = 0; k < 9; ++k) M[k] = rgb_to_xyz ? (double)rgb_to_xyz[k] : srgb[k];
    std::vector<double> A((size_t)L * 3);
    double ysum = 0.0;
    for (int i = 0; i < L; ++i) ysum += (double)ctx->quad_w[i] * ctx->cmf[3 * i + 1];
    if (!(ysum > 0.0)) return fail(SDDM_ERR_INVALID_ARG, "sddm_rgb_to_spectrum: the spectrum has no luminance");
    for (int i = 0; i < L; ++i)
        for (int c = 0; c < 3; ++c) A[3 * i + c] = (double)ctx->quad_w[i] * ctx->cmf[3 * i + c] / ysum;
    double G[9] = {0};   // A^T A
    for (int i = 0; i < L; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[3 * a + b] += A[3 * i + a] * A[3 * i + b];
    const double det = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                       G[2] * (G[3] * G[7] - G[4] * G[6]);
    if (!(std::fabs(det) > 0.0)) return fail(SDDM_ERR_INVALID_ARG, "sddm_rgb_to_spectrum: singular colour basis");
    const double Gi[9] = {(G[4] * G[8] - G[5] * G[7]) / det, (G[2] * G[7] - G[1] * G[8]) / det,
                          (G[1] * G[5] - G[2] * G[4]) / det, (G[5] * G[6] - G[3] * G[8]) / det,
                          (G[0] * G[8] - G[2] * G[6]) / det, (G[2] * G[3] - G[0] * G[5]) / det,
                          (G[3] * G[7] - G[4] * G[6]) / det, (G[1] * G[6] - G[0] * G[7]) / det,
                          (G[0] * G[4] - G[1] * G[3]) / det};
    std::vector<float> Q((size_t)L * 3);
    for (int i = 0; i < L; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) v += A[3 * i + a] * Gi[3 * a + b] * M[3 * b + k];
            Q[3 * i + k] = (float)v;
        }
    if (n == 0) return SDDM_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    DevBuf dq, din, dout;
    cudaStream_t s = ctx->stream;
    if (e == cudaSuccess) e = dq.upload(Q, s);
    if (e == cudaSuccess) e = din.ensure(sizeof(float) * 3 * (size_t)n);
    if (e == cudaSuccess) e = dout.ensure(sizeof(float) * (size_t)n * L);
    if (e == cudaSuccess) e = cudaMemcpyAsync(din.p, rgb, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_rgb_to_spectrum(n, L, dq.as<float>(), din.as<float>(), dout.as<float>(), clamp01, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(spectra, dout.p, sizeof(float) * (size_t)n * L, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SDDM_OK : cuda_fail(e, "sddm_rgb_to_spectrum");
}

int sddm_philox(sddm_ctx *ctx, int n, const uint32_t *ctr, uint32_t key0, uint32_t key1, uint32_t *out) {
    if (!ctx || n < 0 || (n > 0 && (!ctr || !out))) return fail(SDDM_ERR_INVALID_ARG, "sddm_philox: bad arguments");
    if ((reinterpret_cast<uintptr_t>(ctr) | reinterpret_cast<uintptr_t>(out)) & 15)
        return fail(SDDM_ERR_INVALID_ARG, "sddm_philox: ctr and out must be 16-byte aligned");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = launch_philox(n, ctr, key0, key1, out, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? SDDM_OK : cuda_fail(e, "sddm_philox");
}

}  // extern "C"
