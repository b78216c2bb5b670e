// Internal types of libsddm shared by the host C++ and the CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sddm.h"

namespace sddm {

// Statistics counters of a render call, u64 each (layout at DevScene users'
// `counters` fields): ext, shadow, glass, crossings, fallbacks, nodes, tris,
// visits, surrogate batches, surrogate rows, crossings carried on by the
// tracing thread; the rest spare.
constexpr int kNumCounters = 16;

constexpr int kMaxL = 256;
constexpr int kMaxCross = 4;        // distinct glass slabs a shadow ray may pass through
constexpr int kMaxDepth = 64;
constexpr int kLeafBits = 4;        // leaf child = ~((first << 4) | count)
constexpr int kMaxLeaf = 15;
constexpr int kStackSize = 96;   // > the builder's maximum tree depth

// Material kinds (numbering shared with the C ABI's add order semantics).
enum MatKind : int { kLambert = 0, kConductor = 1, kGlass = 2, kEmitter = 3, kDiffuseEmitter = 4 };

// Random stream slots of the counter (pixel, sample, vertex, slot).
constexpr uint32_t kSlotCamera = 0x10000u;
constexpr uint32_t kSlotBsdf = 0x10001u;
constexpr uint32_t kSlotLight = 0x10002u;
constexpr uint32_t kSlotGlass = 0x10003u;
constexpr uint32_t kSlotProbe = 0x10004u;

constexpr float kRayOffset = 1e-4f;       // metres along the geometric normal
constexpr float kShadowShorten = 1e-4f;   // shadow rays end at (1 - 1e-4) * distance

// Triangle flag bits stored in the .w of the third float4 of a packed triangle.
constexpr uint32_t kTriGlass = 1u;

// Device view of the scene: plain pointers into context-owned device memory.
struct DevScene {
    int L;
    int n_mat;
    const float4 *wcmf;       // [L] (quad_w * cmf_x, quad_w * cmf_y, quad_w * cmf_z, 0)
    const float *lam;         // [L]
    const int *mat_kind;      // [n_mat]
    const float *mat_a;       // [n_mat][L] rho | n | n(glass) | Le
    const float *mat_b;       // [n_mat][L] -   | k | alpha_clear | rho (diffuse emitter)
    const float *mat_c;       // [n_mat][L] -   | - | dalpha
    const float *mat_thick;   // [n_mat]
    // thin-film coatings of glass materials (both faces; NULL when no material has one)
    const int *mat_nfilm;     // [n_mat] films per face, 0..SDDM_MAX_FILMS
    const float *film_n;      // [n_mat][SDDM_MAX_FILMS][L] real index
    const float *film_k;      // [n_mat][SDDM_MAX_FILMS][L] extinction at s = 0
    const float *film_dk;     // [n_mat][SDDM_MAX_FILMS][L] extinction added at s = 1
    const float *film_t;      // [n_mat][SDDM_MAX_FILMS] thickness, nm
    const float4 *tri_n;      // [nt] unit CCW normal, .w = material id (int bits)
    const int *tri_obj;       // [nt]
    int n_light;
    const float4 *light_v;    // [n_light][3] vertices (xyz), .w of first = triangle id bits
    const float *light_cdf;   // [n_light]
    float light_area;
    // global BVH (single domain)
    const float4 *g_nodes;    // [n][4]
    const float4 *g_tris;     // [refs][3]
};

// Per-render constants (device copy in a table).
struct RenderInfo {
    int64_t path_begin;       // first global path index of this render
    int64_t pixel_begin;      // first global pixel index of this render
    int width, height, spp, max_depth;
    uint32_t seed, render_id;
    int nee, s_offset;        // s_offset: index of this render's [n_mat] state table
    float cam_o[3];
    float cam_f[3];           // forward (ortho) / forward (pinhole)
    float cam_x[3];           // right * tan(vfov/2) * aspect   (or * half width for ortho)
    float cam_y[3];           // up * tan(vfov/2)               (or * half height for ortho)
    int ortho;
    int pad;
};

struct RenderBatch {
    const RenderInfo *info;   // [n]
    int n;
    const float *state_s;     // [n][n_mat] coloration state per render and material
};

// Host-side material record.
struct Material {
    int kind;
    std::vector<float> a, b, c;
    float thick = 0.f, s_default = 0.f;
    // coating films (glass): per film n, k, dk curves [L] and thickness (nm)
    int n_film = 0;
    std::vector<float> film_n, film_k, film_dk;   // [n_film][L]
    float film_t[SDDM_MAX_FILMS] = {};
};

// A built BVH in device-ready packed form.
struct PackedBVH {
    std::vector<float4> nodes;   // 4 per node
    std::vector<float4> tris;    // 3 per reference
};

struct GridInfo {
    int dims[3];
    float lo[3], hi[3], cell[3], inv_cell[3];
    float eps;                   // window slack for accepting hits, metres
};

// Host BVH build (bvh_build.cpp).
struct BuildTri {
    float v[3][3];
    uint32_t id, obj, flags;
};
void build_bvh(const std::vector<BuildTri> &tris, const std::vector<uint32_t> &refs, const float clip_lo[3],
               const float clip_hi[3], int leaf_size, int bins, PackedBVH &out);
void build_grid(const std::vector<BuildTri> &tris, const int dims[3], const float lo[3], const float hi[3],
                int leaf_size, int bins, float eps, std::vector<PackedBVH> &cells, int n_threads);

// Errors
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Read-only access to a context from other translation units.
struct CtxView {
    int device;
    cudaStream_t stream;
    bool built;
    DevScene dev;
    int n_mat;
    cudaEvent_t ev0, ev1;
};
int ctx_view(sddm_ctx *ctx, CtxView *v);
int check_render_desc(const sddm_ctx *ctx, const sddm_render_desc *d, int n);
void render_info_for(const sddm_ctx *ctx, const sddm_render_desc &x, RenderInfo &ri);
float material_state(const sddm_ctx *ctx, const sddm_render_desc &x, int m);

}  // namespace sddm

// Kernel launchers (defined in .cu files), all asynchronous on `stream`.
namespace sddm {
// Stored photons of a photon map (Sec. 4 global illumination) sorted into a
// uniform grid of cubic cells of side `cell` >= radius starting at lo.
struct PhotonGridView {
    int on;                   // 0: no photon map in this render
    const float4 *pos;        // [slots] (x, 1 = stored / 0 = empty slot)
    const float4 *dir;        // [slots] incoming direction
    const float *pow;         // [slots][L] power
    const int *cell_start;    // [cells + 1]
    const int *order;         // stored slots sorted by cell
    float lo[3];
    int dims[3];
    float cell, radius;
};

struct MegaArgs {
    DevScene sc;
    RenderBatch rb;
    int64_t path_begin, path_count;    // global path range of this launch
    float *sample_xyz;                 // [path_count][3]
    int32_t *first_prim;               // [path_count] or null
    unsigned long long *counters;      // [16]: ext, shadow, glass, crossings, fallbacks, nodes, tris, visits,
                                       // surrogate batches, spare
    int *error_flag;
    int count_traversal;
    PhotonGridView pm = {};            // photon map gathered at the first diffuse vertex (pm.on)
    PhotonGridView pmc = {};           // caustic map gathered there too (pmc.on)
};
cudaError_t launch_megakernel(const MegaArgs &a, cudaStream_t stream);

struct ReduceArgs {
    RenderBatch rb;
    int64_t path_begin;                // global path index of sample_xyz row 0
    const float *sample_xyz;           // [paths][3]
    const int32_t *first_prim;         // [paths] or null
    float *const *xyz_out;             // device table [n] of output pointers
    float *const *aov_xyz;             // device table [n], entries may be null
    int32_t *const *aov_prim;          // device table [n], entries may be null
};
cudaError_t launch_reduce_pixels(const ReduceArgs &a, int64_t pixel_begin, int64_t pixel_count,
                                 cudaStream_t stream);

cudaError_t launch_philox(int n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                          cudaStream_t stream);
cudaError_t launch_blend(int64_t n, float a, float b, const float *in, float *out, cudaStream_t stream);
cudaError_t launch_rgb_to_spectrum(int n, int L, const float *Q, const float *rgb, float *out, int clamp01,
                                   cudaStream_t stream);
cudaError_t launch_glass_eval(const DevScene &sc, uint32_t mat, int n, const float *cos_t, const int32_t *bin,
                              const float *s, const float *thick, float *R, float *T, cudaStream_t stream);
}  // namespace sddm
