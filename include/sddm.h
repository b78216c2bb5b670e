/*
 * sddm.h -- C ABI of libsddm.so, a GB300 (sm_103a) spectral path tracer whose
 * ray tracing is parallelised by domain decomposition, after
 * Gbikpi-Benissan, Callet, Magoules, "Spectral domain decomposition method for
 * physically-based rendering of photochromic/electrochromic glass windows"
 * (arXiv:1912.06474).
 *
 * The problem, as the paper states it (Sec. 1, Sec. 2, Sec. 6): render a room
 * under natural light from the materials' optical properties -- spectral
 * reflectance, complex index n + ik (Eq. 1) for metals and glass, glass panes
 * whose absorption depends on a coloration state -- through the rendering
 * equation (Eq. 2) with its light-source sum (Eq. 3), by ray tracing (Sec. 4),
 * parallelised by splitting the scene into subdomains that hand rays to each
 * other across interfaces (Sec. 5).
 *
 * Conventions for every call:
 *   - returns SDDM_OK (0) or a negative sddm_status; never aborts or traps;
 *   - sddm_last_error() gives a message for the calling thread's last failure;
 *   - host arrays are read during the call and copied; the caller keeps them;
 *   - pointers documented as DEVICE are caller-owned device memory of the
 *     context's device (e.g. a PyTorch tensor's data_ptr());
 *   - a stream is a cudaStream_t passed as void* (NULL = legacy default);
 *   - units: metres, nanometres, 1/m for absorption; all floats are FP32.
 * A context is not thread-safe: one host thread at a time per context.
 */
#ifndef SDDM_H
#define SDDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sddm_ctx sddm_ctx;

typedef enum {
    SDDM_OK = 0,
    SDDM_ERR_INVALID_ARG = -1,     /* argument out of range, NULL, inconsistent sizes */
    SDDM_ERR_OOM = -2,             /* host or device allocation failed */
    SDDM_ERR_CUDA = -3,            /* a CUDA runtime call failed (message has the CUDA error) */
    SDDM_ERR_QUEUE_OVERFLOW = -4,  /* a subdomain ray queue filled up; rebuild with more capacity */
    SDDM_ERR_TIMEOUT = -5,         /* a device wait hit its iteration cap; the kernel returned */
    SDDM_ERR_NOT_BUILT = -6,       /* sddm_render before sddm_build, or after the scene changed */
    SDDM_ERR_MLP_UNTRAINED = -7,   /* SDDM_BSDF_MLP requested with no trained weights */
    SDDM_ERR_DEVICE_CHECK = -8     /* a device-side bounds check tripped (no access was made) */
} sddm_status;

typedef enum {
    SDDM_BSDF_EXACT = 0,      /* the exact absorbing-slab model */
    SDDM_BSDF_MLP = 1,        /* the trained surrogate, with probe and exact fallback */
    SDDM_BSDF_MLP_RAW = 2     /* sddm_glass_eval only: the network output alone (testing) */
} sddm_bsdf_mode;

typedef enum {
    SDDM_METHOD_MEGAKERNEL = 0,    /* one thread per path over the global BVH (Sec. 5, classical split) */
    SDDM_METHOD_DDM = 1            /* subdomain queues drained by persistent blocks (Sec. 5, DDM) */
} sddm_method;

/* Acceleration structure and scheduling options (sddm_build). */
typedef struct {
    int grid[3];              /* subdomains per axis, each >= 1; {1,1,1} = a single domain */
    int leaf_size;            /* max triangles per BVH leaf, 1..15 (0 = 4) */
    int sah_bins;             /* binned-SAH bins per axis, 4..64 (0 = 16) */
    int64_t queue_capacity;   /* rays per subdomain queue (0 = automatic) */
    int blocks_per_sm;        /* persistent blocks per SM for the DDM trace (0 = automatic) */
    int64_t paths_in_flight;  /* path slots processed at once (0 = automatic) */
    int bvh_in_host_memory;   /* 1: the subdomain BVHs (nodes and triangle references) stay in pinned host
                                 memory that the trace kernel reads over the coherent host link (NVLink-C2C
                                 on Grace-based GPUs) instead of a copy in HBM -- for scenes whose subdomains
                                 exceed device memory (Sec. 5 loads subdomains up to a memory limit); 0 = HBM */
    int64_t cell_cache_bytes; /* > 0: the subdomain BVHs stay in pinned host memory and a device cache of this
                                 many bytes holds the subdomains being traced (Sec. 5: subdomains are loaded
                                 up to a memory limit and unloaded when their rays have run out). Before each
                                 wave the cells holding rays are loaded, fullest first, least recently used
                                 cells evicted; a wave whose cells do not fit at once is traced in groups, the
                                 copies of the next group overlapping the trace of the current one. DDM
                                 renders only (not photon maps), launched eagerly (one host synchronisation
                                 per wave). Images are bit-identical to the all-resident build. Must hold the
                                 largest subdomain (else SDDM_ERR_INVALID_ARG); excludes bvh_in_host_memory.
                                 0 = all subdomains resident in HBM */
    int continue_cells;       /* 1: a ray that leaves its subdomain without a hit is carried on by the same
                                 thread into the neighbour's BVH within the wave (one wave per bounce, no
                                 hand-off through the neighbour's queue); results are identical. 0 = the
                                 ray record is handed to the neighbour's queue for the next wave (Sec. 5's
                                 interface exchange). Not with cell_cache_bytes */
    int handoff_waves;        /* with continue_cells = 0: 0 = every wave of a bounce hands the rays that leave
                                 a subdomain to the neighbour's queue (dims x + y + z - 2 waves); k > 0 =
                                 the first k waves do, then one more wave traces every remaining ray to its
                                 end, the thread carrying it across subdomain faces (the few rays that
                                 cross many faces no longer cost a wave each); results are identical. Not
                                 with cell_cache_bytes */
} sddm_build_opts;

typedef struct {
    float pos[3], look[3], up[3];
    float vfov_deg;           /* vertical field of view of the pinhole camera */
    float ortho_height;       /* > 0: orthographic camera of this image-plane height (Sec. 4) */
} sddm_camera;

/* One render of the scene. Several renders may go to one sddm_render call
 * (one batched launch); they must share method and bsdf_mode. */
typedef struct {
    int width, height, spp;   /* >= 1 each */
    int max_depth;            /* path vertices, 1..64 (Sec. 4's bounce limit) */
    uint32_t seed;            /* Philox key word 0 */
    uint32_t render_id;       /* Philox key word 1 */
    int nee;                  /* 1: shadow rays to the lights (Eq. 3); 0: emission counted at every vertex */
    int bsdf_mode;            /* sddm_bsdf_mode for glass slabs */
    int method;               /* sddm_method */
    sddm_camera camera;
    const float *glass_s;     /* HOST [n_materials] coloration state per material, entries < 0 keep
                                 the material's default; NULL = all defaults */
    float *xyz_out;           /* DEVICE [height][width][3] CIE XYZ, mean over spp (written) */
    float *aov_sample_xyz;    /* DEVICE optional [height*width*spp][3] per-sample XYZ, sample-minor */
    int32_t *aov_first_prim;  /* DEVICE optional [height*width*spp] first-hit triangle id, -1 = miss */
} sddm_render_desc;

/* Counters of the last sddm_render (all renders of the call). */
typedef struct {
    int64_t paths;
    int64_t segments_ext;     /* closest-hit queries (one per path vertex reached) */
    int64_t segments_shadow;  /* shadow (any-hit) queries */
    int64_t crossings;        /* DDM interface hand-offs between subdomains */
    int64_t glass_queries;    /* glass slab (R,T) evaluations, per hit (all bins) */
    int64_t mlp_fallbacks;    /* MLP batches that fell back to the exact slab */
    double gpu_ms;            /* device time of the whole call, CUDA events on the context stream */
    int64_t kernel_launches;  /* kernels this call launched */
    double trace_ms;          /* SDDM_PROFILE_TIME_TRACE: summed device time of the trace kernels */
    int64_t trace_launches;   /* SDDM_PROFILE_TIME_TRACE: launches those times cover */
    int64_t node_visits;      /* SDDM_PROFILE_COUNT_TRAVERSAL: BVH interior nodes visited */
    int64_t tri_tests;        /* SDDM_PROFILE_COUNT_TRAVERSAL: ray/triangle tests */
    int64_t ray_visits;       /* SDDM_PROFILE_COUNT_TRAVERSAL: (ray, subdomain) visits traced */
    int64_t mlp_batches;      /* surrogate batches evaluated (each probed once); mlp_fallbacks of them fell back */
    int64_t cache_loads;      /* cell_cache_bytes > 0: subdomain BVHs copied into the cache */
    int64_t cache_hits;       /* ... (cell, wave) uses that found the subdomain already resident */
    int64_t cache_bytes_loaded; /* ... bytes copied from host memory */
    double mlp_ms;            /* SDDM_PROFILE_TIME_TRACE: summed device time of the surrogate network kernel */
    int64_t mlp_rows;         /* (query, bin) rows the surrogate network evaluated */
    int64_t ray_continues;    /* SDDM_PROFILE_COUNT_TRAVERSAL: crossings the tracing thread carried on itself
                                 (continue_cells, handoff_waves): no ray record staged or read back */
} sddm_stats;

/* Profiling switches (sddm_set_profiling), off by default. */
enum {
    SDDM_PROFILE_TIME_TRACE = 1,        /* CUDA events around every trace and surrogate-network launch */
    SDDM_PROFILE_COUNT_TRAVERSAL = 2,   /* count nodes, triangle tests and ray visits */
    SDDM_PROFILE_EAGER = 4,             /* launch every kernel from the host (no CUDA graph replay) */
    SDDM_PROFILE_TEST_MLP_TIMEOUT = 8   /* test of the failure path: the first CTA of the surrogate network
                                           issues no layer-1 MMA, so its bounded wait on the tensor core runs
                                           out (after 2^10 tries); the call returns SDDM_ERR_TIMEOUT */
};

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA `device` using `stream` (cudaStream_t or NULL).
 * *out receives the context; SDDM_ERR_CUDA if the device cannot be used. */
int sddm_create(sddm_ctx **out, int device, void *stream);

/* Free every device and host resource of the context. NULL is accepted. */
int sddm_destroy(sddm_ctx *ctx);

/* Message of the calling thread's last failed call ("" if none). The pointer
 * stays valid until the next sddm_* call on the same thread. */
const char *sddm_last_error(void);

/* Library version string ("sddm <major>.<minor> sm_103a"). */
const char *sddm_version(void);

/* ---------------------------------------------------------------- scene */

/* Spectral sampling of the rendering model (Sec. 1: the model carries
 * spectral properties; Sec. 3). L bins (1..256) at lambda_nm[L], quadrature
 * weights quad_w[L] (nm), colour matching functions cmf_xyz[L][3]. Resets the
 * material list, which is defined per bin. */
int sddm_set_spectrum(sddm_ctx *ctx, int L, const float *lambda_nm, const float *quad_w,
                      const float *cmf_xyz);

/* Lambertian reflector with spectral reflectance rho[L] in [0,1] (the other
 * room materials of Sec. 2, whose spectra stand for the RGB-derived ones).
 * *mat receives the material id (ids count up from 0 in call order). */
int sddm_add_lambertian(sddm_ctx *ctx, const float *rho, uint32_t *mat);

/* Metal described by its optical constants n[L] + i k[L] (Eq. 1; Sec. 2
 * characterises metals by these constants): a smooth
 * mirror weighted by the Fresnel reflectance. n > 0, k >= 0. */
int sddm_add_conductor(sddm_ctx *ctx, const float *n, const float *k, uint32_t *mat);

/* Glass pane as an absorbing plane-parallel slab (Sec. 2 glass samples; Sec. 6
 * evaluates glass with the Fresnel equations; photochromic/electrochromic state):
 * real index n[L] >= 1, absorption alpha(s) = alpha_clear[L] + s * dalpha[L]
 * in 1/m (k = alpha * lambda / 4 pi), thickness in metres, default state
 * s_default in [0,1]. The slab's triangles must form one closed convex object
 * (one obj_id). */
int sddm_add_glass_slab(sddm_ctx *ctx, const float *n, const float *alpha_clear,
                        const float *dalpha, float thickness_m, float s_default, uint32_t *mat);

/* Glass slab coated on both outer faces with the same stack of n_films thin
 * films (an electrochromic device; a multilayer extension of the slab of
 * Sec. 6): the substrate as in sddm_add_glass_slab, films
 * outermost first, film_n / film_k / film_dk HOST [n_films][L] (real index,
 * extinction at s = 0, extinction added at s = 1: k = k + s dk),
 * film_t_nm[n_films] thicknesses in nm. Each face is evaluated exactly by
 * its characteristic (transfer) matrix per polarisation; the faces combine
 * incoherently through the substrate. 0 <= n_films <= SDDM_MAX_FILMS; with no
 * film this is sddm_add_glass_slab. The paper gives the glass by its "Fresnel
 * definition" (Sec. 6) and has no thin-film model: this call extends it. */
#define SDDM_MAX_FILMS 10
int sddm_add_coated_glass(sddm_ctx *ctx, const float *n, const float *alpha_clear, const float *dalpha,
                          float thickness_m, float s_default, int n_films, const float *film_n, const float *film_k,
                          const float *film_dk, const float *film_t_nm, uint32_t *mat);

/* One-sided area light of radiance Le[L] >= 0 toward its counter-clockwise
 * normal, black to reflection (the light sources of Eq. 3, here with area). */
int sddm_add_emitter(sddm_ctx *ctx, const float *Le, uint32_t *mat);

/* One-sided area light that also reflects diffusely with rho[L] (used by the
 * white-furnace check; no counterpart in the paper). */
int sddm_add_diffuse_emitter(sddm_ctx *ctx, const float *rho, const float *Le, uint32_t *mat);

/* Triangle mesh: vertices v[nv][3], triangles tri[nt][3] (vertex indices,
 * counter-clockwise about the outward normal), material mat_id[nt] and
 * object obj_id[nt] per triangle (Sec. 4: objects are made of polygons). nt >= 1,
 * at most 2^26 triangles. Invalidates a previous build. */
int sddm_set_mesh(sddm_ctx *ctx, const float *v, int nv, const uint32_t *tri, int nt,
                  const uint32_t *mat_id, const uint32_t *obj_id);

/* Build the acceleration structures on the host and upload them (Sec. 5: the
 * scene domain is cut into small subdomains): a global
 * binned-SAH BVH for the megakernel and, for grid != {1,1,1}, a grid of
 * subdomains each with its own BVH over the triangles that overlap it
 * (duplicated by reference, node boxes clipped to the subdomain). o may be
 * NULL for defaults. Synchronous. */
int sddm_build(sddm_ctx *ctx, const sddm_build_opts *o);

/* Render n >= 1 images (Sec. 4 algorithm, Eq. 2-3 model) in one batched
 * call on the context stream; returns when the device has finished. Every
 * output pointer is DEVICE memory owned by the caller. st may be NULL. */
int sddm_render(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_stats *st);

/* Host-buffer variant of sddm_render for callers without device memory:
 * xyz_out / aov pointers in d are HOST pointers here; the library copies
 * results back before returning. Same semantics otherwise. */
int sddm_render_host(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_stats *st);

/* Render one image with the plain megakernel without allocating any memory.
 * The paper has no counterpart: this serves callers that cannot call
 * cudaMalloc while rendering -- an application whose own pool allocator owns
 * the device memory (a library allocating beside it can run out even though
 * the pool has room), or a render loop whose latency budget has no room for
 * cudaMalloc / cudaFree, which may wait for the whole device. All scratch
 * (per-path results, counters, the render record) lives in one fixed 16 MiB
 * device array that the library defines and every GPU that loads it holds
 * until exit, so a call is limited to width * height * spp <= 1,397,418 paths
 * and 1920 materials; larger renders return SDDM_ERR_INVALID_ARG with a
 * message. d->method must be SDDM_METHOD_MEGAKERNEL, d->bsdf_mode
 * SDDM_BSDF_EXACT, and the per-sample outputs NULL. The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and keeps it:
 * make that first call before any stream capture, and do not use this entry
 * point after cudaDeviceReset. Every call shares the array and finds the last
 * call's contents there (each call rewrites what it reads); calls whose work
 * overlaps on the GPU (several streams or threads) race on it. Returns when
 * the device has finished. Output: d->xyz_out, DEVICE, as sddm_render. */
int sddm_render_noalloc(sddm_ctx *ctx, const sddm_render_desc *d, sddm_stats *st);

/* Photon pass of a photon-mapping render (filled by sddm_render_photon_map). */
typedef struct {
    int64_t photons;          /* photons emitted */
    int64_t photon_segments;  /* closest-hit queries of the photon pass */
    int64_t stored;           /* photons stored in the map (the global map when caustic_radius > 0) */
    int64_t grid_cells;       /* cells of the uniform grid(s) the map(s) are sorted into */
    double photon_ms;         /* device time of the photon pass and grid build */
    int64_t kernel_launches;  /* kernels of the photon pass and grid build */
    int64_t stored_caustic;   /* photons in the caustic map (caustic_radius > 0), else 0 */
} sddm_photon_stats;

/* Render one image by photon mapping (Sec. 4: global illumination computed
 * with photons emitted from the light sources), by d->method: with
 * SDDM_METHOD_DDM the photons travel through the same subdomain ray queues and
 * trace kernel as camera paths (Sec. 5), in chunks of paths_in_flight photons;
 * with SDDM_METHOD_MEGAKERNEL one thread traces each photon over the global
 * BVH. First n_photons photons leave
 * the area lights -- triangle chosen by area, uniform point, cosine-distributed
 * direction about the front face, power pi Le A_total / n_photons each --
 * and follow the interactions camera paths follow (diffuse bounce weighted by
 * rho, Fresnel mirror for conductors, the glass branch with the same branch
 * probability and R/P, T/(1-P) weights, absorbing glass at its state in
 * d->glass_s) for at most max_depth - 1 hits over the global BVH. A photon is
 * stored at each diffuse hit reached after a diffuse bounce or a reflection
 * changed its direction (light arriving in a straight line, through glass or
 * not, is next-event light). Random numbers: Philox counter (photon,
 * 0xffffffff, hit, slot), key (seed, render_id), slots as for paths. Then the
 * camera pass of sddm_render with the megakernel: emission and the shadow ray
 * at the first diffuse vertex as usual, plus rho/pi times the power of the
 * stored photons within `radius` whose direction points into the visible
 * side, over pi radius^2; the path stops there. With caustic_radius > 0 the
 * stored photons form two maps (Sec. 4 names a global and a caustic map): a
 * photon that only reflections (metal, glass) have turned since the light,
 * without a diffuse bounce, goes to the caustic map, gathered within
 * caustic_radius; the others to the global map, gathered within radius; both
 * are added. caustic_radius = 0 keeps one map of every stored photon. The photon pass evaluates
 * glass exactly; the camera pass follows d->bsdf_mode (the learned model runs
 * with the DDM method only). Needs d->nee 1, d->max_depth >= 2, radius > 0,
 * caustic_radius >= 0, n_photons * (max_depth - 1) < 2^31 (else
 * SDDM_ERR_INVALID_ARG). The map lives in library-owned device memory: 16
 * bytes x 2 + 4 L bytes per photon and bounce, reused by later calls; too
 * little device memory gives SDDM_ERR_OOM. Synchronous; outputs as
 * sddm_render (d->xyz_out DEVICE). st and pst may be NULL. */
int sddm_render_photon_map(sddm_ctx *ctx, const sddm_render_desc *d, int64_t n_photons, float radius,
                           float caustic_radius, sddm_stats *st, sddm_photon_stats *pst);

/* Progressive photon mapping (Sec. 4 names photon mapping; the progressive
 * form is the probabilistic one of Knaus and Zwicker, 2011): n_passes
 * independent photon-mapping renders, pass j (1-based) with render id
 * d->render_id + j - 1 (new photons and camera samples) and gather radii
 * shrinking as r_{j+1}^2 = r_j^2 (j + alpha) / (j + 1) from r_1 = radius (and
 * caustic_radius, 0 = one map), averaged into d->xyz_out (DEVICE). With
 * 0 < alpha < 1 the radii go to zero slowly enough that the averaged estimate
 * converges; alpha = 1 keeps them constant. Same requirements as
 * sddm_render_photon_map, plus n_passes >= 1 and 0 < alpha <= 1 (else
 * SDDM_ERR_INVALID_ARG). Statistics are sums over the passes (grid_cells: the
 * last pass). Synchronous. */
int sddm_render_progressive_photon_map(sddm_ctx *ctx, const sddm_render_desc *d, int n_passes, int64_t n_photons,
                                       float radius, float caustic_radius, float alpha, sddm_stats *st,
                                       sddm_photon_stats *pst);

/* Pick the subdomain grid ({1,1,1}, {2,2,2}, {4,4,2}, {8,4,4}) with its
 * hand-off schedule (neighbour queues every wave, the thread carrying rays
 * across faces, or one queue wave and then the thread), the
 * persistent trace blocks per SM ({4, 8, 16}) and then the paths in flight per
 * chunk ({2^21, 2^22, 2^23}; the ray queues are sized from it, two rays per
 * path, so they cannot overflow) for these renders, by timing short pilot
 * renders (1 spp, at most 512 x 512) of each candidate (Sec. 5 load
 * balancing, settled here by measurement). Writes the best options to *best
 * and leaves the context built with them. */
int sddm_autotune(sddm_ctx *ctx, const sddm_render_desc *d, int n, sddm_build_opts *best);

/* ------------------------------------------------- learned glass surrogate
 * A small network stands in for the exact slab R, T of a glass material (the
 * paper evaluates glass with the Fresnel equations, Sec. 6): inputs
 * (cos theta, lambda, s, thickness), each mapped to [-1, 1]: 2 cos - 1,
 * (lambda - 380)/200 - 1, 2 s - 1, and the thickness d through the normal-
 * incidence internal transmittance 2 exp(-alpha(lambda, s) d) - 1 with the
 * material's alpha = alpha_clear + s dalpha; the trained box is cos in [0,1],
 * lambda in [380,780] nm, s in [0,1], d in [thick_min, thick_max]; 3 hidden
 * layers of 64 SiLU units; 2 outputs y, served as R = max(exp(y0) - 1e-3, 0),
 * T = max(exp(y1) - 1e-3, 0) (trained on log(R + 1e-3), log(T + 1e-3)).
 * Weights and activations are BF16 with FP32 accumulation and FP32 master
 * weights; parameters in this order (8770 floats): W1[64][4], b1[64],
 * W2[64][64], b2[64], W3[64][64], b3[64], W4[2][64], b4[2]. */
#define SDDM_MLP_PARAMS 8770

typedef struct {
    int64_t samples;          /* exact training samples drawn once (0 = 2^22) */
    int steps;                /* Adam steps (0 = 20000) */
    int batch;                /* rows per step, multiple of 64 (0 = 8192) */
    float lr;                 /* peak learning rate, cosine decay to lr/100 (0 = 3e-3) */
    uint32_t seed;            /* Philox key of the samples and the initial weights */
    float thick_min, thick_max; /* trained thickness range, m (0, 0 = 0.002, 0.010) */
    int resume;               /* 1: continue from the current weights and Adam state */
} sddm_mlp_train_opts;

typedef struct {
    double final_loss;        /* mean squared error of the last batch, in the network's log(. + 1e-3) outputs */
    double max_abs_err_R;     /* on a held-out grid of the trained box, vs the exact slab */
    double max_abs_err_T;
    double train_ms;          /* device time of the training steps */
    double tflops;            /* tensor-core FLOP of forward + backward / train time */
    int64_t steps;            /* Adam steps taken so far (with resume) */
} sddm_mlp_report;

/* Train the surrogate of glass material `mat` on samples of its exact slab
 * model (generated on the device), by the library's own forward, backward and
 * Adam kernels. The weights serve every glass material with the same n,
 * alpha_clear and dalpha curves. Requires sddm_build. r may be NULL. */
int sddm_mlp_train(sddm_ctx *ctx, uint32_t mat, const sddm_mlp_train_opts *o, sddm_mlp_report *r);

/* Copy the FP32 weights of glass material `mat` out (HOST [8770]) or in.
 * Setting weights makes the material's surrogate usable (Adam state reset). */
int sddm_mlp_get_weights(sddm_ctx *ctx, uint32_t mat, float *params);
int sddm_mlp_set_weights(sddm_ctx *ctx, uint32_t mat, const float *params, float thick_min, float thick_max);

/* Checkpoint of the surrogate of `mat`: weights, Adam moments and step, to or
 * from a file (little-endian binary, magic "SDDMMLP1"). */
int sddm_mlp_save(sddm_ctx *ctx, uint32_t mat, const char *path);
int sddm_mlp_load(sddm_ctx *ctx, uint32_t mat, const char *path);

/* Test hook: mean squared error and its gradient (FP32, from the BF16
 * forward/backward training kernels) of parameters params[8770] on n rows of
 * features X[n][4] (already mapped to [-1,1]) and targets Y[n][2]. All DEVICE
 * arrays; grad[8770] and loss[1] written. */
int sddm_mlp_grad(sddm_ctx *ctx, int n, const float *X, const float *Y, const float *params, float *grad,
                  float *loss);

/* Enable the SDDM_PROFILE_* measurements of later sddm_render calls
 * (0 = off). Counting uses a separately compiled trace kernel, so the timed
 * kernel is never the counting one within a call. By default the launch
 * sequence of a render is captured into a CUDA graph the second time the same
 * render shapes are seen (same sizes, depth, method, build) and replayed from
 * then on; any profiling flag, or SDDM_PROFILE_EAGER, launches eagerly. */
int sddm_set_profiling(sddm_ctx *ctx, int flags);

/* ---------------------------------------------------------- test hooks */

/* Glass slab R and T (Sec. 6, Fresnel equations) for n queries of glass
 * material `mat`: cos_theta[n] in [0,1], bin index bin[n] in [0,L), state
 * s[n], thickness_m[n]. All four inputs and R[n], T[n] are DEVICE arrays.
 * mode = sddm_bsdf_mode: the exact slab, or the trained surrogate network on
 * the tensor cores with (SDDM_BSDF_MLP) or without (SDDM_BSDF_MLP_RAW) the
 * per-batch probe and exact fallback. SDDM_ERR_MLP_UNTRAINED if the material
 * has no network; SDDM_ERR_TIMEOUT if the network kernel's bounded wait on the
 * tensor core ran out (the kernel stopped and freed its tensor memory). */
int sddm_glass_eval(sddm_ctx *ctx, uint32_t mat, int n, const float *cos_theta, const int32_t *bin,
                    const float *s, const float *thickness_m, float *R, float *T, int mode);

/* Reflectance spectra of RGB values by Cohen and Kappauf's Matrice-R theory
 * (Sec. 3: a spectrum is its fundamental, which carries the colour stimulus,
 * plus a metameric black with X = Y = Z = 0; the fundamental of a stimulus
 * follows from one matrix equation): XYZ = M rgb, then
 * rho = A (A^T A)^-1 XYZ with A_i = w_i cmf(lambda_i) / sum_i w_i ybar_i, the
 * context's bins, weights and colour-matching functions (sddm_set_spectrum;
 * rho = 1 has Y = 1). rgb: HOST [n][3]; rgb_to_xyz: HOST [3][3] row-major, or
 * NULL for linear sRGB with the D65 white; spectra: HOST [n][L] written.
 * clamp01 != 0 limits the result to [0, 1] (physical reflectances; the round
 * trip back to the same RGB then holds only where nothing was clamped). */
int sddm_rgb_to_spectrum(sddm_ctx *ctx, int n, const float *rgb, const float *rgb_to_xyz, float *spectra,
                         int clamp01);

/* Philox4x32-10 block for counters ctr[n][4] under key {key0, key1}: out[n][4]
 * words. ctr and out are DEVICE arrays. */
int sddm_philox(sddm_ctx *ctx, int n, const uint32_t *ctr, uint32_t key0, uint32_t key1,
                uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* SDDM_H */
