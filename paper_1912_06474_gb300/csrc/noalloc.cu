// sddm_render_noalloc: a megakernel render that allocates no memory.
//
// Some callers cannot call cudaMalloc while they render. A host application
// that hands all device memory to its own pool allocator (a caching allocator
// keeps freed blocks for itself, so a cudaMalloc from a library beside it can
// fail for lack of memory the pool is holding) cannot let a library allocate
// behind its back; and a render loop with a fixed latency budget cannot pay
// for cudaMalloc / cudaFree, which may wait for the whole device.
// sddm_render grows its scratch buffers (per-sample results, counters, render
// tables) with cudaMalloc on demand; this entry point instead keeps all of
// that scratch in one file-scope device array of fixed size, so a call
// allocates nothing.
//
// The array is 16 MiB and lives on every GPU that loads the library until the
// process exits. Its first 8 KiB hold the counters, the error word, the render
// record and the per-material state table; the rest holds one XYZ triple per
// path, which limits a call to (16 MiB - 8 KiB) / 12 B = 1,397,418 paths
// (width * height * spp). Every call shares the array and it keeps the last
// call's contents; each call overwrites everything it reads (the header is
// re-uploaded, counters included), but calls whose work overlaps on the GPU --
// two streams, or two host threads -- race on it.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (that device current) and keeps it for the process;
// make that first call before any stream capture. The address is not looked
// up again, so the entry point must not be used after cudaDeviceReset. A call
// returns once the device has finished its work: it reads the counters and
// the error word back and synchronises the stream.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "sddm_internal.h"

namespace sddm {
namespace {

constexpr size_t kNoAllocBytes = 16u << 20;
constexpr size_t kNoAllocHeader = 8192;
constexpr size_t kOffCounters = 0, kOffErr = 64, kOffInfo = 128, kOffOut = 384, kOffAovX = 392, kOffAovP = 400,
                 kOffState = 512;
constexpr int kNoAllocMaxMat = (int)((kNoAllocHeader - kOffState) / sizeof(float));
constexpr int64_t kNoAllocMaxPaths = (int64_t)((kNoAllocBytes - kNoAllocHeader) / (3 * sizeof(float)));
constexpr int kMaxDevices = 64;
static_assert(sizeof(RenderInfo) <= kOffOut - kOffInfo, "render record does not fit the header slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
unsigned char *g_scratch[kMaxDevices] = {};

// Device address of the scratch array on `device` (the current device). The
// host-side name g_noalloc_scratch is only a stand-in: its address must come
// from cudaGetSymbolAddress, once per device, with that device current.
int scratch_on(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) {
        set_error("sddm_render_noalloc: device index beyond 63");
        return SDDM_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "sddm_render_noalloc: cudaGetSymbolAddress");
        g_scratch[device] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch[device];
    return SDDM_OK;
}

}  // namespace
}  // namespace sddm

using namespace sddm;

extern "C" int sddm_render_noalloc(sddm_ctx *ctx, const sddm_render_desc *d, sddm_stats *st) {
    CtxView v;
    int rc = ctx_view(ctx, &v);
    if (rc != SDDM_OK) return rc;
    rc = check_render_desc(ctx, d, 1);
    if (rc != SDDM_OK) return rc;
    if (d->method != SDDM_METHOD_MEGAKERNEL || d->bsdf_mode != SDDM_BSDF_EXACT) {
        set_error("sddm_render_noalloc: only the megakernel with the exact glass model");
        return SDDM_ERR_INVALID_ARG;
    }
    if (d->aov_sample_xyz || d->aov_first_prim) {
        set_error("sddm_render_noalloc: per-sample outputs are not available here (use sddm_render)");
        return SDDM_ERR_INVALID_ARG;
    }
    const int64_t paths = (int64_t)d->width * d->height * d->spp;
    if (paths > kNoAllocMaxPaths) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "sddm_render_noalloc: %lld paths exceed the fixed scratch of %lld paths "
                      "(width * height * spp); use sddm_render",
                      (long long)paths, (long long)kNoAllocMaxPaths);
        set_error(msg);
        return SDDM_ERR_INVALID_ARG;
    }
    if (v.n_mat > kNoAllocMaxMat) {
        set_error("sddm_render_noalloc: more materials than the fixed state table holds (1920)");
        return SDDM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(v.device);
    if (e != cudaSuccess) return cuda_fail(e, "sddm_render_noalloc: cudaSetDevice");
    unsigned char *scratch = nullptr;
    if ((rc = scratch_on(v.device, &scratch)) != SDDM_OK) return rc;

    // header, built on the host stack: zeroed counters and error word, the
    // render record, output pointer table, state table
    alignas(16) unsigned char hdr[kNoAllocHeader];
    std::memset(hdr, 0, sizeof hdr);
    RenderInfo ri;
    render_info_for(ctx, *d, ri);
    ri.path_begin = 0;
    ri.pixel_begin = 0;
    ri.s_offset = 0;
    std::memcpy(hdr + kOffInfo, &ri, sizeof ri);
    float *outp = d->xyz_out;
    std::memcpy(hdr + kOffOut, &outp, sizeof outp);
    for (int m = 0; m < v.n_mat; ++m) {
        float sv = material_state(ctx, *d, m);
        std::memcpy(hdr + kOffState + sizeof(float) * m, &sv, sizeof sv);
    }
    const size_t hdr_bytes = kOffState + sizeof(float) * (size_t)v.n_mat;
    cudaStream_t s = v.stream;
    if ((e = cudaMemcpyAsync(scratch, hdr, hdr_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, "sddm_render_noalloc: header upload");

    RenderBatch rb;
    rb.info = reinterpret_cast<const RenderInfo *>(scratch + kOffInfo);
    rb.n = 1;
    rb.state_s = reinterpret_cast<const float *>(scratch + kOffState);
    float *samples = reinterpret_cast<float *>(scratch + kNoAllocHeader);

    if ((e = cudaEventRecord(v.ev0, s)) != cudaSuccess) return cuda_fail(e, "sddm_render_noalloc: event");
    MegaArgs a;
    a.sc = v.dev;
    a.rb = rb;
    a.path_begin = 0;
    a.path_count = paths;
    a.sample_xyz = samples;
    a.first_prim = nullptr;
    a.counters = reinterpret_cast<unsigned long long *>(scratch + kOffCounters);
    a.error_flag = reinterpret_cast<int *>(scratch + kOffErr);
    a.count_traversal = 0;
    if ((e = launch_megakernel(a, s)) != cudaSuccess) return cuda_fail(e, "sddm_render_noalloc: megakernel");
    ReduceArgs ra;
    ra.rb = rb;
    ra.path_begin = 0;
    ra.sample_xyz = samples;
    ra.first_prim = nullptr;
    ra.xyz_out = reinterpret_cast<float *const *>(scratch + kOffOut);
    ra.aov_xyz = reinterpret_cast<float *const *>(scratch + kOffAovX);
    ra.aov_prim = reinterpret_cast<int32_t *const *>(scratch + kOffAovP);
    if ((e = launch_reduce_pixels(ra, 0, (int64_t)d->width * d->height, s)) != cudaSuccess)
        return cuda_fail(e, "sddm_render_noalloc: reduce");
    if ((e = cudaEventRecord(v.ev1, s)) != cudaSuccess) return cuda_fail(e, "sddm_render_noalloc: event");
    unsigned long long cnt[8];
    int err[4];
    if ((e = cudaMemcpyAsync(cnt, scratch + kOffCounters, sizeof cnt, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(err, scratch + kOffErr, sizeof err, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return cuda_fail(e, "sddm_render_noalloc: kernel execution");
    if (err[0] != 0) {
        set_error("sddm_render_noalloc: device reported an error");
        return SDDM_ERR_DEVICE_CHECK;
    }
    if (st) {
        std::memset(st, 0, sizeof *st);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, v.ev0, v.ev1);
        st->paths = paths;
        st->segments_ext = (int64_t)cnt[0];
        st->segments_shadow = (int64_t)cnt[1];
        st->glass_queries = (int64_t)cnt[2];
        st->gpu_ms = ms;
        st->kernel_launches = 2;
    }
    return SDDM_OK;
}
