// Pixel reduction and small test-hook kernels.
//
// A pixel's value is the mean of its spp samples (Sec. 4: one estimate per
// pixel), summed in sample order with compensation so the result does not
// depend on how paths were scheduled.
#include <cuda_runtime.h>

#include "device_common.cuh"

namespace sddm {

__global__ void k_reduce_pixels(ReduceArgs a, int64_t pixel_begin, int64_t pixel_count) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= pixel_count) return;
    const int64_t gpix = pixel_begin + t;
    const int r = find_render_pixel(a.rb, gpix);
    const RenderInfo &ri = a.rb.info[r];
    const int64_t k = gpix - ri.pixel_begin;
    const int64_t p0 = ri.path_begin + k * ri.spp - a.path_begin;   // index into sample_xyz
    Kahan X, Y, Z;
    for (int j = 0; j < ri.spp; ++j) {
        const float *s = a.sample_xyz + 3 * (p0 + j);
        X.add(s[0]);
        Y.add(s[1]);
        Z.add(s[2]);
    }
    float *ax = a.aov_xyz[r];
    int32_t *ap = a.aov_prim[r];
    if (ax)
        for (int j = 0; j < ri.spp; ++j)
            for (int c = 0; c < 3; ++c) ax[3 * (k * ri.spp + j) + c] = a.sample_xyz[3 * (p0 + j) + c];
    if (ap && a.first_prim)
        for (int j = 0; j < ri.spp; ++j) ap[k * ri.spp + j] = a.first_prim[p0 + j];
    const float inv = 1.0f / (float)ri.spp;
    float *out = a.xyz_out[r] + 3 * k;
    out[0] = X.s * inv;
    out[1] = Y.s * inv;
    out[2] = Z.s * inv;
}

// Reduce the pixels [pixel_begin, pixel_begin + pixel_count) of the batch; their
// samples are the rows of a.sample_xyz starting at global path a.path_begin.
cudaError_t launch_reduce_pixels(const ReduceArgs &a, int64_t pixel_begin, int64_t pixel_count,
                                 cudaStream_t stream) {
    if (pixel_count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (pixel_count + threads - 1) / threads;
    k_reduce_pixels<<<(unsigned)blocks, threads, 0, stream>>>(a, pixel_begin, pixel_count);
    return cudaGetLastError();
}

__global__ void k_philox(int n, const uint4 *ctr, uint32_t k0, uint32_t k1, uint4 *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(ctr[i], k0, k1);
}

cudaError_t launch_philox(int n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                          cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_philox<<<(n + 255) / 256, 256, 0, stream>>>(n, reinterpret_cast<const uint4 *>(ctr), k0, k1,
                                                   reinterpret_cast<uint4 *>(out));
    return cudaGetLastError();
}

__global__ void k_glass_eval(DevScene sc, uint32_t mat, int n, const float *cos_t, const int32_t *bin,
                             const float *s, const float *thick, float *R, float *T) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int L = sc.L;
    int i = bin[q];
    i = i < 0 ? 0 : (i >= L ? L - 1 : i);
    float r_, t_;
    glass_rt(sc, (int)mat, i, cos_t[q], s[q], thick[q], r_, t_);
    R[q] = r_;
    T[q] = t_;
}

// Spectra of RGB values: rho_i = sum_k Q[i][k] rgb_k with Q = A (A^T A)^-1 M
// (Cohen's fundamental of the stimulus XYZ = M rgb), optionally clamped to
// [0, 1]. One thread per (value, bin).
__global__ void k_rgb_to_spectrum(int n, int L, const float *Q, const float *rgb, float *out, int clamp01) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * L) return;
    const int q = (int)(t / L), i = (int)(t - (int64_t)q * L);
    float v = Q[3 * i] * rgb[3 * q];
    v = fmaf(Q[3 * i + 1], rgb[3 * q + 1], v);
    v = fmaf(Q[3 * i + 2], rgb[3 * q + 2], v);
    if (clamp01) v = fminf(fmaxf(v, 0.0f), 1.0f);
    out[t] = v;
}

cudaError_t launch_rgb_to_spectrum(int n, int L, const float *Q, const float *rgb, float *out, int clamp01,
                                   cudaStream_t stream) {
    const int64_t total = (int64_t)n * L;
    if (total == 0) return cudaSuccess;
    k_rgb_to_spectrum<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(n, L, Q, rgb, out, clamp01);
    return cudaGetLastError();
}

// Running mean of images: out = a out + b in, elementwise (a = (j - 1) / j,
// b = 1 / j for the j-th image).
__global__ void k_blend(int64_t n, float a, float b, const float *in, float *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = fmaf(a, out[t], b * in[t]);
}

cudaError_t launch_blend(int64_t n, float a, float b, const float *in, float *out, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_blend<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(n, a, b, in, out);
    return cudaGetLastError();
}

cudaError_t launch_glass_eval(const DevScene &sc, uint32_t mat, int n, const float *cos_t, const int32_t *bin,
                              const float *s, const float *thick, float *R, float *T, cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    k_glass_eval<<<(n + 127) / 128, 128, 0, stream>>>(sc, mat, n, cos_t, bin, s, thick, R, T);
    return cudaGetLastError();
}

}  // namespace sddm
