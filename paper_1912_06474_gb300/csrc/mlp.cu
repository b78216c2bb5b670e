// Learned surrogate of the glass slab's R and T (a stand-in for the exact
// Fresnel-equation glass of Sec. 6): a 4 -> 64 -> 64 -> 64 -> 2 SiLU
// network evaluated and trained with BF16 tensor-core MMAs (m16n8k16, FP32
// accumulation). The layers are 64 wide, so a warp carries a 16-row tile
// through the whole network: the accumulator fragments of one layer, after
// SiLU and rounding to BF16, are exactly the A fragments of the next layer,
// so activations stay in registers from layer to layer and never leave the
// SM. Layer 1 (K = 4) and the output layer (N = 2) run on the FP32 pipes.
//
// Parameters (FP32 master copy, 8770 floats): W1[64][4], b1[64], W2[64][64],
// b2[64], W3[64][64], b3[64], W4[2][64], b4[2]; z = W h + b. Inputs are mapped
// to [-1, 1] over the trained box: 2 sqrt(cos) - 1, (lambda - 380) / 200 - 1, 2 s - 1,
// and the thickness through the slab's internal transmittance at normal
// incidence, 2 exp(-(alpha d + film absorbance)) - 1 (see features()).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "sddm_mlp.h"

namespace sddm {
namespace {

constexpr int H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = 256, OFF_W2 = 320, OFF_B2 = 4416, OFF_W3 = 4480, OFF_B3 = 8576, OFF_W4 = 8640,
              OFF_B4 = 8768;
static_assert(OFF_B4 + 2 == kMlpParams, "parameter layout");
constexpr int LD = 72;   // shared-memory row stride (bf16): conflict-free 32-bit fragment loads
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
// sigmoid(z) = (1 + tanh(z / 2)) / 2 with the hardware tanh (tanh.approx.f32,
// one SFU operation, relative error about 2^-11 -- below the BF16 rounding the
// activations take next); SiLU(z) = z sigmoid(z) = h + h tanh(h), h = z / 2.
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigm(float z) { return fmaf(0.5f, tanh_fast(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu(float z) {
    const float h = 0.5f * z;
    return fmaf(h, tanh_fast(h), h);
}
__device__ __forceinline__ float dsilu(float z) {
    const float g = sigm(z);
    return g * fmaf(z, 1.0f - g, 1.0f);
}

// D += A B for one m16n8k16 BF16 tile, FP32 accumulators.
__device__ __forceinline__ void mma16816(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// acc (16 x 64) += A (16 x K) * W^T, A rows and W rows K-contiguous in shared
// memory with stride LD (W is [64][K], row n = output column n). Fragment
// ownership: acc[j][0..1] = row g, cols 8j + 2t + {0,1}; acc[j][2..3] = row g + 8.
template <int K>
__device__ __forceinline__ void warp_gemm(float acc[8][4], const __nv_bfloat16 *A, const __nv_bfloat16 *W, int lane) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int kk = 0; kk < K / 16; ++kk) {
        const uint32_t *alo = reinterpret_cast<const uint32_t *>(A + g * LD + 16 * kk + 2 * t);
        const uint32_t *ahi = reinterpret_cast<const uint32_t *>(A + (g + 8) * LD + 16 * kk + 2 * t);
        const uint32_t a0 = alo[0], a1 = ahi[0], a2 = alo[4], a3 = ahi[4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t *bp = reinterpret_cast<const uint32_t *>(W + (8 * j + g) * LD + 16 * kk + 2 * t);
            mma16816(acc[j], a0, a1, a2, a3, bp[0], bp[4]);
        }
    }
}

// Activations h (accumulator layout: h[j][0..1] row g, cols 8j + 2t + {0,1};
// h[j][2..3] row g + 8) as BF16 A fragments of the next layer's mma.
__device__ __forceinline__ void pack_afrag(const float h[8][4], uint32_t fa[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        fa[kk][0] = pack_bf16x2(h[2 * kk][0], h[2 * kk][1]);
        fa[kk][1] = pack_bf16x2(h[2 * kk][2], h[2 * kk][3]);
        fa[kk][2] = pack_bf16x2(h[2 * kk + 1][0], h[2 * kk + 1][1]);
        fa[kk][3] = pack_bf16x2(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
}

__device__ __forceinline__ void zero_acc(float acc[8][4]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
}

// The network predicts log(R + eps) and log(T + eps): a fixed error there is a
// fixed relative error of R and T well above eps, so a dark pane's small T and
// a near-normal reflectance keep their relative accuracy.
constexpr float kOutEps = 1e-3f;
__device__ __forceinline__ float out_to_rt(float y) { return fmaxf(expf(y) - kOutEps, 0.0f); }
__device__ __forceinline__ float rt_to_out(float v) { return logf(v + kOutEps); }

// Network inputs from (cos, lambda, s, thickness): sqrt(cos) and s mapped to
// [-1, 1] (the square root spreads the grazing angles, where reflectance and
// transmittance change fastest), lambda over 380-780 nm to [-1, 1], and the
// thickness through the slab's
// internal transmittance at normal incidence, exp(-alpha(lambda, s) d) mapped
// to [-1, 1] (alpha = alpha_clear + s dalpha, the material's absorption law),
// times that of any coating film (exp(-4 pi k t / lambda) each).
// Angle, Fresnel and the multiple reflections are left to the network.
__device__ __forceinline__ void features(float c, float lam, float s, float alpha_d, float x[4]) {
    x[0] = 2.0f * sqrtf(fmaxf(c, 0.0f)) - 1.0f;
    x[1] = (lam - 380.0f) * (1.0f / 200.0f) - 1.0f;
    x[2] = 2.0f * s - 1.0f;
    x[3] = 2.0f * expf(-alpha_d) - 1.0f;
}

// ------------------------------------------------------------- inference
// The hidden layers' weights and biases are stored halved: the layer then
// produces h = z / 2 directly (halving is exact in binary floating point, so
// the activations are bit for bit those of the unscaled layer), and
// SiLU(z) = h + h tanh(h) costs one SFU operation and one FMA.
//
// All four layers run on the tensor cores (m16n8k16, BF16 operands, FP32
// accumulation):
//  * layer 1 (K = 4) as one K = 16 step whose A row is [x_hi(4) | x_lo(4) |
//    1 | 1 | 0 ...] and whose B row for output n is [W1n(4) | W1n(4) | b_hi |
//    b_lo | 0 ...]: each input split into two BF16 parts and the bias into two,
//    so the products keep 16 bits of the FP32 inputs and bias;
//  * layers 2 and 3 (64 x 64) as four K steps;
//  * layer 4 (N = 2) as an N = 8 tile whose rows 2..7 are zero.
// The activations entering layer 4 are split the same way, h = h_hi + h_lo in
// two BF16 parts, each multiplied by the same BF16 weights (two MMAs per
// fragment), so that the outputs do not carry the 8-bit rounding of the last
// hidden layer (training does the same); layers 2 and 3 take single BF16
// activations.
// B fragments come from shared memory by ldmatrix, four 8x8 blocks at a time.
constexpr int LD1 = 24;   // layer-1 B rows: 16 used, stride 48 B (16-byte aligned, conflict-free)
struct alignas(16) InferSmem {   // 16-byte rows for ldmatrix
    __nv_bfloat16 w1[H * LD1];              // [64][16]: W1 / 2 twice, b1 / 2 as hi + lo
    __nv_bfloat16 w2[H * LD], w3[H * LD];   // W / 2
    __nv_bfloat16 w4[8 * LD];               // rows 0, 1: W4; rows 2..7: 0
    float b2[H], b3[H];                     // b / 2
    float b4[2];
};

__device__ void load_infer_weights(InferSmem &s, const float *__restrict__ p) {
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) {
        const int r = i >> 6, c = i & 63;
        s.w2[r * LD + c] = __float2bfloat16_rn(0.5f * p[OFF_W2 + i]);
        s.w3[r * LD + c] = __float2bfloat16_rn(0.5f * p[OFF_W3 + i]);
    }
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
        const int n = i >> 4, k = i & 15;
        float v = 0.0f;
        if (k < 8) {
            v = 0.5f * bf16r(p[OFF_W1 + 4 * n + (k & 3)]);
        } else if (k < 10) {
            const float b = 0.5f * p[OFF_B1 + n];
            const float hi = bf16r(b);
            v = k == 8 ? hi : b - hi;
        }
        s.w1[n * LD1 + k] = __float2bfloat16_rn(v);
    }
    for (int i = threadIdx.x; i < 8 * H; i += blockDim.x) {
        const int n = i >> 6, k = i & 63;
        s.w4[n * LD + k] = __float2bfloat16_rn(n < 2 ? p[OFF_W4 + H * n + k] : 0.0f);
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        s.b2[i] = 0.5f * p[OFF_B2 + i];
        s.b3[i] = 0.5f * p[OFF_B3 + i];
    }
    if (threadIdx.x < 2) s.b4[threadIdx.x] = p[OFF_B4 + threadIdx.x];
}

// Four 8x8 BF16 blocks from shared memory (ldmatrix): lane l gives the
// address of row l & 7 of block l >> 3 and receives, of every block, row
// (l >> 2), elements 2 (l & 3) and 2 (l & 3) + 1.
__device__ __forceinline__ void ldmatrix_x4(const void *row_addr, uint32_t &r0, uint32_t &r1, uint32_t &r2,
                                            uint32_t &r3) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row_addr);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

// acc (16 x 64) += A (16 x 16 kk_steps) W^T, A in registers as mma A
// fragments (fa, and with LO a second part fb of the same A), W [64][ld]
// bf16 in shared memory (row n = output n). The B fragments of output tiles
// j, j + 1 for one K step are one ldmatrix.x4.
template <int KSTEPS, bool LO>
__device__ __forceinline__ void warp_gemm_ldm(float acc[8][4], const uint32_t fa[][4], const uint32_t fb[][4],
                                              const __nv_bfloat16 *W, int ld, int lane) {
    const int q = lane >> 3, r = lane & 7;
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk) {
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
            uint32_t b0, b1, c0, c1;
            ldmatrix_x4(W + (8 * (j + (q >> 1)) + r) * ld + 16 * kk + 8 * (q & 1), b0, b1, c0, c1);
            mma16816(acc[j], fa[kk][0], fa[kk][1], fa[kk][2], fa[kk][3], b0, b1);
            mma16816(acc[j + 1], fa[kk][0], fa[kk][1], fa[kk][2], fa[kk][3], c0, c1);
            if (LO) {
                mma16816(acc[j], fb[kk][0], fb[kk][1], fb[kk][2], fb[kk][3], b0, b1);
                mma16816(acc[j + 1], fb[kk][0], fb[kk][1], fb[kk][2], fb[kk][3], c0, c1);
            }
        }
    }
}

// Activations h (accumulator layout) as two BF16 A-fragment parts, h_hi =
// bf16(h) and h_lo = bf16(h - h_hi).
__device__ __forceinline__ uint32_t pack_lo_bf16x2(float a, float b) {
    return pack_bf16x2(a - bf16r(a), b - bf16r(b));
}
__device__ __forceinline__ void pack_afrag2(const float h[8][4], uint32_t fa[4][4], uint32_t fb[4][4]) {
    pack_afrag(h, fa);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        fb[kk][0] = pack_lo_bf16x2(h[2 * kk][0], h[2 * kk][1]);
        fb[kk][1] = pack_lo_bf16x2(h[2 * kk][2], h[2 * kk][3]);
        fb[kk][2] = pack_lo_bf16x2(h[2 * kk + 1][0], h[2 * kk + 1][1]);
        fb[kk][3] = pack_lo_bf16x2(h[2 * kk + 1][2], h[2 * kk + 1][3]);
    }
}

// SiLU of z given h = z / 2.
__device__ __forceinline__ float silu_h(float h) { return fmaf(h, tanh_fast(h), h); }

// Layer-1 A fragment of rows g (xl) and g + 8 (xh): this lane's K columns
// 2t, 2t + 1 (t = 0, 1: high parts of inputs 2t, 2t + 1; t = 2, 3: low parts
// of inputs 2t - 4, 2t - 3) and 2t + 8, 2t + 9 (t = 0: the two bias ones).
__device__ __forceinline__ void layer1_afrag(const float xl[4], const float xh[4], int t, uint32_t fa[4]) {
    const int i = 2 * (t & 1);
    const bool lo = t >= 2;
    auto part = [&](float v) {
        const float hi = bf16r(v);
        return lo ? v - hi : hi;
    };
    fa[0] = pack_bf16x2(part(xl[i]), part(xl[i + 1]));
    fa[1] = pack_bf16x2(part(xh[i]), part(xh[i + 1]));
    const uint32_t ones = pack_bf16x2(1.0f, 1.0f);
    fa[2] = t == 0 ? ones : 0u;
    fa[3] = t == 0 ? ones : 0u;
}

// The network on the 16 rows of a warp tile; this thread supplies the inputs
// of rows g and g + 8 and receives their outputs (on the lanes with t = 0).
// Activations stay in registers: each layer's accumulators are packed into
// the next layer's BF16 A fragments.
__device__ void tile_forward(const InferSmem &s, const float xl[4], const float xh[4], int lane, float yl[2],
                             float yh[2]) {
    const int t = lane & 3;
    float acc[8][4];
    uint32_t fa[4][4], fb[4][4];
    layer1_afrag(xl, xh, t, fa[0]);
    zero_acc(acc);
    warp_gemm_ldm<1, false>(acc, fa, fb, s.w1, LD1, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = silu_h(acc[j][e]);
    pack_afrag(acc, fa);
    zero_acc(acc);
    warp_gemm_ldm<4, false>(acc, fa, fb, s.w2, LD, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        const float2 bb = *reinterpret_cast<const float2 *>(s.b2 + c);
        acc[j][0] = silu_h(acc[j][0] + bb.x);
        acc[j][1] = silu_h(acc[j][1] + bb.y);
        acc[j][2] = silu_h(acc[j][2] + bb.x);
        acc[j][3] = silu_h(acc[j][3] + bb.y);
    }
    pack_afrag(acc, fa);
    zero_acc(acc);
    warp_gemm_ldm<4, false>(acc, fa, fb, s.w3, LD, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        const float2 bb = *reinterpret_cast<const float2 *>(s.b3 + c);
        acc[j][0] = silu_h(acc[j][0] + bb.x);
        acc[j][1] = silu_h(acc[j][1] + bb.y);
        acc[j][2] = silu_h(acc[j][2] + bb.x);
        acc[j][3] = silu_h(acc[j][3] + bb.y);
    }
    pack_afrag2(acc, fa, fb);
    // layer 4: one N = 8 tile, K = 64 in four steps (two ldmatrix.x4, each
    // the B fragments of two K steps)
    float o[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int q = lane >> 3, r = lane & 7;
#pragma unroll
    for (int kk = 0; kk < 4; kk += 2) {
        uint32_t b0, b1, c0, c1;
        ldmatrix_x4(s.w4 + r * LD + 16 * (kk + (q >> 1)) + 8 * (q & 1), b0, b1, c0, c1);
        mma16816(o, fa[kk][0], fa[kk][1], fa[kk][2], fa[kk][3], b0, b1);
        mma16816(o, fb[kk][0], fb[kk][1], fb[kk][2], fb[kk][3], b0, b1);
        mma16816(o, fa[kk + 1][0], fa[kk + 1][1], fa[kk + 1][2], fa[kk + 1][3], c0, c1);
        mma16816(o, fb[kk + 1][0], fb[kk + 1][1], fb[kk + 1][2], fb[kk + 1][3], c0, c1);
    }
    // o[0..1]: row g, outputs 2t, 2t + 1; o[2..3]: row g + 8 (outputs 0, 1 on t = 0)
    yl[0] = o[0] + s.b4[0];
    yl[1] = o[1] + s.b4[1];
    yh[0] = o[2] + s.b4[0];
    yh[1] = o[3] + s.b4[1];
}

struct RowIn {
    float c, lam, s, d;
    int mat, bin;
};

// Normal-incidence absorbance of a row's glass: alpha(lambda, s) d of the
// substrate plus, for coated glass, 4 pi k_j(lambda, s) t_j / lambda of each
// film (Beer-Lambert through every absorbing layer, interference left out).
template <bool FILMS = true>
__device__ __forceinline__ float row_alpha_d(const DevScene &sc, const RowIn &in) {
    const size_t k = (size_t)in.mat * sc.L + in.bin;
    float a = (__ldg(sc.mat_b + k) + in.s * __ldg(sc.mat_c + k)) * in.d;
    if constexpr (FILMS) {
        const int J = sc.mat_nfilm ? __ldg(sc.mat_nfilm + in.mat) : 0;
        for (int j = 0; j < J; ++j) {
            const size_t f = ((size_t)in.mat * kMaxFilms + j) * sc.L + in.bin;
            const float kj = __ldg(sc.film_k + f) + in.s * __ldg(sc.film_dk + f);
            a = fmaf(12.566370614359172f * kj, __ldg(sc.film_t + (size_t)in.mat * kMaxFilms + j) / in.lam, a);
        }
    }
    return a;
}

__device__ __forceinline__ bool row_input(const MlpRows &a, int64_t r, int64_t total, RowIn &in) {
    if (r >= total) {
        in.c = 0.5f;
        in.lam = 580.0f;
        in.s = 0.5f;
        in.d = 0.5f * (a.thick_min + a.thick_max);
        in.mat = 0;
        in.bin = 0;
        return false;
    }
    const int L = a.sc.L;
    if (a.mode == 0) {
        int b = a.bin[r];
        b = b < 0 ? 0 : (b >= L ? L - 1 : b);
        in.c = a.cos_t[r];
        in.s = a.s[r];
        in.d = a.thick[r];
        in.mat = (int)a.mat;
        in.bin = b;
    } else {
        const int64_t q = r / L;
        const float4 qq = a.queries[q];
        in.c = qq.x;
        in.s = qq.y;
        in.d = qq.z;
        in.mat = __float_as_int(qq.w);
        in.bin = (int)(r - q * L);
    }
    in.lam = __ldg(a.sc.lam + in.bin);
    return true;
}

template <bool FILMS = true>
__device__ __forceinline__ float2 exact_row(const MlpRows &a, const RowIn &in) {
    float R_, T_;
    glass_rt<FILMS>(a.sc, in.mat, in.bin, in.c, in.s, in.d, R_, T_);
    return make_float2(R_, T_);
}

// Rows are taken 32 at a time by a warp (two 16-row tiles). One row of each
// batch, chosen by Philox, is also evaluated exactly; if it is off by more
// than 1e-3 in R or T, or if any row lies outside the trained box, the whole
// batch is evaluated exactly instead. The probes of 32 batches run together,
// one per lane, so that a probe costs one lane's share of an exact evaluation
// rather than a whole warp's.
#ifndef SDDM_MLP_MINB
#define SDDM_MLP_MINB 4   // resident inference blocks per SM asked of the register allocator: 64
                          // registers with ~80 B of spills, 32 warps per SM
#endif
#ifndef SDDM_MLP_UNROLL_HALVES
#define SDDM_MLP_UNROLL_HALVES 1   // the two 16-row tiles of a batch as one unrolled sequence
#endif
template <bool FILMS>
__global__ void __launch_bounds__(256, SDDM_MLP_MINB) k_mlp_rows(MlpRows a) {
    __shared__ InferSmem s;
    __shared__ float2 out[8][32];
    __shared__ float4 xin[8][32];   // per warp: the encoded inputs of its 32 rows
    load_infer_weights(s, a.params);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    // A batch is 32 rows of one query's bins (renderer queries: a batch never
    // mixes two glass evaluations, so its probe speaks for rows that share
    // angle, state and thickness) or 32 consecutive explicit rows.
    const int L = a.sc.L;
    int64_t total = a.n, n_batches = (a.n + 31) / 32;
    int nb = 1;
    if (a.mode == 1) {
        const int64_t nq0 = (int64_t)*a.n_queries;
        const int64_t nq = nq0 < a.q_cap ? nq0 : a.q_cap;
        total = nq * L;
        nb = (L + 31) / 32;
        n_batches = nq * nb;
    }
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t b_first = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;   // this warp's batches: b_first + k nwarps
    unsigned long long n_fb = 0;
    auto batch_rows = [&](int64_t b, int64_t &r0, int &nvalid) {
        if (a.mode == 1) {
            const int64_t qi = b / nb;
            const int j = (int)(b - qi * nb);
            r0 = qi * L + 32 * j;
            nvalid = L - 32 * j < 32 ? L - 32 * j : 32;
        } else {
            r0 = b * 32;
            nvalid = total - r0 < 32 ? (int)(total - r0) : 32;
        }
    };
    auto store = [&](int64_t r, float2 y) {
        if (a.mode == 0) {
            a.R[r] = y.x;
            a.T[r] = y.y;
        } else {
            a.results[r] = y;
        }
    };
    // Rounds of up to 32 of the warp's batches: the network serves every row
    // of them, then lane k probes batch k (one exact row each, all lanes at
    // once), then every batch whose probe or trained box failed is evaluated
    // exactly, row per lane.
    for (int64_t k0 = 0; b_first + k0 * nwarps < n_batches; k0 += 32) {
        unsigned box_bad = 0;
        int n_round = 0;
        for (int k = 0; k < 32; ++k) {
            const int64_t b = b_first + (k0 + k) * nwarps;
            if (b >= n_batches) break;
            ++n_round;
            int64_t r0;
            int nvalid;
            batch_rows(b, r0, nvalid);
            // each lane encodes the row of its own index once (the coating
            // films' absorbance loop included); the tiles read their rows'
            // inputs from the warp's staging row
            {
                RowIn in;
                row_input(a, lane < nvalid ? r0 + lane : total, total, in);
                float xr[4];
                features(in.c, in.lam, in.s, row_alpha_d<FILMS>(a.sc, in), xr);
                xin[w][lane] = make_float4(xr[0], xr[1], xr[2], xr[3]);
            }
            __syncwarp();
#if SDDM_MLP_UNROLL_HALVES
#pragma unroll
#else
#pragma unroll 1
#endif
            for (int half = 0; half < 2; ++half) {
                if (half == 1 && nvalid <= 16) break;   // warp-uniform: no valid row in the second tile
                const int kl = 16 * half + g, kh = kl + 8;
                float yl[2], yh[2];
                const float4 ql = xin[w][kl], qh = xin[w][kh];
                const float xl[4] = {ql.x, ql.y, ql.z, ql.w}, xh[4] = {qh.x, qh.y, qh.z, qh.w};
                tile_forward(s, xl, xh, lane, yl, yh);
                if (t == 0) {
                    out[w][kl] = make_float2(out_to_rt(yl[0]), out_to_rt(yl[1]));
                    out[w][kh] = make_float2(out_to_rt(yh[0]), out_to_rt(yh[1]));
                }
            }
            __syncwarp();
            RowIn in;
            const bool valid = row_input(a, lane < nvalid ? r0 + lane : total, total, in);
            const bool in_box = in.c >= 0.0f && in.c <= 1.0f && in.lam >= 380.0f && in.lam <= 780.0f &&
                                in.s >= 0.0f && in.s <= 1.0f && in.d >= a.thick_min && in.d <= a.thick_max;
            if (!__all_sync(kFull, !valid || in_box)) box_bad |= 1u << k;
            if (valid) store(r0 + lane, out[w][lane]);
            __syncwarp();
        }
        if (a.raw) continue;
        // probes: lane k takes the Philox-chosen row of batch k of the round
        int bad = 0;
        if (lane < n_round) {
            const int64_t b = b_first + (k0 + lane) * nwarps;
            int64_t r0;
            int nvalid;
            batch_rows(b, r0, nvalid);
            const uint4 pr = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0u, kSlotProbe),
                                           a.probe_key, 0x50524f42u);
            const int64_t r = r0 + (int)(pr.x % (uint32_t)nvalid);
            RowIn in;
            row_input(a, r, total, in);
            const float2 e = exact_row<FILMS>(a, in);
            const float2 y = a.mode == 0 ? make_float2(a.R[r], a.T[r]) : a.results[r];
            bad = fabsf(e.x - y.x) > kMlpProbeTol || fabsf(e.y - y.y) > kMlpProbeTol;
        }
        unsigned fall = __ballot_sync(kFull, bad) | box_bad;
        while (fall) {
            const int k = __ffs(fall) - 1;
            fall &= fall - 1;
            int64_t r0;
            int nvalid;
            batch_rows(b_first + (k0 + k) * nwarps, r0, nvalid);
            RowIn in;
            if (row_input(a, lane < nvalid ? r0 + lane : total, total, in)) store(r0 + lane, exact_row<FILMS>(a, in));
            if (lane == 0) ++n_fb;
        }
        __syncwarp();
    }
    if (a.fallbacks && n_fb) atomicAdd(a.fallbacks, n_fb);
    if (a.batches && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.batches, (unsigned long long)n_batches);
}

// The exact slab for the same query rows, one thread per (query, bin): the
// glass evaluations of a bounce as one dense, divergence-free pass.
template <bool FILMS>
__global__ void __launch_bounds__(256) k_slab_rows(MlpRows a) {
    int64_t total = a.n;
    if (a.mode == 1) {
        const int64_t nq = (int64_t)*a.n_queries;
        total = (nq < a.q_cap ? nq : a.q_cap) * a.sc.L;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
        RowIn in;
        row_input(a, r, total, in);
        const float2 y = exact_row<FILMS>(a, in);
        if (a.mode == 0) {
            a.R[r] = y.x;
            a.T[r] = y.y;
        } else {
            a.results[r] = y;
        }
    }
}

// ---------------------------------------------------------------- training
// One CTA = 64 rows = 4 warps x 16 rows: forward, loss gradient, backward,
// and the CTA's share of every weight gradient, written to grad_cta[cta].
struct TrainSmem {
    __nv_bfloat16 w2[H * LD], w3[H * LD], w2t[H * LD], w3t[H * LD];
    __nv_bfloat16 h1[H * LD], h2[H * LD], h1t[H * LD], h2t[H * LD];
    __nv_bfloat16 dz3[H * LD], dz2[H * LD], dz3t[H * LD], dz2t[H * LD];
    float z1[H * H], z2[H * H], z3[H * H];
    float w1[H * 4], w4[2 * H], b1[H], b2[H], b3[H], b4[2];
    float x[kMlpRowsPerCta * 4], y[kMlpRowsPerCta * 2];
    // per-warp partial sums of the small gradients, added in warp order at the
    // end (no float atomics: the same rows give the same gradient bits)
    float gw1[4][H * 4], gb1[4][H], gb2[4][H], gb3[4][H], gw4[4][2 * H], gb4[4][2], loss[4];
};

__global__ void __launch_bounds__(128) k_mlp_train_tile(MlpTrainArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &s = *reinterpret_cast<TrainSmem *>(smem_raw);
    const float *__restrict__ p = a.params;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
    const int cta = blockIdx.x;
    for (int i = tid; i < H * H; i += blockDim.x) {
        const int r = i >> 6, c = i & 63;
        const __nv_bfloat16 v2 = __float2bfloat16_rn(p[OFF_W2 + i]), v3 = __float2bfloat16_rn(p[OFF_W3 + i]);
        s.w2[r * LD + c] = v2;
        s.w3[r * LD + c] = v3;
        s.w2t[c * LD + r] = v2;
        s.w3t[c * LD + r] = v3;
    }
    for (int i = tid; i < H * 4; i += blockDim.x) {
        s.w1[i] = bf16r(p[OFF_W1 + i]);
    }
    for (int i = tid; i < 2 * H; i += blockDim.x) {
        s.w4[i] = bf16r(p[OFF_W4 + i]);
    }
    for (int i = tid; i < H; i += blockDim.x) {
        s.b1[i] = p[OFF_B1 + i];
        s.b2[i] = p[OFF_B2 + i];
        s.b3[i] = p[OFF_B3 + i];
    }
    if (tid < 2) s.b4[tid] = p[OFF_B4 + tid];
    const int cta_row0 = cta * kMlpRowsPerCta;
    for (int i = tid; i < kMlpRowsPerCta; i += blockDim.x) {
        const bool ok = cta_row0 + i < a.n_rows;
        const int64_t gr = (a.row0 + cta_row0 + i) % a.n_samples;
        for (int k = 0; k < 4; ++k) s.x[4 * i + k] = ok ? a.X[4 * gr + k] : 0.f;
        for (int k = 0; k < 2; ++k) s.y[2 * i + k] = ok ? a.Y[2 * gr + k] : 0.f;
    }
    __syncthreads();

    const int rl = 16 * w + g, rh = rl + 8;   // this thread's two rows in the CTA
    const bool okl = cta_row0 + rl < a.n_rows, okh = cta_row0 + rh < a.n_rows;
    // ---- layer 1 (FP32 pipes, K = 4)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float hl[2], hh[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * j + 2 * t + e;
            float zl = s.b1[c], zh = s.b1[c];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                zl = fmaf(s.w1[4 * c + k], s.x[4 * rl + k], zl);
                zh = fmaf(s.w1[4 * c + k], s.x[4 * rh + k], zh);
            }
            s.z1[rl * H + c] = zl;
            s.z1[rh * H + c] = zh;
            hl[e] = silu(zl);
            hh[e] = silu(zh);
            s.h1t[c * LD + rl] = __float2bfloat16_rn(hl[e]);
            s.h1t[c * LD + rh] = __float2bfloat16_rn(hh[e]);
        }
        *reinterpret_cast<uint32_t *>(s.h1 + rl * LD + 8 * j + 2 * t) = pack_bf16x2(hl[0], hl[1]);
        *reinterpret_cast<uint32_t *>(s.h1 + rh * LD + 8 * j + 2 * t) = pack_bf16x2(hh[0], hh[1]);
    }
    __syncwarp();
    // ---- layer 2
    float acc[8][4];
    zero_acc(acc);
    warp_gemm<H>(acc, s.h1 + 16 * w * LD, s.w2, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        const float zl0 = acc[j][0] + s.b2[c], zl1 = acc[j][1] + s.b2[c + 1];
        const float zh0 = acc[j][2] + s.b2[c], zh1 = acc[j][3] + s.b2[c + 1];
        s.z2[rl * H + c] = zl0;
        s.z2[rl * H + c + 1] = zl1;
        s.z2[rh * H + c] = zh0;
        s.z2[rh * H + c + 1] = zh1;
        const float a0 = silu(zl0), a1 = silu(zl1), a2 = silu(zh0), a3 = silu(zh1);
        *reinterpret_cast<uint32_t *>(s.h2 + rl * LD + c) = pack_bf16x2(a0, a1);
        *reinterpret_cast<uint32_t *>(s.h2 + rh * LD + c) = pack_bf16x2(a2, a3);
        s.h2t[c * LD + rl] = __float2bfloat16_rn(a0);
        s.h2t[(c + 1) * LD + rl] = __float2bfloat16_rn(a1);
        s.h2t[c * LD + rh] = __float2bfloat16_rn(a2);
        s.h2t[(c + 1) * LD + rh] = __float2bfloat16_rn(a3);
    }
    __syncwarp();
    // ---- layer 3 and the output layer
    zero_acc(acc);
    warp_gemm<H>(acc, s.h2 + 16 * w * LD, s.w3, lane);
    float h3l[16], h3h[16];
    float yl0 = 0.f, yl1 = 0.f, yh0 = 0.f, yh1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * j + 2 * t + e;
            const float zl = acc[j][e] + s.b3[c], zh = acc[j][2 + e] + s.b3[c];
            s.z3[rl * H + c] = zl;
            s.z3[rh * H + c] = zh;
            h3l[2 * j + e] = silu(zl);   // layer 4 takes the activations in two BF16 parts: ~16 bits
            h3h[2 * j + e] = silu(zh);
            yl0 = fmaf(s.w4[c], h3l[2 * j + e], yl0);
            yl1 = fmaf(s.w4[H + c], h3l[2 * j + e], yl1);
            yh0 = fmaf(s.w4[c], h3h[2 * j + e], yh0);
            yh1 = fmaf(s.w4[H + c], h3h[2 * j + e], yh1);
        }
    }
#pragma unroll
    for (int o = 1; o <= 2; o <<= 1) {
        yl0 += __shfl_xor_sync(kFull, yl0, o);
        yl1 += __shfl_xor_sync(kFull, yl1, o);
        yh0 += __shfl_xor_sync(kFull, yh0, o);
        yh1 += __shfl_xor_sync(kFull, yh1, o);
    }
    yl0 += s.b4[0];
    yl1 += s.b4[1];
    yh0 += s.b4[0];
    yh1 += s.b4[1];
    // ---- loss gradient: d/dy of mean over (rows x 2 outputs) of squared error
    const float scale = 1.0f / (float)a.n_rows;
    const float el0 = okl ? yl0 - s.y[2 * rl] : 0.f, el1 = okl ? yl1 - s.y[2 * rl + 1] : 0.f;
    const float eh0 = okh ? yh0 - s.y[2 * rh] : 0.f, eh1 = okh ? yh1 - s.y[2 * rh + 1] : 0.f;
    const float dyl0 = scale * el0, dyl1 = scale * el1, dyh0 = scale * eh0, dyh1 = scale * eh1;
    if (t == 0) {
        float lsum = el0 * el0 + el1 * el1 + eh0 * eh0 + eh1 * eh1;
        float b0 = dyl0 + dyh0, b1 = dyl1 + dyh1;
        for (int o = 4; o <= 16; o <<= 1) {
            lsum += __shfl_xor_sync(0x11111111u, lsum, o);
            b0 += __shfl_xor_sync(0x11111111u, b0, o);
            b1 += __shfl_xor_sync(0x11111111u, b1, o);
        }
        if (lane == 0) {
            s.loss[w] = lsum;
            s.gb4[w][0] = b0;
            s.gb4[w][1] = b1;
        }
    }
    // dW4 and dz3
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * j + 2 * t + e;
            float g0 = dyl0 * h3l[2 * j + e] + dyh0 * h3h[2 * j + e];
            float g1 = dyl1 * h3l[2 * j + e] + dyh1 * h3h[2 * j + e];
            for (int o = 4; o <= 16; o <<= 1) {
                g0 += __shfl_xor_sync(kFull, g0, o);
                g1 += __shfl_xor_sync(kFull, g1, o);
            }
            if (g == 0) {
                s.gw4[w][c] = g0;
                s.gw4[w][H + c] = g1;
            }
            const float dzl = (dyl0 * s.w4[c] + dyl1 * s.w4[H + c]) * dsilu(s.z3[rl * H + c]);
            const float dzh = (dyh0 * s.w4[c] + dyh1 * s.w4[H + c]) * dsilu(s.z3[rh * H + c]);
            s.dz3[rl * LD + c] = __float2bfloat16_rn(dzl);
            s.dz3[rh * LD + c] = __float2bfloat16_rn(dzh);
            s.dz3t[c * LD + rl] = __float2bfloat16_rn(dzl);
            s.dz3t[c * LD + rh] = __float2bfloat16_rn(dzh);
            float gb = dzl + dzh;
            for (int o = 4; o <= 16; o <<= 1) gb += __shfl_xor_sync(kFull, gb, o);
            if (g == 0) s.gb3[w][c] = gb;
        }
    }
    __syncthreads();
    float *gout = a.grad_cta + (size_t)cta * kMlpParams;
    // ---- dW3 = dz3^T h2 (warp w: output units 16w .. 16w + 15, K = the CTA's 64 rows)
    zero_acc(acc);
    warp_gemm<kMlpRowsPerCta>(acc, s.dz3t + 16 * w * LD, s.h2t, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        gout[OFF_W3 + rl * H + c] = acc[j][0];
        gout[OFF_W3 + rl * H + c + 1] = acc[j][1];
        gout[OFF_W3 + rh * H + c] = acc[j][2];
        gout[OFF_W3 + rh * H + c + 1] = acc[j][3];
    }
    // ---- dh2 = dz3 W3, dz2
    zero_acc(acc);
    warp_gemm<H>(acc, s.dz3 + 16 * w * LD, s.w3t, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * j + 2 * t + e;
            const float dzl = acc[j][e] * dsilu(s.z2[rl * H + c]), dzh = acc[j][2 + e] * dsilu(s.z2[rh * H + c]);
            s.dz2[rl * LD + c] = __float2bfloat16_rn(dzl);
            s.dz2[rh * LD + c] = __float2bfloat16_rn(dzh);
            s.dz2t[c * LD + rl] = __float2bfloat16_rn(dzl);
            s.dz2t[c * LD + rh] = __float2bfloat16_rn(dzh);
            float gb = dzl + dzh;
            for (int o = 4; o <= 16; o <<= 1) gb += __shfl_xor_sync(kFull, gb, o);
            if (g == 0) s.gb2[w][c] = gb;
        }
    }
    __syncthreads();
    // ---- dW2 = dz2^T h1
    zero_acc(acc);
    warp_gemm<kMlpRowsPerCta>(acc, s.dz2t + 16 * w * LD, s.h1t, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        gout[OFF_W2 + rl * H + c] = acc[j][0];
        gout[OFF_W2 + rl * H + c + 1] = acc[j][1];
        gout[OFF_W2 + rh * H + c] = acc[j][2];
        gout[OFF_W2 + rh * H + c + 1] = acc[j][3];
    }
    // ---- dh1 = dz2 W2, dz1, dW1, db1
    zero_acc(acc);
    warp_gemm<H>(acc, s.dz2 + 16 * w * LD, s.w2t, lane);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int c = 8 * j + 2 * t + e;
            const float dzl = acc[j][e] * dsilu(s.z1[rl * H + c]), dzh = acc[j][2 + e] * dsilu(s.z1[rh * H + c]);
            float gb = dzl + dzh;
            float gk[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) gk[k] = dzl * s.x[4 * rl + k] + dzh * s.x[4 * rh + k];
            for (int o = 4; o <= 16; o <<= 1) {
                gb += __shfl_xor_sync(kFull, gb, o);
#pragma unroll
                for (int k = 0; k < 4; ++k) gk[k] += __shfl_xor_sync(kFull, gk[k], o);
            }
            if (g == 0) {
                s.gb1[w][c] = gb;
#pragma unroll
                for (int k = 0; k < 4; ++k) s.gw1[w][4 * c + k] = gk[k];
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < H * 4; i += blockDim.x)
        gout[OFF_W1 + i] = ((s.gw1[0][i] + s.gw1[1][i]) + s.gw1[2][i]) + s.gw1[3][i];
    for (int i = tid; i < 2 * H; i += blockDim.x)
        gout[OFF_W4 + i] = ((s.gw4[0][i] + s.gw4[1][i]) + s.gw4[2][i]) + s.gw4[3][i];
    for (int i = tid; i < H; i += blockDim.x) {
        gout[OFF_B1 + i] = ((s.gb1[0][i] + s.gb1[1][i]) + s.gb1[2][i]) + s.gb1[3][i];
        gout[OFF_B2 + i] = ((s.gb2[0][i] + s.gb2[1][i]) + s.gb2[2][i]) + s.gb2[3][i];
        gout[OFF_B3 + i] = ((s.gb3[0][i] + s.gb3[1][i]) + s.gb3[2][i]) + s.gb3[3][i];
    }
    if (tid < 2) gout[OFF_B4 + tid] = ((s.gb4[0][tid] + s.gb4[1][tid]) + s.gb4[2][tid]) + s.gb4[3][tid];
    if (tid == 0) a.loss_cta[cta] = ((s.loss[0] + s.loss[1]) + s.loss[2]) + s.loss[3];
}

// Sum of the per-CTA gradients in CTA order (deterministic), then Adam with
// bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t. With grad_out the
// summed gradient is only written out (no update).
__global__ void k_mlp_adam(float *params, float *m, float *v, const float *grad_cta, const float *loss_cta, int n_cta,
                           float lr, float bc1, float bc2, float *grad_out, float *loss_out, float loss_scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_out) {
        float l = 0.f;
        for (int c = 0; c < n_cta; ++c) l += loss_cta[c];
        *loss_out = l * loss_scale;
    }
    if (i >= kMlpParams) return;
    float gsum = 0.f;
    for (int c = 0; c < n_cta; ++c) gsum += grad_cta[(size_t)c * kMlpParams + i];
    if (grad_out) {
        grad_out[i] = gsum;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mi = b1 * m[i] + (1.0f - b1) * gsum;
    const float vi = b2 * v[i] + (1.0f - b2) * gsum * gsum;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Exact training samples: (cos, lambda, s, d) uniform over the trained box,
// lambda continuous (material curves linearly interpolated between bins).
__global__ void k_mlp_data(DevScene sc, uint32_t mat, int64_t n, uint32_t seed, float dmin, float dmax, float *X,
                           float *Y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 u = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)(i >> 32), 0u, 0x20001u), seed, 0x4d4c5044u);
    const float c = u01(u.x), lam = 380.0f + 400.0f * u01(u.y), st = u01(u.z), d = dmin + (dmax - dmin) * u01(u.w);
    const int L = sc.L;
    int lo = 0, hi = L - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(sc.lam + mid) <= lam) lo = mid; else hi = mid;
    }
    const float l0 = __ldg(sc.lam + lo), l1 = __ldg(sc.lam + hi);
    const float f = l1 > l0 ? fminf(fmaxf((lam - l0) / (l1 - l0), 0.0f), 1.0f) : 0.0f;
    const size_t k0 = (size_t)mat * L + lo, k1 = (size_t)mat * L + hi;
    const float nn = (1.0f - f) * __ldg(sc.mat_a + k0) + f * __ldg(sc.mat_a + k1);
    const float ac = (1.0f - f) * __ldg(sc.mat_b + k0) + f * __ldg(sc.mat_b + k1);
    const float da = (1.0f - f) * __ldg(sc.mat_c + k0) + f * __ldg(sc.mat_c + k1);
    float R_, T_;
    const int J = sc.mat_nfilm ? __ldg(sc.mat_nfilm + mat) : 0;
    float film_a = 0.0f;   // the films' normal-incidence absorbance (feature x3)
    if (J == 0) {
        slab_RT(c, lam, nn, ac + st * da, d, R_, T_);
    } else {   // coated glass: film curves interpolated between the same bins
        float nf[kMaxFilms], kf[kMaxFilms], tf[kMaxFilms];
        for (int j = 0; j < J; ++j) {
            const size_t f0 = ((size_t)mat * kMaxFilms + j) * L + lo, f1 = ((size_t)mat * kMaxFilms + j) * L + hi;
            nf[j] = (1.0f - f) * __ldg(sc.film_n + f0) + f * __ldg(sc.film_n + f1);
            kf[j] = (1.0f - f) * (__ldg(sc.film_k + f0) + st * __ldg(sc.film_dk + f0)) +
                    f * (__ldg(sc.film_k + f1) + st * __ldg(sc.film_dk + f1));
            tf[j] = __ldg(sc.film_t + (size_t)mat * kMaxFilms + j);
        }
        coated_RT(c, lam, nn, ac + st * da, d, J, nf, kf, tf, R_, T_);
        for (int j = 0; j < J; ++j) film_a = fmaf(12.566370614359172f * kf[j], tf[j] / lam, film_a);
    }
    float x[4];
    features(c, lam, st, (ac + st * da) * d + film_a, x);
    for (int k = 0; k < 4; ++k) X[4 * i + k] = x[k];
    Y[2 * i] = rt_to_out(R_);
    Y[2 * i + 1] = rt_to_out(T_);
}

// Xavier-uniform initial weights from Philox, zero biases.
__global__ void k_mlp_init(float *p, uint32_t seed) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    float bound = 0.0f;
    if (i < OFF_B1) bound = sqrtf(6.0f / (4 + H));
    else if (i >= OFF_W2 && i < OFF_B2) bound = sqrtf(6.0f / (H + H));
    else if (i >= OFF_W3 && i < OFF_B3) bound = sqrtf(6.0f / (H + H));
    else if (i >= OFF_W4 && i < OFF_B4) bound = sqrtf(6.0f / (H + 2));
    const uint4 u = philox4x32_10(make_uint4((uint32_t)i, 0u, 0u, 0x20002u), seed, 0x494e4954u);
    p[i] = bound * (2.0f * u01(u.x) - 1.0f);
}

// Max |error| of R and T over a held-out grid of the trained box (cos, bin, s, d).
__global__ void k_mlp_grid_error(MlpRows a, unsigned int *max_err) {
    __shared__ InferSmem s;
    load_infer_weights(s, a.params);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int L = a.sc.L;
    const int nc = 17, ns = 5, nd = 5;
    const int64_t total = (int64_t)nc * L * ns * nd;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    auto grid_in = [&](int64_t r, RowIn &in) {
        int64_t q = r;
        const int ic = (int)(q % nc);
        q /= nc;
        const int ib = (int)(q % L);
        q /= L;
        const int is = (int)(q % ns);
        q /= ns;
        const int id = (int)q;
        in.c = (ic + 0.5f) / nc;
        in.bin = ib;
        in.lam = __ldg(a.sc.lam + ib);
        in.s = (is + 0.5f) / ns;
        in.d = a.thick_min + (a.thick_max - a.thick_min) * (id + 0.5f) / nd;
        in.mat = (int)a.mat;
    };
    for (int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + w; b * 16 < total; b += nwarps) {
        const int64_t r0 = b * 16;
        RowIn il, ih;
        grid_in(min(r0 + g, total - 1), il);
        grid_in(min(r0 + g + 8, total - 1), ih);
        float xl[4], xh[4], yl[2], yh[2];
        features(il.c, il.lam, il.s, row_alpha_d(a.sc, il), xl);
        features(ih.c, ih.lam, ih.s, row_alpha_d(a.sc, ih), xh);
        tile_forward(s, xl, xh, lane, yl, yh);
        if (t == 0) {
            const float2 el = exact_row(a, il), eh = exact_row(a, ih);
            atomicMax(max_err + 0,
                      __float_as_uint(fmaxf(fabsf(el.x - out_to_rt(yl[0])), fabsf(eh.x - out_to_rt(yh[0])))));
            atomicMax(max_err + 1,
                      __float_as_uint(fmaxf(fabsf(el.y - out_to_rt(yl[1])), fabsf(eh.y - out_to_rt(yh[1])))));
        }
        __syncwarp();
    }
}

}  // namespace

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

#ifndef SDDM_MLP_BLOCKS_PER_SM
#define SDDM_MLP_BLOCKS_PER_SM 4   // inference blocks (8 warps, ~41 KB shared memory) per SM
#endif
// Blocks of a grid-stride row kernel: per SM, the most that fit at once (at
// most `cap`), so that the grid is one whole wave.
template <typename K>
static int resident_per_sm(K kernel, int cap) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, 256, 0) != cudaSuccess || n < 1) return cap;
    return n < cap ? n : cap;
}

cudaError_t launch_mlp_rows(const MlpRows &a, int sm_count, cudaStream_t stream) {
    const int blocks = sm_count * (a.sc.mat_nfilm ? resident_per_sm(k_mlp_rows<true>, SDDM_MLP_BLOCKS_PER_SM)
                                                  : resident_per_sm(k_mlp_rows<false>, SDDM_MLP_BLOCKS_PER_SM));
    if (a.sc.mat_nfilm)
        k_mlp_rows<true><<<blocks, 256, 0, stream>>>(a);
    else
        k_mlp_rows<false><<<blocks, 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_slab_rows(const MlpRows &a, int sm_count, cudaStream_t stream) {
    if (a.sc.mat_nfilm)
        k_slab_rows<true><<<sm_count * resident_per_sm(k_slab_rows<true>, 8), 256, 0, stream>>>(a);
    else
        k_slab_rows<false><<<sm_count * resident_per_sm(k_slab_rows<false>, 8), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train_tile(const MlpTrainArgs &a, cudaStream_t stream) {
    static bool attr_set = false;
    const size_t bytes = sizeof(TrainSmem);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int n_cta = (a.n_rows + kMlpRowsPerCta - 1) / kMlpRowsPerCta;
    k_mlp_train_tile<<<n_cta, 128, bytes, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *params, float *m, float *v, const float *grad_cta, const float *loss_cta, int n_cta,
                            float lr, float bc1, float bc2, float *grad_out, float *loss_out, float loss_scale,
                            cudaStream_t stream) {
    k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, m, v, grad_cta, loss_cta, n_cta, lr, bc1, bc2,
                                                             grad_out, loss_out, loss_scale);
    return cudaGetLastError();
}

cudaError_t launch_mlp_data(const DevScene &sc, uint32_t mat, float, int64_t n, uint32_t seed, float dmin, float dmax,
                            float *X, float *Y, cudaStream_t stream) {
    k_mlp_data<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(sc, mat, n, seed, dmin, dmax, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_init(float *params, uint32_t seed, cudaStream_t stream) {
    k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grid_error(const float *params, const DevScene &sc, uint32_t mat, float dmin, float dmax,
                                  unsigned int *max_err, cudaStream_t stream) {
    MlpRows a{};
    a.params = params;
    a.sc = sc;
    a.mat = mat;
    a.thick_min = dmin;
    a.thick_max = dmax;
    k_mlp_grid_error<<<152, 256, 0, stream>>>(a, max_err);
    return cudaGetLastError();
}

}  // namespace sddm
