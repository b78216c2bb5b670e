// Learned surrogate of the glass slab's R and T (a stand-in for the exact
// Fresnel-equation glass of Sec. 6): a 4 -> 64 -> 64 -> 64 -> 2 SiLU
// network with BF16 weights and FP32 accumulation. Inference runs its three
// 64-wide layers on the tcgen05 tensor cores, 128 rows per CTA with the
// accumulators in tensor memory; training uses warp-level m16n8k16 MMAs on
// 16-row tiles whose activations stay in registers from layer to layer.
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
// The network runs on the fifth-generation tensor cores (tcgen05): a CTA of
// four warps carries a tile of 128 rows through the hidden layers, one row
// per thread. For each layer one thread issues the MMAs (M = 128, N = 64,
// K = 16 each, BF16 operands from shared memory, FP32 accumulators in tensor
// memory), the CTA waits on an mbarrier that the tensor core arrives on when
// they are done, and every warp reads back its 32 rows of accumulators
// (tensor-memory lanes 32w .. 32w + 31 belong to warp w), applies SiLU and
// writes the BF16 activations into the A operand of the next layer.
//
// The hidden layers' weights and biases are stored halved: a layer then
// produces h = z / 2 directly (halving is exact in binary floating point, so
// the activations are bit for bit those of the unscaled layer), and SiLU(z) =
// h + h tanh(h) costs one SFU operation and one FMA.
//  * Layer 1 (K = 4) is one K = 16 step whose A row is [x_hi(4) | x_lo(4) | 1 |
//    1 | 0 ...] and whose B row for output n is [W1n(4) | W1n(4) | b_hi | b_lo |
//    0 ...]: inputs and bias each split into two BF16 parts, so the products
//    keep 16 bits of the FP32 inputs and bias.
//  * Layers 2 and 3 (64 x 64) are four K steps over the activations plus one
//    over a constant A chunk [1 | 1 | 0 ...] against [b_hi | b_lo | 0 ...]:
//    the bias in two BF16 parts, added by the tensor core.
//  * Layer 4 (N = 2) runs in FP32 on the CUDA cores from the FP32 activations
//    of layer 3 and the BF16-rounded output weights (training multiplies the
//    same weights by the activations split into two BF16 parts).
//
// Operands sit in shared memory in the tensor core's K-major layout without
// swizzle: 8-row x 16-byte core matrices, the core matrices of one 8-row group
// side by side along K (128 B apart, the leading-dimension offset) and the
// 8-row groups one after the other (the stride offset).
constexpr int kTcRows = 128;          // rows per tile = threads per CTA = TMEM lanes
constexpr int kTcCols = 64;           // TMEM columns: one 128 x 64 FP32 accumulator
constexpr int kChA = 10;              // A chunks per 8-row group: 8 activations + bias ones + zero
constexpr int kChB1 = 2;              // layer-1 B: K = 16
constexpr int kChB = 10;              // layers 2, 3 B: K = 64 + bias step
constexpr uint32_t kMbarTries = 1u << 22;   // bounded waits: ~seconds, then the CTA reports and stops
constexpr uint32_t kMbarTriesTest = 1u << 10;   // the failure-path test's wait on an MMA never issued

// The weights in the CTA's operand layout, packed once in global memory
// (k_mlp_pack, after every change of the parameters) and copied into each
// CTA's shared memory by one bulk TMA copy.
struct __align__(128) TcWeights {
    __nv_bfloat16 b1[H * kChB1 * 8];        // B of layer 1: W1 / 2 twice, b1 / 2 as hi + lo
    __nv_bfloat16 b2[H * kChB * 8], b3[H * kChB * 8];   // W / 2, bias / 2 as hi + lo in K columns 64, 65
    float w4[2][H];                         // BF16-rounded output weights (FP32 layer 4)
    float b4[2];
};
static_assert(sizeof(TcWeights) % 16 == 0, "bulk copies move multiples of 16 bytes");
struct __align__(128) TcSmem {
    TcWeights w;
    __nv_bfloat16 a[kTcRows * kChA * 8];    // activations / inputs, K-major core matrices
    unsigned long long mbar, mbar_w;        // MMA completion; weights arrived
    uint32_t tmem;
};

// Element offset of (row, k) in a K-major operand of `nch` 16-byte chunks per row.
__device__ __forceinline__ int kmaj(int row, int k, int nch) {
    return (row >> 3) * (nch * 64) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading- and stride-dimension
// byte offsets (16-byte units), descriptor version 1 (bits 46-47), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 D (bits 4-5 = 1), BF16 A and B
// (bits 7-9 = 1, 10-12 = 1), both K-major, N / 8 at bit 17, M / 16 at bit 24.
constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kIdescHidden = tc_idesc(kTcRows, H);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued so far is complete.
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Generic-proxy shared-memory writes made visible to the tensor core's reads.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t tries) {
    for (uint32_t i = 0; i < tries; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 64 consecutive FP32 accumulator columns of this thread's TMEM lane; the
// wait is in the same statement, so no use of the registers can precede it.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float v[64]) {
    uint32_t r[64];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n\t"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
          "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
          "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
          "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
          "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// SiLU of z given h = z / 2.
__device__ __forceinline__ float silu_h(float h) { return fmaf(h, tanh_fast(h), h); }

// The FP32 parameters into the operand layout of TcWeights (one CTA).
__global__ void __launch_bounds__(256) k_mlp_pack(const float *__restrict__ p, TcWeights *out) {
    TcWeights &s = *out;
    for (int i = threadIdx.x; i < H * kChB * 8; i += blockDim.x) {
        const int n = i / (kChB * 8), k = i % (kChB * 8);
        float v2 = 0.0f, v3 = 0.0f;
        if (k < H) {
            v2 = 0.5f * p[OFF_W2 + H * n + k];
            v3 = 0.5f * p[OFF_W3 + H * n + k];
        } else if (k < H + 2) {
            const float c2 = 0.5f * p[OFF_B2 + n], c3 = 0.5f * p[OFF_B3 + n];
            v2 = k == H ? bf16r(c2) : c2 - bf16r(c2);
            v3 = k == H ? bf16r(c3) : c3 - bf16r(c3);
        }
        s.b2[kmaj(n, k, kChB)] = __float2bfloat16_rn(v2);
        s.b3[kmaj(n, k, kChB)] = __float2bfloat16_rn(v3);
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
        s.b1[kmaj(n, k, kChB1)] = __float2bfloat16_rn(v);
    }
    for (int i = threadIdx.x; i < 2 * H; i += blockDim.x) s.w4[i / H][i % H] = bf16r(p[OFF_W4 + i]);
    if (threadIdx.x < 2) s.b4[threadIdx.x] = p[OFF_B4 + threadIdx.x];
}

// A columns 64..79 of every row: [1, 1, 0, ...] against the biases' two parts.
__device__ void tc_put_bias_columns(TcSmem &s) {
    for (int i = threadIdx.x; i < kTcRows * 16; i += blockDim.x) {
        const int r = i >> 4, k = 64 + (i & 15);
        s.a[kmaj(r, k, kChA)] = __float2bfloat16_rn(k < 66 ? 1.0f : 0.0f);
    }
}

// Byte offset of the packed image behind the FP32 parameters in one buffer.
constexpr size_t kImageOffset = (kMlpParams * sizeof(float) + 127) / 128 * 128;
__device__ __forceinline__ const TcWeights *weight_image(const float *params) {
    return reinterpret_cast<const TcWeights *>(reinterpret_cast<const char *>(params) + kImageOffset);
}

// This thread's row of layer-1 A: [x_hi | x_lo], then [1, 1, 0 ...].
__device__ __forceinline__ void tc_put_inputs(TcSmem &s, int row, const float x[4]) {
    float hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        hi[i] = bf16r(x[i]);
        lo[i] = x[i] - hi[i];
    }
    const uint4 c0 = make_uint4(pack_bf16x2(hi[0], hi[1]), pack_bf16x2(hi[2], hi[3]), pack_bf16x2(lo[0], lo[1]),
                                pack_bf16x2(lo[2], lo[3]));
    const uint4 c1 = make_uint4(pack_bf16x2(1.0f, 1.0f), 0u, 0u, 0u);
    *reinterpret_cast<uint4 *>(s.a + kmaj(row, 0, kChA)) = c0;
    *reinterpret_cast<uint4 *>(s.a + kmaj(row, 8, kChA)) = c1;
}

// SiLU of this thread's 64 accumulators (h = z / 2), as BF16 into its A row.
__device__ __forceinline__ void tc_put_hidden(TcSmem &s, int row, const float v[64]) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint4 u;
        u.x = pack_bf16x2(silu_h(v[8 * c + 0]), silu_h(v[8 * c + 1]));
        u.y = pack_bf16x2(silu_h(v[8 * c + 2]), silu_h(v[8 * c + 3]));
        u.z = pack_bf16x2(silu_h(v[8 * c + 4]), silu_h(v[8 * c + 5]));
        u.w = pack_bf16x2(silu_h(v[8 * c + 6]), silu_h(v[8 * c + 7]));
        *reinterpret_cast<uint4 *>(s.a + kmaj(row, 8 * c, kChA)) = u;
    }
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

// The held-out grid of the trained box (mode 2): cos, bin, s and thickness at
// cell centres of a 17 x L x 5 x 5 grid.
constexpr int kGridCos = 17, kGridS = 5, kGridD = 5;

// Rows to evaluate: mode 0 explicit rows, mode 1 the renderer's queries
// expanded over the L bins, mode 2 the held-out grid.
__device__ __forceinline__ int64_t mlp_total_rows(const MlpRows &a) {
    if (a.mode == 1) {
        const int64_t nq0 = (int64_t)*a.n_queries;
        return (nq0 < a.q_cap ? nq0 : a.q_cap) * a.sc.L;
    }
    if (a.mode == 2) return (int64_t)kGridCos * a.sc.L * kGridS * kGridD;
    return a.n;
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
    } else if (a.mode == 1) {
        const int64_t q = r / L;
        const float4 qq = a.queries[q];
        in.c = qq.x;
        in.s = qq.y;
        in.d = qq.z;
        in.mat = __float_as_int(qq.w);
        in.bin = (int)(r - q * L);
    } else {
        int64_t q = r;
        const int ic = (int)(q % kGridCos);
        q /= kGridCos;
        const int ib = (int)(q % L);
        q /= L;
        const int is = (int)(q % kGridS);
        const int id = (int)(q / kGridS);
        in.c = (ic + 0.5f) / kGridCos;
        in.bin = ib;
        in.s = (is + 0.5f) / kGridS;
        in.d = a.thick_min + (a.thick_max - a.thick_min) * (id + 0.5f) / kGridD;
        in.mat = (int)a.mat;
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

__device__ __forceinline__ bool row_in_box(const MlpRows &a, const RowIn &in) {
    return in.c >= 0.0f && in.c <= 1.0f && in.lam >= 380.0f && in.lam <= 780.0f && in.s >= 0.0f && in.s <= 1.0f &&
           in.d >= a.thick_min && in.d <= a.thick_max;
}

__device__ __forceinline__ void store_row(const MlpRows &a, int64_t r, float2 y) {
    if (a.mode == 0) {
        a.R[r] = y.x;
        a.T[r] = y.y;
    } else {
        a.results[r] = y;
    }
}

// The network over all rows, tile by tile (see the top of this section).
// Writes the served (R, T) of every row; mode 2 instead records the largest
// |error| against the exact slab. On a wait that runs out (the tensor core
// never signalled completion) the CTA reports error 2 and stops.
#ifndef SDDM_MLP_MINB
#define SDDM_MLP_MINB 5   // resident 128-thread tile CTAs per SM (96 registers; shared memory admits 5)
#endif
template <bool FILMS>
__global__ void __launch_bounds__(kTcRows, SDDM_MLP_MINB) k_mlp_net(MlpRows a) {
    __shared__ TcSmem s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t mbar = smem_addr(&s.mbar), mbar_w = smem_addr(&s.mbar_w);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s.tmem)),
                     "r"((uint32_t)kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(mbar);
        mbar_init(mbar_w);
    }
    __syncthreads();
    // the packed weights by one bulk copy (the TMA engine), completion on mbar_w
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_w),
                     "r"((uint32_t)sizeof(TcWeights))
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_addr(&s.w)),
                     "l"(weight_image(a.params)), "r"((uint32_t)sizeof(TcWeights)), "r"(mbar_w)
                     : "memory");
    }
    tc_put_bias_columns(s);
    const bool w_ok = mbar_wait(mbar_w, 0u, kMbarTries);
    fence_async_smem();
    tc_fence_before();
    const bool w_failed = __syncthreads_or(!w_ok) != 0;
    tc_fence_after();
    const uint32_t tmem = s.tmem;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
    const uint32_t sa = smem_addr(s.a), sb1 = smem_addr(s.w.b1), sb2 = smem_addr(s.w.b2), sb3 = smem_addr(s.w.b3);
    constexpr uint32_t kSboA = kChA * 128, kSboB1 = kChB1 * 128, kSboB = kChB * 128;
    const int64_t total = mlp_total_rows(a);
    const int64_t n_tiles = (total + kTcRows - 1) / kTcRows;
    if (a.rows && blockIdx.x == 0 && tid == 0) atomicAdd(a.rows, (unsigned long long)total);
    uint32_t phase = 0;
    bool failed = w_failed;   // this thread's wait on the tensor core (or on the weights) ran out
    // failure-path test: CTA 0 issues nothing, so its first wait runs out
    const bool skip = a.test_timeout && blockIdx.x == 0;
    const uint32_t tries = skip ? kMbarTriesTest : kMbarTries;
    // One layer: the A rows written by every thread are made visible to the
    // tensor core, the CTA synchronises (and learns whether any thread's
    // previous wait ran out: then it stops, false), one thread issues the
    // MMAs, and every thread waits on the mbarrier for their completion.
    auto layer = [&](int l) -> bool {
        fence_async_smem();
        tc_fence_before();
        if (__syncthreads_or(failed)) return false;
        if (tid == 0 && !skip) {
            tc_fence_after();
            if (l == 1) {
                tc_mma(tmem, tc_desc(sa, 128, kSboA), tc_desc(sb1, 128, kSboB1), kIdescHidden, 0u);
            } else {
                const uint32_t sb = l == 2 ? sb2 : sb3;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks)
                    tc_mma(tmem, tc_desc(sa + 256 * ks, 128, kSboA), tc_desc(sb + 256 * ks, 128, kSboB), kIdescHidden,
                           ks > 0 ? 1u : 0u);
                tc_mma(tmem, tc_desc(sa + 1024, 128, kSboA), tc_desc(sb + 1024, 128, kSboB), kIdescHidden, 1u);
            }
            tc_commit(mbar);
        }
        failed = !mbar_wait(mbar, phase, tries);
        phase ^= 1u;
        tc_fence_after();
        return true;
    };
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r = tile * kTcRows + tid;
        RowIn in;
        const bool valid = row_input(a, r, total, in);
        float x[4];
        features(in.c, in.lam, in.s, row_alpha_d<FILMS>(a.sc, in), x);
        tc_put_inputs(s, tid, x);
        float v[64];
        if (!layer(1)) break;
        tmem_ld64(taddr, v);
        tc_put_hidden(s, tid, v);
        if (!layer(2)) break;
        tmem_ld64(taddr, v);
        tc_put_hidden(s, tid, v);
        if (!layer(3)) break;
        tmem_ld64(taddr, v);
        float y0 = s.w.b4[0], y1 = s.w.b4[1];
#pragma unroll
        for (int j = 0; j < H; ++j) {
            const float h = silu_h(v[j]);
            y0 = fmaf(s.w.w4[0][j], h, y0);
            y1 = fmaf(s.w.w4[1][j], h, y1);
        }
        const float2 y = make_float2(out_to_rt(y0), out_to_rt(y1));
        if (valid) {
            if (a.mode == 2) {
                const float2 e = exact_row<FILMS>(a, in);
                atomicMax(a.grid_err + 0, __float_as_uint(fabsf(e.x - y.x)));
                atomicMax(a.grid_err + 1, __float_as_uint(fabsf(e.y - y.y)));
            } else {
                store_row(a, r, y);
            }
        }
    }
    if (failed && a.err && atomicCAS(a.err, 0, 2) == 0) {
        a.err[1] = 20;   // surrogate inference: the tensor core did not complete
        a.err[2] = (int)blockIdx.x;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)kTcCols)
                     : "memory");
    }
}

// Probe and fallback, after the network has served every row. A batch is up
// to 32 rows of one query's bins (renderer queries: a batch never mixes two
// glass evaluations, so its probe speaks for rows that share angle, state and
// thickness) or 32 consecutive explicit rows. One row of each batch, chosen by
// Philox, is evaluated exactly; if it is off by more than 1e-3 in R or T, or
// if a row of the batch lies outside the trained box, the whole batch is
// evaluated exactly instead. Lane k of a warp probes batch k of a round of 32
// batches, so a probe costs one lane's share of an exact evaluation; failing
// batches are then redone by the whole warp, one row per lane.
template <bool FILMS>
__global__ void __launch_bounds__(256) k_mlp_probe(MlpRows a) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int L = a.sc.L;
    const int64_t total = mlp_total_rows(a);
    const int nb = a.mode == 1 ? (L + 31) / 32 : 1;
    const int64_t n_batches = a.mode == 1 ? total / L * nb : (total + 31) / 32;
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
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t b_first = (int64_t)blockIdx.x * (blockDim.x >> 5) + w;
    unsigned long long n_fb = 0;
    for (int64_t k0 = 0; b_first + k0 * nwarps < n_batches; k0 += 32) {
        const int64_t b = b_first + (k0 + lane) * nwarps;
        int bad = 0;
        if (b < n_batches) {
            int64_t r0;
            int nvalid;
            batch_rows(b, r0, nvalid);
            RowIn in;
            // the trained box: one query's rows share cos, s and thickness and
            // their wavelengths rise with the bin, so its first and last rows
            // decide; explicit rows are checked one by one
            if (a.mode == 1) {
                row_input(a, r0, total, in);
                bad = !row_in_box(a, in);
                row_input(a, r0 + nvalid - 1, total, in);
                bad |= !row_in_box(a, in);
            } else {
                for (int i = 0; i < nvalid; ++i) {
                    row_input(a, r0 + i, total, in);
                    bad |= !row_in_box(a, in);
                }
            }
            const uint4 pr = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0u, kSlotProbe),
                                           a.probe_key, 0x50524f42u);
            const int64_t r = r0 + (int)(pr.x % (uint32_t)nvalid);
            row_input(a, r, total, in);
            const float2 e = exact_row<FILMS>(a, in);
            const float2 y = a.mode == 0 ? make_float2(a.R[r], a.T[r]) : a.results[r];
            bad |= fabsf(e.x - y.x) > kMlpProbeTol || fabsf(e.y - y.y) > kMlpProbeTol;
        }
        unsigned fall = __ballot_sync(kFull, bad);
        while (fall) {
            const int k = __ffs(fall) - 1;
            fall &= fall - 1;
            int64_t r0;
            int nvalid;
            batch_rows(b_first + (k0 + k) * nwarps, r0, nvalid);
            RowIn in;
            if (lane < nvalid && row_input(a, r0 + lane, total, in)) store_row(a, r0 + lane, exact_row<FILMS>(a, in));
            if (lane == 0) ++n_fb;
        }
    }
    if (a.fallbacks && n_fb) atomicAdd(a.fallbacks, n_fb);
    if (a.batches && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.batches, (unsigned long long)n_batches);
}

// The exact slab for the same query rows, one thread per (query, bin): the
// glass evaluations of a bounce as one dense, divergence-free pass.
template <bool FILMS>
__global__ void __launch_bounds__(256) k_slab_rows(MlpRows a) {
    const int64_t total = mlp_total_rows(a);
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

}  // namespace

size_t mlp_train_smem_bytes() { return sizeof(TrainSmem); }

// Blocks of a grid-stride row kernel: per SM, the most that fit at once (at
// most `cap`), so that the grid is one whole wave.
template <typename K>
static int resident_per_sm(K kernel, int threads, int cap) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) return cap;
    return n < cap ? n : cap;
}

// Tile CTAs per SM: as many as the registers and shared memory allow
// (__launch_bounds__ asks for SDDM_MLP_MINB). Tensor memory has 512 columns
// per SM and each CTA holds kTcCols of them, so up to 512 / kTcCols resident
// CTAs never wait on one another's allocation.
static_assert(SDDM_MLP_MINB * kTcCols <= 512, "tensor-memory columns of the resident tile CTAs");
template <bool FILMS>
static cudaError_t launch_mlp_net(const MlpRows &a, int sm_count, cudaStream_t stream) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_net<FILMS>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_mlp_net<FILMS><<<sm_count * SDDM_MLP_MINB, kTcRows, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mlp_rows(const MlpRows &a, int sm_count, cudaStream_t stream, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e = ev0 ? cudaEventRecord(ev0, stream) : cudaSuccess;
    if (e == cudaSuccess)
        e = a.sc.mat_nfilm ? launch_mlp_net<true>(a, sm_count, stream) : launch_mlp_net<false>(a, sm_count, stream);
    if (e == cudaSuccess && ev1) e = cudaEventRecord(ev1, stream);
    if (e != cudaSuccess || a.raw) return e;
    if (a.sc.mat_nfilm)
        k_mlp_probe<true><<<sm_count * resident_per_sm(k_mlp_probe<true>, 256, 8), 256, 0, stream>>>(a);
    else
        k_mlp_probe<false><<<sm_count * resident_per_sm(k_mlp_probe<false>, 256, 8), 256, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_slab_rows(const MlpRows &a, int sm_count, cudaStream_t stream) {
    if (a.sc.mat_nfilm)
        k_slab_rows<true><<<sm_count * resident_per_sm(k_slab_rows<true>, 256, 8), 256, 0, stream>>>(a);
    else
        k_slab_rows<false><<<sm_count * resident_per_sm(k_slab_rows<false>, 256, 8), 256, 0, stream>>>(a);
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

size_t mlp_param_buffer_bytes() { return kImageOffset + sizeof(TcWeights); }

cudaError_t launch_mlp_pack(float *params, cudaStream_t stream) {
    k_mlp_pack<<<1, 256, 0, stream>>>(params, reinterpret_cast<TcWeights *>(reinterpret_cast<char *>(params) +
                                                                           kImageOffset));
    return cudaGetLastError();
}

cudaError_t launch_mlp_init(float *params, uint32_t seed, cudaStream_t stream) {
    k_mlp_init<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(params, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grid_error(const float *params, const DevScene &sc, uint32_t mat, float dmin, float dmax,
                                  unsigned int *max_err, int *err, int sm_count, cudaStream_t stream) {
    MlpRows a{};
    a.params = params;
    a.sc = sc;
    a.mat = mat;
    a.thick_min = dmin;
    a.thick_max = dmax;
    a.mode = 2;
    a.raw = 1;
    a.grid_err = max_err;
    a.err = err;
    return launch_mlp_rows(a, sm_count, stream);
}

}  // namespace sddm
