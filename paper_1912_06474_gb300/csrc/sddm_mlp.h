// Glass-slab surrogate network: device entry points (mlp.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sddm_internal.h"

namespace sddm {

constexpr int kMlpParams = 8770;
constexpr int kMlpRowsPerCta = 64;       // training tile
constexpr float kMlpProbeTol = 1e-3f;    // |dR|, |dT| above which a 32-row batch falls back to exact

// Rows to evaluate: explicit per-row inputs (mode 0, the test hook), the
// renderer's glass queries, each expanded over the L wavelength bins (mode
// 1), or a held-out grid of the trained box (mode 2, training report).
struct MlpRows {
    const float *params;              // FP32 master weights [8770]
    DevScene sc;
    float thick_min, thick_max;       // trained thickness box
    uint32_t probe_key;               // Philox key word of the probe choice
    // explicit rows (mode 0)
    int n;
    uint32_t mat;
    const float *cos_t, *s, *thick;
    const int32_t *bin;
    float *R, *T;
    // renderer queries (mode 1): query = (cos, s, thickness, material bits)
    const float4 *queries;
    const unsigned long long *n_queries;
    int64_t q_cap;                    // queries beyond it were not stored
    float2 *results;                  // [query][L] (R, T)
    int mode;
    int raw;                          // 1: network output only, no probe or fallback
    unsigned long long *fallbacks;    // 32-row batches that fell back to the exact slab
    unsigned long long *batches;      // 32-row batches evaluated (probe batches; NULL: not counted)
    int *err;                         // device error word [4] (NULL: not reported); 2 = a wait ran out
    unsigned int *grid_err;           // mode 2: largest |dR|, |dT| as float bits [2]
    unsigned long long *rows;         // rows the network evaluated (NULL: not counted)
    int test_timeout;                 // 1: CTA 0 issues no layer-1 MMA and waits 2^10 tries (failure-path test)
};
// The network over every row (tensor cores), then, unless raw, the probes
// and the exact fallback of failing batches: two kernels on `stream`. With
// ev0 / ev1 given, they are recorded around the network kernel.
cudaError_t launch_mlp_rows(const MlpRows &a, int sm_count, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                            cudaEvent_t ev1 = nullptr);
// The exact slab over the same rows (no network).
cudaError_t launch_slab_rows(const MlpRows &a, int sm_count, cudaStream_t stream);

// Training.
struct MlpTrainArgs {
    const float *params;              // [8770]
    const float *X, *Y;               // [n_samples][4], [n_samples][2]
    int64_t n_samples, row0;          // rows row0 .. row0 + n_rows - 1 (mod n_samples)
    int n_rows;                       // rows of this step
    float *grad_cta;                  // [n_cta][8770]
    float *loss_cta;                  // [n_cta]
};
cudaError_t launch_mlp_train_tile(const MlpTrainArgs &a, cudaStream_t stream);
cudaError_t launch_mlp_adam(float *params, float *m, float *v, const float *grad_cta, const float *loss_cta, int n_cta,
                            float lr, float bc1, float bc2, float *grad_out, float *loss_out, float loss_scale,
                            cudaStream_t stream);
cudaError_t launch_mlp_data(const DevScene &sc, uint32_t mat, float state_unused, int64_t n, uint32_t seed,
                            float thick_min, float thick_max, float *X, float *Y, cudaStream_t stream);
cudaError_t launch_mlp_init(float *params, uint32_t seed, cudaStream_t stream);
// The parameter buffer holds the FP32 parameters and, behind them, the weights
// packed in the inference kernel's tensor-core operand layout; launch_mlp_pack
// rewrites the packed copy from the parameters (after every change of them).
size_t mlp_param_buffer_bytes();
cudaError_t launch_mlp_pack(float *params, cudaStream_t stream);
cudaError_t launch_mlp_grid_error(const float *params, const DevScene &sc, uint32_t mat, float thick_min,
                                  float thick_max, unsigned int *max_err2, int *err, int sm_count,
                                  cudaStream_t stream);
size_t mlp_train_smem_bytes();

}  // namespace sddm
