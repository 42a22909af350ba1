// Input and output marshalling of the learned-initialisation network (no
// counterpart in the paper): per-Gaussian features in BF16, targets and
// outputs as w = amplitude e^{j phase} per wavelength (Re, Im), which keeps
// the regression smooth across the phase wrap.
#include "common.cuh"

namespace hcgs {

__device__ __forceinline__ uint16_t to_bf16(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (uint16_t)((u >> 16) | 0x40u);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// x[n] = (mean 3, (log_scale + 4) / 0.5 (3), unit quaternion 4, opacity logit,
//         rgb 3, 0, 0) in bfloat16
__global__ void k_init_features(hcgs_gaussians g, const float* __restrict__ rgb, uint16_t* __restrict__ x) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= g.N) return;
    float f[16];
    for (int k = 0; k < 3; k++) {
        f[k] = g.means[3 * n + k];
        f[3 + k] = (g.log_scales[3 * n + k] + 4.f) * 2.f;
    }
    const float* q = g.quats + 4 * n;
    const float qn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; k++) f[6 + k] = q[k] * qn;
    f[10] = g.opacity_logits[n];
    for (int k = 0; k < 3; k++) f[11 + k] = rgb[3 * n + k];
    f[14] = f[15] = 0.f;
    for (int k = 0; k < 16; k++) x[16 * n + k] = to_bf16(f[k]);
}

// target[n] = (a_c cos phi_c, a_c sin phi_c) for c < C, zeros after
__global__ void k_init_targets(const float* __restrict__ amp, const float* __restrict__ ph, int N, int C,
                               float* __restrict__ t) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    for (int k = 0; k < 16; k++) t[16 * n + k] = 0.f;
    for (int c = 0; c < C; c++) {
        float s, co;
        sincosf(ph[C * n + c], &s, &co);
        t[16 * n + 2 * c] = amp[C * n + c] * co;
        t[16 * n + 2 * c + 1] = amp[C * n + c] * s;
    }
}

// amplitude = |w|, phase = arg w from the network output y[n][2c], y[n][2c+1]
__global__ void k_init_apply(const float* __restrict__ y, int N, int C, float* __restrict__ amp,
                             float* __restrict__ ph) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    for (int c = 0; c < C; c++) {
        const float re = y[16 * n + 2 * c], im = y[16 * n + 2 * c + 1];
        amp[C * n + c] = sqrtf(re * re + im * im);
        ph[C * n + c] = atan2f(im, re);
    }
}

}  // namespace hcgs

using namespace hcgs;

extern "C" {

hcgs_status hcgs_init_features(hcgs_ctx* ctx, const hcgs_gaussians* g, const float* rgb, uint16_t* x,
                               void* stream) {
    if (!ctx || !g || !rgb || !x) return HCGS_ERR_INVALID_ARG;
    if (g->N <= 0) return HCGS_OK;
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits) return HCGS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    HCGS_KERNEL(ctx, "k_init_features", st, k_init_features<<<(g->N + 255) / 256, 256, 0, st>>>(*g, rgb, x));
    return HCGS_OK;
}

hcgs_status hcgs_init_targets(hcgs_ctx* ctx, const float* amplitude, const float* phase, int N, int C,
                              float* target, void* stream) {
    if (!ctx || !amplitude || !phase || !target || N < 0 || C < 1 || C > 8) return HCGS_ERR_INVALID_ARG;
    if (N == 0) return HCGS_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    HCGS_KERNEL(ctx, "k_init_targets", st, k_init_targets<<<(N + 255) / 256, 256, 0, st>>>(amplitude, phase, N, C, target));
    return HCGS_OK;
}

hcgs_status hcgs_init_apply(hcgs_ctx* ctx, const float* y, int N, int C, float* amplitude, float* phase,
                            void* stream) {
    if (!ctx || !y || !amplitude || !phase || N < 0 || C < 1 || C > 8) return HCGS_ERR_INVALID_ARG;
    if (N == 0) return HCGS_OK;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    HCGS_KERNEL(ctx, "k_init_apply", st, k_init_apply<<<(N + 255) / 256, 256, 0, st>>>(y, N, C, amplitude, phase));
    return HCGS_OK;
}

}  // extern "C"
