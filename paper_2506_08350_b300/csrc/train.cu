// Training-step pieces: fused Adam update and a deterministic sum of loss
// partials.
#include "common.cuh"

namespace hcgs {

// p -= lr m^/(sqrt(v^)+eps) with bias-corrected moments; float4 when aligned.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

hcgs_status adam(hcgs_ctx* ctx, float* p, const float* g, float* m, float* v, int64_t n, int step, float lr,
                 float b1, float b2, float eps, cudaStream_t st) {
    if (n <= 0) return HCGS_OK;
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)b2, step)));
    int64_t blocks = (n + 255) / 256;
    if (blocks > 148 * 16) blocks = 148 * 16;
    HCGS_KERNEL(ctx, "k_adam", st, k_adam<<<(unsigned)blocks, 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2));
    HCGS_LAUNCH(ctx, "k_adam");
    return HCGS_OK;
}

// out[0] = scale * sum(partials[0..n)), one block, fixed order.
__global__ void k_reduce_sum(const float* __restrict__ partials, int n, float scale, float* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[0] = (float)(t * scale);
    }
}

hcgs_status reduce_sum(hcgs_ctx* ctx, const float* partials, int n, float scale, float* out, cudaStream_t st) {
    HCGS_KERNEL(ctx, "k_reduce_sum", st, k_reduce_sum<<<1, 1024, 0, st>>>(partials, n, scale, out));
    HCGS_LAUNCH(ctx, "k_reduce_sum");
    return HCGS_OK;
}

}  // namespace hcgs
