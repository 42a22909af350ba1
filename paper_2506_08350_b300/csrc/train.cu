// Training-step pieces: fused Adam update and a deterministic sum of loss
// partials.
#include "common.cuh"

namespace hcgs {

// One element of the Adam update: p -= lr m^/(sqrt(v^)+eps) with
// bias-corrected moments (c1 = 1/(1-b1^t), c2 = 1/(1-b2^t)).
__device__ __forceinline__ void adam_elem(float* __restrict__ p, const float* __restrict__ g,
                                          float* __restrict__ m, float* __restrict__ v, int64_t i, float lr,
                                          float b1, float b2, float eps, float c1, float c2) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        adam_elem(p, g, m, v, i, lr, b1, b2, eps, c1, c2);
}

// Several parameter arrays in one launch: block b works on array a with
// first[a] <= b < first[a + 1], on its OPT_EPB elements from
// (b - first[a]) OPT_EPB; the arithmetic is adam_elem's, so the result is
// the same as one k_adam launch per array.
__global__ void __launch_bounds__(OPT_THREADS) k_adam_multi(OptArrays A, float b1, float b2, float eps, float c1,
                                                            float c2) {
    int a = 0;
    while (a + 1 < A.k && (int64_t)blockIdx.x >= A.first[a + 1]) a++;
    const int64_t base = ((int64_t)blockIdx.x - A.first[a]) * OPT_EPB;
    for (int e = threadIdx.x; e < OPT_EPB; e += OPT_THREADS) {
        const int64_t i = base + e;
        if (i < A.count[a]) adam_elem(A.p[a], A.g[a], A.m[a], A.v[a], i, A.lr[a], b1, b2, eps, c1, c2);
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

// Block prefix of the arrays of A (OPT_EPB elements per block); returns the
// total number of blocks.
int64_t opt_blocks(OptArrays& A) {
    A.first[0] = 0;
    for (int a = 0; a < A.k; a++) A.first[a + 1] = A.first[a] + (A.count[a] + OPT_EPB - 1) / OPT_EPB;
    return A.first[A.k];
}

hcgs_status adam_multi(hcgs_ctx* ctx, OptArrays& A, int step, float b1, float b2, float eps, cudaStream_t st) {
    const int64_t blocks = opt_blocks(A);
    if (blocks == 0) return HCGS_OK;
    const float c1 = (float)(1.0 / (1.0 - pow((double)b1, step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)b2, step)));
    HCGS_KERNEL(ctx, "k_adam", st, k_adam_multi<<<(unsigned)blocks, OPT_THREADS, 0, st>>>(A, b1, b2, eps, c1, c2));
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
