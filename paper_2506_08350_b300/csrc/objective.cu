// The paper's training objective on sm_103a: L = L_recon + L_SSIM on the
// focal stack (the loss paragraph of Sec. 3), and the Adan optimiser step
// (Sec. 5, implementation).
//
//   L_recon = mean over (view, plane, channel, pixel) of d^2 (1 + M + I_gt^2),
//             d = I - I_gt, M the binary plane mask (|I M - I_gt M|^2 and
//             |I I_gt - I_gt I_gt|^2 are d^2 M and d^2 I_gt^2);
//   L_SSIM  = lambda_1 mean over (view, plane, channel) of (1 - SSIM).
// SSIM is the structural similarity of Wang et al.: local means, variances
// and covariance under an 11 x 11 Gaussian window (standard deviation 1.5,
// the image continued by zeros), constants C1 = 0.01^2, C2 = 0.03^2.  With
// n the number of intensity values, L = lambda_1 + (1/n) sum (d^2 w -
// lambda_1 S) and dL/dI = (2 d w - lambda_1 (G(dS/dmx) + 2 I G(dS/d<x^2>) +
// I_gt G(dS/d<xy>))) / n, G the (self-adjoint) window average.
#include <cmath>

#include "common.cuh"

namespace hcgs {

constexpr int SS_R = 5;                 // window radius
constexpr int SS_T = 32;                // output tile (SS_T x SS_T pixels)
constexpr int SS_E = SS_T + 2 * SS_R;   // tile with halo
constexpr int SS_TY = 8;                // threads: SS_T x SS_TY, four rows each
constexpr float SS_C1 = 0.01f * 0.01f, SS_C2 = 0.03f * 0.03f;

// the normalised 1D factor of the window, formed on the host in double
__constant__ float c_ssim_g[2 * SS_R + 1];

static cudaError_t ssim_window_upload() {
    static bool done = false;  // one upload per process (the table never changes)
    if (done) return cudaSuccess;
    double g[2 * SS_R + 1], s = 0.0;
    for (int k = 0; k <= 2 * SS_R; k++) {
        const double x = k - SS_R;
        g[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    float gf[2 * SS_R + 1];
    for (int k = 0; k <= 2 * SS_R; k++) gf[k] = (float)(g[k] / s);
    const cudaError_t e = cudaMemcpyToSymbol(c_ssim_g, gf, sizeof(gf));
    if (e == cudaSuccess) done = true;
    return e;
}

// Window averages of NQ quantities at the tile's pixels: q holds the NQ
// inputs on the halo tile [NQ][SS_E][SS_E] (zeros outside the image); the
// horizontal pass goes to h [NQ][SS_E][SS_T], the vertical one to the caller.
template <int NQ>
__device__ __forceinline__ void window_rows(const float (*q)[SS_E][SS_E], float (*h)[SS_E][SS_T]) {
    for (int e = threadIdx.y * SS_T + threadIdx.x; e < SS_E * SS_T; e += SS_T * SS_TY) {
        const int r = e / SS_T, cc = e % SS_T;
#pragma unroll
        for (int k = 0; k < NQ; k++) {
            float s = 0.f;
#pragma unroll
            for (int t = 0; t <= 2 * SS_R; t++) s = fmaf(c_ssim_g[t], q[k][r][cc + t], s);
            h[k][r][cc] = s;
        }
    }
}

template <int NQ>
__device__ __forceinline__ void window_col(const float (*h)[SS_E][SS_T], int r, int cc, float (&out)[NQ]) {
#pragma unroll
    for (int k = 0; k < NQ; k++) {
        float s = 0.f;
#pragma unroll
        for (int t = 0; t <= 2 * SS_R; t++) s = fmaf(c_ssim_g[t], h[k][r + t][cc], s);
        out[k] = s;
    }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = (threadIdx.y * SS_T + threadIdx.x) >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0 && threadIdx.y == 0)
        for (int i = 0; i < SS_T * SS_TY / 32; i++) s += red[i];  // fixed order: deterministic
    return s;
}

// Pass 1 over each (view, plane, channel) image: the SSIM map's partial
// derivatives dS/dmx, dS/d<x^2>, dS/d<xy> (written to dmap[3][n]) and the
// block's part of sum (d^2 w + lambda (1 - S)).  The intensities come either
// from I or, when V is given, as |V|^2 of the propagated field (then also
// written to I for pass 2).  grid (tiles x, tiles y, B L C).
template <bool FROM_FIELD>
__global__ void __launch_bounds__(SS_T * SS_TY)
    k_ssim_partials(const float2* __restrict__ V, float* __restrict__ I, const float* __restrict__ Igt,
                    const float* __restrict__ M, int C, int H, int W, float lam, float* __restrict__ dmap,
                    float* __restrict__ partials) {
    __shared__ float q[2][SS_E][SS_E];
    __shared__ float h[5][SS_E][SS_T];
    __shared__ float red[SS_T * SS_TY / 32];
    const int img = blockIdx.z;
    const size_t HW = (size_t)H * W, n = (size_t)gridDim.z * HW;
    const float* y = Igt + (size_t)img * HW;
    const float* m = M ? M + (size_t)(img / C) * HW : nullptr;  // masks per (view, plane)
    const int x0 = blockIdx.x * SS_T - SS_R, y0 = blockIdx.y * SS_T - SS_R;
    for (int e = threadIdx.y * SS_T + threadIdx.x; e < SS_E * SS_E; e += SS_T * SS_TY) {
        const int r = e / SS_E, cc = e % SS_E, gy = y0 + r, gx = x0 + cc;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        float xv = 0.f;
        if (in) {
            if constexpr (FROM_FIELD) {
                const float2 v = V[p];
                xv = fmaf(v.x, v.x, v.y * v.y);
            } else {
                xv = I[p];
            }
        }
        q[0][r][cc] = xv;
        q[1][r][cc] = in ? y[(size_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    // horizontal window sums of x, y, x^2, y^2, x y
    for (int e = threadIdx.y * SS_T + threadIdx.x; e < SS_E * SS_T; e += SS_T * SS_TY) {
        const int r = e / SS_T, cc = e % SS_T;
        float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= 2 * SS_R; t++) {
            const float a = q[0][r][cc + t], b = q[1][r][cc + t], g = c_ssim_g[t];
            s[0] = fmaf(g, a, s[0]);
            s[1] = fmaf(g, b, s[1]);
            s[2] = fmaf(g, a * a, s[2]);
            s[3] = fmaf(g, b * b, s[3]);
            s[4] = fmaf(g, a * b, s[4]);
        }
#pragma unroll
        for (int k = 0; k < 5; k++) h[k][r][cc] = s[k];
    }
    __syncthreads();
    float acc = 0.f;
    const int cc = threadIdx.x, gx = blockIdx.x * SS_T + cc;
#pragma unroll
    for (int k = 0; k < SS_T / SS_TY; k++) {
        const int r = threadIdx.y + k * SS_TY, gy = blockIdx.y * SS_T + r;
        if (gx >= W || gy >= H) continue;
        float mu[5];
        window_col<5>(h, r, cc, mu);
        const float mx = mu[0], my = mu[1];
        const float sxx = mu[2] - mx * mx, syy = mu[3] - my * my, sxy = mu[4] - mx * my;
        const float a = 2.f * mx * my + SS_C1, b = 2.f * sxy + SS_C2;
        const float c = mx * mx + my * my + SS_C1, d = sxx + syy + SS_C2;
        const float icd = 1.f / (c * d);
        const float S = a * b * icd;
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        dmap[p] = 2.f * my * (b - a) * icd - 2.f * mx * S / c + 2.f * mx * S / d;
        dmap[n + p] = -S / d;
        dmap[2 * n + p] = 2.f * a * icd;
        const float xv = q[0][r + SS_R][cc + SS_R], yv = q[1][r + SS_R][cc + SS_R];
        if constexpr (FROM_FIELD) I[p] = xv;
        const float dl = xv - yv;
        const float w = 1.f + (m ? m[(size_t)gy * W + gx] : 0.f) + yv * yv;
        acc += dl * dl * w + lam * (1.f - S);
    }
    const float s = block_sum(acc, red);
    if (threadIdx.x == 0 && threadIdx.y == 0)
        partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

// Pass 2: g = dL/dI = (2 d w - lambda (G dmap0 + 2 I G dmap1 + I_gt G dmap2)) / n,
// written to gI, or (TO_FIELD) turned into dL/dV = 2 g V in place over V.
template <bool TO_FIELD>
__global__ void __launch_bounds__(SS_T * SS_TY)
    k_ssim_grad(const float* __restrict__ I, const float* __restrict__ Igt, const float* __restrict__ M, int C,
                int H, int W, float lam, float inv_n, const float* __restrict__ dmap, float* __restrict__ gI,
                float2* __restrict__ V) {
    __shared__ float q[3][SS_E][SS_E];
    __shared__ float h[3][SS_E][SS_T];
    const int img = blockIdx.z;
    const size_t HW = (size_t)H * W, n = (size_t)gridDim.z * HW;
    const int x0 = blockIdx.x * SS_T - SS_R, y0 = blockIdx.y * SS_T - SS_R;
    for (int e = threadIdx.y * SS_T + threadIdx.x; e < SS_E * SS_E; e += SS_T * SS_TY) {
        const int r = e / SS_E, cc = e % SS_E, gy = y0 + r, gx = x0 + cc;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
#pragma unroll
        for (int k = 0; k < 3; k++) q[k][r][cc] = in ? dmap[k * n + p] : 0.f;
    }
    __syncthreads();
    window_rows<3>(q, h);
    __syncthreads();
    const int cc = threadIdx.x, gx = blockIdx.x * SS_T + cc;
    const float* m = M ? M + (size_t)(img / C) * HW : nullptr;
#pragma unroll
    for (int k = 0; k < SS_T / SS_TY; k++) {
        const int r = threadIdx.y + k * SS_TY, gy = blockIdx.y * SS_T + r;
        if (gx >= W || gy >= H) continue;
        float gd[3];
        window_col<3>(h, r, cc, gd);
        const size_t p = (size_t)img * HW + (size_t)gy * W + gx;
        const float xv = I[p], yv = Igt[p];
        const float w = 1.f + (m ? m[(size_t)gy * W + gx] : 0.f) + yv * yv;
        const float g = inv_n * (2.f * (xv - yv) * w - lam * (gd[0] + 2.f * xv * gd[1] + yv * gd[2]));
        if constexpr (TO_FIELD) {
            const float2 v = V[p];
            V[p] = make_float2(2.f * g * v.x, 2.f * g * v.y);
        } else {
            gI[p] = g;
        }
    }
}

// Loss partials and gradient of L_recon + L_SSIM for B L C images of H x W.
// V != nullptr: intensities |V|^2 (written to I), gradient dL/dV over V;
// otherwise intensities read from I and dL/dI written to gI.  dmap holds
// 3 B L C H W floats; partials one float per block (query with partials = NULL).
hcgs_status ssim_recon_loss(hcgs_ctx* ctx, float2* V, float* I, const float* Igt, const float* M, int B, int L,
                            int C, int H, int W, float lam, float* dmap, float* partials, int* nblocks_out,
                            float* gI, cudaStream_t st) {
    const dim3 grid((W + SS_T - 1) / SS_T, (H + SS_T - 1) / SS_T, B * L * C);
    *nblocks_out = (int)(grid.x * grid.y * grid.z);
    if (!partials) return HCGS_OK;  // size query
    HCGS_CUDA(ctx, ssim_window_upload());
    const dim3 blk(SS_T, SS_TY);
    const float inv_n = (float)(1.0 / ((double)B * L * C * H * W));
    if (V) {
        HCGS_KERNEL(ctx, "k_ssim_partials", st,
                    k_ssim_partials<true><<<grid, blk, 0, st>>>(V, I, Igt, M, C, H, W, lam, dmap, partials));
        HCGS_KERNEL(ctx, "k_ssim_grad", st,
                    k_ssim_grad<true><<<grid, blk, 0, st>>>(I, Igt, M, C, H, W, lam, inv_n, dmap, nullptr, V));
    } else {
        HCGS_KERNEL(ctx, "k_ssim_partials", st,
                    k_ssim_partials<false><<<grid, blk, 0, st>>>(nullptr, I, Igt, M, C, H, W, lam, dmap, partials));
        HCGS_KERNEL(ctx, "k_ssim_grad", st,
                    k_ssim_grad<false><<<grid, blk, 0, st>>>(I, Igt, M, C, H, W, lam, inv_n, dmap, gI, nullptr));
    }
    return HCGS_OK;
}

// ---------------------------------------------------------------------------
// Adan (Xie et al., Algorithm 1), decay-factor form: first step m = g, v = 0,
// n = g^2; second step v = g - g_prev; then the moving averages
//   m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2)(g - g_prev),
//   n <- b3 n + (1 - b3)(g + b2 (g - g_prev))^2;
// p <- (p - lr (m + b2 v) / (sqrt(n) + eps)) / (1 + wd lr); g_prev <- g.
// ---------------------------------------------------------------------------
__global__ void k_adan(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ gp,
                       float* __restrict__ m, float* __restrict__ v, float* __restrict__ nn, int64_t count,
                       int step, float lr, float b1, float b2, float b3, float eps, float wd) {
    const float shrink = 1.f / (1.f + wd * lr);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        float mi, vi, ni;
        if (step == 1) {
            mi = gi;
            vi = 0.f;
            ni = gi * gi;
        } else {
            const float dg = gi - gp[i];
            mi = fmaf(b1, m[i], (1.f - b1) * gi);
            vi = step == 2 ? dg : fmaf(b2, v[i], (1.f - b2) * dg);
            const float u = fmaf(b2, dg, gi);
            ni = fmaf(b3, nn[i], (1.f - b3) * u * u);
        }
        m[i] = mi;
        v[i] = vi;
        nn[i] = ni;
        gp[i] = gi;
        p[i] = (p[i] - lr * fmaf(b2, vi, mi) / (sqrtf(ni) + eps)) * shrink;
    }
}

hcgs_status adan(hcgs_ctx* ctx, float* p, const float* g, float* gp, float* m, float* v, float* n, int64_t count,
                 int step, float lr, float b1, float b2, float b3, float eps, float wd, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>(148 * 16, (count + 255) / 256);
    HCGS_KERNEL(ctx, "k_adan", st, k_adan<<<blocks, 256, 0, st>>>(p, g, gp, m, v, n, count, step, lr, b1, b2, b3, eps, wd));
    return HCGS_OK;
}

}  // namespace hcgs
